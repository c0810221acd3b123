"""Seeded synthetic inputs for the RS-SRI-GF2 self-energy path.

This module only *draws inputs*; it holds none of the method's arithmetic
(no screening, no metric root, no Green's function, no self-energy).  Both the
CUDA path and the fp64 oracle are fed from here, so the two sides see the same
arrays.

The inputs stand in for the paper's hydrogen-dimer chains (Sec. IV: STO-3G AO
basis, cc-pVDZ-RI auxiliary basis, beta = 50 1/Eh).  The real integrals and
basis sets are not available, so a chain-like law is used instead:

* 3-index integrals (ij|A) = N_aux^{-1/2} g_ijA exp(-|i-j|/decay), g ~ N(0,1)
  drawn for i <= j and mirrored, so (ij|A) = (ji|A) (Eq. 5 symmetry);
* Coulomb metric V = B B^T / N_aux + 0.5 I with B ~ N(0,1): symmetric positive
  definite, condition number about 9 (Eq. 6 is SPD);
* orbital energies: occupied linspace(-1.0, -0.2), virtual linspace(0.2, 2.0),
  a 0.4 Eh gap with the chemical potential mu = 0 in the middle;
* orbital coefficients: the orthogonal factor of the QR decomposition of an
  N(0,1) matrix with diag(R) > 0, i.e. an orthonormal AO basis (S = I, Eq. 2);
* imaginary-time grid: Gauss-Legendre in u = ln(1 + tau/tau_s) on
  [0, ln(1 + beta/tau_s)], so dense near tau = 0 where G varies fastest; the
  weights carry the Jacobian d tau / d u = tau + tau_s.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

__all__ = ["System", "make_system", "make_system_torch", "tau_grid", "CONFIGS", "MANY", "C4",
           "many_sizes"]


@dataclass
class System:
    """One synthetic problem, all arrays float64, C-contiguous."""

    n: int
    n_occ: int
    n_aux: int
    eri3: np.ndarray  # [n][n][n_aux], (ij|A)
    metric: np.ndarray  # [n_aux][n_aux], V_AB
    orb_e: np.ndarray  # [n], ascending; first n_occ occupied
    orb_c: np.ndarray  # [n][n], AO x MO
    mu: float
    beta: float
    tau: np.ndarray  # [n_tau] nodes in (0, beta)
    tau_w: np.ndarray  # [n_tau] quadrature weights

    @property
    def n_tau(self) -> int:
        return int(self.tau.shape[0])


def tau_grid(n_tau: int, beta: float = 50.0, tau_s: float = 0.5):
    """Gauss-Legendre nodes/weights in u = ln(1 + tau/tau_s) mapped to tau."""
    x, w = np.polynomial.legendre.leggauss(n_tau)
    umax = np.log1p(beta / tau_s)
    u = 0.5 * (x + 1.0) * umax
    wu = 0.5 * umax * w
    tau = tau_s * np.expm1(u)
    return np.ascontiguousarray(tau), np.ascontiguousarray(wu * (tau + tau_s))


def make_system(n: int, n_occ: int, n_aux: int, n_tau: int, input_seed: int = 0,
                beta: float = 50.0, tau_s: float = 0.5, decay: float = 3.0,
                gap_lo: float = -0.2, gap_hi: float = 0.2) -> System:
    if not (0 < n_occ < n):
        raise ValueError("need 0 < n_occ < n")
    rng = np.random.default_rng(input_seed)
    # (ij|A): one draw per unordered pair i <= j, mirrored
    g = rng.standard_normal((n, n, n_aux))
    iu, ju = np.triu_indices(n, 1)
    g[ju, iu, :] = g[iu, ju, :]
    idx = np.arange(n)
    damp = np.exp(-np.abs(idx[:, None] - idx[None, :]) / decay) / np.sqrt(n_aux)
    g *= damp[:, :, None]  # in place: one [n][n][n_aux] array on the host at a time
    eri3 = g
    # SPD metric
    b = rng.standard_normal((n_aux, n_aux))
    metric = b @ b.T / n_aux + 0.5 * np.eye(n_aux)
    metric = np.ascontiguousarray(0.5 * (metric + metric.T))
    # orbitals
    orb_e = np.concatenate([np.linspace(-1.0, gap_lo, n_occ),
                            np.linspace(gap_hi, 2.0, n - n_occ)])
    q, r = np.linalg.qr(rng.standard_normal((n, n)))
    q = q * np.sign(np.diag(r))[None, :]
    tau, tau_w = tau_grid(n_tau, beta, tau_s)
    return System(n=n, n_occ=n_occ, n_aux=n_aux, eri3=eri3, metric=metric,
                  orb_e=np.ascontiguousarray(orb_e), orb_c=np.ascontiguousarray(q),
                  mu=0.5 * (gap_lo + gap_hi), beta=beta, tau=tau, tau_w=tau_w)


def make_system_torch(n: int, n_occ: int, n_aux: int, n_tau: int, input_seed: int = 0,
                      device: str = "cuda", beta: float = 50.0, tau_s: float = 0.5,
                      decay: float = 3.0, gap_lo: float = -0.2, gap_hi: float = 0.2) -> System:
    """The recipe of make_system drawn on `device` with a seeded torch
    generator (other numbers than make_system's, the same distribution and
    structure): for the many-chain workload, whose largest (ij|A) (12 GB at
    N = 800) would take minutes to draw and copy from the host.  Arrays are
    float64 torch tensors on `device`; tau and its weights as in tau_grid."""
    import torch

    if not (0 < n_occ < n):
        raise ValueError("need 0 < n_occ < n")
    gen = torch.Generator(device=device)
    gen.manual_seed(int(input_seed))
    f64 = dict(dtype=torch.float64, device=device)
    eri3 = torch.randn((n, n, n_aux), generator=gen, **f64)
    iu, ju = torch.triu_indices(n, n, 1, device=device)
    eri3[ju, iu, :] = eri3[iu, ju, :]
    idx = torch.arange(n, **f64)
    damp = torch.exp(-torch.abs(idx[:, None] - idx[None, :]) / decay) / float(np.sqrt(n_aux))
    eri3 *= damp[:, :, None]
    b = torch.randn((n_aux, n_aux), generator=gen, **f64)
    metric = b @ b.T / n_aux + 0.5 * torch.eye(n_aux, **f64)
    metric = (0.5 * (metric + metric.T)).contiguous()
    del b
    orb_e = torch.cat([torch.linspace(-1.0, gap_lo, n_occ, **f64),
                       torch.linspace(gap_hi, 2.0, n - n_occ, **f64)])
    # the QR on the host (small; no dependence on the device linear-algebra library)
    q, r = torch.linalg.qr(torch.randn((n, n), generator=gen, **f64).cpu())
    q = (q * torch.sign(torch.diagonal(r))[None, :]).contiguous().to(device)
    tau, tau_w = tau_grid(n_tau, beta, tau_s)
    return System(n=n, n_occ=n_occ, n_aux=n_aux, eri3=eri3.contiguous(), metric=metric,
                  orb_e=orb_e.contiguous(), orb_c=q, mu=0.5 * (gap_lo + gap_hi), beta=beta,
                  tau=torch.from_numpy(tau).to(device), tau_w=torch.from_numpy(tau_w).to(device))


def mlp_init(seed: int = 0, zero_output: bool = True) -> np.ndarray:
    """Initial parameters of the control-variate network as the flat float32
    layout W0[256][10] b0[256] W1[256][256] b1 W2[256][256] b2 W3[1][256] b3[1]:
    He-normal hidden weights, zero biases, and a zero output layer (so the
    network starts at c = 1) unless zero_output is False."""
    rng = np.random.default_rng(seed)
    sizes = [10, 256, 256, 256, 1]
    parts = []
    for k in range(4):
        w = rng.standard_normal((sizes[k + 1], sizes[k])) * np.sqrt(2.0 / sizes[k])
        if k == 3 and zero_output:
            w[:] = 0.0
        parts += [w.ravel(), np.zeros(sizes[k + 1])]
    return np.concatenate(parts).astype(np.float32)


def mlp_unflatten(flat: np.ndarray):
    """The flat layout of mlp_init as [(W, b), ...] float64 arrays."""
    sizes = [10, 256, 256, 256, 1]
    out, o = [], 0
    for k in range(4):
        nw = sizes[k + 1] * sizes[k]
        w = flat[o:o + nw].astype(np.float64).reshape(sizes[k + 1], sizes[k])
        o += nw
        b = flat[o:o + sizes[k + 1]].astype(np.float64)
        o += sizes[k + 1]
        out.append((w, b))
    return out


# The five workloads the method is exercised on (sizes only; eps is the K^L cut
# of Eq. 13, eps_prime the (ij|A) screen of Eq. 11 at the paper's 0.02).
CONFIGS = {
    "c1_n20": dict(n=20, n_occ=10, n_aux=60, n_tau=32, n_s=64, eps=1e-2,
                   eps_prime=0.02, seeds=(0,)),
    "c2_n200": dict(n=200, n_occ=100, n_aux=600, n_tau=64, n_s=300, eps=1e-3,
                    eps_prime=0.02, seeds=tuple(range(10))),
    "c3_n1000": dict(n=1000, n_occ=500, n_aux=3000, n_tau=128, n_s=500, eps=1e-3,
                     eps_prime=0.02, seeds=(0,)),
}

# Many independent chains of uneven size (a reduced form of the 64-chain
# batch, N from 100 to 800, whose deterministic blocks alone would take tens
# of minutes): K chains with N_k spread evenly over [n_min, n_max], N_aux = 3N,
# n_occ = N/2, input seed k.
MANY = dict(k=16, n_min=64, n_max=256, n_tau=16, n_s=64, eps=1e-3, eps_prime=0.02)
# The many-chain workload: 64 chains, N_k = 100 + round(700 k / 63), n_occ = N/2,
# N_aux = 3N, 64 tau points, 200 sample pairs each, eps = 1e-3.
C4 = dict(k=64, n_min=100, n_max=800, n_tau=64, n_s=200, eps=1e-3, eps_prime=0.02)


def many_sizes(k: int, n_min: int, n_max: int):
    """N_k = n_min + round((n_max - n_min) k / (K - 1)), k = 0..K-1."""
    if k == 1:
        return [n_min]
    return [n_min + int(round((n_max - n_min) * i / (k - 1))) for i in range(k)]
