"""RS-SRI-GF2 self-energy and correlation energy, plain fp64 numpy.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Notation follows the paper: N basis functions, N_aux auxiliary functions,
(ij|A) the 3-index integrals (Eq. 5), V the Coulomb metric (Eq. 6),
K^Q_ij = sum_A (ij|A) V^{-1/2}_AQ (Eq. 7), theta^xi the stochastic orbitals,
R^xi (Eq. 9), [K^Q]^L and R^L, R^S (Eqs. 12-15), G(tau) (Eq. 17),
Sigma(tau) (Eq. 20 / Eq. 25) and E_corr (Eq. 26).  Gb(tau) denotes
G(beta - tau).

Readings of the paper taken here (each is also listed in the design notes):
  * Eq. 11 "max for each j": M_j = max_{i,A} |(ij|A)|; an element is kept
    when it passes the test of either of its two orbital indices, i.e.
    |(ij|A)| >= (eps'/N) min(M_i, M_j).  This keeps (ij|A)^L symmetric.
  * Eq. 13: the maximum is the global one over (i, j, Q); ties are kept.
  * G at zero temperature from given orbitals (Eq. 17 with occupations 1/0):
    G(tau) = -C_v exp(-(e_v - mu) tau) C_v^T and
    G(beta - tau) = -C_o exp((e_o - mu) tau) C_o^T, tau in (0, beta).
  * theta and theta' of Eq. 25 are independent; sample xi of theta is paired
    with sample xi of theta' (N_s pairs, O(N_s N^3) work as in Sec. II).
  * Default estimator ("cv"): Sigma = Sigma_DD + (1/N_s) sum_xi
    [F(R^xi, R'^xi) - F(R^Lxi, R'^Lxi)], where Sigma_DD is Eq. 20 with
    v = sum_Q [K^Q]^L [K^Q]^L.  Every bracket of Eq. 25 equals
    D + <R R> - <R^L R^L>; the cv form keeps D D exactly and pairs the
    stochastic products.  The "literal" mode expands Eq. 25's product of
    brackets term by term instead.  Both have the RI self-energy as mean.
  * Sign of Eq. 26: E_corr = -(1/N_e) int_0^beta Tr[Sigma(tau) G(beta-tau)],
    which is the MP2 energy per electron for a Hartree-Fock G.
  * The reported self-energy is symmetrised, (Sigma + Sigma^T)/2, which does
    not change its mean nor Tr[Sigma Gb].
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .rng import rademacher

__all__ = [
    "metric_inv_sqrt", "ri_factor", "eri4_from_factor", "screen",
    "large_factor", "stochastic_factors", "green", "sigma_eri4",
    "factor_pair", "sigma_from_factor", "energy_trace", "RsSriResult",
    "rs_sri", "pair_energies_split",
]


# ---------------------------------------------------------------- Sec. II ---
def metric_inv_sqrt(metric: np.ndarray) -> np.ndarray:
    """V^{-1/2}: the symmetric inverse square root used in Eq. 7.

    Eigen-decomposition V = U diag(lam) U^T, V^{-1/2} = U diag(lam^-1/2) U^T.
    Raises ValueError if V is not positive definite.
    """
    lam, u = np.linalg.eigh(metric)
    if not np.all(lam > 0):
        raise ValueError("metric not positive definite")
    return (u * lam ** -0.5) @ u.T


def ri_factor(eri3: np.ndarray, w: np.ndarray) -> np.ndarray:
    """Eq. 7: K^Q_ij = sum_A (ij|A) V^{-1/2}_AQ, returned as [N, N, N_aux]."""
    n, _, naux = eri3.shape
    return (eri3.reshape(n * n, naux) @ w).reshape(n, n, naux)


def eri4_from_factor(k: np.ndarray) -> np.ndarray:
    """Eq. 8: v_ijkl = sum_Q K^Q_ij K^Q_kl (chemists' order (ij|kl))."""
    n = k.shape[0]
    kf = k.reshape(n * n, -1)
    return (kf @ kf.T).reshape(n, n, n, n)


def screen(eri3: np.ndarray, eps_prime: float):
    """Eq. 11: keep (ij|A) where |(ij|A)| >= (eps'/N) min(M_i, M_j).

    M_j = max over (i, A) of |(ij|A)|.  Returns ((ij|A)^L, mask, M).
    """
    n = eri3.shape[0]
    a = np.abs(eri3)
    m = a.max(axis=(0, 2))
    thr = (eps_prime / n) * np.minimum(m[:, None], m[None, :])
    mask = a >= thr[:, :, None]
    return np.where(mask, eri3, 0.0), mask, m


def large_factor(eri3_l: np.ndarray, w: np.ndarray, eps: float):
    """Eqs. 12-13: [K^Q_ij]^L = sum_A (ij|A)^L V^{-1/2}_AQ, then entries below
    eps times the global maximum of |[K^Q_ij]^L| are set to zero.

    Returns (K^L [N, N, N_aux], max |K^L| before the cut).
    """
    kl = ri_factor(eri3_l, w)
    kmax = float(np.abs(kl).max()) if kl.size else 0.0
    kl = np.where(np.abs(kl) >= eps * kmax, kl, 0.0)
    return kl, kmax


def stochastic_factors(eri3: np.ndarray, w: np.ndarray, k_l: np.ndarray,
                       theta: np.ndarray):
    """Eq. 9 and Eqs. 14-15 for a block of stochastic orbitals.

    R^xi_ij = sum_A (ij|A) sum_Q V^{-1/2}_AQ theta^xi_Q,
    [R^xi_ij]^L = sum_Q [K^Q_ij]^L theta^xi_Q, R^S = R - R^L.
    theta: [N_s, N_aux].  Returns (R, R^L), each [N_s, N, N].
    """
    n, _, naux = eri3.shape
    ns = theta.shape[0]
    u = w @ theta.T  # [N_aux, N_s]
    r = (eri3.reshape(n * n, naux) @ u).T.reshape(ns, n, n)
    rl = (k_l.reshape(n * n, naux) @ theta.T).T.reshape(ns, n, n)
    return r, rl


# --------------------------------------------------------------- Sec. III ---
def green(orb_e, orb_c, n_occ: int, mu: float, tau: float):
    """Eq. 17 for a non-interacting G at zero temperature, S = I.

    G(tau)        = -sum_{a virtual}  C_ia C_ja exp(-(e_a - mu) tau)
    G(beta - tau) = -sum_{i occupied} C_ii' C_ji' exp(+(e_i' - mu) tau)
    (the second from antiperiodicity, G(beta - tau) = -G(-tau)).
    """
    co, cv = orb_c[:, :n_occ], orb_c[:, n_occ:]
    eo, ev = orb_e[:n_occ], orb_e[n_occ:]
    g = -(cv * np.exp(-(ev - mu) * tau)[None, :]) @ cv.T
    gb = -(co * np.exp((eo - mu) * tau)[None, :]) @ co.T
    return g, gb


def sigma_eri4(v: np.ndarray, g: np.ndarray, gb: np.ndarray) -> np.ndarray:
    """Eq. 20 written out on 4-index integrals (brute force, tiny N only):

    Sigma_ij = sum_{klmnpq} v_imqk (2 v_lpnj - v_nplj) G_kl G_mn Gb_pq.
    """
    d = np.einsum("imqk,lpnj,kl,mn,pq->ij", v, v, g, g, gb, optimize="greedy")
    x = np.einsum("imqk,nplj,kl,mn,pq->ij", v, v, g, g, gb, optimize="greedy")
    return 2.0 * d - x


def factor_pair(x: np.ndarray, y: np.ndarray, g: np.ndarray, gb: np.ndarray):
    """Eq. 20 with rank-one integrals v_imqk = X_im X_qk, v_lpnj = Y_lp Y_nj.

    Walking the indices of Eq. 20: the direct term is
    2 (X G Y)_ij Tr(X G Y Gb), the exchange term (X G Y Gb X G Y)_ij.
    With C = X G Y, t = Tr(C Gb), B = C Gb:
        F = 2 t C - B C,   Tr(F Gb) = 2 t^2 - Tr(B B).
    Returns (F, t, Tr(B B)).
    """
    c = x @ g @ y
    b = c @ gb
    t = float(np.trace(b))
    s = float(np.sum(b * b.T))
    return 2.0 * t * c - b @ c, t, s


def sigma_from_factor(k: np.ndarray, g: np.ndarray, gb: np.ndarray, outer=None) -> np.ndarray:
    """Eq. 20 with v = sum_Q K^Q K^Q (Eq. 8): since Eq. 20 is bilinear in its
    two integrals, Sigma = sum_{Q, Q'} F(K^Q, K^Q').  Used for the RI
    self-energy and, with K = [K]^L, for the deterministic block of Eq. 25.
    outer: optionally restrict the first auxiliary index Q to these positions
    among the non-zero K^Q (partial sums, for timing samples).
    """
    kq = np.ascontiguousarray(np.moveaxis(k, 2, 0))  # [N_aux, N, N]
    keep = np.flatnonzero(np.abs(kq).reshape(kq.shape[0], -1).max(axis=1) > 0)
    kq = kq[keep]
    out = np.zeros_like(g)
    for q in (range(kq.shape[0]) if outer is None else outer):
        c = (kq[q] @ g) @ kq  # [N_aux', N, N]: C = K^Q G K^Q' for all Q'
        b = c @ gb
        t = np.trace(b, axis1=1, axis2=2)
        out += 2.0 * np.einsum("q,qij->ij", t, c) - (b @ c).sum(axis=0)
    return out


def energy_trace(sigma_tau: np.ndarray, gb_tau, tau_w: np.ndarray, n_occ: int) -> float:
    """Eq. 26 (sign reading above): -(1/N_e) sum_tau w_tau Tr[Sigma Gb]."""
    ne = 2 * n_occ
    tr = np.array([np.sum(s * gb.T) for s, gb in zip(sigma_tau, gb_tau)])
    return float(-np.dot(tau_w, tr) / ne)


# ------------------------------------------------------------ the estimator --
@dataclass
class RsSriResult:
    sigma: np.ndarray  # [N_tau, N, N], symmetrised
    sigma_raw: np.ndarray  # [N_tau, N, N], before symmetrisation
    sigma_dd: np.ndarray  # [N_tau, N, N], deterministic block
    e_corr: float  # Eq. 26 from sigma
    e_stderr: float  # sample std of e_pair / sqrt(N_s)
    e_pair: np.ndarray  # [N_s] per-pair estimates; mean(e_pair) == e_corr
    e_dd: float  # Eq. 26 for the deterministic block alone
    extra: dict = field(default_factory=dict)


def pair_energies_split(r, rl, r1, rl1, g, gb):
    """Range-separated split of one sample pair (Eqs. 14-15, R = R^L + R^S).

    With C^L = R^L G R'^L and dC = R^S G R' + R^L G R'^S (so C = C^L + dC):
        F(R, R') - F(R^L, R'^L) = 2 (dC t + C^L dt) - (dC Gb C + C^L Gb dC)
    where t = Tr(C Gb), dt = Tr(dC Gb).  Returns (that difference,
    (2 t^2 - s) - (2 t_L^2 - s_L)).
    """
    rs, rs1 = r - rl, r1 - rl1
    cl = rl @ g @ rl1
    dc = rs @ g @ r1 + rl @ g @ rs1
    c = cl + dc
    tl = float(np.sum(cl * gb.T))
    dt = float(np.sum(dc * gb.T))
    t = tl + dt
    dcg, clg = dc @ gb, cl @ gb
    diff = 2.0 * (dc * t + cl * dt) - (dcg @ c + clg @ dc)
    de = 2.0 * dt * (t + tl) - (float(np.sum(dcg * (c @ gb).T)) + float(np.sum(clg * dcg.T)))
    return diff, de


def rs_sri(eri3, metric, orb_e, orb_c, n_occ: int, mu: float, tau, tau_w,
           eps_prime: float, eps: float, n_s: int, seed: int, xi_offset: int = 0,
           mode: str = "cv", form: str = "difference", empty_large: bool = False,
           tau_index=None, theta=None) -> RsSriResult:
    """The RS-SRI-GF2 self-energy on a tau grid and E_corr (Eqs. 11-15, 25, 26).

    mode: "cv" (default reading) or "literal" (Eq. 25 expanded term by term).
    form: "difference" evaluates F(R,R') - F(R^L,R'^L) directly, "split" uses
          the R^S split of Eq. 15 (same value up to rounding).
    empty_large: force [K]^L = 0, the pure stochastic-RI limit (Sec. II).
    tau_index: optional subset of tau points to evaluate (energies then cover
          only that subset).
    theta: optional explicit (theta, theta') pair of [N_s, N_aux] arrays that
          replaces the seeded draws (used to enumerate all sign vectors).
    """
    n, _, naux = eri3.shape
    tau = np.asarray(tau, dtype=np.float64)
    tau_w = np.asarray(tau_w, dtype=np.float64)
    if tau_index is not None:
        tau, tau_w = tau[list(tau_index)], tau_w[list(tau_index)]
    ne = 2 * n_occ
    w = metric_inv_sqrt(metric)
    eri3_l, mask, mcol = screen(eri3, eps_prime)
    k_l, kmax = large_factor(eri3_l, w, eps)
    if empty_large:
        k_l = np.zeros_like(k_l)
    if theta is None:
        th0 = rademacher(seed, 0, n_s, naux, xi_offset)
        th1 = rademacher(seed, 1, n_s, naux, xi_offset)
    else:
        th0, th1 = (np.asarray(t, dtype=np.float64) for t in theta)
        n_s = th0.shape[0]
    r0, rl0 = stochastic_factors(eri3, w, k_l, th0)
    r1, rl1 = stochastic_factors(eri3, w, k_l, th1)

    nt = tau.shape[0]
    sig = np.zeros((nt, n, n))
    sdd = np.zeros((nt, n, n))
    gbs = []
    e_st = np.zeros(n_s)  # stochastic part of the per-pair energies
    for it in range(nt):
        g, gb = green(orb_e, orb_c, n_occ, mu, tau[it])
        gbs.append(gb)
        sdd[it] = sigma_from_factor(k_l, g, gb)
        acc = np.zeros((n, n))
        for xi in range(n_s):
            if mode == "cv":
                if form == "split":
                    diff, de = pair_energies_split(r0[xi], rl0[xi], r1[xi], rl1[xi], g, gb)
                else:
                    f, t, s = factor_pair(r0[xi], r1[xi], g, gb)
                    fl, tl, sl = factor_pair(rl0[xi], rl1[xi], g, gb)
                    diff, de = f - fl, (2 * t * t - s) - (2 * tl * tl - sl)
            elif mode == "literal":
                # Eq. 25 brackets: D + S_xi with S_xi = R(x)R - R^L(x)R^L.
                # Phi(D, S') + Phi(S, D) + Phi(S, S'), Phi bilinear.
                diff = np.zeros((n, n))
                for (x, sx) in ((r0[xi], 1.0), (rl0[xi], -1.0)):
                    for (y, sy) in ((r1[xi], 1.0), (rl1[xi], -1.0)):
                        f, _, _ = factor_pair(x, y, g, gb)
                        diff += sx * sy * f
                for q in range(naux):
                    kq = k_l[:, :, q]
                    if not np.any(kq):
                        continue
                    for (y, sy) in ((r1[xi], 1.0), (rl1[xi], -1.0)):
                        f1, _, _ = factor_pair(kq, y, g, gb)  # Phi(D, S')
                        diff += sy * f1
                    for (x, sx) in ((r0[xi], 1.0), (rl0[xi], -1.0)):
                        f2, _, _ = factor_pair(x, kq, g, gb)  # Phi(S, D)
                        diff += sx * f2
                de = float(np.sum(diff * gb.T))
            else:
                raise ValueError(mode)
            acc += diff
            e_st[xi] += -tau_w[it] * de / ne
        sig[it] = sdd[it] + acc / n_s
    e_dd = energy_trace(sdd, gbs, tau_w, n_occ)
    e_pair = e_dd + e_st
    sym = 0.5 * (sig + np.transpose(sig, (0, 2, 1)))
    e_corr = energy_trace(sym, gbs, tau_w, n_occ)
    stderr = float(np.std(e_pair, ddof=1) / np.sqrt(n_s)) if n_s > 1 else float("nan")
    extra = dict(w=w, mask=mask, m_col=mcol, k_l=k_l, k_l_max=kmax,
                 theta0=th0, theta1=th1, r0=r0, rl0=rl0, r1=r1, rl1=rl1,
                 nnz_eri_l=int(mask.sum()), nnz_k_l=int(np.count_nonzero(k_l)))
    return RsSriResult(sigma=sym, sigma_raw=sig, sigma_dd=sdd, e_corr=e_corr,
                       e_stderr=stderr, e_pair=e_pair, e_dd=e_dd, extra=extra)
