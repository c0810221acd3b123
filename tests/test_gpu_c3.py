"""GPU parity at N = 1000 (N_aux = 3000): the largest single-GPU workload.

The selection work (Eq. 11 screen, Eq. 13 cut) is compared exactly with the
oracle over every element; [K]^L over every kept row; R and R^L (Eqs. 9, 14)
over every element for a few sample pairs; and the stochastic remainder of
Sigma (Eq. 25 minus its deterministic block) at one tau point for those
pairs.  The oracle's [K]^L product runs on the kept rows of (ij|A)^L only
(a screened-out row of (ij|A)^L is zero, so its [K]^L row is zero and
changes neither the global maximum nor the cut).  The deterministic block
itself is not evaluated by the oracle here (its plain sum over Q, Q' costs
~1e17 flops at this size); the N = 200 tests cover it element by element.

The tau grid has 4 points instead of the workload's 128 (parity does not
depend on the grid; the setup's deterministic block is built for every tau).
Tolerance as everywhere: 1e-10 relative (Frobenius), exact for integer work.
"""
import numpy as np
import pytest

import oracle as O
from paper_2005_12338_gb300 import synth

pytestmark = [pytest.mark.gpu, pytest.mark.slow]
TOL = 1e-10
N_S = 4

torch = pytest.importorskip("torch")


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2005_12338_gb300 import binding, build
    build.build()
    return binding


@pytest.fixture(scope="module")
def ref():
    cfg = synth.CONFIGS["c3_n1000"]
    s = synth.make_system(cfg["n"], cfg["n_occ"], cfg["n_aux"], 4, input_seed=0)
    n, na = s.n, s.n_aux
    w = O.metric_inv_sqrt(s.metric)
    el, mask, m = O.screen(s.eri3, cfg["eps_prime"])
    rows = np.flatnonzero(mask.reshape(n * n, na).any(axis=1))
    # the kept rows, zero-padded to a square count so that they form an
    # [m, m, N_aux] array the oracle's Eq. 12-13 step accepts
    side = int(np.ceil(np.sqrt(len(rows))))
    el_rows = np.zeros((side * side, na))
    el_rows[:len(rows)] = el.reshape(n * n, na)[rows]
    del el
    kl_rows, kmax = O.large_factor(el_rows.reshape(side, side, na), w, cfg["eps"])
    kl_rows = kl_rows.reshape(side * side, na)[:len(rows)]
    kl = np.zeros((n * n, na))
    kl[rows] = kl_rows
    kl = kl.reshape(n, n, na)
    th0 = O.rademacher(0, 0, N_S, na)
    th1 = O.rademacher(0, 1, N_S, na)
    r0, rl0 = O.stochastic_factors(s.eri3, w, kl, th0)
    r1, rl1 = O.stochastic_factors(s.eri3, w, kl, th1)
    t = s.n_tau - 1
    g, gb = O.green(s.orb_e, s.orb_c, s.n_occ, s.mu, s.tau[t])
    rem = np.zeros((n, n))
    for x in range(N_S):
        rem += O.factor_pair(r0[x], r1[x], g, gb)[0] - O.factor_pair(rl0[x], rl1[x], g, gb)[0]
    return dict(cfg=cfg, s=s, w=w, mask_count=int(mask.sum()), m=m, rows=rows,
                kl_rows=kl_rows, kmax=kmax, nnz_kl=int(np.count_nonzero(kl_rows)),
                n_large=int((np.abs(kl_rows).max(axis=1) > 0).sum()),
                r=(r0, r1), rl=(rl0, rl1), t=t, g=g, gb=gb, rem=rem / N_S)


# (chain precision, deterministic-block arithmetic): IEEE fp64 and double-float
FORMS = {"plain": (0, 0), "df64": (3, 1)}


@pytest.fixture(scope="module", params=sorted(FORMS))
def gpu(B, ref, request):
    s, cfg = ref["s"], ref["cfg"]
    prec, dd = FORMS[request.param]
    h = B.Handle(0)
    opts = B.Handle.options(cfg["eps_prime"], cfg["eps"], N_S, 0, precision=prec, dd_arith=dd)
    arrs = [torch.from_numpy(a).cuda() for a in (s.eri3, s.metric, s.orb_e, s.orb_c, s.tau,
                                                  s.tau_w)]
    h.setup(*arrs, n_occ=s.n_occ, mu=s.mu, beta=s.beta, opts=opts)
    sig = torch.empty((s.n_tau, s.n, s.n), dtype=torch.float64, device="cuda")
    ep = torch.empty(N_S, dtype=torch.float64, device="cuda")
    e, se, st = h.sigma(opts, sig, ep)
    torch.cuda.synchronize()
    out = dict(h=h, st=st, sigma=sig.cpu().numpy(), e_pair=ep.cpu().numpy(), e=e)
    del arrs, sig, ep
    yield out
    h.close()
    torch.cuda.empty_cache()


def test_c3_selection_exact(ref, gpu):
    st, h = gpu["st"], gpu["h"]
    assert st["nnz_eri_l"] == ref["mask_count"]
    assert st["n_pairs_screened"] == len(ref["rows"])
    assert st["nnz_k_l"] == ref["nnz_kl"]
    assert st["n_pairs_large"] == ref["n_large"]
    assert st["k_l_max"] == pytest.approx(ref["kmax"], rel=1e-12)
    assert np.array_equal(h.export("COLMAX"), ref["m"])


def test_c3_metric_root_and_large_factor(ref, gpu):
    h, s = gpu["h"], ref["s"]
    na = s.n_aux
    w = ref["w"]
    assert np.abs(h.export("W").reshape(na, na) - w).max() < 1e-11 * np.abs(w).max()
    kg = h.export("K_L").reshape(s.n * s.n, na)
    rows = ref["rows"]
    # the kept rows match, and every row outside the screened pairs is zero
    kr = kg[rows]
    nnz_all = np.count_nonzero(kg)
    del kg
    assert nnz_all == np.count_nonzero(kr)
    assert np.array_equal(kr != 0, ref["kl_rows"] != 0)
    assert rel(kr, ref["kl_rows"]) < 1e-12


def test_c3_factors(ref, gpu):
    h, s = gpu["h"], ref["s"]
    n = s.n
    rg = h.export("R").reshape(2, N_S, n, n)
    rlg = h.export("R_L").reshape(2, N_S, n, n)
    for k in range(2):
        assert rel(rg[k], ref["r"][k]) < 1e-12
        assert rel(rlg[k], ref["rl"][k]) < 1e-12


def test_c3_stochastic_remainder_one_tau(ref, gpu):
    h, s = gpu["h"], ref["s"]
    n, t = s.n, ref["t"]
    g = h.export("G").reshape(s.n_tau, n, n)[t]
    gb = h.export("GB").reshape(s.n_tau, n, n)[t]
    assert rel(g, ref["g"]) < 1e-13 and rel(gb, ref["gb"]) < 1e-13
    sdd = h.export("SIGMA_DD").reshape(s.n_tau, n, n)[t]
    raw = h.export("SIGMA_RAW").reshape(s.n_tau, n, n)[t]
    assert rel(raw - sdd, ref["rem"]) < TOL
    assert np.abs(raw - sdd - ref["rem"]).max() < TOL * np.abs(ref["rem"]).max()
    # the deterministic block is symmetric, and so is the output
    assert np.abs(sdd - sdd.T).max() <= 1e-13 * np.abs(sdd).max()
    assert np.array_equal(gpu["sigma"], np.transpose(gpu["sigma"], (0, 2, 1)))
