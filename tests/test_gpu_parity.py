"""GPU parity of the RS-SRI-GF2 path against the fp64 oracle, through the C ABI.

Tolerance: the path computes in fp64; results must agree with the oracle to
1e-10 relative (Frobenius norm per tau point for matrices, |dE|/|E| for
energies).  Integer and selection work (masks, pair lists, counts, the
Rademacher signs) must agree exactly.
"""
import numpy as np
import pytest

import oracle as O
from paper_2005_12338_gb300 import synth

pytestmark = pytest.mark.gpu
TOL = 1e-10

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2005_12338_gb300 import binding, build
    build.build()
    return binding


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def run_gpu(B, s, eps_prime, eps, n_s, seed, host=False, estimator=0, xi_offset=0, pair_batch=0,
            g=None, gb=None, dd_arith=0, precision=0):
    h = B.Handle(0)
    opts = B.Handle.options(eps_prime, eps, n_s, seed, xi_offset, estimator, pair_batch,
                            dd_arith=dd_arith, precision=precision)
    arrs = [s.eri3, s.metric, s.orb_e, s.orb_c, s.tau, s.tau_w]
    if host:
        sig = np.empty((s.n_tau, s.n, s.n))
        ep = np.empty(n_s)
    else:
        arrs = [dev(a) for a in arrs]
        sig = torch.empty((s.n_tau, s.n, s.n), dtype=torch.float64, device="cuda")
        ep = torch.empty(n_s, dtype=torch.float64, device="cuda")
    h.setup(*arrs, n_occ=s.n_occ, mu=s.mu, beta=s.beta, opts=opts)
    if g is not None and not host:
        g, gb = dev(g), dev(gb)
    e, se, st = h.sigma(opts, sig, ep, g=g, gb=gb)
    torch.cuda.synchronize()
    sig = sig if host else sig.cpu().numpy()
    ep = ep if host else ep.cpu().numpy()
    return h, dict(sigma=sig, e_pair=ep, e_corr=e, e_stderr=se, stats=st)


def run_oracle(s, eps_prime, eps, n_s, seed, **kw):
    return O.rs_sri(s.eri3, s.metric, s.orb_e, s.orb_c, s.n_occ, s.mu, s.tau, s.tau_w,
                    eps_prime, eps, n_s, seed, **kw)


def compare_all(h, got, ref, s):
    n, na, nt = s.n, s.n_aux, s.n_tau
    x = ref.extra
    st = got["stats"]
    # exact selection work
    assert st["nnz_eri_l"] == x["nnz_eri_l"]
    assert st["nnz_k_l"] == x["nnz_k_l"]
    assert np.array_equal(h.export("COLMAX"), x["m_col"])
    el_ref = np.where(x["mask"], s.eri3, 0.0)
    assert np.array_equal(h.export("ERI_L").reshape(n, n, na), el_ref)
    assert st["k_l_max"] == pytest.approx(x["k_l_max"], rel=1e-12)
    kl = h.export("K_L").reshape(n, n, na)
    assert np.array_equal(kl != 0, x["k_l"] != 0)
    assert rel(kl, x["k_l"]) < 1e-12
    th = h.export("THETA").reshape(2, -1, na)
    assert np.array_equal(th[0], x["theta0"]) and np.array_equal(th[1], x["theta1"])
    # fp64 work
    assert np.abs(h.export("W").reshape(na, na) - x["w"]).max() < 1e-11 * np.abs(x["w"]).max()
    r = h.export("R").reshape(2, -1, n, n)
    rl = h.export("R_L").reshape(2, -1, n, n)
    assert rel(r[0], x["r0"]) < 1e-12 and rel(r[1], x["r1"]) < 1e-12
    assert rel(rl[0], x["rl0"]) < 1e-12 and rel(rl[1], x["rl1"]) < 1e-12
    g = h.export("G").reshape(nt, n, n)
    gb = h.export("GB").reshape(nt, n, n)
    sdd = h.export("SIGMA_DD").reshape(nt, n, n)
    raw = h.export("SIGMA_RAW").reshape(nt, n, n)
    for t in range(nt):
        gr, gbr = O.green(s.orb_e, s.orb_c, s.n_occ, s.mu, s.tau[t])
        assert rel(g[t], gr) < 1e-13 and rel(gb[t], gbr) < 1e-13
        assert rel(sdd[t], ref.sigma_dd[t]) < TOL
        assert rel(raw[t], ref.sigma_raw[t]) < TOL
        assert rel(got["sigma"][t], ref.sigma[t]) < TOL
    assert np.array_equal(got["sigma"], np.transpose(got["sigma"], (0, 2, 1)))
    assert abs(got["e_corr"] - ref.e_corr) < TOL * abs(ref.e_corr)
    assert abs(st["e_dd"] - ref.e_dd) < TOL * abs(ref.e_dd)
    assert np.abs(got["e_pair"] - ref.e_pair).max() < TOL * abs(ref.e_corr)
    assert got["e_stderr"] == pytest.approx(ref.e_stderr, rel=1e-8)


CASES = {
    # the N = 20 correctness workload (all steps run by the oracle in full)
    "n20": dict(sys=(20, 10, 60, 32), eps_prime=0.02, eps=1e-2, n_s=64, seed=0),
    # ragged: two 64-wide tiles plus a tail, odd sample count, several tau
    "n72_ragged": dict(sys=(72, 31, 150, 5), eps_prime=0.02, eps=1e-2, n_s=7, seed=12345),
    # odd N and odd N_aux: unaligned rows everywhere (scalar paths of the vector loads)
    "n37_odd": dict(sys=(37, 16, 45, 3), eps_prime=0.02, eps=1e-2, n_s=5, seed=99),
    # short contractions (N N_aux < 1024): no split over K anywhere
    "n16_short": dict(sys=(16, 7, 40, 3), eps_prime=0.02, eps=1e-2, n_s=4, seed=5),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_parity_all_steps(B, case):
    c = CASES[case]
    s = synth.make_system(*c["sys"], input_seed=1)
    ref = run_oracle(s, c["eps_prime"], c["eps"], c["n_s"], c["seed"])
    h, got = run_gpu(B, s, c["eps_prime"], c["eps"], c["n_s"], c["seed"])
    compare_all(h, got, ref, s)
    h.close()


@pytest.mark.parametrize("case", sorted(CASES))
def test_parity_double_float_deterministic_block(B, case):
    """The exchange contraction in double-float (fp32 pairs) meets the same
    1e-10 bar as the fp64 one."""
    c = CASES[case]
    s = synth.make_system(*c["sys"], input_seed=1)
    ref = run_oracle(s, c["eps_prime"], c["eps"], c["n_s"], c["seed"])
    h, got = run_gpu(B, s, c["eps_prime"], c["eps"], c["n_s"], c["seed"], dd_arith=1)
    compare_all(h, got, ref, s)
    h.close()


@pytest.mark.parametrize("case", sorted(CASES))
def test_parity_double_float_everywhere(B, case):
    """The fp64-accurate fast form: chain products and deterministic block in
    double-float (RSSRI_PREC_DF64 with RSSRI_DD_DF64) meet the fp64 bar of 1e-10."""
    c = CASES[case]
    s = synth.make_system(*c["sys"], input_seed=1)
    ref = run_oracle(s, c["eps_prime"], c["eps"], c["n_s"], c["seed"])
    h, got = run_gpu(B, s, c["eps_prime"], c["eps"], c["n_s"], c["seed"], dd_arith=1,
                     precision=B.RSSRI_PREC_DF64)
    compare_all(h, got, ref, s)
    h.close()


@pytest.mark.parametrize("case", sorted(CASES))
def test_parity_sliced_block(B, case):
    """The deterministic block on the tensor cores (RSSRI_DD_OZ: fp64 operands
    split into bf16 digits, exact digit products) with the double-float chain
    meets the fp64 bar of 1e-10."""
    c = CASES[case]
    s = synth.make_system(*c["sys"], input_seed=1)
    ref = run_oracle(s, c["eps_prime"], c["eps"], c["n_s"], c["seed"])
    h, got = run_gpu(B, s, c["eps_prime"], c["eps"], c["n_s"], c["seed"], dd_arith=B.RSSRI_DD_OZ,
                     precision=B.RSSRI_PREC_DF64)
    compare_all(h, got, ref, s)
    h.close()


def test_double_float_chain_pair_batches(B):
    s = synth.make_system(30, 12, 60, 3, input_seed=6)
    _, a = run_gpu(B, s, 0.02, 1e-2, 9, 4, dd_arith=1, precision=B.RSSRI_PREC_DF64)
    _, b = run_gpu(B, s, 0.02, 1e-2, 9, 4, dd_arith=1, precision=B.RSSRI_PREC_DF64,
                   pair_batch=4)
    assert rel(b["sigma"], a["sigma"]) < 1e-13
    assert np.abs(b["e_pair"] - a["e_pair"]).max() < 1e-13 * abs(a["e_corr"])


def test_host_pointers_deterministic_and_batched(B):
    s = synth.make_system(24, 11, 50, 6, input_seed=2)
    h1, a = run_gpu(B, s, 0.02, 1e-2, 9, 3)
    h2, b = run_gpu(B, s, 0.02, 1e-2, 9, 3, host=True)
    h3, c = run_gpu(B, s, 0.02, 1e-2, 9, 3)
    assert np.array_equal(a["sigma"], b["sigma"]) and np.array_equal(a["sigma"], c["sigma"])
    assert np.array_equal(a["e_pair"], b["e_pair"]) and a["e_corr"] == c["e_corr"]
    # smaller pair batches change only the summation order of Sigma
    h4, d = run_gpu(B, s, 0.02, 1e-2, 9, 3, pair_batch=4)
    assert np.array_equal(a["e_pair"], d["e_pair"])
    assert rel(a["sigma"], d["sigma"]) < 1e-13
    for h in (h1, h2, h3, h4):
        h.close()


def test_resume_concatenates(B):
    s = synth.make_system(16, 8, 40, 4, input_seed=3)
    _, full = run_gpu(B, s, 0.02, 1e-2, 8, 77)
    _, lo = run_gpu(B, s, 0.02, 1e-2, 4, 77)
    _, hi = run_gpu(B, s, 0.02, 1e-2, 4, 77, xi_offset=4)
    assert np.array_equal(np.concatenate([lo["e_pair"], hi["e_pair"]]), full["e_pair"])


def test_threshold_zero_is_exact_ri(B):
    s = synth.make_system(18, 7, 36, 4, input_seed=4)
    _, got = run_gpu(B, s, 0.0, 0.0, 4, 5)
    k = O.ri_factor(s.eri3, O.metric_inv_sqrt(s.metric))
    for t in range(s.n_tau):
        g, gb = O.green(s.orb_e, s.orb_c, s.n_occ, s.mu, s.tau[t])
        assert rel(got["sigma"][t], O.sigma_from_factor(k, g, gb)) < TOL


def test_sri_estimator(B):
    s = synth.make_system(20, 10, 40, 5, input_seed=5)
    ref = run_oracle(s, 0.02, 1e-2, 6, 9, empty_large=True)
    h, got = run_gpu(B, s, 0.02, 1e-2, 6, 9, estimator=1)
    for t in range(s.n_tau):
        assert rel(got["sigma"][t], ref.sigma[t]) < TOL
    assert abs(got["e_corr"] - ref.e_corr) < TOL * abs(ref.e_corr)
    h.close()


def test_sigma_from_given_g(B):
    s = synth.make_system(22, 9, 44, 3, input_seed=6)
    gs, gbs = zip(*(O.green(s.orb_e, s.orb_c, s.n_occ, s.mu, t) for t in s.tau))
    _, a = run_gpu(B, s, 0.02, 1e-2, 5, 2)
    _, b = run_gpu(B, s, 0.02, 1e-2, 5, 2, g=np.array(gs), gb=np.array(gbs))
    assert rel(b["sigma"], a["sigma"]) < 1e-13
    assert abs(a["e_corr"] - b["e_corr"]) < 1e-13 * abs(a["e_corr"])


def test_errors_are_reported(B):
    s = synth.make_system(12, 5, 20, 3, input_seed=7)
    opts = B.Handle.options(0.02, 1e-2, 4, 0)
    h = B.Handle(0)
    sig = torch.empty((3, 12, 12), dtype=torch.float64, device="cuda")
    with pytest.raises(B.RssriError) as e:
        h.sigma(opts, sig)
    assert e.value.code == -7  # NOT_READY
    args = [dev(a) for a in (s.eri3, s.metric, s.orb_e, s.orb_c, s.tau, s.tau_w)]
    bad = s.eri3.copy()
    bad[0, 1, 3] += 1e-9
    with pytest.raises(B.RssriError) as e:
        h.setup(dev(bad), *args[1:], n_occ=5, mu=0.0, beta=50.0, opts=opts)
    assert e.value.code == -3
    v = s.metric.copy()
    v[0, 0] = -5.0
    with pytest.raises(B.RssriError) as e:
        h.setup(args[0], dev(v), *args[2:], n_occ=5, mu=0.0, beta=50.0, opts=opts)
    assert e.value.code == -2
    nan = s.orb_c.copy()
    nan[2, 2] = np.nan
    with pytest.raises(B.RssriError) as e:
        h.setup(*args[:3], dev(nan), *args[4:], n_occ=5, mu=0.0, beta=50.0, opts=opts)
    assert e.value.code == -8
    with pytest.raises(B.RssriError) as e:
        h.setup(*args, n_occ=5, mu=0.0, beta=1.0, opts=opts)  # tau beyond beta
    assert e.value.code == -1
    with pytest.raises(B.RssriError) as e:
        h.setup(*args, n_occ=12, mu=0.0, beta=50.0, opts=opts)
    assert e.value.code == -1
    # the handle still works after rejected calls
    h.setup(*args, n_occ=5, mu=0.0, beta=50.0, opts=opts)
    h.sigma(opts, sig)
    h.close()


# ---------------------------------------------------- the N = 200 workload ---
# Forms: (chain precision, deterministic-block arithmetic).  "plain" is IEEE
# fp64 throughout; "sliced" has the block's products on the tensor cores
# (RSSRI_DD_OZ) and the double-float chain; "df64" is the double-float form
# (chain and block), whose
# N = 200 launches pick other tile geometries than the small cases (padded
# 16x16 / 8x8 double-float tiles, the symmetric upper-tile Sigma_DD product,
# N_aux = 600 split into five aux chunks in the exchange contraction).
C2_FORMS = {"plain": (0, 0), "df64": (3, 1), "sliced": (3, 2)}


@pytest.fixture(scope="module", params=sorted(C2_FORMS))
def c2(B, request):
    cfg = synth.CONFIGS["c2_n200"]
    s = synth.make_system(cfg["n"], cfg["n_occ"], cfg["n_aux"], cfg["n_tau"], input_seed=0)
    prec, dd = C2_FORMS[request.param]
    h, got = run_gpu(B, s, cfg["eps_prime"], cfg["eps"], cfg["n_s"], 0, dd_arith=dd,
                     precision=prec)
    yield cfg, s, h, got
    h.close()


@pytest.fixture(scope="module")
def c2_oracle_dd():
    """The oracle's deterministic block (Eq. 20 on v^L, summed over Q, Q') at
    one tau point of the N = 200 workload: a few host minutes."""
    cfg = synth.CONFIGS["c2_n200"]
    s = synth.make_system(cfg["n"], cfg["n_occ"], cfg["n_aux"], cfg["n_tau"], input_seed=0)
    w = O.metric_inv_sqrt(s.metric)
    el, _, _ = O.screen(s.eri3, cfg["eps_prime"])
    kl, _ = O.large_factor(el, w, cfg["eps"])
    t = s.n_tau // 2
    g, gb = O.green(s.orb_e, s.orb_c, s.n_occ, s.mu, s.tau[t])
    return t, O.sigma_from_factor(kl, g, gb)


def test_c2_deterministic_block_elementwise(c2, c2_oracle_dd):
    """S7 at full size, every element of Sigma_DD(tau) at one tau point (the
    trace check below would miss a wrong off-diagonal block, e.g. a bad mirror
    of the symmetric upper-tile product)."""
    cfg, s, h, got = c2
    t, ref = c2_oracle_dd
    sdd = h.export("SIGMA_DD").reshape(s.n_tau, s.n, s.n)[t]
    assert rel(sdd, ref) < TOL
    assert np.abs(sdd - ref).max() < TOL * np.abs(ref).max()


def test_c2_selection_and_factors(c2):
    cfg, s, h, got = c2
    n, na = s.n, s.n_aux
    w = O.metric_inv_sqrt(s.metric)
    el, mask, m = O.screen(s.eri3, cfg["eps_prime"])
    kl, kmax = O.large_factor(el, w, cfg["eps"])
    st = got["stats"]
    assert st["nnz_eri_l"] == int(mask.sum())
    assert st["nnz_k_l"] == int(np.count_nonzero(kl))
    assert st["n_pairs_large"] == int((np.abs(kl).max(axis=2) > 0).sum())
    assert np.array_equal(h.export("COLMAX"), m)
    assert np.abs(h.export("W").reshape(na, na) - w).max() < 1e-11 * np.abs(w).max()
    kg = h.export("K_L").reshape(n, n, na)
    assert np.array_equal(kg != 0, kl != 0) and rel(kg, kl) < 1e-12
    th0 = O.rademacher(0, 0, cfg["n_s"], na)
    th1 = O.rademacher(0, 1, cfg["n_s"], na)
    th = h.export("THETA").reshape(2, cfg["n_s"], na)
    assert np.array_equal(th[0], th0) and np.array_equal(th[1], th1)
    r0, rl0 = O.stochastic_factors(s.eri3, w, kl, th0)
    rg = h.export("R").reshape(2, cfg["n_s"], n, n)
    rlg = h.export("R_L").reshape(2, cfg["n_s"], n, n)
    assert rel(rg[0], r0) < 1e-12 and rel(rlg[0], rl0) < 1e-12


def test_c2_stochastic_part_sampled_tau(c2):
    """S8 at full size: the stochastic part of Sigma at two sampled tau points."""
    cfg, s, h, got = c2
    n, na, ns = s.n, s.n_aux, cfg["n_s"]
    w = O.metric_inv_sqrt(s.metric)
    el, _, _ = O.screen(s.eri3, cfg["eps_prime"])
    kl, _ = O.large_factor(el, w, cfg["eps"])
    r0, rl0 = O.stochastic_factors(s.eri3, w, kl, O.rademacher(0, 0, ns, na))
    r1, rl1 = O.stochastic_factors(s.eri3, w, kl, O.rademacher(0, 1, ns, na))
    sdd = h.export("SIGMA_DD").reshape(s.n_tau, n, n)
    raw = h.export("SIGMA_RAW").reshape(s.n_tau, n, n)
    for t in (0, s.n_tau - 1):
        g, gb = O.green(s.orb_e, s.orb_c, s.n_occ, s.mu, s.tau[t])
        acc = np.zeros((n, n))
        for x in range(ns):
            acc += O.factor_pair(r0[x], r1[x], g, gb)[0] - O.factor_pair(rl0[x], rl1[x], g, gb)[0]
        assert rel(raw[t] - sdd[t], acc / ns) < TOL
        assert np.abs(raw[t] - sdd[t] - acc / ns).max() < TOL * np.abs(acc / ns).max()
        sym = sdd[t] + 0.5 * (acc + acc.T) / ns
        assert rel(got["sigma"][t], sym) < TOL


def test_c2_deterministic_energy_closed_form(c2):
    """S7 + S9 at full size: -(1/N_e) sum_tau w Tr[Sigma_DD Gb] equals the
    MP2-form energy of the large-part integrals on the same grid."""
    cfg, s, h, got = c2
    n, na, o = s.n, s.n_aux, s.n_occ
    w = O.metric_inv_sqrt(s.metric)
    el, _, _ = O.screen(s.eri3, cfg["eps_prime"])
    kl, _ = O.large_factor(el, w, cfg["eps"])
    co, cv = s.orb_c[:, :o], s.orb_c[:, o:]
    kov = np.einsum("pi,pqQ->iqQ", co, kl)
    kov = np.einsum("iqQ,qa->iaQ", kov, cv).reshape(o * (n - o), na)
    iajb = (kov @ kov.T).reshape(o, n - o, o, n - o)
    num = iajb * (2 * iajb - iajb.transpose(0, 3, 2, 1))
    eo, ev = s.orb_e[:o], s.orb_e[o:]
    x = np.exp(-(ev[None, :, None] - eo[:, None, None]) * s.tau[None, None, :])  # [o, v, tau]
    x = x.reshape(o * (n - o), s.n_tau)
    e2 = -np.einsum("t,pt,pt->", s.tau_w, x, num.reshape(o * (n - o), -1) @ x)
    e_dd_ref = e2 / (2 * o)
    assert abs(got["stats"]["e_dd"] - e_dd_ref) < TOL * abs(e_dd_ref)


def test_c2_sampled_pair_energies(c2):
    cfg, s, h, got = c2
    n, na, ns = s.n, s.n_aux, cfg["n_s"]
    w = O.metric_inv_sqrt(s.metric)
    el, _, _ = O.screen(s.eri3, cfg["eps_prime"])
    kl, _ = O.large_factor(el, w, cfg["eps"])
    xs = [0, 137, ns - 1]
    r0, rl0 = O.stochastic_factors(s.eri3, w, kl, O.rademacher(0, 0, ns, na)[xs])
    r1, rl1 = O.stochastic_factors(s.eri3, w, kl, O.rademacher(0, 1, ns, na)[xs])
    e_st = np.zeros(len(xs))
    for t in range(s.n_tau):
        g, gb = O.green(s.orb_e, s.orb_c, s.n_occ, s.mu, s.tau[t])
        for k in range(len(xs)):
            _, ta, sa = O.factor_pair(r0[k], r1[k], g, gb)
            _, tb, sb = O.factor_pair(rl0[k], rl1[k], g, gb)
            e_st[k] += -s.tau_w[t] * ((2 * ta * ta - sa) - (2 * tb * tb - sb)) / (2 * s.n_occ)
    e_dd = got["stats"]["e_dd"]
    for k, x in enumerate(xs):
        assert abs(got["e_pair"][x] - (e_dd + e_st[k])) < TOL * abs(got["e_corr"])
    # E_corr is the mean of the pair estimates; Sigma is symmetric
    assert got["e_corr"] == pytest.approx(np.mean(got["e_pair"]), rel=1e-12)
    assert np.array_equal(got["sigma"], np.transpose(got["sigma"], (0, 2, 1)))
