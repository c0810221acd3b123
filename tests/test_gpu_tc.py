"""The reduced-precision chains (RSSRI_PREC_BF16, RSSRI_PREC_TF32): tensor-core
products in the range-separated split, against the fp64 oracle.

Stated tolerance.  Every operand of the split chain is rounded to the operand
type (bf16: 8 significant bits, unit roundoff u = 2^-8; tf32: 11 bits,
u = 2^-11) and accumulated in fp32; the rounding errors of the operands on
the longest path add up to about one u of the stochastic remainder
Sigma - Sigma_DD.  The tests allow 5 u of that remainder (Frobenius norm per
tau point) and of the remainder's share of E_corr; the deterministic block
stays fp64, so it must still match to 1e-10.
"""
import numpy as np
import pytest

import oracle as O
from paper_2005_12338_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
# 5 u per operand type
TOL = {"bf16": 5 * 2.0 ** -8, "tf32": 5 * 2.0 ** -11}
PRECS = ["bf16", "tf32"]


def prec(B, name):
    return {"bf16": B.RSSRI_PREC_BF16, "tf32": B.RSSRI_PREC_TF32}[name]


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2005_12338_gb300 import binding, build
    build.build()
    return binding


def run(B, s, eps_prime, eps, n_s, seed, precision, estimator=0):
    h = B.Handle(0)
    opts = B.Handle.options(eps_prime, eps, n_s, seed, estimator=estimator, precision=precision)
    dev = [torch.from_numpy(a).cuda() for a in (s.eri3, s.metric, s.orb_e, s.orb_c, s.tau,
                                                 s.tau_w)]
    h.setup(*dev, n_occ=s.n_occ, mu=s.mu, beta=s.beta, opts=opts)
    sig = torch.empty((s.n_tau, s.n, s.n), dtype=torch.float64, device="cuda")
    ep = torch.empty(n_s, dtype=torch.float64, device="cuda")
    e, se, st = h.sigma(opts, sig, ep)
    sdd = h.export("SIGMA_DD").reshape(s.n_tau, s.n, s.n)
    out = dict(sigma=sig.cpu().numpy(), e_pair=ep.cpu().numpy(), e=e, se=se, st=st, sdd=sdd)
    h.close()
    return out


@pytest.fixture(scope="module")
def n72():
    dims, epsp, eps, ns, seed = (72, 31, 150, 5), 0.02, 1e-2, 7, 12345
    s = synth.make_system(*dims, input_seed=1)
    ref = O.rs_sri(s.eri3, s.metric, s.orb_e, s.orb_c, s.n_occ, s.mu, s.tau, s.tau_w, epsp, eps,
                   ns, seed)
    return s, ref, (epsp, eps, ns, seed)


@pytest.mark.parametrize("pname", PRECS)
def test_tc_chain_against_oracle(B, n72, pname):
    s, ref, (epsp, eps, ns, seed) = n72
    TOL_ST = TOL[pname]
    got = run(B, s, epsp, eps, ns, seed, prec(B, pname))
    for t in range(s.n_tau):
        assert np.linalg.norm(got["sdd"][t] - ref.sigma_dd[t]) < 1e-10 * np.linalg.norm(
            ref.sigma_dd[t])
        st_ref = ref.sigma[t] - 0.5 * (ref.sigma_dd[t] + ref.sigma_dd[t].T)
        st_got = got["sigma"][t] - 0.5 * (got["sdd"][t] + got["sdd"][t].T)
        err = np.linalg.norm(st_got - st_ref) / np.linalg.norm(st_ref)
        assert err < TOL_ST, (t, err)
    e_st = ref.e_corr - ref.e_dd
    assert abs(got["e"] - ref.e_corr) < TOL_ST * abs(e_st)
    assert np.abs(got["e_pair"] - ref.e_pair).max() < TOL_ST * np.abs(ref.e_pair - ref.e_dd).max()
    # the reduced-precision error is far below the statistical error
    assert abs(got["e"] - ref.e_corr) < 0.1 * ref.e_stderr


@pytest.mark.parametrize("pname", PRECS)
def test_tc_chain_odd_size(B, pname):
    """N = 37: operand rows padded to 40 elements for the TMA descriptors, a
    ragged last tile in every product."""
    s = synth.make_system(37, 16, 45, 3, input_seed=8)
    ref = O.rs_sri(s.eri3, s.metric, s.orb_e, s.orb_c, s.n_occ, s.mu, s.tau, s.tau_w, 0.02, 1e-2,
                   5, 99)
    got = run(B, s, 0.02, 1e-2, 5, 99, prec(B, pname))
    for t in range(s.n_tau):
        st_ref = ref.sigma[t] - 0.5 * (ref.sigma_dd[t] + ref.sigma_dd[t].T)
        st_got = got["sigma"][t] - 0.5 * (got["sdd"][t] + got["sdd"][t].T)
        assert np.linalg.norm(st_got - st_ref) / np.linalg.norm(st_ref) < TOL[pname], t


def test_tf32_closer_than_bf16(B, n72):
    """The tf32 operands carry 3 more bits: its remainder error must be well
    below the bf16 one on the same draws."""
    s, ref, (epsp, eps, ns, seed) = n72
    errs = {}
    for pname in PRECS:
        got = run(B, s, epsp, eps, ns, seed, prec(B, pname))
        d = [np.linalg.norm(got["sigma"][t] - ref.sigma[t]) for t in range(s.n_tau)]
        errs[pname] = max(d)
    assert errs["tf32"] < 0.5 * errs["bf16"], errs


@pytest.mark.parametrize("pname", PRECS)
def test_tc_chain_full_size_sampled(B, pname):
    """N = 200 workload: the stochastic part at two tau points against the
    oracle's paired sums of F(R,R') - F(R^L,R'^L) (the oracle's deterministic
    block is too slow at this size; it is the same fp64 code as the fp64 mode)."""
    TOL_ST = TOL[pname]
    cfg = synth.CONFIGS["c2_n200"]
    s = synth.make_system(cfg["n"], cfg["n_occ"], cfg["n_aux"], 4, input_seed=0)
    ns, seed = 40, 3
    got = run(B, s, cfg["eps_prime"], cfg["eps"], ns, seed, prec(B, pname))
    f64 = run(B, s, cfg["eps_prime"], cfg["eps"], ns, seed, B.RSSRI_PREC_FP64)
    w = O.metric_inv_sqrt(s.metric)
    el, _, _ = O.screen(s.eri3, cfg["eps_prime"])
    kl, _ = O.large_factor(el, w, cfg["eps"])
    r0, rl0 = O.stochastic_factors(s.eri3, w, kl, O.rademacher(seed, 0, ns, s.n_aux))
    r1, rl1 = O.stochastic_factors(s.eri3, w, kl, O.rademacher(seed, 1, ns, s.n_aux))
    for t in (0, s.n_tau - 1):
        g, gb = O.green(s.orb_e, s.orb_c, s.n_occ, s.mu, s.tau[t])
        acc = np.zeros((s.n, s.n))
        for x in range(ns):
            acc += O.factor_pair(r0[x], r1[x], g, gb)[0] - O.factor_pair(rl0[x], rl1[x], g, gb)[0]
        ref = 0.5 * (acc + acc.T) / ns
        st = got["sigma"][t] - 0.5 * (got["sdd"][t] + got["sdd"][t].T)
        assert np.linalg.norm(st - ref) / np.linalg.norm(ref) < TOL_ST
    assert np.abs(got["sdd"] - f64["sdd"]).max() == 0.0  # same fp64 block
    e_st = f64["e"] - f64["st"]["e_dd"]
    assert abs(got["e"] - f64["e"]) < TOL_ST * abs(e_st)
    assert abs(got["e"] - f64["e"]) < 0.1 * f64["se"]


@pytest.mark.parametrize("pname", PRECS)
def test_tc_sri_mode(B, pname):
    TOL_ST = TOL[pname]
    s = synth.make_system(40, 20, 80, 3, input_seed=2)
    ref = O.rs_sri(s.eri3, s.metric, s.orb_e, s.orb_c, s.n_occ, s.mu, s.tau, s.tau_w, 0.02, 1e-2,
                   6, 9, empty_large=True)
    got = run(B, s, 0.02, 1e-2, 6, 9, prec(B, pname), estimator=1)
    for t in range(s.n_tau):
        err = np.linalg.norm(got["sigma"][t] - ref.sigma[t]) / np.linalg.norm(ref.sigma[t])
        assert err < TOL_ST, (t, err)


@pytest.mark.parametrize("pname", PRECS)
def test_tc_deterministic(B, pname):
    s = synth.make_system(48, 20, 96, 3, input_seed=3)
    a = run(B, s, 0.02, 1e-2, 8, 1, prec(B, pname))
    b = run(B, s, 0.02, 1e-2, 8, 1, prec(B, pname))
    assert np.array_equal(a["sigma"], b["sigma"]) and a["e"] == b["e"]


def test_tc_graph_replay_matches_fresh_capture(B):
    """The chain is captured as a CUDA graph on the first call and replayed
    after; a replay with a new seed must equal a fresh handle's result."""
    s = synth.make_system(64, 30, 128, 4, input_seed=4)
    dev = [torch.from_numpy(a).cuda() for a in (s.eri3, s.metric, s.orb_e, s.orb_c, s.tau,
                                                 s.tau_w)]
    sig = torch.empty((s.n_tau, s.n, s.n), dtype=torch.float64, device="cuda")
    h = B.Handle(0)
    outs = []
    # a switch of operand kind must rebuild the graph, a seed change must not
    plan = [(5, "bf16"), (6, "bf16"), (7, "bf16"), (7, "tf32"), (8, "tf32")]
    for seed, pname in plan:
        o = B.Handle.options(0.02, 1e-2, 12, seed, precision=prec(B, pname))
        h.setup(*dev, n_occ=s.n_occ, mu=s.mu, beta=s.beta, opts=o)
        e, _, st = h.sigma(o, sig)
        outs.append((sig.cpu().numpy().copy(), e, st["kernel_launches"]))
    h.close()
    fresh = run(B, s, 0.02, 1e-2, 12, 7, B.RSSRI_PREC_BF16)
    assert np.array_equal(outs[2][0], fresh["sigma"]) and outs[2][1] == fresh["e"]
    assert outs[1][2] == outs[2][2] > 0
    fresh = run(B, s, 0.02, 1e-2, 12, 8, B.RSSRI_PREC_TF32)
    assert np.array_equal(outs[4][0], fresh["sigma"]) and outs[4][1] == fresh["e"]
    assert not np.array_equal(outs[2][0], outs[3][0])
