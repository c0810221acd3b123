"""Exponent range of the fp64-accurate forms.

Double-float pairs carry ~48 bits only inside fp32's exponent range, so the
double-float forms check every input matrix they convert (per tau point for
G) and return RSSRI_ERR_RANGE when its largest magnitude lies outside
[2^-40, 2^40], instead of losing precision silently.  (The N=200 workload's
block intermediates at its largest tau points lie below 2^-40 with no loss:
the parity tests of the double-float forms cover them.)  The sliced tensor-core
block (RSSRI_DD_OZ) scales each row of every operand by a power of two, so it
keeps fp64's range: with G(tau) and G(beta - tau) scaled by 2^-100 (entries
near 1e-35 and below) it must still match the oracle to 1e-10, as the IEEE
fp64 form does."""
import numpy as np
import pytest

import oracle as O
from paper_2005_12338_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
RANGE = -9
TOL = 1e-10


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2005_12338_gb300 import binding, build
    build.build()
    return binding


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def run(B, s, eri3, opts, g=None, gb=None):
    dev = [torch.from_numpy(a).cuda() for a in (eri3, s.metric, s.orb_e, s.orb_c, s.tau,
                                                 s.tau_w)]
    h = B.Handle(0)
    try:
        h.setup(*dev, n_occ=s.n_occ, mu=s.mu, beta=s.beta, opts=opts)
        sig = torch.empty((s.n_tau, s.n, s.n), dtype=torch.float64, device="cuda")
        e, se, st = h.sigma(opts, sig, g=None if g is None else torch.from_numpy(g).cuda(),
                            gb=None if gb is None else torch.from_numpy(gb).cuda())
        torch.cuda.synchronize()
        return sig.cpu().numpy(), e
    finally:
        h.close()


def test_tiny_green_function(B):
    s = synth.make_system(24, 11, 48, 3, input_seed=9)
    ns, seed, epsp, eps = 5, 3, 0.02, 1e-2
    scale = 2.0 ** -100
    gs, gbs = zip(*(O.green(s.orb_e, s.orb_c, s.n_occ, s.mu, t) for t in s.tau))
    g, gb = np.array(gs) * scale, np.array(gbs) * scale
    # the oracle's estimator on the same draws with the scaled G
    w = O.metric_inv_sqrt(s.metric)
    el, _, _ = O.screen(s.eri3, epsp)
    kl, _ = O.large_factor(el, w, eps)
    r0, rl0 = O.stochastic_factors(s.eri3, w, kl, O.rademacher(seed, 0, ns, s.n_aux))
    r1, rl1 = O.stochastic_factors(s.eri3, w, kl, O.rademacher(seed, 1, ns, s.n_aux))
    ref = []
    for t in range(s.n_tau):
        acc = O.sigma_from_factor(kl, g[t], gb[t])
        for x in range(ns):
            acc = acc + (O.factor_pair(r0[x], r1[x], g[t], gb[t])[0] -
                         O.factor_pair(rl0[x], rl1[x], g[t], gb[t])[0]) / ns
        ref.append(0.5 * (acc + acc.T))
    ref = np.array(ref)
    e_ref = O.energy_trace(ref, gb, s.tau_w, s.n_occ)
    for prec, dd in ((B.RSSRI_PREC_FP64, B.RSSRI_DD_FP64), (B.RSSRI_PREC_FP64, B.RSSRI_DD_OZ)):
        o = B.Handle.options(epsp, eps, ns, seed, precision=prec, dd_arith=dd)
        sig, e = run(B, s, s.eri3, o, g=g, gb=gb)
        for t in range(s.n_tau):
            assert rel(sig[t], ref[t]) < TOL, (dd, t)
        assert abs(e - e_ref) < TOL * abs(e_ref)
    # double-float: refused
    for prec, dd in ((B.RSSRI_PREC_DF64, B.RSSRI_DD_DF64), (B.RSSRI_PREC_DF64, B.RSSRI_DD_OZ),
                     (B.RSSRI_PREC_FP64, B.RSSRI_DD_DF64)):
        o = B.Handle.options(epsp, eps, ns, seed, precision=prec, dd_arith=dd)
        with pytest.raises(B.RssriError) as err:
            run(B, s, s.eri3, o, g=g, gb=gb)
        assert err.value.code == RANGE, (prec, dd)


def test_tiny_integrals_refused_by_the_double_float_setup(B):
    s = synth.make_system(20, 9, 40, 2, input_seed=10)
    tiny = s.eri3 * 2.0 ** -80
    o = B.Handle.options(0.02, 1e-2, 4, 1, precision=B.RSSRI_PREC_DF64, dd_arith=B.RSSRI_DD_DF64)
    with pytest.raises(B.RssriError) as err:
        run(B, s, tiny, o)
    assert err.value.code == RANGE
    # the IEEE fp64 form takes it (and its result is the unscaled one times 2^-320:
    # Sigma is of degree 4 in the integrals)
    o = B.Handle.options(0.02, 1e-2, 4, 1)
    sig_tiny, _ = run(B, s, tiny, o)
    sig, _ = run(B, s, s.eri3, o)
    assert rel(sig_tiny * 2.0 ** 320, sig) < 1e-12
