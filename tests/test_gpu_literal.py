"""GPU parity of the literal Eq. 25 estimator (RSSRI_EST_LITERAL) against the
oracle's literal mode, through the C ABI.

The literal estimator expands the product of the two brackets of Eq. 25
with D exact inside each bracket, so besides the four chains
F(R, R'), F(R^L, R'^L), F(R, R'^L), F(R^L, R') it needs the cross terms
Phi(D, S') and Phi(S, D), which the GPU builds per sample from the pair-space
v^L (exchange) and [K]^L (direct).  Everything is fp64 (or double-float for
the pair-space build), so the bar is the fp64 one: 1e-10 relative per tau
point and for the energies.
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


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def run(B, s, eps_prime, eps, n_s, seed, estimator, dd_arith=0, pair_batch=0):
    h = B.Handle(0)
    opts = B.Handle.options(eps_prime, eps, n_s, seed, estimator=estimator,
                            pair_batch=pair_batch, dd_arith=dd_arith)
    dev = [torch.from_numpy(a).cuda() for a in (s.eri3, s.metric, s.orb_e, s.orb_c, s.tau,
                                                 s.tau_w)]
    h.setup(*dev, n_occ=s.n_occ, mu=s.mu, beta=s.beta, opts=opts)
    sig = torch.empty((s.n_tau, s.n, s.n), dtype=torch.float64, device="cuda")
    ep = torch.empty(n_s, dtype=torch.float64, device="cuda")
    e, se, st = h.sigma(opts, sig, ep)
    out = dict(sigma=sig.cpu().numpy(), e_pair=ep.cpu().numpy(), e=e, se=se, st=st)
    h.close()
    return out


@pytest.fixture(scope="module")
def case():
    s = synth.make_system(24, 10, 48, 3, input_seed=11)
    args = (0.02, 1e-2, 5, 4242)
    ref = O.rs_sri(s.eri3, s.metric, s.orb_e, s.orb_c, s.n_occ, s.mu, s.tau, s.tau_w, *args,
                   mode="literal")
    return s, args, ref


@pytest.mark.parametrize("dd_arith", [0, 1], ids=["fp64", "df64"])
def test_literal_against_oracle(B, case, dd_arith):
    s, args, ref = case
    got = run(B, s, *args, B.RSSRI_EST_LITERAL, dd_arith=dd_arith)
    for t in range(s.n_tau):
        assert rel(got["sigma"][t], ref.sigma[t]) < TOL, t
    assert abs(got["e"] - ref.e_corr) < TOL * abs(ref.e_corr)
    assert rel(got["e_pair"], ref.e_pair) < TOL
    assert abs(got["se"] - ref.e_stderr) < 1e-8 * abs(ref.e_stderr)


def test_literal_differs_from_cv_on_the_same_draws(B, case):
    """Both estimators are unbiased but they are different functions of the
    draws: on the same seed their results must differ, by about one stderr."""
    s, args, ref = case
    lit = run(B, s, *args, B.RSSRI_EST_LITERAL)
    cv = run(B, s, *args, B.RSSRI_EST_CV)
    assert rel(lit["sigma"], cv["sigma"]) > 1e-8
    assert abs(lit["e"] - cv["e"]) < 6 * (lit["se"] ** 2 + cv["se"] ** 2) ** 0.5


def test_literal_pair_batches(B, case):
    s, args, _ = case
    a = run(B, s, *args, B.RSSRI_EST_LITERAL)
    b = run(B, s, *args, B.RSSRI_EST_LITERAL, pair_batch=2)
    assert rel(b["sigma"], a["sigma"]) < 1e-13
    assert rel(b["e_pair"], a["e_pair"]) < 1e-13


def test_literal_threshold_zero_is_exact_ri(B):
    """eps = eps' = 0: R^L = R, so every S_xi vanishes and the literal
    estimator reduces to the RI self-energy for any draw."""
    s = synth.make_system(18, 7, 36, 3, input_seed=4)
    got = run(B, s, 0.0, 0.0, 4, 5, B.RSSRI_EST_LITERAL)
    k = O.ri_factor(s.eri3, O.metric_inv_sqrt(s.metric))
    for t in range(s.n_tau):
        g, gb = O.green(s.orb_e, s.orb_c, s.n_occ, s.mu, s.tau[t])
        assert rel(got["sigma"][t], O.sigma_from_factor(k, g, gb)) < TOL


def test_literal_rejects_reduced_precision(B, case):
    s, args, _ = case
    h = B.Handle(0)
    opts = B.Handle.options(*args, estimator=B.RSSRI_EST_LITERAL, precision=B.RSSRI_PREC_BF16)
    dev = [torch.from_numpy(a).cuda() for a in (s.eri3, s.metric, s.orb_e, s.orb_c, s.tau,
                                                 s.tau_w)]
    h.setup(*dev, n_occ=s.n_occ, mu=s.mu, beta=s.beta, opts=B.Handle.options(*args))
    sig = torch.empty((s.n_tau, s.n, s.n), dtype=torch.float64, device="cuda")
    with pytest.raises(B.RssriError) as e:
        h.sigma(opts, sig)
    assert e.value.code == -1
    h.close()
