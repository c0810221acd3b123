"""Pins of the learned-control-variate oracle (CPU only)."""
import itertools

import numpy as np

import oracle as O
from oracle import cv
from paper_2005_12338_gb300 import synth


def test_mlp_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    params = [(rng.standard_normal((o, i)) * 0.3, rng.standard_normal(o) * 0.1)
              for i, o in ((cv.N_FEAT, 7), (7, 6), (6, 5), (5, 1))]
    x = rng.standard_normal((13, cv.N_FEAT))
    t = rng.standard_normal(13)
    w = rng.random(13) + 0.1
    loss, grads = cv.mlp_loss_grad(params, x, t, w)
    h = 1e-6
    for k in range(4):
        for which in (0, 1):
            arr = params[k][which]
            g = grads[k][which]
            for idx in [tuple(rng.integers(0, s) for s in arr.shape) for _ in range(4)]:
                old = arr[idx]
                arr[idx] = old + h
                lp, _ = cv.mlp_loss_grad(params, x, t, w)
                arr[idx] = old - h
                lm, _ = cv.mlp_loss_grad(params, x, t, w)
                arr[idx] = old
                fd = (lp - lm) / (2 * h)
                assert abs(fd - g[idx]) < 1e-6 * max(1.0, abs(fd)), (k, which, idx, fd, g[idx])


def test_optimal_coefficient_recovers_linear_relation():
    rng = np.random.default_rng(1)
    fl = rng.standard_normal((4000, 3))
    f = np.array([0.5, 1.0, 2.0]) * fl + 0.01 * rng.standard_normal((4000, 3))
    c, var = cv.cv_optimal(f, fl)
    assert np.allclose(c, [0.5, 1.0, 2.0], atol=2e-3)
    assert np.allclose(var, 1.0, atol=0.1)


def per_sample_terms(s, eps_prime, eps, th0, th1, t):
    w = O.metric_inv_sqrt(s.metric)
    el, _, _ = O.screen(s.eri3, eps_prime)
    kl, _ = O.large_factor(el, w, eps)
    r0, rl0 = O.stochastic_factors(s.eri3, w, kl, th0)
    r1, rl1 = O.stochastic_factors(s.eri3, w, kl, th1)
    g, gb = O.green(s.orb_e, s.orb_c, s.n_occ, s.mu, s.tau[t])
    f = np.array([O.factor_pair(r0[x], r1[x], g, gb)[0] for x in range(th0.shape[0])])
    fl = np.array([O.factor_pair(rl0[x], rl1[x], g, gb)[0] for x in range(th0.shape[0])])
    return f, fl, O.sigma_from_factor(kl, g, gb), O.ri_factor(s.eri3, w), g, gb


def test_unit_coefficient_is_the_default_estimator():
    s = synth.make_system(10, 4, 24, 3, input_seed=3)
    r = O.rs_sri(s.eri3, s.metric, s.orb_e, s.orb_c, s.n_occ, s.mu, s.tau, s.tau_w, 0.02, 0.05,
                 6, 2)
    f, fl, sdd, _, _, _ = per_sample_terms(s, 0.02, 0.05, r.extra["theta0"], r.extra["theta1"], 1)
    sig = cv.cv_sigma(f.sum(0), fl.sum(0), 6, sdd, np.ones_like(sdd))
    assert np.abs(sig - r.sigma_raw[1]).max() < 1e-12 * np.abs(sig).max()


def test_any_fixed_coefficient_is_unbiased_exhaustive():
    s = synth.make_system(6, 3, 4, 2, input_seed=4)
    signs = np.array(list(itertools.product((-1.0, 1.0), repeat=4)))
    th0 = np.repeat(signs, len(signs), axis=0)
    th1 = np.tile(signs, (len(signs), 1))
    f, fl, sdd, k, g, gb = per_sample_terms(s, 0.3, 0.2, th0, th1, 1)
    c = np.random.default_rng(5).uniform(-1.0, 3.0, size=sdd.shape)
    sig = cv.cv_sigma(f.sum(0), fl.sum(0), f.shape[0], sdd, c)
    ref = O.sigma_from_factor(k, g, gb)
    assert np.abs(sig - ref).max() < 1e-12 * np.abs(ref).max()


def test_features_shape_and_range():
    s = synth.make_system(8, 3, 16, 2, input_seed=6)
    w = O.metric_inv_sqrt(s.metric)
    el, _, _ = O.screen(s.eri3, 0.02)
    kl, _ = O.large_factor(el, w, 0.05)
    g, gb = O.green(s.orb_e, s.orb_c, s.n_occ, s.mu, s.tau[0])
    sdd = O.sigma_from_factor(kl, g, gb)
    rn = np.sqrt((kl ** 2).sum(axis=(1, 2)))
    f = cv.features(sdd, g, gb, s.tau[0], s.beta, rn)
    assert f.shape == (64, cv.N_FEAT)
    assert np.all(np.abs(f[:, [0, 2, 3, 4, 5, 6, 7, 8]]) <= 1.0 + 1e-15)
    assert f[9, 0] == 0.0 and f[9, 9] == 1.0  # element (1, 1)
    assert f[1, 0] == 1 / 8 and f[1, 9] == 0.0  # element (0, 1)


def test_features_hand_computed_3x3():
    """Every feature of three elements of a 3 x 3 case, worked by hand: which
    index (i or j) each feature reads and what it is normalised by."""
    sdd = np.array([[2.0, -1.0, 0.0], [-1.0, 4.0, 0.5], [0.0, 0.5, -1.0]])  # max |.| = 4
    g = np.array([[-0.5, 0.3, 0.1], [0.3, -1.0, 0.2], [0.1, 0.2, -0.25]])  # max |diag| = 1
    gb = np.array([[-2.0, 0.7, 0.0], [0.7, -1.0, 0.0], [0.0, 0.0, -4.0]])  # max |diag| = 4
    rn = np.array([3.0, 6.0, 1.5])  # max 6
    tau, beta = np.e, np.e ** 2  # ln tau / ln beta = 1/2
    f = cv.features(sdd, g, gb, tau, beta, rn)
    want = {
        # (i, j): [|i-j|/N, ln tau/ln beta, Sdd_ij/4, G_ii, G_jj, Gb_ii/4, Gb_jj/4, r_i/6, r_j/6, i==j]
        (0, 2): [2 / 3, 0.5, 0.0, -0.5, -0.25, -0.5, -1.0, 0.5, 0.25, 0.0],
        (1, 0): [1 / 3, 0.5, -0.25, -1.0, -0.5, -0.25, -0.5, 1.0, 0.5, 0.0],
        (2, 2): [0.0, 0.5, -0.25, -0.25, -0.25, -1.0, -1.0, 0.25, 0.25, 1.0],
        (1, 2): [1 / 3, 0.5, 0.125, -1.0, -0.25, -0.25, -1.0, 1.0, 0.25, 0.0],
    }
    for (i, j), row in want.items():
        assert np.allclose(f[3 * i + j], row, rtol=0, atol=1e-15), ((i, j), f[3 * i + j])
