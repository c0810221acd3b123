"""Pins of the fp64 oracle against facts fixed by the paper and the mathematics
(not against the oracle itself).  CPU only."""
import itertools
import json
import os

import numpy as np
import pytest

import oracle as O
from paper_2005_12338_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def small(n=10, n_occ=4, n_aux=24, n_tau=16, seed=3):
    return synth.make_system(n, n_occ, n_aux, n_tau, input_seed=seed)


def ri_sigma(s, k, taus=None):
    taus = s.tau if taus is None else taus
    out, gbs = [], []
    for t in taus:
        g, gb = O.green(s.orb_e, s.orb_c, s.n_occ, s.mu, t)
        out.append(O.sigma_from_factor(k, g, gb))
        gbs.append(gb)
    return np.array(out), gbs


# ---------------------------------------------------------------- RNG -------
def test_splitmix64_published_stream():
    # SplitMix64 (Steele, Lea & Flood 2014) reference outputs.
    assert O.splitmix64_stream(0, 3) == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4,
                                         0x06C45D188009454F]
    assert O.splitmix64_stream(1234567, 5) == [
        6457827717110365317, 3203168211198807973, 9817491932198370423,
        4593380528125082431, 16408922859458223821]


def test_rademacher_counter_layout():
    seed = 0xDEADBEEF12345
    th = O.rademacher(seed, 1, 7, 33, xi_offset=11)
    for xi in (0, 3, 6):
        for q in (0, 17, 32):
            c = (1 << 60) | ((11 + xi) << 20) | q
            z = O.splitmix64_stream(seed ^ c, 1)[0]
            assert th[xi, q] == (-1.0 if z >> 63 else 1.0)
    # resume: an offset block is the tail of a longer block
    a = O.rademacher(5, 0, 40, 50)
    b = O.rademacher(5, 0, 30, 50, xi_offset=10)
    assert np.array_equal(a[10:], b)
    # the two sets are different streams, both balanced
    t0 = O.rademacher(0, 0, 400, 500)
    t1 = O.rademacher(0, 1, 400, 500)
    assert not np.array_equal(t0, t1)
    for t in (t0, t1):
        assert set(np.unique(t)) == {-1.0, 1.0}
        assert abs(t.mean()) < 0.01
    assert abs((t0 * t1).mean()) < 0.01


# ------------------------------------------------------ Sec. II factors -----
def test_metric_inv_sqrt_is_the_spd_root():
    s = small()
    w = O.metric_inv_sqrt(s.metric)
    eye = np.eye(s.n_aux)
    assert np.allclose(w, w.T, atol=1e-14)
    assert np.linalg.eigvalsh(w).min() > 0
    assert np.abs(w @ s.metric @ w - eye).max() < 1e-12
    assert np.abs(w @ w @ s.metric - eye).max() < 1e-12
    with pytest.raises(ValueError):
        O.metric_inv_sqrt(np.diag([1.0, -1.0, 2.0]))


def test_ri_factor_matches_metric_inverse_form():
    # Eq. 8 (sum_Q K K) against Eq. 4 (sum_AB (ij|A) V^-1_AB (B|kl)).
    s = small(n=6, n_aux=14)
    k = O.ri_factor(s.eri3, O.metric_inv_sqrt(s.metric))
    v8 = O.eri4_from_factor(k)
    e = s.eri3.reshape(36, 14)
    v4 = (e @ np.linalg.solve(s.metric, e.T)).reshape(6, 6, 6, 6)
    assert np.abs(v8 - v4).max() < 1e-13 * np.abs(v4).max()
    # permutational symmetry of real integrals
    assert np.allclose(v8, v8.transpose(1, 0, 2, 3), atol=1e-15)
    assert np.allclose(v8, v8.transpose(2, 3, 0, 1), atol=1e-15)


def test_screen_and_cut_golden():
    with open(os.path.join(GOLDEN, "screen_cut_n2.json")) as f:
        gd = json.load(f)
    eri3 = np.array(gd["eri3"])
    eri3_l, mask, m = O.screen(eri3, gd["eps_prime"])
    assert np.array_equal(m, gd["m_col"])
    assert np.array_equal(mask, np.array(gd["mask"]))
    assert np.array_equal(eri3_l, np.where(np.array(gd["mask"]), eri3, 0.0))
    w = O.metric_inv_sqrt(np.array(gd["metric"]))
    k_l, kmax = O.large_factor(eri3_l, w, gd["eps"])
    assert kmax == pytest.approx(gd["k_l_max"], rel=1e-15)
    assert np.allclose(k_l, np.array(gd["k_l_cut"]), atol=1e-15)
    # eps = 0 keeps every entry: the product before the cut
    k_all, _ = O.large_factor(eri3_l, w, 0.0)
    assert np.allclose(k_all, np.array(gd["k_l_before_cut"]), atol=1e-15)


def test_screen_limits_and_symmetry():
    s = small(n=12, n_aux=30)
    e_l, mask, _ = O.screen(s.eri3, 0.0)
    assert mask.all()
    e_l, mask, _ = O.screen(s.eri3, 0.05)
    assert np.array_equal(mask, mask.transpose(1, 0, 2))
    assert 0 < mask.sum() < mask.size
    # larger eps' keeps a subset
    _, mask2, _ = O.screen(s.eri3, 0.5)
    assert not np.any(mask2 & ~mask)
    # every column keeps its own maximum (threshold <= eps'/N * M_j <= M_j)
    a = np.abs(s.eri3)
    for j in range(s.n):
        i, q = np.unravel_index(np.argmax(a[:, j, :]), a[:, j, :].shape)
        assert mask[i, j, q]


def test_sri_expectation_exhaustive():
    # Eq. 10: averaging R_ij R_kl over all 2^N_aux sign vectors gives v_ijkl.
    s = small(n=5, n_aux=4)
    w = O.metric_inv_sqrt(s.metric)
    theta = np.array(list(itertools.product((-1.0, 1.0), repeat=4)))
    r, _ = O.stochastic_factors(s.eri3, w, np.zeros_like(s.eri3), theta)
    v_sri = np.einsum("xij,xkl->ijkl", r, r) / theta.shape[0]
    v = O.eri4_from_factor(O.ri_factor(s.eri3, w))
    assert np.abs(v_sri - v).max() < 1e-13 * np.abs(v).max()


# ------------------------------------------------------- Sec. III / Eq. 20 --
def test_green_jump_particle_number_and_eom():
    s = small(n=9, n_occ=4)
    g0, gb0 = O.green(s.orb_e, s.orb_c, s.n_occ, s.mu, 0.0)
    # Eq. 2 with S = I: G(0+) - G(0-) = -I and G(beta - 0) = -G(0-)
    assert np.abs(g0 + gb0 + np.eye(s.n)).max() < 1e-14
    # particle number N_e = -2 sum_ij G_ij(beta^-) S_ij
    assert -2.0 * np.trace(gb0) == pytest.approx(2 * s.n_occ, rel=1e-14)
    # Eq. 18 without Sigma (S = I): -dG/dtau = (F - mu) G, F = C diag(e) C^T
    f = (s.orb_c * s.orb_e) @ s.orb_c.T - s.mu * np.eye(s.n)
    t, h = 0.7, 1e-5
    gp, gbp = O.green(s.orb_e, s.orb_c, s.n_occ, s.mu, t + h)
    gm, gbm = O.green(s.orb_e, s.orb_c, s.n_occ, s.mu, t - h)
    g, gb = O.green(s.orb_e, s.orb_c, s.n_occ, s.mu, t)
    assert np.abs(-(gp - gm) / (2 * h) - f @ g).max() < 1e-8
    # Gb(tau) = G(beta - tau) obeys d/dtau Gb = (F - mu) Gb
    assert np.abs((gbp - gbm) / (2 * h) - f @ gb).max() < 1e-8


def test_sigma_factor_form_matches_bruteforce_eq20():
    s = small(n=7, n_occ=3, n_aux=10)
    k = O.ri_factor(s.eri3, O.metric_inv_sqrt(s.metric))
    v = O.eri4_from_factor(k)
    for t in (0.05, 1.3, 17.0):
        g, gb = O.green(s.orb_e, s.orb_c, s.n_occ, s.mu, t)
        a = O.sigma_eri4(v, g, gb)
        b = O.sigma_from_factor(k, g, gb)
        assert np.abs(a - b).max() < 1e-12 * np.abs(a).max()
        assert np.abs(b - b.T).max() < 1e-13 * np.abs(b).max()


def mp2_on_grid(s, k, tau, tau_w):
    """Closed-form MP2 integrand in the MO basis, integrated on the grid."""
    o, c = s.n_occ, s.orb_c
    kmo = np.einsum("pi,pqQ,qa->iaQ", c[:, :o], k, c[:, o:])
    iajb = np.einsum("iaQ,jbQ->iajb", kmo, kmo)
    eo, ev = s.orb_e[:o], s.orb_e[o:]
    delta = ev[None, :, None, None] + ev[None, None, None, :] - eo[:, None, None, None] - eo[None, None, :, None]
    num = iajb * (2 * iajb - iajb.transpose(0, 3, 2, 1))
    e_grid = -sum(w * np.sum(num * np.exp(-delta * t)) for t, w in zip(tau, tau_w))
    e_exact = -np.sum(num / delta)
    return e_grid, e_exact


def test_energy_matches_mp2_closed_form():
    s = small(n=12, n_occ=5, n_aux=30, n_tau=48)
    k = O.ri_factor(s.eri3, O.metric_inv_sqrt(s.metric))
    sig, gbs = ri_sigma(s, k)
    e_corr = O.energy_trace(sig, gbs, s.tau_w, s.n_occ)
    e_grid, e_exact = mp2_on_grid(s, k, s.tau, s.tau_w)
    ne = 2 * s.n_occ
    assert ne * e_corr == pytest.approx(e_grid, rel=1e-12)
    assert e_corr < 0
    # the log-spaced Gauss-Legendre tau grid converges to the textbook MP2 energy
    tau, tw = synth.tau_grid(160, s.beta)
    e_fine, _ = mp2_on_grid(s, k, tau, tw)
    assert e_fine == pytest.approx(e_exact, rel=1e-9)


# -------------------------------------------------------- the estimator -----
def run(s, **kw):
    args = dict(eps_prime=0.02, eps=1e-2, n_s=16, seed=0)
    args.update(kw)
    return O.rs_sri(s.eri3, s.metric, s.orb_e, s.orb_c, s.n_occ, s.mu, s.tau, s.tau_w, **args)


@pytest.mark.parametrize("mode", ["cv", "literal"])
def test_estimator_unbiased_exhaustive(mode):
    # Mean over every (theta, theta') pair of sign vectors equals the RI Sigma.
    s = small(n=6, n_occ=3, n_aux=4, n_tau=3)
    signs = np.array(list(itertools.product((-1.0, 1.0), repeat=4)))
    th0 = np.repeat(signs, len(signs), axis=0)
    th1 = np.tile(signs, (len(signs), 1))
    r = run(s, eps_prime=0.3, eps=0.2, theta=(th0, th1), mode=mode)
    k_l = r.extra["k_l"]
    assert 0 < np.count_nonzero(k_l) < k_l.size  # a real split
    k = O.ri_factor(s.eri3, r.extra["w"])
    ref, _ = ri_sigma(s, k)
    assert np.abs(r.sigma_raw - ref).max() < 1e-12 * np.abs(ref).max()


def test_threshold_zero_gives_exact_ri():
    s = small(n=10, n_occ=4, n_aux=24, n_tau=6)
    r = run(s, eps_prime=0.0, eps=0.0, n_s=8, seed=7)
    k = O.ri_factor(s.eri3, r.extra["w"])
    ref, gbs = ri_sigma(s, k)
    assert np.abs(r.sigma - ref).max() < 1e-12 * np.abs(ref).max()
    assert np.abs(r.e_pair - r.e_corr).max() < 1e-12 * abs(r.e_corr)


def test_empty_large_part_is_plain_sri():
    s = small(n=8, n_occ=4, n_aux=16, n_tau=4)
    r = run(s, empty_large=True, n_s=6, seed=2)
    assert np.abs(r.sigma_dd).max() == 0.0
    w = r.extra["w"]
    r0, _ = O.stochastic_factors(s.eri3, w, np.zeros_like(s.eri3), O.rademacher(2, 0, 6, 16))
    r1, _ = O.stochastic_factors(s.eri3, w, np.zeros_like(s.eri3), O.rademacher(2, 1, 6, 16))
    for it, t in enumerate(s.tau):
        g, gb = O.green(s.orb_e, s.orb_c, s.n_occ, s.mu, t)
        sri = sum(O.factor_pair(r0[x], r1[x], g, gb)[0] for x in range(6)) / 6
        assert np.abs(r.sigma_raw[it] - sri).max() < 1e-13 * np.abs(sri).max()


def test_split_form_equals_difference_form():
    s = small(n=10, n_occ=4, n_aux=24, n_tau=5)
    a = run(s, eps=0.05, n_s=5, seed=4)
    b = run(s, eps=0.05, n_s=5, seed=4, form="split")
    assert np.abs(a.sigma - b.sigma).max() < 1e-12 * np.abs(a.sigma).max()
    assert np.abs(a.e_pair - b.e_pair).max() < 1e-12 * abs(a.e_corr)


def test_energy_is_mean_of_pairs_and_sigma_symmetric():
    s = small(n=10, n_occ=4, n_aux=24, n_tau=5)
    r = run(s, n_s=9, seed=1)
    assert r.e_corr == pytest.approx(np.mean(r.e_pair), rel=1e-12)
    assert np.array_equal(r.sigma, np.transpose(r.sigma, (0, 2, 1)))
    sdd = r.sigma_dd
    assert np.abs(sdd - np.transpose(sdd, (0, 2, 1))).max() < 1e-13 * np.abs(sdd).max()


@pytest.mark.slow
def test_error_law_and_agreement_with_ri():
    # Sec. IV: the statistical error falls as 1/sqrt(N_s); stochastic results
    # agree with deterministic RI within their error bars; the range-separated
    # form has a much smaller error than plain SRI at the same N_s.
    s = small(n=12, n_occ=6, n_aux=36, n_tau=12, seed=1)
    k = O.ri_factor(s.eri3, O.metric_inv_sqrt(s.metric))
    sig, gbs = ri_sigma(s, k)
    e_ri = O.energy_trace(sig, gbs, s.tau_w, s.n_occ)
    se = {}
    for ns in (32, 512):
        r = run(s, eps=0.05, n_s=ns, seed=11)
        se[ns] = r.e_stderr
        assert abs(r.e_corr - e_ri) < 4 * r.e_stderr
    ratio = se[32] / se[512]
    assert 2.8 < ratio < 5.6  # sqrt(16) = 4
    sri = run(s, eps=0.05, n_s=32, seed=11, empty_large=True)
    assert abs(sri.e_corr - e_ri) < 4 * sri.e_stderr
    assert sri.e_stderr > 3 * se[32]
