"""The device-side synthetic generator (used by the many-chain workload) draws
the same structure as the host one: (ij|A) symmetric in (i, j) with the
exp(-|i - j| / 3) / sqrt(N_aux) envelope on standard normal draws, an SPD
metric B B^T / N_aux + 0.5 I, orthonormal orbitals with positive R diagonal,
the same orbital energies and tau grid.  Run here on the CPU device."""
import numpy as np
import pytest

from paper_2005_12338_gb300 import synth

torch = pytest.importorskip("torch")


def test_device_generator_structure():
    n, n_occ, n_aux, n_tau = 24, 11, 72, 5
    s = synth.make_system_torch(n, n_occ, n_aux, n_tau, input_seed=7, device="cpu")
    ref = synth.make_system(n, n_occ, n_aux, n_tau, input_seed=7)
    eri = s.eri3.numpy()
    assert eri.shape == (n, n, n_aux)
    assert np.array_equal(eri, eri.transpose(1, 0, 2))
    idx = np.arange(n)
    env = np.exp(-np.abs(idx[:, None] - idx[None, :]) / 3.0) / np.sqrt(n_aux)
    g = eri / env[:, :, None]
    iu = np.triu_indices(n)
    draws = g[iu[0], iu[1], :].ravel()
    assert abs(draws.mean()) < 0.02 and abs(draws.std() - 1.0) < 0.02
    v = s.metric.numpy()
    assert np.array_equal(v, v.T)
    assert np.linalg.eigvalsh(v).min() > 0.5 - 1e-12
    c = s.orb_c.numpy()
    assert np.abs(c.T @ c - np.eye(n)).max() < 1e-12
    assert np.abs(s.orb_e.numpy() - ref.orb_e).max() < 1e-15  # linspace, to rounding
    assert np.array_equal(s.tau.numpy(), ref.tau) and np.array_equal(s.tau_w.numpy(), ref.tau_w)
    assert s.mu == ref.mu and s.beta == ref.beta


def test_many_chain_sizes():
    sizes = synth.many_sizes(synth.C4["k"], synth.C4["n_min"], synth.C4["n_max"])
    assert len(sizes) == 64 and sizes[0] == 100 and sizes[-1] == 800
    assert all(b > a for a, b in zip(sizes, sizes[1:]))
