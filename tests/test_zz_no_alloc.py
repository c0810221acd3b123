"""rssri_energy_static: the allocation-free Eq. 26 energy for callers that may
not allocate device memory (graph capture, host-owned memory pools).

Runs last (file name) so that a failure here does not hide the other tests.
Checks, through the C ABI, that two calls in a row reproduce the energy that
rssri_sigma reports for the same self-energy and the oracle's Eq. 26 trace of
the same arrays (a bug shared by the library's trace kernels would not pass
the second check), for tau counts below, at and above the 32-wide reduction
blocks, and that sizes beyond the static scratch are rejected before any
work is launched.
"""
import ctypes as C

import numpy as np
import pytest

import oracle as O
from paper_2005_12338_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2005_12338_gb300 import binding, build
    build.build()
    return binding


@pytest.mark.parametrize("n_tau", [6, 32, 45])
def test_static_energy_matches_sigma_energy_twice(B, n_tau):
    s = synth.make_system(24, 11, 48, n_tau, input_seed=8)
    dev = [torch.from_numpy(a).cuda() for a in (s.eri3, s.metric, s.orb_e, s.orb_c, s.tau,
                                                 s.tau_w)]
    h = B.Handle(0)
    opts = B.Handle.options(0.02, 1e-2, 6, 4)
    h.setup(*dev, n_occ=s.n_occ, mu=s.mu, beta=s.beta, opts=opts)
    sig = torch.empty((s.n_tau, s.n, s.n), dtype=torch.float64, device="cuda")
    e_ref, _, _ = h.sigma(opts, sig)
    gb_h = h.export("GB").reshape(s.n_tau, s.n, s.n)
    gb = torch.from_numpy(gb_h).cuda()
    # the oracle's Eq. 26 trace of the same arrays
    e_oracle = O.energy_trace(sig.cpu().numpy(), gb_h, s.tau_w, s.n_occ)
    assert abs(e_ref - e_oracle) <= 1e-12 * abs(e_oracle)
    stream = torch.cuda.current_stream().cuda_stream
    lib = B.lib()
    for _ in range(2):
        out = torch.full((1,), np.nan, dtype=torch.float64, device="cuda")
        rc = lib.rssri_energy_static(sig.data_ptr(), gb.data_ptr(), dev[5].data_ptr(), s.n,
                                     s.n_tau, s.n_occ, out.data_ptr(), C.c_void_p(stream))
        assert rc == 0
        torch.cuda.synchronize()
        e = float(out.item())
        assert abs(e - e_ref) <= 1e-10 * abs(e_ref), (e, e_ref)
        assert abs(e - e_oracle) <= 1e-12 * abs(e_oracle), (e, e_oracle)
    h.close()


def test_static_energy_rejects_oversize(B):
    x = torch.zeros(4, dtype=torch.float64, device="cuda")
    lib = B.lib()
    too_many = B.RSSRI_STATIC_MAX_TAU + 1
    rc = lib.rssri_energy_static(x.data_ptr(), x.data_ptr(), x.data_ptr(), 1, too_many, 1,
                                 x.data_ptr(), None)
    assert rc == -1
    rc = lib.rssri_energy_static(None, x.data_ptr(), x.data_ptr(), 1, 1, 1, x.data_ptr(), None)
    assert rc == -1
