"""The deterministic block (G(tau), G(beta - tau), Sigma_DD(tau); S6 and S7)
is built once by rssri_setup and reused by every sampling call.

A handle set up once must give, for draws A, B and A resumed at an offset,
bit for bit what a fresh setup gives for each; no sampling call on it may
spend time on the block; and a call with a caller-supplied G in between must
not leave its block behind for the next call."""
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


def run(B, h, s, opts, setup=True, g=None, gb=None):
    if setup:
        arrs = [torch.from_numpy(a).cuda() for a in (s.eri3, s.metric, s.orb_e, s.orb_c, s.tau,
                                                      s.tau_w)]
        h.setup(*arrs, n_occ=s.n_occ, mu=s.mu, beta=s.beta, opts=opts)
    sig = torch.empty((s.n_tau, s.n, s.n), dtype=torch.float64, device="cuda")
    ep = torch.empty(opts.n_s, dtype=torch.float64, device="cuda")
    if g is not None:
        g, gb = torch.from_numpy(g).cuda(), torch.from_numpy(gb).cuda()
    e, se, st = h.sigma(opts, sig, ep, g=g, gb=gb)
    torch.cuda.synchronize()
    return sig.cpu().numpy(), ep.cpu().numpy(), e, st


@pytest.mark.parametrize("prec,dd", [(0, 0), (3, 1), (1, 1)], ids=["fp64", "df64", "bf16"])
def test_block_reused_bitwise(B, prec, dd):
    s = synth.make_system(37, 16, 45, 5, input_seed=11)
    mk = lambda seed, ns=6, off=0: B.Handle.options(0.02, 1e-2, ns, seed, xi_offset=off,
                                                     precision=prec, dd_arith=dd)
    h = B.Handle(0)
    a1 = run(B, h, s, mk(101))
    b1 = run(B, h, s, mk(202), setup=False)
    c1 = run(B, h, s, mk(101, ns=3, off=3), setup=False)
    a2 = run(B, h, s, mk(101), setup=False)
    for r in (a1, b1, c1, a2):
        assert r[3]["t_green_dd_ms"] == 0.0
    # a caller-supplied G in between: its block is rebuilt, then the orbitals' block again
    gs, gbs = zip(*(O.green(s.orb_e, s.orb_c, s.n_occ, s.mu, 0.9 * t) for t in s.tau))
    gx = run(B, h, s, mk(101), setup=False, g=np.array(gs), gb=np.array(gbs))
    assert gx[3]["t_green_dd_ms"] > 0.0
    assert not np.array_equal(gx[0], a1[0])
    a3 = run(B, h, s, mk(101), setup=False)
    assert a3[3]["t_green_dd_ms"] > 0.0
    h.close()
    for got, opts in ((a1, mk(101)), (b1, mk(202)), (c1, mk(101, ns=3, off=3)), (a2, mk(101)),
                      (a3, mk(101))):
        hf = B.Handle(0)
        ref = run(B, hf, s, opts)
        hf.close()
        assert np.array_equal(got[0], ref[0])
        assert np.array_equal(got[1], ref[1])
        assert got[2] == ref[2]
    # resuming at an offset reproduces the tail of the pair energies
    assert np.array_equal(c1[1], a1[1][3:])


def test_sri_after_cached_block(B):
    """The plain stochastic-RI estimator adds to a zero block, also on a handle
    whose setup built a non-zero one; the next default call still sees it."""
    s = synth.make_system(20, 10, 40, 3, input_seed=5)
    h = B.Handle(0)
    o_cv = B.Handle.options(0.02, 1e-2, 6, 9)
    o_sri = B.Handle.options(0.02, 1e-2, 6, 9, estimator=B.RSSRI_EST_SRI)
    a = run(B, h, s, o_cv)
    b = run(B, h, s, o_sri, setup=False)
    c = run(B, h, s, o_cv, setup=False)
    ref = O.rs_sri(s.eri3, s.metric, s.orb_e, s.orb_c, s.n_occ, s.mu, s.tau, s.tau_w, 0.02,
                   1e-2, 6, 9, empty_large=True)
    for t in range(s.n_tau):
        assert np.linalg.norm(b[0][t] - ref.sigma[t]) < 1e-10 * np.linalg.norm(ref.sigma[t])
    assert np.array_equal(a[0], c[0])
    assert np.abs(h.export("SIGMA_DD")).max() > 0
    h.close()


def test_destroy_returns_every_device_allocation():
    """A handle frees all its device memory: after one warm-up handle (the
    context and per-process state), setting up and sampling with fresh
    handles in every form and destroying them leaves free device memory
    where it was."""
    from paper_2005_12338_gb300 import binding as B, build
    build.build()
    s = synth.make_system(48, 20, 120, 3, input_seed=8)
    dev = [torch.from_numpy(a).cuda() for a in (s.eri3, s.metric, s.orb_e, s.orb_c, s.tau,
                                                 s.tau_w)]
    sig = torch.empty((s.n_tau, s.n, s.n), dtype=torch.float64, device="cuda")
    forms = [(B.RSSRI_PREC_BF16, B.RSSRI_DD_OZ), (B.RSSRI_PREC_DF64, B.RSSRI_DD_DF64),
             (B.RSSRI_PREC_FP64, B.RSSRI_DD_FP64)]

    def cycle():
        for prec, dd in forms:
            o = B.Handle.options(0.02, 1e-2, 8, 3, precision=prec, dd_arith=dd)
            h = B.Handle(0)
            h.setup(*dev, n_occ=s.n_occ, mu=s.mu, beta=s.beta, opts=o)
            h.sigma(o, sig)
            h.close()
        torch.cuda.synchronize()

    cycle()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        cycle()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 >= free0 - (2 << 20), (free0 - free1) / 2 ** 20
