"""Failure paths, made on the host: a bounded device wait that expires and a
device allocation that fails.  Neither faults, traps or hangs the GPU.

* rssri_options.test_wait_polls > 0 makes the tensor-core kernels of the call
  issue no copy and no product and give up their first wait after that many
  polls: nothing is in flight when they flag the expiry.  The call must
  return RSSRI_ERR_TIMEOUT, and the same handle must then give, bit for bit,
  what a fresh handle gives.
* rssri_options.test_fail_alloc = k makes the k-th device allocation of the
  call fail without calling the allocator.  Every k up to the number of
  allocations must return RSSRI_ERR_OOM, and the handle must recover.
"""
import numpy as np
import pytest

from paper_2005_12338_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
TIMEOUT, OOM = -6, -4


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2005_12338_gb300 import binding, build
    build.build()
    return binding


@pytest.fixture(scope="module")
def sysd():
    s = synth.make_system(40, 18, 80, 4, input_seed=21)
    dev = [torch.from_numpy(a).cuda() for a in (s.eri3, s.metric, s.orb_e, s.orb_c, s.tau,
                                                 s.tau_w)]
    return s, dev


def run(B, h, s, dev, opts, setup=True):
    if setup:
        h.setup(*dev, n_occ=s.n_occ, mu=s.mu, beta=s.beta, opts=opts)
    sig = torch.empty((s.n_tau, s.n, s.n), dtype=torch.float64, device="cuda")
    ep = torch.empty(opts.n_s, dtype=torch.float64, device="cuda")
    e, se, _ = h.sigma(opts, sig, ep)
    torch.cuda.synchronize()
    return sig.cpu().numpy(), ep.cpu().numpy(), e


def fresh(B, s, dev, opts):
    h = B.Handle(0)
    out = run(B, h, s, dev, opts)
    h.close()
    return out


def same(a, b):
    return np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]) and a[2] == b[2]


def test_expired_wait_in_the_tensor_core_chain(B, sysd):
    s, dev = sysd
    o = B.Handle.options(0.02, 1e-2, 6, 3, precision=B.RSSRI_PREC_BF16)
    bad = B.Handle.options(0.02, 1e-2, 6, 3, precision=B.RSSRI_PREC_BF16, test_wait_polls=1)
    h = B.Handle(0)
    h.setup(*dev, n_occ=s.n_occ, mu=s.mu, beta=s.beta, opts=o)
    sig = torch.empty((s.n_tau, s.n, s.n), dtype=torch.float64, device="cuda")
    with pytest.raises(B.RssriError) as e:
        h.sigma(bad, sig)
    assert e.value.code == TIMEOUT
    got = run(B, h, s, dev, o, setup=False)
    h.close()
    assert same(got, fresh(B, s, dev, o))


def test_expired_wait_in_the_sliced_block(B, sysd):
    s, dev = sysd
    o = B.Handle.options(0.02, 1e-2, 6, 3, precision=B.RSSRI_PREC_DF64, dd_arith=B.RSSRI_DD_OZ)
    bad = B.Handle.options(0.02, 1e-2, 6, 3, precision=B.RSSRI_PREC_DF64, dd_arith=B.RSSRI_DD_OZ,
                           test_wait_polls=1)
    h = B.Handle(0)
    with pytest.raises(B.RssriError) as e:
        h.setup(*dev, n_occ=s.n_occ, mu=s.mu, beta=s.beta, opts=bad)
    assert e.value.code == TIMEOUT
    sig = torch.empty((s.n_tau, s.n, s.n), dtype=torch.float64, device="cuda")
    with pytest.raises(B.RssriError) as e:  # no usable setup
        h.sigma(o, sig)
    assert e.value.code == -7
    got = run(B, h, s, dev, o)
    h.close()
    assert same(got, fresh(B, s, dev, o))


@pytest.mark.parametrize("call", ["setup", "sigma"])
def test_failed_allocation_is_reported_and_recovered(B, sysd, call):
    s, dev = sysd
    o = B.Handle.options(0.02, 1e-2, 6, 3, precision=B.RSSRI_PREC_DF64, dd_arith=B.RSSRI_DD_OZ)
    ref = fresh(B, s, dev, o)
    failures = 0
    for k in range(1, 400):
        bad = B.Handle.options(0.02, 1e-2, 6, 3, precision=B.RSSRI_PREC_DF64,
                               dd_arith=B.RSSRI_DD_OZ, test_fail_alloc=k)
        h = B.Handle(0)
        if call == "sigma":
            h.setup(*dev, n_occ=s.n_occ, mu=s.mu, beta=s.beta, opts=o)
        sig = torch.empty((s.n_tau, s.n, s.n), dtype=torch.float64, device="cuda")
        try:
            if call == "setup":
                h.setup(*dev, n_occ=s.n_occ, mu=s.mu, beta=s.beta, opts=bad)
            else:
                h.sigma(bad, sig)
            ok = True
        except B.RssriError as e:
            assert e.code == OOM, (k, e)
            ok = False
        if ok:
            h.close()
            break
        failures += 1
        # the same handle recovers with a normal call
        assert same(run(B, h, s, dev, o), ref)
        h.close()
    assert failures > 5  # the calls do allocate, and every allocation was made to fail once
