"""Many independent systems at once (rssri_sigma_async / rssri_sigma_wait /
rssri_sigma_batch): each handle on its own stream, all work enqueued before
any is waited for.  Every result must equal, bit for bit, the same handle's
synchronous rssri_sigma, and one of them the fp64 oracle to 1e-10."""
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


SIZES = [(24, 10, 48), (32, 14, 64), (40, 18, 80), (56, 25, 112)]


def make(B, dims, seed, opts):
    s = synth.make_system(*dims, 3, input_seed=seed)
    stream = torch.cuda.Stream()
    h = B.Handle(0, stream=stream.cuda_stream)
    dev = [torch.from_numpy(a).cuda() for a in (s.eri3, s.metric, s.orb_e, s.orb_c, s.tau,
                                                 s.tau_w)]
    torch.cuda.synchronize()
    h.setup(*dev, n_occ=s.n_occ, mu=s.mu, beta=s.beta, opts=opts)
    sig = torch.empty((s.n_tau, s.n, s.n), dtype=torch.float64, device="cuda")
    ep = torch.empty(opts.n_s, dtype=torch.float64, device="cuda")
    return s, h, dev, sig, ep


@pytest.mark.parametrize("precision", ["fp64", "bf16"])
def test_batch_equals_one_by_one(B, precision):
    prec = B.RSSRI_PREC_FP64 if precision == "fp64" else B.RSSRI_PREC_BF16
    opts = B.Handle.options(0.02, 1e-2, 6, 31, precision=prec, dd_arith=B.RSSRI_DD_DF64)
    sysm = [make(B, d, 20 + i, opts) for i, d in enumerate(SIZES)]
    ref = []
    for s, h, _, sig, ep in sysm:
        e, se, _ = h.sigma(opts, sig, ep)
        torch.cuda.synchronize()
        ref.append((sig.cpu().numpy().copy(), ep.cpu().numpy().copy(), e, se))
        sig.zero_()
        ep.zero_()
    torch.cuda.synchronize()
    es, ses = B.sigma_batch([x[1] for x in sysm], opts, [x[3] for x in sysm],
                            [x[4] for x in sysm])
    torch.cuda.synchronize()
    for i, (s, h, _, sig, ep) in enumerate(sysm):
        assert np.array_equal(sig.cpu().numpy(), ref[i][0]), i
        assert np.array_equal(ep.cpu().numpy(), ref[i][1]), i
        assert es[i] == ref[i][2] and ses[i] == ref[i][3], i
    if precision == "fp64":
        s = sysm[0][0]
        o = O.rs_sri(s.eri3, s.metric, s.orb_e, s.orb_c, s.n_occ, s.mu, s.tau, s.tau_w, 0.02,
                     1e-2, 6, 31)
        for t in range(s.n_tau):
            d = np.linalg.norm(ref[0][0][t] - o.sigma[t]) / np.linalg.norm(o.sigma[t])
            assert d < 1e-10
        assert abs(es[0] - o.e_corr) < 1e-10 * abs(o.e_corr)
    for x in sysm:
        x[1].close()


def test_async_wait_and_pending_rules(B):
    opts = B.Handle.options(0.02, 1e-2, 5, 7)
    s, h, dev, sig, ep = make(B, SIZES[1], 3, opts)
    e0, se0, _ = h.sigma(opts, sig, ep)
    a = sig.cpu().numpy().copy()
    sig.zero_()
    torch.cuda.synchronize()
    h.sigma_async(opts, sig, ep)
    with pytest.raises(B.RssriError) as err:  # one pending call per handle
        h.sigma_async(opts, sig, ep)
    assert err.value.code == -1
    with pytest.raises(B.RssriError) as err:  # no setup while a call is pending
        h.setup(*dev, n_occ=s.n_occ, mu=s.mu, beta=s.beta, opts=opts)
    assert err.value.code == -1
    e1, se1, st = h.sigma_wait()
    torch.cuda.synchronize()
    assert np.array_equal(sig.cpu().numpy(), a) and e1 == e0 and se1 == se0
    assert st["kernel_launches"] > 0
    with pytest.raises(B.RssriError) as err:  # nothing pending any more
        h.sigma_wait()
    assert err.value.code == -1
    h.close()
