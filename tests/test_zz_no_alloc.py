"""ff_match_pair_noalloc, the entry point for callers that must not allocate device memory while they run
(a real-time frame loop that cudaMalloc/cudaFree would stall, memory owned by another framework's fixed pool,
a hot path that must not run out of memory half way).

It must give exactly what ff_match_pair gives (the matching is integer, so the tolerance is zero), on calls in
a row that carve the shared scratch array differently (a smaller pair after a larger one), at the 1242x375 size
of the KITTI-shaped workload against the oracle itself, and near the array's size limit (1.41 Mpx).  Across
every call the device's free memory and the library's count of the bytes it holds must not change: the array
and the kernels were set up when the context was created.  This file is named so that pytest collects it last.
"""
import numpy as np
import pytest

from paper_1805_03517_gb300 import configs
from tests import oracle_pins as P

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ffm():
    from paper_1805_03517_gb300 import build, ff

    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return ff


def _pair(seed, h, w, dx, dy):
    a = P.smooth_texture(seed, h, w)
    b = P.shifted(a, dx, dy, seed + 1)
    b[h // 4:h // 2, w // 5:w // 2] = P.smooth_texture(seed + 2, h // 2 - h // 4, w // 2 - w // 5)
    return a, b


def _noalloc_call(ffm, M, X, Y, dir, h, w):
    """One call into fresh poisoned outputs; asserts that it allocated nothing on the device."""
    with torch.cuda.stream(M.stream):  # poison the outputs on the stream the library uses
        flow = torch.full((h, w, 2), -7, dtype=torch.int16, device="cuda")
        cost = torch.full((h, w), -7, dtype=torch.int32, device="cuda")
    M.sync()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    held0 = ffm.ff_get_stats(M.ctx)["scratch_bytes"]
    ffm.ff_match_pair_noalloc(M.ctx, X.handle, Y.handle, dir, flow.data_ptr(), cost.data_ptr())
    M.sync()
    assert ffm.ff_get_stats(M.ctx)["scratch_bytes"] == held0, "the library allocated during the call"
    assert torch.cuda.mem_get_info()[0] == free0, "device memory was allocated during the call"
    return flow, cost


def test_noalloc_equals_match_pair_on_calls_in_a_row(ffm):
    prm = configs.MatchParams(n_scales=4, iters=3, eps=1)
    M = ffm.Matcher(prm, 0)
    # two pairs of one size (the second call reuses the first one's carving), then a smaller one (a new carving)
    pairs = [_pair(900, 150, 230, 7, -3), _pair(910, 150, 230, -5, 4), _pair(920, 70, 96, 3, 2)]
    for call, (a, b) in enumerate(pairs):
        h, w, _ = a.shape
        pa = M.features(torch.from_numpy(a).cuda())
        pb = M.features(torch.from_numpy(b).cuda())
        for dir, (X, Y) in enumerate(((pa, pb), (pb, pa))):
            ref_flow, ref_cost = M.match_pair(X, Y, dir)
            flow, cost = _noalloc_call(ffm, M, X, Y, dir, h, w)
            assert torch.equal(flow, ref_flow), (call, dir)
            assert torch.equal(cost, ref_cost), (call, dir)
        M.release(pa)
        M.release(pb)
    M.close()


def test_noalloc_kitti_size_against_the_oracle(ffm, orc):
    """The 1242x375 pair of the KITTI-shaped workload (L=5, T=6), each direction against the oracle."""
    import oracle
    from paper_1805_03517_gb300 import synth

    spec = configs.workload("kitti_1242x375").pairs[0]
    a, b, _ = synth.make_pair(spec.kind, spec.seed, spec.w, spec.h)
    p = spec.params
    want = orc.match_bidir(a, b, oracle.params(p.n_scales, p.iters, p.rs_radius, p.eps, p.seed))
    M = ffm.Matcher(p, 0)
    pa = M.features(torch.from_numpy(a).cuda())
    pb = M.features(torch.from_numpy(b).cuda())
    for dir, (X, Y) in enumerate(((pa, pb), (pb, pa))):
        flow, cost = _noalloc_call(ffm, M, X, Y, dir, spec.h, spec.w)
        assert np.array_equal(flow.cpu().numpy(), want[dir]), dir
        assert np.array_equal(cost.cpu().numpy(), want[2 + dir]), dir
    M.release(pa)
    M.release(pb)
    M.close()


def test_noalloc_near_its_scratch_limit(ffm):
    """A 1600x880 pair (1.41 Mpx, L=5, T=6): its per-level flow and cost buffers take about 30 MB of the
    32 MiB array.  Each direction equals ff_match_pair, and nothing is allocated during the calls."""
    from paper_1805_03517_gb300 import synth

    M = ffm.Matcher(configs.KITTI, 0)
    a, b, _ = synth.make_pair("kitti", 7700, 1600, 880)
    pa = M.features(torch.from_numpy(a).cuda())
    pb = M.features(torch.from_numpy(b).cuda())
    for dir, (X, Y) in enumerate(((pa, pb), (pb, pa))):
        ref_flow, ref_cost = M.match_pair(X, Y, dir)
        flow, cost = _noalloc_call(ffm, M, X, Y, dir, 880, 1600)
        assert torch.equal(flow, ref_flow), dir
        assert torch.equal(cost, ref_cost), dir
    M.release(pa)
    M.release(pb)
    M.close()


def test_noalloc_rejects_pyramids_beyond_its_scratch(ffm):
    M = ffm.Matcher(configs.MatchParams(n_scales=2, iters=1), 0)
    img = torch.zeros((1200, 2000, 3), dtype=torch.uint8, device="cuda")  # 2.4 Mpx > the fixed scratch
    pa = M.features(img)
    flow = torch.zeros((1200, 2000, 2), dtype=torch.int16, device="cuda")
    with pytest.raises(ffm.FFError) as e:
        ffm.ff_match_pair_noalloc(M.ctx, pa.handle, pa.handle, 0, flow.data_ptr(), None)
    assert e.value.status == ffm.FF_ERR_ARG
    M.release(pa)
    M.close()


def test_noalloc_census_cost_equals_match_pair(ffm):
    """Under the Census cost (Sec. 3.1) the entry point matches on the pyramids' Census patterns as well."""
    prm = configs.MatchParams(n_scales=3, iters=2, eps=1, cost=1)
    M = ffm.Matcher(prm, 0)
    a, b = _pair(930, 90, 140, 4, -2)
    pa = M.features(torch.from_numpy(a).cuda())
    pb = M.features(torch.from_numpy(b).cuda())
    for dir, (X, Y) in enumerate(((pa, pb), (pb, pa))):
        ref_flow, ref_cost = M.match_pair(X, Y, dir)
        flow, cost = _noalloc_call(ffm, M, X, Y, dir, 90, 140)
        assert torch.equal(flow, ref_flow), dir
        assert torch.equal(cost, ref_cost), dir
    M.release(pa)
    M.release(pb)
    M.close()
