"""ff_match_pair_noalloc, the entry point for callers that must not allocate device memory while they run.

It must give exactly what ff_match_pair gives (the matching is integer, so the tolerance is zero), on two
calls in a row: the second call reuses the fixed scratch array the first one left behind.  This file is
named so that pytest collects it last.
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


def test_noalloc_equals_match_pair_on_two_calls_in_a_row(ffm):
    prm = configs.MatchParams(n_scales=4, iters=3, eps=1)
    M = ffm.Matcher(prm, 0)
    pairs = [_pair(900, 150, 230, 7, -3), _pair(910, 150, 230, -5, 4)]  # same size: the second call reuses it all
    for call, (a, b) in enumerate(pairs):
        pa = M.features(torch.from_numpy(a).cuda())
        pb = M.features(torch.from_numpy(b).cuda())
        for dir, (X, Y) in enumerate(((pa, pb), (pb, pa))):
            ref_flow, ref_cost = M.match_pair(X, Y, dir)
            with torch.cuda.stream(M.stream):  # poison the outputs on the stream the library uses
                flow = torch.full((150, 230, 2), -7, dtype=torch.int16, device="cuda")
                cost = torch.full((150, 230), -7, dtype=torch.int32, device="cuda")
            ffm.ff_match_pair_noalloc(M.ctx, X.handle, Y.handle, dir, flow.data_ptr(), cost.data_ptr())
            M.sync()
            assert torch.equal(flow, ref_flow), (call, dir)
            assert torch.equal(cost, ref_cost), (call, dir)
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
        with torch.cuda.stream(M.stream):
            flow = torch.full((90, 140, 2), -7, dtype=torch.int16, device="cuda")
            cost = torch.full((90, 140), -7, dtype=torch.int32, device="cuda")
        ffm.ff_match_pair_noalloc(M.ctx, X.handle, Y.handle, dir, flow.data_ptr(), cost.data_ptr())
        M.sync()
        assert torch.equal(flow, ref_flow), dir
        assert torch.equal(cost, ref_cost), dir
    M.release(pa)
    M.release(pb)
    M.close()
