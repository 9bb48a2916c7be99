"""Sub-scales and sub-sub-scales (Sec. 3.1, under the reading the oracle states: every level below the coarsest is
first matched on the grid of every 4th / 2nd pixel of the level, then on every pixel): the CUDA path through the
C-ABI against the oracle, bit for bit, on sizes that span several tiles with ragged tails, under both costs, in a
batch of mixed sizes, at the full 1242x375 size, and with the second consistency check."""
import dataclasses

import numpy as np
import pytest

from paper_1805_03517_gb300 import configs, synth
from tests import gpu_helpers as G
from tests import oracle_pins as P

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

NAMES = ("flow_fwd", "flow_bwd", "cost_fwd", "cost_bwd", "mask")


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


@pytest.mark.parametrize("sub_scales", [1, 2])
@pytest.mark.parametrize("cost", [0, 1])
@pytest.mark.parametrize("shape", [(97, 131), (61, 45), (150, 230)])
def test_sub_scales_against_the_oracle(ffm, orc, sub_scales, cost, shape):
    h, w = shape
    prm = configs.MatchParams(n_scales=3, iters=3, eps=1, cost=cost, sub_scales=sub_scales)
    a, b = _pair(1100 + h + sub_scales, h, w, 5, -3)
    M = ffm.Matcher(prm, 0)
    got = G.gpu_bidir(M, a, b, torch)
    M.close()
    G.assert_same(got, orc.match_bidir(a, b, G.oracle_params(prm)))


def test_sub_scales_batch_of_mixed_sizes_equals_alone_and_oracle(ffm, orc):
    prm = configs.MatchParams(n_scales=4, iters=2, eps=1, sub_scales=2)
    shapes = [(120, 200), (77, 93), (120, 200), (40, 56), (97, 131)]
    pairs = [_pair(1200 + i, h, w, (i % 5) - 2, (i % 3) - 1) for i, (h, w) in enumerate(shapes)]
    M = ffm.Matcher(prm, 0)
    dev = [(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()) for a, b in pairs]
    torch.cuda.synchronize()
    pyrs = [(M.features(a), M.features(b)) for a, b in dev]
    outs = M.match_batch(pyrs)
    outs = M.match_batch(pyrs, outs=outs)  # replayed from the captured graph
    M.sync()
    got = [tuple(o[k].cpu().numpy() for k in NAMES) for o in outs]
    for i, pp in enumerate(pyrs):
        alone = M.match_batch([pp])[0]
        M.sync()
        G.assert_same(got[i], tuple(alone[k].cpu().numpy() for k in NAMES))
    want = G.oracle_bidir_many(pairs, prm)
    for i in range(len(pairs)):
        G.assert_same(got[i], want[i])
    for pa, pb in pyrs:
        M.release(pa)
        M.release(pb)
    M.close()


def test_sub_scales_full_size_kitti(ffm, orc):
    """The 1242x375 KITTI-shaped pair (L=5, T=6) with sub-scales and sub-sub-scales, in the benchmark's launch
    configuration for the levels (the package table); grids take the default configuration for their size."""
    import json
    import os

    spec = configs.workload("kitti_1242x375").pairs[0]
    prm = dataclasses.replace(spec.params, sub_scales=2)
    a, b, _ = synth.make_pair(spec.kind, spec.seed, spec.w, spec.h)
    M = ffm.Matcher(prm, 0)
    with open(os.path.join(os.path.dirname(configs.__file__), "tuned.json")) as f:
        for lvl, cfg in enumerate(json.load(f)["kitti_1242x375"]):
            ffm.ff_set_tuning(M.ctx, lvl, cfg)
    got = G.gpu_bidir(M, a, b, torch)
    M.close()
    G.assert_same(got, orc.match_bidir(a, b, G.oracle_params(prm)))


def test_sub_scales_second_consistency_check(ffm, orc):
    prm = configs.MatchParams(n_scales=3, iters=2, eps=1, sub_scales=1, rs_radius2=4)
    a, b = _pair(1300, 90, 120, 3, 2)
    M = ffm.Matcher(prm, 0)
    ta, tb = torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()
    torch.cuda.synchronize()
    pa, pb = M.features(ta), M.features(tb)
    out = M.match_batch([(pa, pb)], second_check=True)[0]
    M.sync()
    ff_, fb_, fb2_, mask_ = orc.match_bidir2(a, b, G.oracle_params(prm), prm.rs_radius2)
    assert np.array_equal(out["flow_fwd"].cpu().numpy(), ff_)
    assert np.array_equal(out["flow_bwd"].cpu().numpy(), fb_)
    assert np.array_equal(out["flow_bwd2"].cpu().numpy(), fb2_)
    assert np.array_equal(out["mask"].cpu().numpy(), mask_)
    M.release(pa)
    M.release(pb)
    M.close()


def test_sub_scales_work_counts_and_rejections(ffm):
    prm = configs.MatchParams(n_scales=3, iters=2, sub_scales=2)
    M = ffm.Matcher(prm, 0)
    pix_iters, pixels = ffm.ff_work_counts(M.ctx, 101, 57)
    # level 0: 101x57 + grids 51x29 and 26x15; level 1: 50x28 + 25x14 + 13x7; level 2 (coarsest): 25x14
    want = 2 * (101 * 57 + 51 * 29 + 26 * 15 + 50 * 28 + 25 * 14 + 13 * 7 + 25 * 14)
    assert (pix_iters, pixels) == (want, 101 * 57)
    img = torch.zeros((40, 48, 3), dtype=torch.uint8, device="cuda")
    pa = M.features(img)
    flow = torch.zeros((40, 48, 2), dtype=torch.int16, device="cuda")
    with pytest.raises(ffm.FFError) as e:  # the entry point with the fixed scratch runs no sub-scale grids
        ffm.ff_match_pair_noalloc(M.ctx, pa.handle, pa.handle, 0, flow.data_ptr(), None)
    assert e.value.status == ffm.FF_ERR_ARG
    M.release(pa)
    M.close()
    bad = dataclasses.replace(prm, sub_scales=3)
    with pytest.raises(ffm.FFError) as e:
        ffm.Matcher(bad, 0)
    assert e.value.status == ffm.FF_ERR_ARG


def _outputs(M, h, w):
    with torch.cuda.stream(M.stream):
        return {"flow_fwd": torch.full((h, w, 2), -9, dtype=torch.int16, device="cuda"),
                "flow_bwd": torch.full((h, w, 2), -9, dtype=torch.int16, device="cuda"),
                "cost_fwd": torch.full((h, w), -9, dtype=torch.int32, device="cuda"),
                "cost_bwd": torch.full((h, w), -9, dtype=torch.int32, device="cuda"),
                "mask": torch.full((h, w), 9, dtype=torch.uint8, device="cuda")}


@pytest.mark.parametrize("max_active", [4, 12])
def test_sub_scales_served_mix_equals_alone_and_oracle(ffm, orc, max_active):
    """The server runs the grid passes too: a staggered mix of sizes (whole passes per tick with few requests in
    flight, one chunk per tick with many) equals matching each pair alone, and the oracle."""
    prm = configs.MatchParams(n_scales=3, iters=3, eps=1, sub_scales=2)
    sizes = [(60, 90), (97, 131), (33, 47), (60, 90), (80, 80), (97, 131), (45, 70), (60, 90), (33, 47), (80, 80)]
    pairs = [_pair(1800 + i, h, w, (i % 5) - 2, (i % 3) - 1) for i, (h, w) in enumerate(sizes)]
    M = ffm.Matcher(prm, 0)
    dev = [(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()) for a, b in pairs]
    torch.cuda.synchronize()
    S = ffm.Server(M, mem_budget_bytes=1 << 30, max_active=max_active)
    outs = {i: _outputs(M, h, w) for i, (h, w) in enumerate(sizes)}
    done, nxt = [], 0
    for step in range(2000):
        if nxt < len(dev) and step % 2 == 0:
            S.submit(nxt, dev[nxt][0], dev[nxt][1], outs[nxt])
            nxt += 1
        S.step()
        done += S.poll()
        if len(done) == len(dev):
            break
    while len(done) < len(dev):
        S.step()
        done += S.poll(wait=True)
    M.sync()
    got = [tuple(outs[i][k].cpu().numpy() for k in NAMES) for i in range(len(dev))]
    for i, (da, db) in enumerate(dev):
        pa, pb = M.features(da), M.features(db)
        alone = M.match_batch([(pa, pb)])[0]
        M.sync()
        G.assert_same(got[i], tuple(alone[k].cpu().numpy() for k in NAMES))
        M.release(pa)
        M.release(pb)
    want = G.oracle_bidir_many(pairs, prm)
    for i in range(len(dev)):
        G.assert_same(got[i], want[i])
    S.close()
    M.close()
