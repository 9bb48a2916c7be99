"""ff_match_frames: the features and the matching of frame pairs in one call (Sec. 3 and 3.1), with the descriptors
of pyramid levels 0 and 1 written on a branch of the matching's graph beside the coarse levels' matching.  Its results equal the
oracle's and those of ff_features_batch followed by ff_match_batch, bit for bit, at every fork point, on repeated
calls (graph replays), at the full 1242x375 size in the package table's launch configuration, under profiling and
with two levels (where nothing runs beside the matching), and the pyramids it keeps are complete when it returns.
Argument errors launch nothing."""
import json
import os

import numpy as np
import pytest

from paper_1805_03517_gb300 import configs, synth
from tests import gpu_helpers as G
from tests import oracle_pins as P

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

KEYS = ("flow_fwd", "flow_bwd", "cost_fwd", "cost_bwd", "mask")


@pytest.fixture(scope="module")
def ffm():
    from paper_1805_03517_gb300 import build, ff

    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return ff


def small_pairs(shapes, seed):
    pairs = []
    for i, (h, w) in enumerate(shapes):
        a = P.smooth_texture(seed + i, h, w)
        pairs.append((a, P.shifted(a, 3 - i, i - 1, seed + 10 + i)))
    return pairs


def to_dev(pairs):
    dev = [(torch.from_numpy(np.ascontiguousarray(a)).cuda(), torch.from_numpy(np.ascontiguousarray(b)).cuda())
           for a, b in pairs]
    torch.cuda.synchronize()
    return dev


def host(outs, keys=KEYS):
    return [tuple(o[k].cpu().numpy() for k in keys) for o in outs]


def two_calls(M, dev, with_cost=True):
    """The same step as ff_features_batch followed by ff_match_batch."""
    fp = M.features_batch([x for pr in dev for x in pr])
    outs = M.match_batch(list(zip(fp[0::2], fp[1::2])), with_cost=with_cost)
    M.sync()
    for p in fp:
        M.release(p)
    return outs


@pytest.mark.parametrize("overlap", [0, 1, 2])
def test_mixed_sizes_equal_oracle_on_every_replay(ffm, overlap):
    prm = configs.MatchParams(n_scales=4, iters=3, eps=1)
    pairs = small_pairs([(120, 200), (77, 93), (64, 80), (33, 47)], 1900)
    want = G.oracle_bidir_many(pairs, prm)
    M = ffm.Matcher(prm, 0)
    ffm.ff_set_option(M.ctx, ffm.FF_OPT_OVERLAP, overlap)
    dev = to_dev(pairs)
    outs = None
    for rep in range(3):  # the first call builds the plan and its graphs, the others replay them
        if outs is not None:
            for o in outs:
                for v in o.values():
                    v.fill_(7)
        s0 = M.stats()
        outs = M.match_frames(dev, outs=outs)
        M.sync()
        s1 = M.stats()
        for i, got in enumerate(host(outs)):
            G.assert_same(got, want[i])
        assert s1["graph_replays"] - s0["graph_replays"] == 1
        assert s1["plans_built"] - s0["plans_built"] == (1 if rep == 0 else 0)
    M.close()


def test_launch_count_and_results_match_the_two_calls(ffm):
    """With the fine levels beside the matching the step takes one more launch (the descriptors in two), and
    without (FF_OPT_OVERLAP 0) the same launches as the two calls; the outputs are the two calls' in both."""
    prm = configs.MatchParams(n_scales=5, iters=2, eps=1)
    pairs = small_pairs([(150, 260), (96, 128)], 1950)
    dev = to_dev(pairs)
    R = ffm.Matcher(prm, 0)
    two_calls(R, dev)
    s0 = R.stats()
    ref = host(two_calls(R, dev))
    per_step = R.stats()["kernel_launches"] - s0["kernel_launches"]
    R.close()
    for overlap, extra in ((0, 0), (1, 1), (2, 1)):
        M = ffm.Matcher(prm, 0)
        ffm.ff_set_option(M.ctx, ffm.FF_OPT_OVERLAP, overlap)
        M.match_frames(dev)
        M.sync()
        s0 = M.stats()
        outs = M.match_frames(dev)
        M.sync()
        assert M.stats()["kernel_launches"] - s0["kernel_launches"] == per_step + extra, overlap
        for g, w in zip(host(outs), ref):
            G.assert_same(g, w)
        M.close()


def test_fork_point_changes_between_calls(ffm):
    prm = configs.MatchParams(n_scales=4, iters=2, eps=1)
    pairs = small_pairs([(90, 140)], 1970)
    dev = to_dev(pairs)
    M = ffm.Matcher(prm, 0)
    ref = host(two_calls(M, dev))
    outs = None
    for overlap in (2, 1, 0, 2, 1):
        ffm.ff_set_option(M.ctx, ffm.FF_OPT_OVERLAP, overlap)
        outs = M.match_frames(dev, outs=outs)
        M.sync()
        G.assert_same(host(outs)[0], ref[0])
    M.close()


def test_full_size_in_the_benchmark_configuration(ffm):
    """The 1242x375 pair with the package table's per-level configurations (cluster form at level 4, dataflow
    forms below): every output equals the two calls' at both fork points."""
    name = "kitti_1242x375"
    table = json.load(open(os.path.join(os.path.dirname(ffm.__file__), "tuned.json")))
    spec = configs.workload(name).pairs[0]
    a, b, _ = synth.make_pair(spec.kind, spec.seed, spec.w, spec.h)
    dev = to_dev([(a, b)])
    M = ffm.Matcher(spec.params, 0)
    for lvl, cfg in enumerate(table[name]):
        ffm.ff_set_tuning(M.ctx, lvl, tuple(cfg))
    ref = host(two_calls(M, dev))
    outs = None
    for overlap in (1, 2, 2):
        ffm.ff_set_option(M.ctx, ffm.FF_OPT_OVERLAP, overlap)
        outs = M.match_frames(dev, outs=outs)
        M.sync()
        G.assert_same(host(outs)[0], ref[0])
    M.close()


def test_profiling_and_two_levels_run_in_order(ffm):
    """Profiling brackets phases on one stream and two levels leave no coarse level to overlap: both take the
    sequential path, with the two calls' launches and results (the oracle's)."""
    for L, profile in ((2, False), (4, True)):
        prm = configs.MatchParams(n_scales=L, iters=2, eps=1)
        pairs = small_pairs([(64, 96)], 1980 + L)
        want = G.oracle_bidir_many(pairs, prm)
        dev = to_dev(pairs)
        M = ffm.Matcher(prm, 0)
        ffm.ff_profile_enable(M.ctx, profile)
        two_calls(M, dev)
        s0 = M.stats()
        two_calls(M, dev)
        per_step = M.stats()["kernel_launches"] - s0["kernel_launches"]
        s0 = M.stats()
        outs = M.match_frames(dev)
        M.sync()
        assert M.stats()["kernel_launches"] - s0["kernel_launches"] == per_step
        G.assert_same(host(outs)[0], want[0])
        M.close()


def test_kept_pyramids_are_complete_at_return(ffm, orc):
    """The pyramids kept by the call hold every level's descriptors once the context's stream reaches the end of
    the call (levels 0 and 1 come from the graph's branch); released, they are recycled by the next call."""
    prm = configs.MatchParams(n_scales=4, iters=1, eps=1)
    pairs = small_pairs([(100, 150), (60, 70)], 1990)
    dev = to_dev(pairs)
    M = ffm.Matcher(prm, 0)
    outs, pyrs = M.match_frames(dev, keep_pyramids=True)
    for (img_a, img_b), (pa, pb) in zip(pairs, pyrs):
        for img, pyr in ((img_a, pa), (img_b, pb)):
            for s, lv in enumerate(orc.pyramid(img, prm.n_scales)):
                got = M.level_features(pyr, s)
                M.sync()
                assert np.array_equal(got.cpu().numpy(), orc.wht(lv)), s
    handles = {p.handle.value for pr in pyrs for p in pr}
    for pa, pb in pyrs:
        M.release(pa)
        M.release(pb)
    _, pyrs2 = M.match_frames(dev, outs=outs, keep_pyramids=True)
    assert {p.handle.value for pr in pyrs2 for p in pr} == handles
    for pa, pb in pyrs2:
        M.release(pa)
        M.release(pb)
    M.close()


def test_argument_errors_launch_nothing(ffm):
    prm = configs.MatchParams(n_scales=3, iters=1, eps=1)
    M = ffm.Matcher(prm, 0)
    a = torch.zeros((20, 30, 3), dtype=torch.uint8, device="cuda")
    b = torch.zeros((21, 30, 3), dtype=torch.uint8, device="cuda")
    flow = torch.zeros((20, 30, 2), dtype=torch.int16, device="cuda")
    flow_b = torch.zeros((20, 30, 2), dtype=torch.int16, device="cuda")
    mask = torch.zeros((20, 30), dtype=torch.uint8, device="cuda")
    frames = [(a.data_ptr(), 30, 20, 90), (a.data_ptr(), 30, 20, 90), (b.data_ptr(), 30, 21, 90)]
    fp, bp, mp_ = flow.data_ptr(), flow_b.data_ptr(), mask.data_ptr()
    bad_jobs = [
        [ffm.FrameJob(0, 3, fp, bp, None, None, mp_, None)],   # frame index out of range
        [ffm.FrameJob(-1, 1, fp, bp, None, None, mp_, None)],  # negative index
        [ffm.FrameJob(0, 2, fp, bp, None, None, mp_, None)],   # frames differ in size
        [ffm.FrameJob(0, 1, fp, None, None, None, mp_, None)],  # NULL output
        [ffm.FrameJob(0, 1, fp + 2, bp, None, None, mp_, None)],  # misaligned output
    ]
    torch.cuda.synchronize()
    s0 = M.stats()
    for jobs in bad_jobs:
        with pytest.raises(ffm.FFError) as e:
            ffm.ff_match_frames(M.ctx, frames, jobs)
        assert e.value.status == ffm.FF_ERR_ARG
    with pytest.raises(ffm.FFError):
        ffm.ff_match_frames(M.ctx, frames, [])
    assert M.stats()["kernel_launches"] == s0["kernel_launches"]
    # nothing was taken: a valid call afterwards runs
    ffm.ff_match_frames(M.ctx, frames[:2], [ffm.FrameJob(0, 1, fp, bp, None, None, mp_, None)])
    M.sync()
    assert M.stats()["kernel_launches"] > s0["kernel_launches"]
    M.close()


def test_out_of_memory_keeps_no_pyramid(ffm):
    """An allocation failure while the matching is prepared returns FF_ERR_OOM; the call's pyramids go back to the
    pool (the next call gets the same ones) and the next call matches as before."""
    prm = configs.MatchParams(n_scales=4, iters=2, eps=1)
    dev = to_dev(small_pairs([(90, 140)], 2010))
    M = ffm.Matcher(prm, 0)
    outs, pyrs = M.match_frames(dev, keep_pyramids=True)
    M.sync()
    ref = host(outs)
    handles = {p.handle.value for pr in pyrs for p in pr}
    for pa, pb in pyrs:
        M.release(pa)
        M.release(pb)
    ffm.ff_set_option(M.ctx, ffm.FF_OPT_TEST_FAIL_ALLOCS, 1)
    with pytest.raises(ffm.FFError) as e:
        M.match_frames(dev, keep_pyramids=True)  # new outputs: a new plan, whose scratch allocation fails
    assert e.value.status == ffm.FF_ERR_OOM
    ffm.ff_set_option(M.ctx, ffm.FF_OPT_TEST_FAIL_ALLOCS, 0)
    outs2, pyrs2 = M.match_frames(dev, keep_pyramids=True)
    M.sync()
    assert {p.handle.value for pr in pyrs2 for p in pr} == handles
    G.assert_same(host(outs2)[0], ref[0])
    for pa, pb in pyrs2:
        M.release(pa)
        M.release(pb)
    M.close()
