"""Propagation launch configurations (tile shape, iterations fused per launch, the cluster form) never change the
results.

Every configuration -- including odd tile shapes, halos wider than the level, and the cluster form with every
cluster size and partition shape -- must give flows, costs and masks bit-identical to the oracle; so must the
configuration the autotuner picks.
"""
import numpy as np
import pytest

import oracle
from paper_1805_03517_gb300 import configs
from tests import gpu_helpers as G
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


def mp(L, T, eps=1):
    return configs.MatchParams(n_scales=L, iters=T, eps=eps)


@pytest.mark.parametrize("cfg", [(64, 32, 1, 256, 0), (32, 16, 2, 256, 0), (16, 16, 3, 256, 1), (8, 8, 6, 256, 0),
                                 (7, 5, 4, 256, 1), (13, 9, 2, 128, 0), (3, 2, 1, 128, 1), (128, 8, 5, 512, 0),
                                 (16, 64, 1, 512, 1), (24, 24, 1, 512, 0), (16, 8, 3, 128, 1), (32, 32, 1, 256, 1)])
def test_every_configuration_is_bit_exact(ffm, cfg):
    prm = mp(3, 5)
    h, w = 70, 133
    a = P.smooth_texture(400, h, w)
    b = P.shifted(a, 5, -3, 401)
    b[10:30, 20:50] = P.smooth_texture(402, 20, 30)
    M = ffm.Matcher(prm, 0)
    for lvl in range(3):
        ffm.ff_set_tuning(M.ctx, lvl, cfg)
        assert ffm.ff_get_tuning(M.ctx, lvl) == cfg
    got = G.gpu_bidir(M, a, b, torch)
    G.assert_same(got, oracle.default().match_bidir(a, b, G.oracle_params(prm)))
    M.close()


def test_autotune_then_bit_exact(ffm):
    prm = mp(4, 3)
    M = ffm.Matcher(prm, 0)
    imgs = []
    for i, (h, w) in enumerate(((96, 160), (96, 160))):
        a = P.smooth_texture(500 + i, h, w)
        imgs.append((a, P.shifted(a, 6 - 3 * i, 2, 510 + i)))
    pyrs = [(M.features(torch.from_numpy(a).cuda()), M.features(torch.from_numpy(b).cuda())) for a, b in imgs]
    chosen = M.autotune(pyrs, reps=1)
    assert len(chosen) == 4
    for cfg in chosen:
        tw, th, k, n, spec = cfg[:5]
        if len(cfg) == 7:  # the dataflow form
            assert tw >= 4 and th >= 4 and k == 1 and n in (128, 256, 512) and spec == 0 and cfg[5] == 0
            assert cfg[6] in (1, 2)
        elif len(cfg) == 6:  # the cluster form
            assert tw == th == 0 and 1 <= cfg[5] <= 16 and n in (256, 512) and k >= 1 and spec == 0
        else:
            assert tw >= 1 and th >= 1 and 1 <= k <= 3 and n in (128, 256, 512) and spec in (0, 1)
    outs = M.match_batch(pyrs)
    M.sync()
    names = ("flow_fwd", "flow_bwd", "cost_fwd", "cost_bwd", "mask")
    o = oracle.default()
    for (a, b), out in zip(imgs, outs):
        G.assert_same(tuple(out[k].cpu().numpy() for k in names), o.match_bidir(a, b, G.oracle_params(prm)))
    for pa, pb in pyrs:
        M.release(pa)
        M.release(pb)
    M.close()


def test_set_tuning_rejects_bad_configurations(ffm):
    M = ffm.Matcher(mp(2, 1), 0)
    ffm.ff_set_tuning(M.ctx, 0, (8, 8, 1, 256, 0))  # valid
    assert ffm.ff_get_tuning(M.ctx, 0) == (8, 8, 1, 256, 0)
    for level, cfg in ((-1, (8, 8, 1, 256, 0)), (24, (8, 8, 1, 256, 0)), (0, (0, 8, 1, 256, 0)),
                       (0, (8, 8, 0, 256, 0)), (0, (1024, 1024, 1, 256, 0)), (0, (64, 64, 40, 256, 0)),
                       (0, (8, 8, 1, 100, 0)), (0, (8, 8, 1, 1024, 0)), (0, (8, 8, 1, 256, 2)),
                       (0, (0, 0, 3, 128, 0, 16)), (0, (0, 0, 3, 256, 0, 17)), (0, (8, 8, 3, 256, 0, 16)),
                       (0, (0, 0, 3, 256, 0, -1)), (0, (0, 0, 0, 256, 0, 8)), (0, (0, 0, 3, 256, 1, 8)),
                       (0, (16, 16, 2, 256, 0, 0, 1)), (0, (16, 16, 1, 256, 1, 0, 1)), (0, (3, 16, 1, 256, 0, 0, 1)),
                       (0, (16, 16, 1, 256, 0, 8, 1)), (0, (16, 16, 1, 256, 0, 0, 3))):
        with pytest.raises(ffm.FFError) as e:
            ffm.ff_set_tuning(M.ctx, level, cfg)
        assert e.value.status == ffm.FF_ERR_ARG
    ffm.ff_set_tuning(M.ctx, 1, None)  # clearing an absent override is fine
    with pytest.raises(ffm.FFError):
        ffm.ff_get_tuning(M.ctx, 1)
    M.close()


def _pair_70x133():
    h, w = 70, 133
    a = P.smooth_texture(400, h, w)
    b = P.shifted(a, 5, -3, 401)
    b[10:30, 20:50] = P.smooth_texture(402, 20, 30)
    return a, b


@pytest.mark.parametrize("cfg", [(0, 0, 255, 256, 0, 16), (0, 0, 2, 512, 0, 8), (0, 0, 5, 256, 0, 4),
                                 (0, 0, 3, 512, 0, 6), (0, 0, 1, 256, 0, 1), (0, 0, 4, 512, 0, 16),
                                 (0, 0, 5, 256, 0, 12), (0, 0, 2, 256, 0, 2)])
def test_cluster_form_is_bit_exact(ffm, cfg):
    """The cluster form (one cluster of n CTAs per direction, blocks exchanging their edges through distributed
    shared memory, a cluster barrier between half-sweeps) on every level of a 70x133 pair, against the oracle;
    every propagation launch of the plan is of the cluster form."""
    prm = mp(3, 5)
    a, b = _pair_70x133()
    M = ffm.Matcher(prm, 0)
    for lvl in range(3):
        ffm.ff_set_tuning(M.ctx, lvl, cfg)
        assert ffm.ff_get_tuning(M.ctx, lvl) == cfg
    c0 = M.stats()["cluster_launches"]
    got = G.gpu_bidir(M, a, b, torch)
    per_level = -(-prm.iters // min(cfg[2], prm.iters))
    assert M.stats()["cluster_launches"] - c0 == 3 * per_level
    G.assert_same(got, oracle.default().match_bidir(a, b, G.oracle_params(prm)))
    M.close()


def test_cluster_form_falls_back_where_a_level_has_no_partition(ffm):
    """A 12x20 frame with 3 levels: 16 CTAs partition the 10x6 level (4 x 4 blocks) and the 20x12 one, not the 5x3
    level, which takes the tile form; the results are the oracle's either way."""
    prm = mp(3, 4)
    a = P.smooth_texture(430, 12, 20)
    b = P.shifted(a, 1, -1, 431)
    M = ffm.Matcher(prm, 0)
    for lvl in range(3):
        ffm.ff_set_tuning(M.ctx, lvl, (0, 0, 2, 256, 0, 16))
    c0 = M.stats()["cluster_launches"]
    got = G.gpu_bidir(M, a, b, torch)
    assert M.stats()["cluster_launches"] - c0 == 2 * 2  # two levels, two launches each
    G.assert_same(got, oracle.default().match_bidir(a, b, G.oracle_params(prm)))
    M.close()


@pytest.mark.parametrize("cost", [0, 1])
def test_cluster_form_on_sub_scale_grids(ffm, cost):
    """The grid instantiation of the cluster form: every level and every sub-scale / sub-sub-scale grid pass
    (pass index s + 8k) in the cluster form, under both costs, against the oracle."""
    prm = configs.MatchParams(n_scales=3, iters=3, eps=1, cost=cost, sub_scales=2)
    a, b = _pair_70x133()
    M = ffm.Matcher(prm, 0)
    passes = [0, 1, 2, 8, 9, 16, 17]  # the coarsest level has no grids
    for i, p in enumerate(passes):
        ffm.ff_set_tuning(M.ctx, p, (0, 0, 3 - i % 2, (256, 512)[i % 2], 0, (16, 8, 4)[i % 3]))
    c0 = M.stats()["cluster_launches"]
    got = G.gpu_bidir(M, a, b, torch)
    want_launches = sum(-(-3 // (3 - i % 2)) for i in range(len(passes)))
    assert M.stats()["cluster_launches"] - c0 == want_launches
    G.assert_same(got, oracle.default().match_bidir(a, b, G.oracle_params(prm)))
    M.close()


def test_cluster_form_in_a_batch_of_mixed_sizes(ffm):
    """Clusters of different problems in one launch (pairs of three sizes, both directions): each pair equals the
    oracle."""
    prm = mp(3, 4)
    shapes = [(70, 133), (41, 57), (96, 96)]
    pairs = []
    for i, (h, w) in enumerate(shapes):
        a = P.smooth_texture(440 + i, h, w)
        pairs.append((a, P.shifted(a, 3 - i, i - 1, 450 + i)))
    M = ffm.Matcher(prm, 0)
    for lvl in range(3):
        ffm.ff_set_tuning(M.ctx, lvl, (0, 0, 255, 512, 0, 8))
    dev = [(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()) for a, b in pairs]
    torch.cuda.synchronize()
    pyrs = [(M.features(x), M.features(y)) for x, y in dev]
    c0 = M.stats()["cluster_launches"]
    outs = M.match_batch(pyrs)
    M.sync()
    assert M.stats()["cluster_launches"] - c0 == 3
    want = G.oracle_bidir_many(pairs, prm)
    names = ("flow_fwd", "flow_bwd", "cost_fwd", "cost_bwd", "mask")
    for i, o in enumerate(outs):
        G.assert_same(tuple(o[k].cpu().numpy() for k in names), want[i])
    for pa, pb in pyrs:
        M.release(pa)
        M.release(pb)
    M.close()


def test_cluster_form_bounded_wait_reports_expiry_and_context_recovers(ffm):
    """With the block edges withheld, every wait of the cluster form expires after its poll limit: ff_sync reports
    FF_ERR_TIMEOUT, nothing hangs, and the same context then matches bit-exactly again."""
    prm = mp(3, 2)
    a, b = _pair_70x133()
    M = ffm.Matcher(prm, 0)
    ffm.ff_set_option(M.ctx, ffm.FF_OPT_SEED_KERNEL, ffm.FF_SEED_MMA_SYNC)  # only the propagation waits
    for lvl in range(3):
        ffm.ff_set_tuning(M.ctx, lvl, (0, 0, 255, 256, 0, 8))
    ffm.ff_set_option(M.ctx, ffm.FF_OPT_WAIT_LIMIT, 2000)
    ffm.ff_set_option(M.ctx, ffm.FF_OPT_TEST_WITHHOLD_COPIES, 1)  # no CTA sends its edges
    ta, tb = torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()
    torch.cuda.synchronize()
    pa, pb = M.features(ta), M.features(tb)
    M.match_batch([(pa, pb)])
    with pytest.raises(ffm.FFError) as e:
        M.sync()
    assert e.value.status == ffm.FF_ERR_TIMEOUT
    assert "cluster-form" in str(e.value)
    M.release(pa)
    M.release(pb)
    ffm.ff_set_option(M.ctx, ffm.FF_OPT_TEST_WITHHOLD_COPIES, 0)
    ffm.ff_set_option(M.ctx, ffm.FF_OPT_WAIT_LIMIT, 1 << 22)
    got = G.gpu_bidir(M, a, b, torch)
    G.assert_same(got, oracle.default().match_bidir(a, b, G.oracle_params(prm)))
    M.close()


@pytest.mark.parametrize("cfg,T", [((50, 32, 1, 256, 0, 0, 1), 5), ((16, 16, 1, 128, 0, 0, 1), 4),
                                   ((7, 5, 1, 512, 0, 0, 1), 3), ((64, 27, 1, 512, 0, 0, 1), 6),
                                   ((4, 4, 1, 256, 0, 0, 1), 2), ((33, 9, 1, 256, 0, 0, 1), 1),
                                   ((16, 8, 1, 512, 0, 0, 2), 6), ((4, 4, 1, 128, 0, 0, 2), 3),
                                   ((50, 32, 1, 256, 0, 0, 2), 4), ((13, 7, 1, 256, 0, 0, 2), 1)])
def test_dataflow_form_is_bit_exact(ffm, cfg, T):
    """The dataflow form (every iteration of a level in one persistent launch, a tile starting iteration t once the
    3x3 tiles around it have finished t - 1) on every level, with odd and even iteration counts (the buffer the
    last iteration writes depends on the parity), against the oracle; one launch per level."""
    prm = mp(3, T)
    a, b = _pair_70x133()
    M = ffm.Matcher(prm, 0)
    for lvl in range(3):
        ffm.ff_set_tuning(M.ctx, lvl, cfg)
        assert ffm.ff_get_tuning(M.ctx, lvl) == cfg
    s0 = M.stats()
    got = G.gpu_bidir(M, a, b, torch)
    s1 = M.stats()
    assert s1["cluster_launches"] == s0["cluster_launches"]
    G.assert_same(got, oracle.default().match_bidir(a, b, G.oracle_params(prm)))
    M.close()


@pytest.mark.parametrize("cost", [0, 1])
def test_dataflow_form_on_sub_scale_grids_and_census(ffm, cost):
    prm = configs.MatchParams(n_scales=3, iters=4, eps=1, cost=cost, sub_scales=2)
    a, b = _pair_70x133()
    M = ffm.Matcher(prm, 0)
    for i, p in enumerate([0, 1, 2, 8, 9, 16, 17]):
        ffm.ff_set_tuning(M.ctx, p, ((16, 8), (8, 8), (32, 16))[i % 3] + (1, (128, 256, 512)[i % 3], 0, 0, 1 + i % 2))
    got = G.gpu_bidir(M, a, b, torch)
    G.assert_same(got, oracle.default().match_bidir(a, b, G.oracle_params(prm)))
    M.close()


def test_dataflow_form_in_a_batch_of_mixed_sizes_and_replayed(ffm):
    """Problems of three sizes share each dataflow launch; the captured graph is replayed (the progress counters
    start from zero on every run)."""
    prm = mp(3, 4)
    shapes = [(70, 133), (41, 57), (96, 96)]
    pairs = []
    for i, (h, w) in enumerate(shapes):
        a = P.smooth_texture(460 + i, h, w)
        pairs.append((a, P.shifted(a, 3 - i, i - 1, 470 + i)))
    M = ffm.Matcher(prm, 0)
    for lvl in range(3):  # level 1 in the affine variant
        ffm.ff_set_tuning(M.ctx, lvl, (16, 16, 1, 256, 0, 0, 2 if lvl == 1 else 1))
    dev = [(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()) for a, b in pairs]
    torch.cuda.synchronize()
    pyrs = [(M.features(x), M.features(y)) for x, y in dev]
    outs = M.match_batch(pyrs)
    outs = M.match_batch(pyrs, outs=outs)  # graph replay
    M.sync()
    want = G.oracle_bidir_many(pairs, prm)
    names = ("flow_fwd", "flow_bwd", "cost_fwd", "cost_bwd", "mask")
    for i, o in enumerate(outs):
        G.assert_same(tuple(o[k].cpu().numpy() for k in names), want[i])
    for pa, pb in pyrs:
        M.release(pa)
        M.release(pb)
    M.close()


@pytest.mark.parametrize("variant", [1, 2])
def test_dataflow_form_bounded_wait_reports_expiry_and_context_recovers(ffm, variant):
    """With the tiles' progress withheld, every wait of the dataflow form expires after its poll limit: ff_sync
    reports FF_ERR_TIMEOUT, nothing hangs, and the same context then matches bit-exactly again."""
    prm = mp(3, 3)
    a, b = _pair_70x133()
    M = ffm.Matcher(prm, 0)
    ffm.ff_set_option(M.ctx, ffm.FF_OPT_SEED_KERNEL, ffm.FF_SEED_MMA_SYNC)  # only the propagation waits
    for lvl in range(3):
        ffm.ff_set_tuning(M.ctx, lvl, (16, 16, 1, 256, 0, 0, variant))
    ffm.ff_set_option(M.ctx, ffm.FF_OPT_WAIT_LIMIT, 2000)
    ffm.ff_set_option(M.ctx, ffm.FF_OPT_TEST_WITHHOLD_COPIES, 1)  # no tile publishes its progress
    ta, tb = torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()
    torch.cuda.synchronize()
    pa, pb = M.features(ta), M.features(tb)
    M.match_batch([(pa, pb)])
    with pytest.raises(ffm.FFError) as e:
        M.sync()
    assert e.value.status == ffm.FF_ERR_TIMEOUT
    assert "dataflow" in str(e.value)
    M.release(pa)
    M.release(pb)
    ffm.ff_set_option(M.ctx, ffm.FF_OPT_TEST_WITHHOLD_COPIES, 0)
    ffm.ff_set_option(M.ctx, ffm.FF_OPT_WAIT_LIMIT, 1 << 22)
    got = G.gpu_bidir(M, a, b, torch)
    G.assert_same(got, oracle.default().match_bidir(a, b, G.oracle_params(prm)))
    M.close()
