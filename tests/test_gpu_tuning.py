"""Propagation launch configurations (tile shape, iterations fused per launch) never change the results.

Every configuration -- including odd tile shapes and halos wider than the level -- must give flows, costs and
masks bit-identical to the oracle; so must the configuration the autotuner picks.
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
    for tw, th, k, n, spec in chosen:
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
    for level, cfg in ((-1, (8, 8, 1, 256, 0)), (8, (8, 8, 1, 256, 0)), (0, (0, 8, 1, 256, 0)),
                       (0, (8, 8, 0, 256, 0)), (0, (1024, 1024, 1, 256, 0)), (0, (64, 64, 40, 256, 0)),
                       (0, (8, 8, 1, 100, 0)), (0, (8, 8, 1, 1024, 0)), (0, (8, 8, 1, 256, 2))):
        with pytest.raises(ffm.FFError) as e:
            ffm.ff_set_tuning(M.ctx, level, cfg)
        assert e.value.status == ffm.FF_ERR_ARG
    ffm.ff_set_tuning(M.ctx, 1, None)  # clearing an absent override is fine
    with pytest.raises(ffm.FFError):
        ffm.ff_get_tuning(M.ctx, 1)
    M.close()
