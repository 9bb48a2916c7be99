"""ff_features_batch: the pyramids and descriptors of many frames of different sizes in one launch per kernel are
the oracle's (Sec. 3 and 3.1), level by level, with 5 and 8 levels (the last level of 8 takes the per-frame
pyramid launch), under the Census cost, and matching from them equals the oracle's whole stage."""
import numpy as np
import pytest

from paper_1805_03517_gb300 import configs
from tests import gpu_helpers as G
from tests import oracle_pins as P

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

SHAPES = [(1, 1), (23, 37), (96, 128), (41, 300), (130, 257), (3, 2), (96, 128)]


@pytest.fixture(scope="module")
def ffm():
    from paper_1805_03517_gb300 import build, ff

    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return ff


@pytest.mark.parametrize("L,cost", [(5, 0), (8, 0), (3, 1)])
def test_features_batch_equals_oracle_per_level(ffm, orc, L, cost):
    M = ffm.Matcher(configs.MatchParams(n_scales=L, iters=1, cost=cost), 0)
    imgs = [P.rand_img(1600 + 7 * i + h * w, h, w) for i, (h, w) in enumerate(SHAPES)]
    dev = [torch.from_numpy(x).cuda() for x in imgs]
    torch.cuda.synchronize()
    launches0 = M.stats()["kernel_launches"]
    pyrs = M.features_batch(dev)
    deep = sum(1 for (h, w) in SHAPES if L > 7)  # one launch per frame for a level past the fused six
    assert M.stats()["kernel_launches"] - launches0 == 2 + deep
    for i, (img, pyr) in enumerate(zip(imgs, pyrs)):
        for s, lv in enumerate(orc.pyramid(img, L)):
            got = M.level_features(pyr, s)
            M.sync()
            assert np.array_equal(got.cpu().numpy(), orc.wht(lv)), (i, s)
            if cost:
                cen = M.level_census(pyr, s)
                M.sync()
                assert np.array_equal(cen.cpu().numpy().astype(np.uint64), orc.census(lv)), (i, s)
    for p in pyrs:
        M.release(p)
    M.close()


def test_matching_from_batched_features_equals_oracle(ffm, orc):
    """Seed rows (written by the coarsest level's tiles) and descriptors of a batch: the whole stage from them."""
    prm = configs.MatchParams(n_scales=4, iters=2, eps=1)
    shapes = [(120, 200), (77, 93), (64, 80), (120, 200)]
    pairs = []
    for i, (h, w) in enumerate(shapes):
        a = P.smooth_texture(1700 + i, h, w)
        pairs.append((a, P.shifted(a, 3 - i, i - 1, 1710 + i)))
    M = ffm.Matcher(prm, 0)
    dev = [torch.from_numpy(x).cuda() for pr in pairs for x in pr]
    torch.cuda.synchronize()
    pyrs = M.features_batch(dev)
    outs = M.match_batch([(pyrs[2 * i], pyrs[2 * i + 1]) for i in range(len(pairs))])
    M.sync()
    want = G.oracle_bidir_many(pairs, prm)
    for i, o in enumerate(outs):
        G.assert_same(tuple(o[k].cpu().numpy() for k in ("flow_fwd", "flow_bwd", "cost_fwd", "cost_bwd", "mask")),
                      want[i])
    for p in pyrs:
        M.release(p)
    # a second batch reuses the released pyramids and the table buffer
    pyrs2 = M.features_batch(dev[:2])
    out2 = M.match_batch([(pyrs2[0], pyrs2[1])])[0]
    M.sync()
    G.assert_same(tuple(out2[k].cpu().numpy() for k in ("flow_fwd", "flow_bwd", "cost_fwd", "cost_bwd", "mask")),
                  want[0])
    for p in pyrs2:
        M.release(p)
    M.close()


def test_features_batch_rejects_and_takes_nothing(ffm):
    M = ffm.Matcher(configs.MatchParams(n_scales=3, iters=1), 0)
    good = torch.zeros((20, 30, 3), dtype=torch.uint8, device="cuda")
    frames = [(good.data_ptr(), 30, 20, 90), (good.data_ptr(), 30, 20, 10)]  # second pitch < 3w
    with pytest.raises(ffm.FFError) as e:
        ffm.ff_features_batch(M.ctx, frames)
    assert e.value.status == ffm.FF_ERR_ARG
    assert ffm.ff_features_batch(M.ctx, []) == []
    # the first frame's pyramid was given back: a batch of two of its size takes the pool's pyramid plus a new one
    pyrs = M.features_batch([good, good])
    assert len({p.handle.value for p in pyrs}) == 2
    for p in pyrs:
        M.release(p)
    M.close()
