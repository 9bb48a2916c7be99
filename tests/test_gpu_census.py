"""The Census matching cost on the GPU (Sec. 3.1 names a Census cost next to SIFT; Sec. 4.1 takes Census for
Sintel): the 7x7 Census patterns of every pyramid level, and the whole bidirectional stage with the Hamming
cost -- seed on the WHT descriptors, hand-over, propagation and random search on Census patterns, consistency.

The cost is an integer (a popcount), so every flow, cost and mask must equal the oracle's bit for bit.  Cases
span several tiles and ragged tails, every propagation configuration family, batches of mixed sizes, the
two-check mode, the continuous-batching server and the full-size Sintel-shaped pair.
"""
import numpy as np
import pytest

import oracle
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
    yield ff
    for m in _matchers.values():
        m.close()
    _matchers.clear()


_matchers = {}


def cp(L, T, eps=1, R=2, seed=configs.HASH_SEED):
    return configs.MatchParams(n_scales=L, iters=T, rs_radius=R, eps=eps, seed=seed, cost=1)


def matcher(ff, prm):
    key = (prm.n_scales, prm.iters, prm.rs_radius, prm.eps, prm.seed, prm.cost)
    if key not in _matchers:
        _matchers[key] = ff.Matcher(prm, 0)
    return _matchers[key]


def check_pair(ff, a, b, prm):
    want = oracle.default().match_bidir(a, b, G.oracle_params(prm))
    got = G.gpu_bidir(matcher(ff, prm), a, b, torch)
    G.assert_same(got, want)
    return got


def test_census_patterns_every_level(ffm):
    o = oracle.default()
    M = matcher(ffm, cp(5, 1))
    for (h, w) in ((1, 1), (3, 2), (7, 9), (23, 37), (96, 128), (41, 300)):
        img = P.rand_img(h * 17 + w, h, w)
        pyr = M.features(torch.from_numpy(img).cuda())
        for s, lv in enumerate(o.pyramid(img, 5)):
            got = M.level_census(pyr, s)
            feat = M.level_features(pyr, s)
            M.sync()
            assert np.array_equal(got.cpu().numpy().view(np.uint64), o.census(lv)), (h, w, s)
            assert np.array_equal(feat.cpu().numpy(), o.wht(lv)), (h, w, s)  # the seed still needs them
        M.release(pyr)


def test_sad_context_has_no_census(ffm):
    M = ffm.Matcher(configs.MatchParams(n_scales=2, iters=1), 0)
    pyr = M.features(torch.zeros((8, 8, 3), dtype=torch.uint8, device="cuda"))
    assert M.level_census(pyr, 0) is None
    M.release(pyr)
    M.close()


def test_create_rejects_unknown_cost(ffm):
    p = ffm.ff_default_params()
    p.cost = 2
    with pytest.raises(ffm.FFError) as e:
        ffm.ff_create(p, 0)
    assert e.value.status == ffm.FF_ERR_ARG


def test_census_small_config(ffm):
    spec = configs.workload("small_128x96").pairs[0]
    a, b, _ = synth.make_pair(spec.kind, spec.seed, spec.w, spec.h)
    check_pair(ffm, a, b, cp(3, 4))


@pytest.mark.parametrize("h,w,L,T", [(1, 1, 1, 1), (1, 9, 2, 2), (9, 1, 2, 2), (5, 7, 1, 3), (23, 37, 3, 2),
                                     (64, 48, 4, 1), (33, 65, 2, 3), (70, 133, 3, 2), (17, 300, 2, 1)])
def test_census_tiny_and_ragged(ffm, h, w, L, T):
    a = P.smooth_texture(h * 11 + w, h, w)
    b = P.shifted(a, -2, 1, h + 3 * w)
    check_pair(ffm, a, b, cp(L, T))


def test_census_random_images_radius(ffm):
    check_pair(ffm, P.rand_img(3, 40, 52), P.rand_img(4, 40, 52), cp(3, 2, eps=2, R=3, seed=777))


def test_census_flat_images(ffm):
    """Flat frames: every Census pattern is zero, every candidate costs 0, nothing is strictly cheaper than
    the seed (which takes the first target pixel on WHT ties)."""
    a = np.full((30, 44, 3), 90, np.uint8)
    got = check_pair(ffm, a, a.copy(), cp(1, 2))
    ys, xs = np.mgrid[0:30, 0:44]
    assert np.array_equal(got[0][..., 0], -xs) and np.array_equal(got[0][..., 1], -ys)
    assert not got[2].any() and not got[3].any()


@pytest.mark.parametrize("cfg", [(64, 32, 1, 256, 0), (32, 16, 2, 256, 0), (16, 16, 3, 256, 1), (8, 8, 5, 256, 0),
                                 (7, 5, 4, 128, 1), (13, 9, 2, 512, 0), (16, 64, 1, 512, 1)])
def test_census_every_configuration_family(ffm, cfg):
    prm = cp(3, 5)
    a = P.smooth_texture(410, 70, 133)
    b = P.shifted(a, 4, -2, 411)
    b[10:30, 20:50] = P.smooth_texture(412, 20, 30)
    M = ffm.Matcher(prm, 0)
    for lvl in range(3):
        ffm.ff_set_tuning(M.ctx, lvl, cfg)
    got = G.gpu_bidir(M, a, b, torch)
    G.assert_same(got, oracle.default().match_bidir(a, b, G.oracle_params(prm)))
    M.close()


def test_census_batch_mixed_sizes(ffm):
    prm = cp(3, 2)
    M = matcher(ffm, prm)
    o = oracle.default()
    imgs = []
    for i, (h, w) in enumerate(((40, 60), (23, 37), (64, 64), (17, 90))):
        a = P.smooth_texture(150 + i, h, w)
        imgs.append((a, P.shifted(a, 2 - i, i - 1, 160 + i)))
    pyrs = [(M.features(torch.from_numpy(a).cuda()), M.features(torch.from_numpy(b).cuda())) for a, b in imgs]
    outs = M.match_batch(pyrs)
    M.sync()
    for (a, b), out in zip(imgs, outs):
        G.assert_same(tuple(out[k].cpu().numpy() for k in NAMES), o.match_bidir(a, b, G.oracle_params(prm)))
    for pa, pb in pyrs:
        M.release(pa)
        M.release(pb)


def test_census_two_consistency_checks(ffm):
    prm = cp(3, 3)
    h, w = 60, 90
    a = P.smooth_texture(920, h, w)
    b = P.shifted(a, -3, 2, 921)
    b[15:30, 30:45] = P.smooth_texture(922, 15, 15)
    M = matcher(ffm, prm)
    pa, pb = M.features(torch.from_numpy(a).cuda()), M.features(torch.from_numpy(b).cuda())
    out = M.match_batch([(pa, pb)], second_check=True)[0]
    M.sync()
    want = oracle.default().match_bidir2(a, b, G.oracle_params(prm), prm.rs_radius2)
    for k, wv in zip(("flow_fwd", "flow_bwd", "flow_bwd2", "mask"), want):
        assert np.array_equal(out[k].cpu().numpy(), wv), k
    M.release(pa)
    M.release(pb)


def test_census_served_equals_oracle(ffm):
    prm = cp(3, 2)
    M = ffm.Matcher(prm, 0)
    sizes = [(48, 64), (30, 50), (64, 96), (48, 64)]
    pairs = []
    for i, (h, w) in enumerate(sizes):
        a = P.smooth_texture(960 + i, h, w)
        pairs.append((a, P.shifted(a, i - 1, 2 - i, 970 + i)))
    dev = [(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()) for a, b in pairs]
    torch.cuda.synchronize()
    S = ffm.Server(M, mem_budget_bytes=1 << 30, max_active=3)
    outs = {}
    for i, (h, w) in enumerate(sizes):
        with torch.cuda.stream(M.stream):
            outs[i] = {"flow_fwd": torch.full((h, w, 2), -9, dtype=torch.int16, device="cuda"),
                       "flow_bwd": torch.full((h, w, 2), -9, dtype=torch.int16, device="cuda"),
                       "cost_fwd": torch.full((h, w), -9, dtype=torch.int32, device="cuda"),
                       "cost_bwd": torch.full((h, w), -9, dtype=torch.int32, device="cuda"),
                       "mask": torch.full((h, w), 9, dtype=torch.uint8, device="cuda")}
        S.submit(i, dev[i][0], dev[i][1], outs[i])
        S.step()
    done = []
    while len(done) < len(sizes):
        S.step()
        done += S.poll(wait=True)
    M.sync()
    o = oracle.default()
    for i, (a, b) in enumerate(pairs):
        G.assert_same(tuple(outs[i][k].cpu().numpy() for k in NAMES), o.match_bidir(a, b, G.oracle_params(prm)))
    S.close()
    M.close()


def test_census_full_size_sintel(ffm):
    """The Sintel-shaped 1024x436 pair with the Census cost (the paper's choice for Sintel), L=5, T=6, eps=7."""
    spec = configs.workload("sintel_1024x436").pairs[0]
    a, b, _ = synth.make_pair(spec.kind, spec.seed, spec.w, spec.h)
    check_pair(ffm, a, b, cp(5, 6, eps=7))
