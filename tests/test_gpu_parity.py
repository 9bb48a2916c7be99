"""Parity of the CUDA path (through the C-ABI) with the CPU oracle: bit-exact flows, costs and masks.

All arithmetic is integer, so the bar is equality for every output.  Cases span several propagation tiles and
ragged tails, 1-pixel images, 1-level pyramids, seed ties (flat images), flows leaving the image, and the
full-size KITTI- and Sintel-shaped pairs in the launch configuration the benchmark times.
"""
import numpy as np
import pytest

import oracle
from paper_1805_03517_gb300 import configs, synth
from tests import gpu_helpers as G
from tests import oracle_pins as P

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib_built():
    from paper_1805_03517_gb300 import build

    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    yield
    for m in _matchers.values():
        m.close()
    _matchers.clear()


_matchers = {}


def matcher(params):
    from paper_1805_03517_gb300 import ff

    key = (params.n_scales, params.iters, params.rs_radius, params.eps, params.seed)
    if key not in _matchers:
        _matchers[key] = ff.Matcher(params, 0)
    return _matchers[key]


def mp(L, T, eps=1, R=2, seed=configs.HASH_SEED):
    return configs.MatchParams(n_scales=L, iters=T, rs_radius=R, eps=eps, seed=seed)


def check_pair(img_a, img_b, prm):
    o = oracle.default()
    want = o.match_bidir(img_a, img_b, G.oracle_params(prm))
    got = G.gpu_bidir(matcher(prm), img_a, img_b, torch)
    G.assert_same(got, want)
    return got


@pytest.mark.parametrize("L", [5, 7, 8])
def test_features_parity(lib_built, L):
    """Pyramid and WHT features of every level; L = 7 and 8 also take the per-level pyramid launches past the
    six levels the fused pyramid kernel derives from one block."""
    o = oracle.default()
    M = matcher(mp(L, 1))
    for (h, w) in ((1, 1), (3, 2), (23, 37), (96, 128), (41, 300), (130, 257)):
        img = P.rand_img(h * 131 + w, h, w)
        t = torch.from_numpy(img).cuda()
        pyr = M.features(t)
        levels = o.pyramid(img, L)
        for s, lv in enumerate(levels):
            got = M.level_features(pyr, s)
            M.sync()
            assert np.array_equal(got.cpu().numpy(), o.wht(lv)), (h, w, s)
        M.release(pyr)


def test_features_pitched_input(lib_built):
    """Rows of the input image may be padded (pitch > 3w)."""
    o = oracle.default()
    M = matcher(mp(3, 1))
    img = P.rand_img(5, 20, 30)
    big = torch.zeros((20, 40, 3), dtype=torch.uint8)
    big[:, :30] = torch.from_numpy(img)
    t = big.cuda()[:, :30]
    pyr = M.features(t)
    for s, lv in enumerate(o.pyramid(img, 3)):
        got = M.level_features(pyr, s)
        M.sync()
        assert np.array_equal(got.cpu().numpy(), o.wht(lv)), s
    M.release(pyr)


def test_small_config(lib_built):
    spec = configs.workload("small_128x96").pairs[0]
    a, b, _ = synth.make_pair(spec.kind, spec.seed, spec.w, spec.h)
    check_pair(a, b, spec.params)


@pytest.mark.parametrize("h,w,L,T", [(1, 1, 1, 1), (1, 9, 2, 2), (9, 1, 2, 2), (5, 7, 1, 3), (23, 37, 3, 2),
                                     (64, 48, 4, 1), (33, 65, 2, 3), (70, 133, 3, 2), (17, 300, 2, 1)])
def test_tiny_and_ragged(lib_built, h, w, L, T):
    a = P.smooth_texture(h * 7 + w, h, w)
    b = P.shifted(a, 2, -1, h + w)
    check_pair(a, b, mp(L, T))


def test_random_parameter_sweep(lib_built):
    """Seeded draws over sizes, scales, iterations, random-search radius (0 disables the random candidates),
    eps, hash seed and cost, on textured pairs with a random shift: every output bit-exact."""
    from paper_1805_03517_gb300 import ff

    rng = np.random.default_rng(2024)
    for k in range(12):
        h, w = int(rng.integers(1, 90)), int(rng.integers(1, 140))
        max_l = 1
        while max_l < 8 and (h >> max_l) >= 1 and (w >> max_l) >= 1:
            max_l += 1
        prm = configs.MatchParams(n_scales=int(rng.integers(1, max_l + 1)), iters=int(rng.integers(1, 5)),
                                  rs_radius=int(rng.integers(0, 17)), eps=int(rng.integers(0, 8)),
                                  seed=int(rng.integers(0, 2**32)), cost=int(rng.integers(0, 2)))
        a = P.smooth_texture(100 + k, h, w)
        b = P.shifted(a, int(rng.integers(-6, 7)), int(rng.integers(-6, 7)), 200 + k)
        M = ff.Matcher(prm, 0)
        got = G.gpu_bidir(M, a, b, torch)
        M.close()
        G.assert_same(got, oracle.default().match_bidir(a, b, G.oracle_params(prm)))
    # radius 0: the random candidate is always the current flow, so only the neighbours can move a match
    prm = configs.MatchParams(n_scales=3, iters=3, rs_radius=0, eps=1)
    a = P.smooth_texture(300, 45, 61)
    b = P.shifted(a, 4, -3, 301)
    M = ff.Matcher(prm, 0)
    got = G.gpu_bidir(M, a, b, torch)
    M.close()
    G.assert_same(got, oracle.default().match_bidir(a, b, G.oracle_params(prm)))


def test_random_images_radius(lib_built):
    a = P.rand_img(1, 40, 52)
    b = P.rand_img(2, 40, 52)
    check_pair(a, b, mp(3, 2, eps=2, R=3, seed=12345))


def test_flat_images_seed_ties(lib_built):
    """Every descriptor ties: the seed takes the first target pixel; no candidate is ever strictly cheaper."""
    a = np.full((30, 44, 3), 77, np.uint8)
    b = np.full((30, 44, 3), 77, np.uint8)
    got = check_pair(a, b, mp(1, 2))
    ys, xs = np.mgrid[0:30, 0:44]
    assert np.array_equal(got[0][..., 0], -xs) and np.array_equal(got[0][..., 1], -ys)


def test_partly_flat_with_large_motion(lib_built):
    a = P.smooth_texture(9, 90, 120)
    a[30:60, 40:80] = 128
    b = P.shifted(a, 37, 11, 10)
    check_pair(a, b, mp(4, 3, eps=1))


def test_match_pair_each_direction(lib_built):
    o = oracle.default()
    prm = mp(3, 2)
    a = P.smooth_texture(3, 50, 70)
    b = P.shifted(a, -4, 3, 4)
    M = matcher(prm)
    pa, pb = M.features(torch.from_numpy(a).cuda()), M.features(torch.from_numpy(b).cuda())
    fa = [o.wht(x) for x in o.pyramid(a, 3)]
    fb = [o.wht(x) for x in o.pyramid(b, 3)]
    for dir, (X, Y, src, dst) in enumerate(((pa, pb, fa, fb), (pb, pa, fb, fa))):
        flow, cost = M.match_pair(X, Y, dir)
        M.sync()
        wf, wc = o.match_dir(src, dst, G.oracle_params(prm), dir)
        assert np.array_equal(flow.cpu().numpy(), wf) and np.array_equal(cost.cpu().numpy(), wc), dir
    flow, _ = M.match_pair(pa, pb, 0, with_cost=False)
    M.sync()
    assert np.array_equal(flow.cpu().numpy(), o.match_dir(fa, fb, G.oracle_params(prm), 0)[0])
    M.release(pa)
    M.release(pb)


def test_consistency_parity(lib_built):
    o = oracle.default()
    M = matcher(mp(1, 1))
    rng = np.random.default_rng(0)
    for (h, w) in ((1, 1), (13, 17), (64, 96)):
        fwd = rng.integers(-5, 6, size=(h, w, 2)).astype(np.int16)
        bwd = rng.integers(-5, 6, size=(h, w, 2)).astype(np.int16)
        for eps in (0, 1, 3):
            got = M.consistency(torch.from_numpy(fwd).cuda(), torch.from_numpy(bwd).cuda(), eps)
            M.sync()
            assert np.array_equal(got.cpu().numpy(), o.consistency(fwd, bwd, eps)), (h, w, eps)


def test_batch_mixed_sizes_equals_alone_and_oracle(lib_built):
    prm = mp(3, 2)
    M = matcher(prm)
    o = oracle.default()
    sizes = [(40, 60), (23, 37), (64, 64), (17, 90)]
    imgs = []
    for i, (h, w) in enumerate(sizes):
        a = P.smooth_texture(50 + i, h, w)
        imgs.append((a, P.shifted(a, i - 2, 1 - i, 60 + i)))
    pyrs = [(M.features(torch.from_numpy(a).cuda()), M.features(torch.from_numpy(b).cuda())) for a, b in imgs]
    outs = M.match_batch(pyrs)
    M.sync()
    names = ("flow_fwd", "flow_bwd", "cost_fwd", "cost_bwd", "mask")
    for (a, b), out in zip(imgs, outs):
        G.assert_same(tuple(out[k].cpu().numpy() for k in names), o.match_bidir(a, b, G.oracle_params(prm)))
    # same jobs again: replayed from the captured graph, identical results
    s0 = M.stats()
    outs2 = M.match_batch(pyrs)
    M.sync()
    assert M.stats()["graph_replays"] == s0["graph_replays"] + 1
    for o1, o2 in zip(outs, outs2):
        for k in names:
            assert torch.equal(o1[k], o2[k])
    for pa, pb in pyrs:
        M.release(pa)
        M.release(pb)


def test_profiled_run_is_identical(lib_built):
    from paper_1805_03517_gb300 import ff

    prm = mp(3, 2)
    a = P.smooth_texture(70, 48, 64)
    b = P.shifted(a, 3, 2, 71)
    base = G.gpu_bidir(matcher(prm), a, b, torch)
    M = ff.Matcher(prm, 0)
    ff.ff_profile_enable(M.ctx, True)
    got = G.gpu_bidir(M, a, b, torch)
    prof = ff.ff_profile_read(M.ctx)
    G.assert_same(got, base)
    # one launch per level covers between 1 and all iterations (the configuration decides)
    assert prof["propagate"][0] > 0 and 3 <= prof["propagate"][1] <= 3 * 2
    assert prof["features"][1] > 0 and prof["seed"][1] >= 1 and prof["consistency"][1] == 1
    M.close()


@pytest.mark.parametrize("name", ["kitti_1242x375", "sintel_1024x436"])
def test_full_size_configs(lib_built, name):
    """Full-size pairs in the launch configuration of the benchmark: every output bit-exact."""
    spec = configs.workload(name).pairs[0]
    a, b, _ = synth.make_pair(spec.kind, spec.seed, spec.w, spec.h)
    check_pair(a, b, spec.params)


def test_full_size_in_the_benchmark_configuration(lib_built):
    """Every workload in the package table of tuned launch configurations (the per-level configurations the
    benchmark times), matched with exactly those configurations: every output bit-exact."""
    import json
    import os

    from paper_1805_03517_gb300 import ff

    table = json.load(open(os.path.join(os.path.dirname(ff.__file__), "tuned.json")))
    names = [k for k in table if k in configs.WORKLOADS]
    assert names
    for name in names:
        spec = configs.workload(name).pairs[0]
        a, b, _ = synth.make_pair(spec.kind, spec.seed, spec.w, spec.h)
        M = ff.Matcher(spec.params, 0)
        for lvl, cfg in enumerate(table[name]):
            ff.ff_set_tuning(M.ctx, lvl, tuple(cfg))
        assert [list(ff.ff_get_tuning(M.ctx, lvl)) for lvl in range(spec.params.n_scales)] == table[name]
        got = G.gpu_bidir(M, a, b, torch)
        G.assert_same(got, oracle.default().match_bidir(a, b, G.oracle_params(spec.params)))
        M.close()


def test_errors_are_reported(lib_built):
    from paper_1805_03517_gb300 import ff

    M = matcher(mp(3, 1))
    img = torch.zeros((10, 12, 3), dtype=torch.uint8, device="cuda")
    with pytest.raises(ff.FFError) as e:
        ff.ff_features(M.ctx, img.data_ptr(), 0, 10, 36)
    assert e.value.status == ff.FF_ERR_ARG
    with pytest.raises(ff.FFError):
        ff.ff_features(M.ctx, img.data_ptr(), 12, 10, 20)  # pitch < 3w
    with pytest.raises(ff.FFError):
        ff.ff_features(M.ctx, img.data_ptr(), 9000, 10, 27000)
    M1 = matcher(mp(1, 1))  # one level: the exhaustive seed would run over all 2048*1024 pixels
    with pytest.raises(ff.FFError) as e:
        ff.ff_features(M1.ctx, img.data_ptr(), 2048, 1024, 3 * 2048)
    assert e.value.status == ff.FF_ERR_ARG and "coarsest level" in ff.ff_last_error(M1.ctx)
    pa = M.features(img)
    pb = M.features(torch.zeros((10, 14, 3), dtype=torch.uint8, device="cuda"))
    flow = torch.zeros((10, 12, 2), dtype=torch.int16, device="cuda")
    with pytest.raises(ff.FFError):  # sizes differ
        ff.ff_match_pair(M.ctx, pa.handle, pb.handle, 0, flow.data_ptr(), None)
    with pytest.raises(ff.FFError):  # misaligned output
        ff.ff_match_pair(M.ctx, pa.handle, pa.handle, 0, flow.data_ptr() + 2, None)
    with pytest.raises(ff.FFError):
        ff.ff_match_pair(M.ctx, pa.handle, pa.handle, 2, flow.data_ptr(), None)
    M.release(pb)
    with pytest.raises(ff.FFError):  # released pyramid
        ff.ff_match_pair(M.ctx, pa.handle, pb.handle, 0, flow.data_ptr(), None)
    M.release(pa)
    M.sync()


def test_filter_argument_errors_launch_nothing(lib_built):
    """ff_consistency and ff_sparsify reject bad arguments with FF_ERR_ARG before launching anything."""
    from paper_1805_03517_gb300 import ff

    M = matcher(mp(3, 1))
    f = torch.zeros((6, 9, 2), dtype=torch.int16, device="cuda")
    out = torch.zeros((6, 9), dtype=torch.uint8, device="cuda")
    L = ff.lib()
    fp, op = f.data_ptr(), out.data_ptr()
    M.sync()
    s0 = M.stats()["kernel_launches"]
    bad_sparsify = [(fp, fp, None, 9, 6, 1, 0, op), (fp, fp, None, 9, 6, 1, 10, op), (fp, fp, None, 9, 6, -1, 7, op),
                    (fp, fp, None, 0, 6, 1, 7, op), (fp, fp, None, 9, 9000, 1, 7, op), (None, fp, None, 9, 6, 1, 7, op),
                    (fp + 2, fp, None, 9, 6, 1, 7, op), (fp, fp, None, 9, 6, 1, 7, None)]
    for args in bad_sparsify:
        assert L.ff_sparsify(M.ctx, *args) == ff.FF_ERR_ARG, args
    bad_consistency = [(fp, fp, 0, 6, 1, op), (fp, fp, 9, 6, -1, op), (None, fp, 9, 6, 1, op), (fp, fp + 2, 9, 6, 1, op),
                       (fp, fp, 9, 6, 1, None)]
    for args in bad_consistency:
        assert L.ff_consistency(M.ctx, *args) == ff.FF_ERR_ARG, args
    M.sync()
    assert M.stats()["kernel_launches"] == s0
    keep = torch.ones((6, 9), dtype=torch.uint8, device="cuda")
    assert L.ff_sparsify(M.ctx, fp, fp, keep.data_ptr(), 9, 6, 1, 7, op) == ff.FF_OK
    M.sync()
    assert M.stats()["kernel_launches"] == s0 + 1
    assert out.cpu().numpy().sum() == 3 * 2  # zero flows: every full 3x3 block keeps its first pixel


def test_empty_batch_launches_nothing(lib_built):
    from paper_1805_03517_gb300 import ff

    M = matcher(mp(3, 1))
    s0 = M.stats()
    assert M.match_batch([]) == []
    M.sync()
    assert M.stats()["kernel_launches"] == s0["kernel_launches"]
    assert ff.lib().ff_match_batch(M.ctx, -1, None) == ff.FF_ERR_ARG


def test_sparsify_parity(lib_built):
    """Sparsification (Sec. 3.1) of random flows (ragged edge blocks) and of real matches, against the oracle."""
    o = oracle.default()
    M = matcher(mp(1, 1))
    rng = np.random.default_rng(4)
    for (h, w) in ((1, 1), (7, 8), (31, 47), (96, 128)):
        fwd = rng.integers(-2, 3, size=(h, w, 2)).astype(np.int16)
        bwd = rng.integers(-2, 3, size=(h, w, 2)).astype(np.int16)
        keep = (rng.random((h, w)) < 0.7).astype(np.uint8)
        for eps, s in ((1, 1), (2, 4), (3, 7), (0, 9)):
            got = M.sparsify(torch.from_numpy(fwd).cuda(), torch.from_numpy(bwd).cuda(), eps, s)
            got_k = M.sparsify(torch.from_numpy(fwd).cuda(), torch.from_numpy(bwd).cuda(), eps, s,
                               keep=torch.from_numpy(keep).cuda())
            M.sync()
            assert np.array_equal(got.cpu().numpy(), o.sparsify(fwd, bwd, eps, s)), (h, w, eps, s)
            assert np.array_equal(got_k.cpu().numpy(), o.sparsify(fwd, bwd, eps, s, keep)), (h, w, eps, s)
    spec = configs.workload("small_128x96").pairs[0]
    a, b, _ = synth.make_pair(spec.kind, spec.seed, spec.w, spec.h)
    ff_, fb_, _, _, _ = check_pair(a, b, spec.params)
    for s in (4, 7):
        got = M.sparsify(torch.from_numpy(ff_).cuda(), torch.from_numpy(fb_).cuda(), 1, s)
        M.sync()
        assert np.array_equal(got.cpu().numpy(), o.sparsify(ff_, fb_, 1, s))


@pytest.mark.parametrize("h,w,L,T", [(48, 64, 3, 2), (96, 128, 3, 4), (70, 133, 2, 3)])
def test_two_consistency_checks(lib_built, h, w, L, T):
    """Two checks of Sec. 3.1: a second inverse field with its own radius and random stream; mask = both pass."""
    prm = mp(L, T)
    a = P.smooth_texture(900 + h, h, w)
    b = P.shifted(a, 3, -2, 901 + h)
    b[h // 4:h // 2, w // 3:w // 2] = P.smooth_texture(902, h // 2 - h // 4, w // 2 - w // 3)
    M = matcher(prm)
    pa, pb = M.features(torch.from_numpy(a).cuda()), M.features(torch.from_numpy(b).cuda())
    out = M.match_batch([(pa, pb)], second_check=True)[0]
    M.sync()
    o = oracle.default()
    want = o.match_bidir2(a, b, G.oracle_params(prm), prm.rs_radius2)
    for k, wv in zip(("flow_fwd", "flow_bwd", "flow_bwd2", "mask"), want):
        assert np.array_equal(out[k].cpu().numpy(), wv), k
    # the whole filter of Sec. 3.1: sparsification of what both checks left (s of Table 3)
    for s in (4, 7):
        got = M.sparsify(out["flow_fwd"], out["flow_bwd"], prm.eps, s, keep=out["mask"])
        M.sync()
        assert np.array_equal(got.cpu().numpy(), o.sparsify(want[0], want[1], prm.eps, s, want[3])), s
    M.release(pa)
    M.release(pb)
