"""Hand-worked examples and the paper's printed parameters (tests/golden/*.json, each with its citation and
derivation) against the oracle and, under the gpu marker, against the CUDA path through the C-ABI."""
import json
import os

import numpy as np
import pytest

import oracle
from paper_1805_03517_gb300 import configs

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def image(spec):
    """uint8 [h][w][3] from a fixture's image description."""
    w, h = spec["w"], spec["h"]
    img = np.zeros((h, w, 3), np.uint8)
    if "cols" in spec:
        for c, ch in enumerate("RGB"):
            img[:, :, c] = np.asarray(spec["cols"][ch], np.uint8)[None, :]
    elif "rows" in spec:
        for c, ch in enumerate("RGB"):
            img[:, :, c] = np.asarray(spec["rows"][ch], np.uint8)[:, None]
    elif "pixels" in spec:
        for c, ch in enumerate("RGB"):
            img[:, :, c] = np.asarray(spec["pixels"][ch], np.uint8)
    elif "quadrants" in spec:
        q = spec["quadrants"]
        ys, xs = np.mgrid[0:h, 0:w]
        same = (xs >= q["x0"]) == (ys >= q["y0"])
        img[same] = q["same"]
        img[~same] = q["diff"]
    else:
        img[:] = spec.get("fill", [0, 0, 0])
    for x, y, rgb in spec.get("set", []):
        img[y, x] = rgb
    return img


def census_image(case):
    return image({"w": 9, "h": 9, "fill": [50, 50, 50], "set": case["set"]})


def wht_expected(px):
    want = np.zeros(48, np.int64)
    for k, v in px["nonzero"].items():
        want[int(k)] = v
    return want


def flows(rows):
    return np.asarray(rows, np.int16).reshape(len(rows), len(rows[0]), 2)


# ------------------------------------------------------------------------------------------------- oracle

def test_table3_parameters():
    g = load("table3_parameters.json")
    assert configs.TABLE3 == g["table3"]
    assert configs.KITTI.eps == g["table3"]["kitti"]["eps"]
    assert configs.SINTEL.eps == g["table3"]["sintel"]["eps"]
    for wl in ("kitti_1242x375", "sintel_1024x436"):
        assert configs.workload(wl).pairs[0].params.eps == g["table3"][wl.split("_")[0]]["eps"]


def test_census_patch_and_sparsification_block_sizes(orc):
    """The 7x7 Census patch and the 3x3 sparsification block of Sec. 3.1, as seen through the oracle."""
    g = load("table3_parameters.json")["sec_3_1"]
    r = g["census_patch"] // 2
    img = np.full((2 * r + 5, 2 * r + 5, 3), 50, np.uint8)
    c = r + 2
    reach = []
    for d in range(1, r + 2):
        im = img.copy()
        im[c, c + d, 0] = 10
        reach.append(int(orc.census(im)[c, c, 0]).bit_count())
    assert reach == [1] * r + [0]
    b = g["sparsification_block"]
    n = 2 * b
    zero = np.zeros((n, n, 2), np.int16)
    kept = orc.sparsify(zero, zero, 0, 1)
    assert kept.sum() == 4 and all(kept[y:y + b, x:x + b].sum() == 1 for y in (0, b) for x in (0, b))


def test_wht_hand_worked(orc):
    for case in load("wht_hand_worked.json")["cases"]:
        f = orc.wht(image(case["image"])).astype(np.int64)
        for px in case["pixels"]:
            assert np.array_equal(f[px["y"], px["x"]], wht_expected(px)), (case["name"], px)


def test_pyramid_hand_worked(orc):
    g = load("pyramid_hand_worked.json")
    pyr = orc.pyramid(image(g["image"]), 3)
    for lv in g["levels"]:
        got = pyr[lv["level"]]
        assert got.shape == (lv["h"], lv["w"], 3)
        for c, ch in enumerate("RGB"):
            assert got[:, :, c].tolist() == lv[ch], (lv["level"], ch)


def test_seed_quantisation_hand_worked(orc):
    for case in load("seed_quantisation_hand_worked.json")["cases"]:
        fa = np.zeros((1, 1, 48), np.int16)
        fa[0, 0, 0] = case["C"]
        flow, dist = orc.seed(fa, np.zeros_like(fa))
        assert flow.tolist() == [[[0, 0]]] and int(dist[0, 0]) == case["dist"] == case["d"] ** 2, case


def test_census_hand_worked(orc):
    for case in load("census_hand_worked.json")["cases"]:
        cen = orc.census(census_image(case))
        got = [int(v).bit_count() for v in cen[case["cy"], case["cx"]]]
        assert got == case["popcount"], case


def test_consistency_and_sparsify_hand_worked(orc):
    g = load("consistency_sparsify_hand_worked.json")
    for case in g["consistency"]:
        fwd, bwd = flows(case["fwd"]), flows(case["bwd"])
        for eps, mask in case["masks"].items():
            assert orc.consistency(fwd, bwd, int(eps)).tolist() == mask, (case["derivation"], eps)
    for case in g["sparsify"]:
        fwd, bwd = flows(case["fwd"]), flows(case["bwd"])
        for s, kept in case["kept"].items():
            assert orc.sparsify(fwd, bwd, case["eps"], int(s)).tolist() == kept, s


# ---------------------------------------------------------------------------------------------- CUDA path

@pytest.fixture(scope="module")
def gpu():
    torch = pytest.importorskip("torch")
    from paper_1805_03517_gb300 import build, ff

    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch, ff


@pytest.mark.gpu
def test_gpu_wht_hand_worked(gpu):
    torch, ff = gpu
    M = ff.Matcher(configs.MatchParams(n_scales=1, iters=1), 0)
    for case in load("wht_hand_worked.json")["cases"]:
        pyr = M.features(torch.from_numpy(image(case["image"])).cuda())
        f = M.level_features(pyr, 0)
        M.sync()
        f = f.cpu().numpy().astype(np.int64)
        for px in case["pixels"]:
            assert np.array_equal(f[px["y"], px["x"]], wht_expected(px)), (case["name"], px)
        M.release(pyr)
    M.close()


@pytest.mark.gpu
def test_gpu_census_hand_worked(gpu):
    torch, ff = gpu
    M = ff.Matcher(configs.MatchParams(n_scales=1, iters=1, cost=1), 0)
    for case in load("census_hand_worked.json")["cases"]:
        pyr = M.features(torch.from_numpy(census_image(case)).cuda())
        cen = M.level_census(pyr, 0)
        M.sync()
        got = [int(v).bit_count() for v in cen.cpu().numpy().view(np.uint64)[case["cy"], case["cx"]]]
        assert got == case["popcount"], case
        M.release(pyr)
    M.close()


@pytest.mark.gpu
def test_gpu_consistency_and_sparsify_hand_worked(gpu):
    torch, ff = gpu
    M = ff.Matcher(configs.MatchParams(n_scales=1, iters=1), 0)
    g = load("consistency_sparsify_hand_worked.json")
    for case in g["consistency"]:
        fwd, bwd = torch.from_numpy(flows(case["fwd"])).cuda(), torch.from_numpy(flows(case["bwd"])).cuda()
        for eps, mask in case["masks"].items():
            got = M.consistency(fwd, bwd, int(eps))
            M.sync()
            assert got.cpu().tolist() == mask, (case["derivation"], eps)
    for case in g["sparsify"]:
        fwd, bwd = torch.from_numpy(flows(case["fwd"])).cuda(), torch.from_numpy(flows(case["bwd"])).cuda()
        for s, kept in case["kept"].items():
            got = M.sparsify(fwd, bwd, case["eps"], int(s))
            M.sync()
            assert got.cpu().tolist() == kept, s
    M.close()
