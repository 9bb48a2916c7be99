"""The largest frames the C-ABI accepts (8192 pixels wide or high), checked where the oracle cannot run the whole
stage: sampled features against the oracle's WHT of crops of its own pyramid, sampled costs against the SAD of
those oracle descriptors at the returned flows, and the full consistency mask against the oracle's check of the
returned flows.  A translated frame must also be recovered almost everywhere with cost 0."""
import numpy as np
import pytest

import oracle
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


def wht_at(o, lv, y, x):
    """Oracle WHT descriptor of pixel (x, y) of a level image, from a crop holding its whole 8x8 patch (crop
    edges that are not image edges lie outside the patch, so the edge repetition is the image's)."""
    h, w, _ = lv.shape
    y0, y1, x0, x1 = max(0, y - 4), min(h, y + 5), max(0, x - 4), min(w, x + 5)
    return o.wht(np.ascontiguousarray(lv[y0:y1, x0:x1]))[y - y0, x - x0].astype(np.int64)


def sample_points(rng, h, w, n):
    pts = [(0, 0), (0, w - 1), (h - 1, 0), (h - 1, w - 1), (h // 2, w // 2), (3, w - 4), (h - 4, 3)]
    pts += [(int(rng.integers(0, h)), int(rng.integers(0, w))) for _ in range(n)]
    return pts


@pytest.mark.parametrize("h,w", [(1200, 8192), (8192, 640)])
def test_maximum_frame_sizes(ffm, h, w):
    o = oracle.default()
    prm = configs.MatchParams(n_scales=5, iters=2, eps=1)
    dx, dy = 5, -3
    a = P.smooth_texture(h + w, h, w)
    b = P.shifted(a, dx, dy, h + w + 1)
    M = ffm.Matcher(prm, 0)
    pa, pb = M.features(torch.from_numpy(a).cuda()), M.features(torch.from_numpy(b).cuda())
    out = M.match_batch([(pa, pb)])[0]
    M.sync()
    rng = np.random.default_rng(h * w)
    # features of the finest and the coarsest level at sampled pixels
    pyr_a = o.pyramid(a, prm.n_scales)
    for s in (0, prm.n_scales - 1):
        got = M.level_features(pa, s)
        M.sync()
        got = got.cpu().numpy()
        lh, lw, _ = pyr_a[s].shape
        for (y, x) in sample_points(rng, lh, lw, 40):
            assert np.array_equal(got[y, x].astype(np.int64), wht_at(o, pyr_a[s], y, x)), (s, y, x)
        del got
    ff_, fb_ = out["flow_fwd"].cpu().numpy(), out["flow_bwd"].cpu().numpy()
    cf = out["cost_fwd"].cpu().numpy()
    # every flow lands in the frame; sampled costs are the SAD of the oracle's descriptors at the flow
    ys, xs = np.mgrid[0:h, 0:w]
    assert ((xs + ff_[..., 0] >= 0) & (xs + ff_[..., 0] < w) & (ys + ff_[..., 1] >= 0) & (ys + ff_[..., 1] < h)).all()
    for (y, x) in sample_points(rng, h, w, 60):
        qy, qx = y + int(ff_[y, x, 1]), x + int(ff_[y, x, 0])
        sad = int(np.abs(wht_at(o, a, y, x) - wht_at(o, b, qy, qx)).sum())
        assert int(cf[y, x]) == sad, (y, x)
    # the whole mask is the oracle's consistency check of the returned fields
    assert np.array_equal(out["mask"].cpu().numpy(), o.consistency(ff_, fb_, prm.eps))
    # the translation is recovered (exactly, cost 0) away from the refilled border
    inner = (slice(16, h - 16), slice(16, w - 16))
    hit = (ff_[inner][..., 0] == dx) & (ff_[inner][..., 1] == dy)
    assert hit.mean() > 0.95, hit.mean()
    assert (cf[inner][hit] == 0).all()
    M.release(pa)
    M.release(pb)
    M.close()
