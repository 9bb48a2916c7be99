"""Seeded synthetic frame pairs standing in for the KITTI 2015 and MPI Sintel data of FlowFields++.

FlowFields++ (arXiv 1805.03517, Sec. 4) is evaluated on KITTI 2015 and MPI Sintel, which are not available
here.  These generators make frame pairs with the same shapes, motion ranges and photometric effects:

* ``translating_rects`` -- multi-octave value noise; two rectangles moved by integer shifts over a static
  background; Gaussian noise on frame 2 (the 128x96 case, and the 640x480 / 320x240 pairs of the batched and
  served workloads);
* ``kitti_like`` -- a textured ground plane seen by a forward-moving pinhole camera (flow up to ~250 px at the
  bottom rows), a static far background above the horizon, four rigid textured boxes with independent
  sub-pixel motion; disoccluded ground gets fresh noise;
* ``sintel_like`` -- six layered textured sprites (rotation up to 10 deg, scale 0.9-1.1, translation up to
  300 px), a global brightness gain of 0.95-1.05 and Gaussian noise on frame 2.

Each returns ``(img1, img2, gt_flow)``: uint8 [h][w][3] frames and an int16 [h][w][2] ground-truth flow of
frame 1, rounded to integer pixels (used only to report end-point error as context).

This module holds only input generation: none of the matching arithmetic lives here, so both the CUDA path
and the oracle can consume its output.  Everything is driven by ``numpy.random.Generator(PCG64(seed))``.
"""
from __future__ import annotations

import numpy as np

__all__ = ["value_noise", "Texture", "translating_rects", "kitti_like", "sintel_like", "make_pair"]


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _smooth(t):
    return t * t * (3.0 - 2.0 * t)


def value_noise(rng, h, w, periods=(32, 16, 8, 4), weights=(1.0, 0.5, 0.25, 0.125)):
    """Multi-octave value noise, one independent field per RGB channel, stretched to 0..255 (uint8)."""
    out = np.empty((h, w, 3), np.uint8)
    ys = np.arange(h, dtype=np.float64)
    xs = np.arange(w, dtype=np.float64)
    for c in range(3):
        acc = np.zeros((h, w))
        for p, wt in zip(periods, weights):
            lat = rng.random((h // p + 2, w // p + 2))
            fy, fx = ys / p, xs / p
            iy, ix = np.floor(fy).astype(np.int64), np.floor(fx).astype(np.int64)
            ty, tx = _smooth(fy - iy)[:, None], _smooth(fx - ix)[None, :]
            a = lat[iy][:, ix]
            b = lat[iy][:, ix + 1]
            cc = lat[iy + 1][:, ix]
            d = lat[iy + 1][:, ix + 1]
            acc += wt * ((a * (1 - tx) + b * tx) * (1 - ty) + (cc * (1 - tx) + d * tx) * ty)
        lo, hi = acc.min(), acc.max()
        out[..., c] = np.clip(np.rint((acc - lo) / max(hi - lo, 1e-9) * 255.0), 0, 255).astype(np.uint8)
    return out


class Texture:
    """Procedural RGB value-noise texture that can be sampled at arbitrary real coordinates."""

    def __init__(self, rng, period=24.0, octaves=4, lo=20.0, hi=235.0):
        self.tab = rng.random((3, octaves, 256, 256)).astype(np.float32)
        self.period = float(period)
        self.octaves = octaves
        self.lo, self.hi = lo, hi

    def sample(self, X, Y):
        X = np.asarray(X, dtype=np.float32)
        Y = np.asarray(Y, dtype=np.float32)
        out = np.zeros(X.shape + (3,), np.float32)
        norm = sum(0.5 ** o for o in range(self.octaves))
        for o in range(self.octaves):
            p = np.float32(self.period / (2.0 ** o))
            u, v = X / p, Y / p
            iu, iv = np.floor(u), np.floor(v)
            tu, tv = _smooth(u - iu), _smooth(v - iv)
            iu = iu.astype(np.int64) & 255
            iv = iv.astype(np.int64) & 255
            iu1, iv1 = (iu + 1) & 255, (iv + 1) & 255
            i00, i01, i10, i11 = iv * 256 + iu, iv * 256 + iu1, iv1 * 256 + iu, iv1 * 256 + iu1
            for c in range(3):
                t = self.tab[c, o].ravel()
                val = (t[i00] * (1 - tu) + t[i01] * tu) * (1 - tv) + (t[i10] * (1 - tu) + t[i11] * tu) * tv
                out[..., c] += np.float32(0.5 ** o) * val
        out /= np.float32(norm)
        # value noise clusters around 0.5: stretch it for texture contrast
        out = np.clip((out - 0.5) * 2.2 + 0.5, 0.0, 1.0)
        return self.lo + (self.hi - self.lo) * out


def _to_u8(img):
    return np.clip(np.rint(img), 0, 255).astype(np.uint8)


def translating_rects(seed, w=128, h=96, n_rects=2, max_shift=12, noise_sigma=2.0):
    """Value-noise frame; frame 2 = frame 1 with ``n_rects`` rectangles moved by integer shifts + noise."""
    rng = _rng(seed)
    img1 = value_noise(rng, h, w)
    img2 = img1.copy()
    gt = np.zeros((h, w, 2), np.int16)
    for _ in range(n_rects):
        rw = int(rng.integers(max(2, w // 6), max(3, w // 3 + 1)))
        rh = int(rng.integers(max(2, h // 6), max(3, h // 3 + 1)))
        x0 = int(rng.integers(0, max(1, w - rw)))
        y0 = int(rng.integers(0, max(1, h - rh)))
        dx, dy = (int(v) for v in rng.integers(-max_shift, max_shift + 1, size=2))
        # destination window, clipped to the frame
        xa, xb = max(0, x0 + dx), min(w, x0 + rw + dx)
        ya, yb = max(0, y0 + dy), min(h, y0 + rh + dy)
        if xa < xb and ya < yb:
            img2[ya:yb, xa:xb] = img1[ya - dy:yb - dy, xa - dx:xb - dx]
        gt[y0:y0 + rh, x0:x0 + rw] = (dx, dy)
    noisy = img2.astype(np.float64) + rng.normal(0.0, noise_sigma, img2.shape)
    return img1, _to_u8(noisy), gt


def kitti_like(seed, w=1242, h=375, max_disp=250.0, n_objects=4, noise_sigma=1.0):
    """Driving-scene stand-in: ground plane under forward camera motion, static far background, 4 boxes."""
    rng = _rng(seed)
    f = 0.58 * w
    cx, cy = 0.5 * w + rng.uniform(-10, 10), 0.42 * h
    cam_h = 1.65
    ppm = 30.0  # texture pixels per metre on the ground
    ground = Texture(rng, period=24.0)
    sky = Texture(rng, period=40.0)
    # forward motion chosen so that the bottom row moves by about max_disp pixels
    yb = (h - 1) - cy
    z_bottom = f * cam_h / yb
    dz = z_bottom - f * cam_h / (yb + max_disp)
    lateral = rng.uniform(-0.15, 0.15)

    ys, xs = np.mgrid[0:h, 0:w].astype(np.float64)
    is_ground = ys > cy + 0.5

    def render_background(frame):
        out = np.empty((h, w, 3))
        out[~is_ground] = sky.sample(xs[~is_ground], ys[~is_ground])
        z = f * cam_h / np.maximum(ys[is_ground] - cy, 1e-3)
        x_w = (xs[is_ground] - cx) * z / f + (lateral if frame == 1 else 0.0)
        z_w = z + (dz if frame == 1 else 0.0)
        out[is_ground] = ground.sample(x_w * ppm, z_w * ppm)
        return out

    img1 = render_background(0)
    img2 = render_background(1)
    gt = np.zeros((h, w, 2), np.float64)
    # ground flow of frame 1: world point seen again by the moved camera
    z1 = f * cam_h / np.maximum(ys - cy, 1e-3)
    x1w = (xs - cx) * z1 / f
    z2 = z1 - dz
    ok = is_ground & (z2 > 0.5)
    x2 = cx + f * (x1w - lateral) / np.where(ok, z2, 1.0)
    y2 = cy + f * cam_h / np.where(ok, z2, 1.0)
    gt[..., 0] = np.where(ok, x2 - xs, 0.0)
    gt[..., 1] = np.where(ok, y2 - ys, 0.0)

    boxes = []
    for _ in range(n_objects):
        bw = rng.uniform(0.06, 0.16) * w
        bh = rng.uniform(0.12, 0.3) * h
        bx = rng.uniform(0.05 * w, 0.95 * w - bw)
        by = rng.uniform(cy - 0.4 * bh, min(h - bh, cy + 0.5 * bh))
        mx, my = rng.uniform(-40.0, 40.0), rng.uniform(-6.0, 6.0)
        boxes.append((bx, by, bw, bh, mx, my, Texture(rng, period=rng.uniform(10, 20))))
    covered1 = np.zeros((h, w), bool)
    for bx, by, bw, bh, mx, my, tex in boxes:
        in1 = (xs >= bx) & (xs < bx + bw) & (ys >= by) & (ys < by + bh)
        img1[in1] = tex.sample(xs[in1] - bx, ys[in1] - by)
        gt[in1] = (mx, my)
        covered1 |= in1
    # frame-2 ground that was hidden behind a box in frame 1 (disoccluded): fresh noise
    zc = f * cam_h / np.maximum(ys - cy, 1e-3)
    back_x = cx + f * ((xs - cx) * zc / f + lateral) / (zc + dz)
    back_y = cy + f * cam_h / (zc + dz)
    bxi = np.clip(np.rint(back_x), 0, w - 1).astype(np.int64)
    byi = np.clip(np.rint(back_y), 0, h - 1).astype(np.int64)
    disocc = is_ground & covered1[byi, bxi]
    fresh = rng.uniform(20, 235, size=(h, w, 3))
    img2[disocc] = fresh[disocc]
    for bx, by, bw, bh, mx, my, tex in boxes:
        in2 = (xs >= bx + mx) & (xs < bx + mx + bw) & (ys >= by + my) & (ys < by + my + bh)
        img2[in2] = tex.sample(xs[in2] - bx - mx, ys[in2] - by - my)
    img2 = img2 + rng.normal(0.0, noise_sigma, img2.shape)
    return _to_u8(img1), _to_u8(img2), np.rint(gt).astype(np.int16)


def sintel_like(seed, w=1024, h=436, n_sprites=6, noise_sigma=3.0):
    """Animation stand-in: 6 layered sprites (rotation <= 10 deg, scale 0.9-1.1, shift <= 300 px), gain, noise."""
    rng = _rng(seed)
    ys, xs = np.mgrid[0:h, 0:w].astype(np.float64)
    layers = []
    for k in range(n_sprites):
        if k == 0:  # backdrop covering the frame
            hw, hh = 0.8 * w, 0.8 * h
            c = np.array([0.5 * w, 0.5 * h])
            t = rng.uniform(-40, 40, size=2)
        else:
            hw, hh = rng.uniform(0.08, 0.25) * w, rng.uniform(0.1, 0.35) * h
            c = np.array([rng.uniform(0, w), rng.uniform(0, h)])
            ang = rng.uniform(0, 2 * np.pi)
            t = rng.uniform(0, 300) * np.array([np.cos(ang), np.sin(ang)])
        a1 = np.deg2rad(rng.uniform(-20, 20))
        da = np.deg2rad(rng.uniform(-10, 10))
        s1 = rng.uniform(0.9, 1.1)
        ds = rng.uniform(0.9, 1.1)
        ellipse = k > 0 and rng.random() < 0.5
        tex = Texture(rng, period=rng.uniform(12, 30))
        layers.append(dict(hw=hw, hh=hh, pose1=(c, a1, s1), pose2=(c + t, a1 + da, s1 * ds), ellipse=ellipse, tex=tex))

    def local(pose):
        c, a, s = pose
        dx, dy = xs - c[0], ys - c[1]
        ca, sa = np.cos(a), np.sin(a)
        return (ca * dx + sa * dy) / s, (-sa * dx + ca * dy) / s

    def inside(L, lx, ly):
        if L["ellipse"]:
            return (lx / L["hw"]) ** 2 + (ly / L["hh"]) ** 2 <= 1.0
        return (np.abs(lx) <= L["hw"]) & (np.abs(ly) <= L["hh"])

    def render(which):
        img = np.full((h, w, 3), 128.0)
        for L in layers:
            lx, ly = local(L[which])
            m = inside(L, lx, ly)
            img[m] = L["tex"].sample(lx[m], ly[m])
        return img

    img1 = render("pose1")
    img2 = render("pose2")
    gt = np.zeros((h, w, 2))
    for L in layers:  # topmost layer wins, as in the render
        lx, ly = local(L["pose1"])
        m = inside(L, lx, ly)
        c, a, s = L["pose2"]
        ca, sa = np.cos(a), np.sin(a)
        x2 = c[0] + s * (ca * lx - sa * ly)
        y2 = c[1] + s * (sa * lx + ca * ly)
        gt[..., 0] = np.where(m, x2 - xs, gt[..., 0])
        gt[..., 1] = np.where(m, y2 - ys, gt[..., 1])
    gain = rng.uniform(0.95, 1.05)
    img2 = img2 * gain + rng.normal(0.0, noise_sigma, img2.shape)
    return _to_u8(img1), _to_u8(img2), np.rint(gt).astype(np.int16)


_KINDS = {"rects": translating_rects, "kitti": kitti_like, "sintel": sintel_like}


def make_pair(kind: str, seed: int, w: int, h: int):
    """Dispatch by workload kind ('rects', 'kitti', 'sintel') at size w x h."""
    return _KINDS[kind](seed, w=w, h=h)
