"""Pins of the CPU oracle: checks against facts that do not come from the oracle itself.

Each ``check_*`` takes an ``oracle.Oracle`` and raises ``AssertionError`` on a violation.  They are used twice:
against the real oracle (tests/test_oracle_pins.py) and against copies of the oracle with a planted mistake
(tests/test_oracle_mutants.py), where at least one check must fail for every planted mistake.

What pins what (FlowFields++, arXiv 1805.03517, Sec. 3.1, under the readings in the design notes):
  * pyramid        -- hand-computed 2x2 box averages, odd sizes, 1-pixel levels;
  * WHT            -- closed forms for step edges and ramps, and the matrix product W P W^T with a
                      sequency-ordered Walsh matrix built from the Sylvester construction (not from the
                      oracle's sign table);
  * seed           -- brute-force argmin over all pixel pairs in NumPy (first index wins ties), on random
                      descriptors with negative values and planted duplicates;
  * SAD/cost       -- NumPy sum of absolute differences; out-of-level targets rejected;
  * propagation    -- invariants: cost never rises, cost == SAD(flow), flows stay in the level, only the
                      active colour changes, the result is no worse than every neighbour candidate, a changed
                      flow strictly lowers the cost;
  * random search  -- where every move comes from: at d = 0 only an upstream neighbour's flow, at d >= 1 a
                      neighbour's flow or a base plus this pixel's hashed offset in [-R, R]^2 (never (0, 0)),
                      and no untaken random candidate was strictly cheaper; a (-1, -2) shift that only the random
                      search can reach is recovered exactly, and nothing moves with R = 0; the same content at
                      two levels, or as forward vs inverse field, draws different offsets (level and direction
                      are in the key of the whole stage);
  * sub-scales     -- (reading: grids of every 2nd / 4th pixel of a level, matched before the level itself)
                      hand-overs against their definitions (twice the parent flow onto a grid; the parent grid
                      pixel's flow clamped into the level), grid propagation moves and costs at the strided level
                      pixels with the hash keyed by level coordinates and the grid's stream, exact recovery of
                      translations through sub-scales and sub-sub-scales;
  * cross-checks   -- a pure-Python restatement of the schedule on tiny inputs and the stage recomposed from its
                      steps (checks against the oracle's own loop, not pins: every planted mistake must also be
                      caught by a pin above, tests/test_oracle_mutants.py);
  * hash           -- a NumPy restatement of the published lowbias32 finaliser, and uniformity of offsets;
  * translation    -- exact recovery (cost 0, consistent) of known integer translations of a texture;
  * consistency    -- NumPy restatement, the f = -b case, and the eps boundary.
"""
from __future__ import annotations

import numpy as np

# ----------------------------------------------------------------------------------------------------------
# independent restatements


def sylvester_sequency_walsh(n=8):
    """Walsh matrix in sequency order: Sylvester Hadamard rows sorted by their number of sign changes."""
    H = np.array([[1]], dtype=np.int64)
    while H.shape[0] < n:
        H = np.block([[H, H], [H, -H]])
    changes = [(np.diff(np.sign(r)) != 0).sum() for r in H]
    return H[np.argsort(changes, kind="stable")]


def wht_numpy(img):
    W = sylvester_sequency_walsh(8)[:4]
    h, w, _ = img.shape
    pad = np.pad(img.astype(np.int64), ((3, 4), (3, 4), (0, 0)), mode="edge")
    win = np.lib.stride_tricks.sliding_window_view(pad, (8, 8), axis=(0, 1))  # [h][w][3][8][8]
    C = np.einsum("ui,yxcij,vj->yxcuv", W, win, W)
    return C.reshape(h, w, 48)


def quant_numpy(f):
    return np.floor_divide(f.astype(np.int64), 128)


def seed_numpy(fa, fb):
    h, w, _ = fa.shape
    A = quant_numpy(fa.reshape(-1, 48))
    B = quant_numpy(fb.reshape(-1, 48))
    D = ((A[:, None, :] - B[None, :, :]) ** 2).sum(-1)
    q = D.argmin(axis=1)  # first occurrence = smallest index on ties
    p = np.arange(h * w)
    flow = np.stack([q % w - p % w, q // w - p // w], -1).reshape(h, w, 2)
    return flow, D[p, q].reshape(h, w)


def sad_numpy(fa, fb, x, y, fx, fy):
    h, w, _ = fa.shape
    qx, qy = x + fx, y + fy
    if not (0 <= qx < w and 0 <= qy < h):
        return -1
    return int(np.abs(fa[y, x].astype(np.int64) - fb[qy, qx].astype(np.int64)).sum())


def sad_field(fa, fb, flow):
    h, w, _ = fa.shape
    out = np.empty((h, w), np.int64)
    for y in range(h):
        for x in range(w):
            out[y, x] = sad_numpy(fa, fb, x, y, int(flow[y, x, 0]), int(flow[y, x, 1]))
    return out


M32 = 0xFFFFFFFF


def lowbias32(x):
    """C. Wellons' published 32-bit finaliser (hash-prospector), restated with Python integers."""
    x &= M32
    x ^= x >> 16
    x = (x * 0x7FEB352D) & M32
    x ^= x >> 15
    x = (x * 0x846CA68B) & M32
    x ^= x >> 16
    return x


def hash_py(seed, dir, level, t, d, x, y, comp):
    k = lowbias32(seed ^ lowbias32(dir * 65536 + level * 256 + t))
    k = lowbias32(k ^ (y * 65536 + x))
    return lowbias32(k ^ (d * 2 + comp))


UPSTREAM = {0: ((-1, 0), (0, -1)), 1: ((1, 0), (0, -1)), 2: ((-1, 0), (0, 1)), 3: ((1, 0), (0, 1))}


def propagate_py(fa, fb, flow, cost, iters, R, seed, dir, level, max_halfsweeps=-1):
    """Pure-Python restatement of the per-level schedule (for tiny inputs)."""
    h, w, _ = fa.shape
    flow = flow.astype(np.int64).copy()
    cost = cost.astype(np.int64).copy()
    done = 0
    for t in range(iters):
        for d in range(4):
            for colour in (0, 1):
                if 0 <= max_halfsweeps <= done:
                    return flow, cost
                before = flow.copy()
                for y in range(h):
                    for x in range(w):
                        if (x + y) % 2 != colour:
                            continue
                        bx, by = int(flow[y, x, 0]), int(flow[y, x, 1])
                        bc = int(cost[y, x])
                        for ox, oy in UPSTREAM[d]:
                            nx, ny = x + ox, y + oy
                            if not (0 <= nx < w and 0 <= ny < h):
                                continue
                            cx, cy = int(before[ny, nx, 0]), int(before[ny, nx, 1])
                            c = sad_numpy(fa, fb, x, y, cx, cy)
                            if 0 <= c < bc:
                                bx, by, bc = cx, cy, c
                        if d >= 1:
                            rx = hash_py(seed, dir, level, t, d, x, y, 0) % (2 * R + 1) - R
                            ry = hash_py(seed, dir, level, t, d, x, y, 1) % (2 * R + 1) - R
                            if (rx, ry) != (0, 0):
                                c = sad_numpy(fa, fb, x, y, bx + rx, by + ry)
                                if 0 <= c < bc:
                                    bx, by, bc = bx + rx, by + ry, c
                        flow[y, x] = (bx, by)
                        cost[y, x] = bc
                done += 1
    return flow, cost


def consistency_numpy(fwd, bwd, eps):
    h, w, _ = fwd.shape
    ys, xs = np.mgrid[0:h, 0:w]
    qx = xs + fwd[..., 0].astype(np.int64)
    qy = ys + fwd[..., 1].astype(np.int64)
    inside = (qx >= 0) & (qx < w) & (qy >= 0) & (qy < h)
    qxc, qyc = np.clip(qx, 0, w - 1), np.clip(qy, 0, h - 1)
    ex = fwd[..., 0].astype(np.int64) + bwd[qyc, qxc, 0]
    ey = fwd[..., 1].astype(np.int64) + bwd[qyc, qxc, 1]
    return (inside & (ex * ex + ey * ey <= eps * eps)).astype(np.uint8)


# ----------------------------------------------------------------------------------------------------------
# inputs


def rand_img(seed, h, w):
    return np.random.default_rng(seed).integers(0, 256, size=(h, w, 3), dtype=np.uint8)


def smooth_texture(seed, h, w):
    """Band-limited random texture (distinctive patches, like natural images) for matching tests."""
    rng = np.random.default_rng(seed)
    acc = np.zeros((h, w, 3))
    for p, wt in ((8, 1.0), (4, 0.6), (2, 0.35)):
        lat = rng.random((h // p + 2, w // p + 2, 3))
        up = np.repeat(np.repeat(lat, p, 0), p, 1)[:h, :w]
        acc += wt * up
    acc += 0.25 * rng.random((h, w, 3))
    acc = (acc - acc.min()) / (acc.max() - acc.min())
    return np.rint(acc * 255).astype(np.uint8)


def shifted(img, dx, dy, seed):
    """Frame 2 = frame 1 moved by (dx, dy); the uncovered border gets fresh noise."""
    h, w, _ = img.shape
    out = np.random.default_rng(seed).integers(0, 256, size=img.shape, dtype=np.uint8)
    ys, yd = (slice(0, h - dy), slice(dy, h)) if dy >= 0 else (slice(-dy, h), slice(0, h + dy))
    xs, xd = (slice(0, w - dx), slice(dx, w)) if dx >= 0 else (slice(-dx, w), slice(0, w + dx))
    out[yd, xd] = img[ys, xs]
    return out


# ----------------------------------------------------------------------------------------------------------
# checks


def check_pyramid(o):
    # hand-computed: (1+2+3+5+2)//4 = 13//4 = 3, (4+4+4+4+2)//4 = 4, (0+0+0+1+2)//4 = 0, (255*4+2)//4 = 255
    img = np.zeros((2, 4, 3), np.uint8)
    img[..., 0] = [[1, 2, 4, 4], [3, 5, 4, 4]]
    img[..., 1] = [[0, 0, 255, 255], [0, 1, 255, 255]]
    img[..., 2] = [[1, 1, 0, 0], [1, 0, 0, 0]]  # (1+1+1+0+2)//4 = 1, 0
    out = o.downsample(img)
    assert out.shape == (1, 2, 3)
    assert out[0, :, 0].tolist() == [3, 4]
    assert out[0, :, 1].tolist() == [0, 255]
    assert out[0, :, 2].tolist() == [1, 0]
    # round half up: (1+1+0+0+2)//4 = 1 (a plain floor average would give 0)
    img2 = np.zeros((2, 2, 3), np.uint8)
    img2[0, 0] = 1
    img2[0, 1] = 1
    assert o.downsample(img2)[0, 0].tolist() == [1, 1, 1]
    # odd sizes floor, the last column/row is dropped
    big = rand_img(3, 7, 5)
    d = o.downsample(big)
    assert d.shape == (3, 2, 3)
    b = big.astype(int)
    ref = (b[0:6:2, 0:4:2] + b[0:6:2, 1:4:2] + b[1:6:2, 0:4:2] + b[1:6:2, 1:4:2] + 2) // 4
    assert np.array_equal(d, ref)
    # 1-pixel-wide level: clamp to the only column
    col = rand_img(4, 4, 1)
    d = o.downsample(col)
    assert d.shape == (2, 1, 3)
    c = col.astype(int)
    ref = (2 * c[0:4:2, 0] + 2 * c[1:4:2, 0] + 2) // 4
    assert np.array_equal(d[:, 0], ref)
    assert o.level_dims(1242, 375, 5) == [(1242, 375), (621, 187), (310, 93), (155, 46), (77, 23)]
    assert o.level_dims(3, 1, 3) == [(3, 1), (1, 1), (1, 1)]


def check_wht(o):
    # closed forms, patch fully inside: vertical step (left 4 columns a, right 4 columns b)
    a, b = 40, 200
    img = np.zeros((16, 16, 3), np.uint8)
    img[:, :8, :] = a
    img[:, 8:, :] = b
    img[..., 1] = 17  # flat channel
    f = o.wht(img).astype(np.int64).reshape(16, 16, 3, 4, 4)
    C = f[8, 7, 0]  # columns 4..11: 4 of a, 4 of b
    assert C[0, 0] == 32 * (a + b) and C[0, 1] == 32 * (a - b)
    assert C[0, 2] == 0 and C[0, 3] == 0 and np.all(C[1:] == 0)
    G = f[8, 7, 1]
    assert G[0, 0] == 64 * 17 and np.count_nonzero(G) == 1
    # horizontal ramp by rows: only the u (vertical) index may be non-zero
    ramp = np.zeros((16, 16, 3), np.uint8)
    ramp[..., 2] = (np.arange(16) * 9)[:, None]
    C = o.wht(ramp).astype(np.int64).reshape(16, 16, 3, 4, 4)[8, 8, 2]
    rows = np.arange(5, 13) * 9  # rows y-3 .. y+4
    W = sylvester_sequency_walsh(8)[:4]
    assert np.all(C[:, 1:] == 0)
    assert np.array_equal(C[:, 0], 8 * (W @ rows))
    # full definition, all pixels including clamped borders, odd sizes
    for s, (h, w) in enumerate(((9, 13), (1, 5), (6, 1), (17, 11))):
        im = rand_img(10 + s, h, w)
        assert np.array_equal(o.wht(im).astype(np.int64), wht_numpy(im)), (h, w)
    # extreme values fit int16 without wrap
    white = np.full((8, 8, 3), 255, np.uint8)
    assert o.wht(white)[4, 4, 0] == 64 * 255


def check_hash(o):
    for x in (0, 1, 0x7FEB352D, 0xFFFFFFFF, 123456789):
        assert o.mix32(x) == lowbias32(x)
    rng = np.random.default_rng(7)
    for _ in range(300):
        seed = int(rng.integers(0, 2**32))
        args = (seed, int(rng.integers(0, 2)), int(rng.integers(0, 8)), int(rng.integers(0, 12)),
                int(rng.integers(0, 4)), int(rng.integers(0, 8192)), int(rng.integers(0, 8192)),
                int(rng.integers(0, 2)))
        assert o.hash(*args) == hash_py(*args), args
    # offsets over a grid of pixels are close to uniform on the 5x5 window
    counts = np.zeros((5, 5), int)
    for y in range(40):
        for x in range(40):
            ox = o.hash(99, 0, 1, 2, 3, x, y, 0) % 5
            oy = o.hash(99, 0, 1, 2, 3, x, y, 1) % 5
            counts[oy, ox] += 1
    assert counts.min() > 64 * 0.5 and counts.max() < 64 * 1.6


def check_sad(o):
    fa = np.random.default_rng(1).integers(-16320, 16321, size=(5, 6, 48)).astype(np.int16)
    fb = np.random.default_rng(2).integers(-16320, 16321, size=(5, 6, 48)).astype(np.int16)
    for (x, y, fx, fy) in ((0, 0, 0, 0), (2, 3, 1, -2), (5, 4, 0, 0), (5, 4, -5, -4), (1, 1, 4, 3)):
        assert o.sad(fa, fb, x, y, fx, fy) == sad_numpy(fa, fb, x, y, fx, fy)
    for (x, y, fx, fy) in ((0, 0, -1, 0), (0, 0, 0, -1), (5, 4, 1, 0), (5, 4, 0, 1), (2, 2, 9, 0)):
        assert o.sad(fa, fb, x, y, fx, fy) == -1
    # maximum cost: 48 * 32640 fits int32
    hi = np.full((1, 1, 48), 16320, np.int16)
    assert o.sad(hi, -hi, 0, 0, 0, 0) == 48 * 32640


def check_seed(o):
    rng = np.random.default_rng(5)
    for (h, w) in ((1, 1), (3, 4), (7, 9), (12, 10)):
        fa = rng.integers(-16320, 16321, size=(h, w, 48)).astype(np.int16)
        fb = rng.integers(-16320, 16321, size=(h, w, 48)).astype(np.int16)
        if h * w >= 4:  # planted exact ties: two identical frame-B descriptors equal to one of frame A
            fb.reshape(-1, 48)[1] = fa.reshape(-1, 48)[2]
            fb.reshape(-1, 48)[3] = fa.reshape(-1, 48)[2]
        flow, dist = o.seed(fa, fb)
        rf, rd = seed_numpy(fa, fb)
        assert np.array_equal(flow, rf) and np.array_equal(dist, rd), (h, w)
        if h * w >= 4:
            p = 2
            assert flow.reshape(-1, 2)[p].tolist() == [1 % w - p % w, 1 // w - p // w]
            assert dist.reshape(-1)[p] == 0
    # descriptors of real images, negative coefficients not multiples of 128 (floor vs truncation)
    fa = o.wht(rand_img(8, 6, 7))
    fb = o.wht(rand_img(9, 6, 7))
    flow, dist = o.seed(fa, fb)
    rf, rd = seed_numpy(fa, fb)
    assert np.array_equal(flow, rf) and np.array_equal(dist, rd)


def check_upsample(o):
    rng = np.random.default_rng(11)
    for (h, w) in ((8, 10), (9, 11), (5, 3)):
        hc, wc = max(1, h // 2), max(1, w // 2)
        fa = o.wht(rand_img(12, h, w))
        fb = o.wht(rand_img(13, h, w))
        fc = np.zeros((hc, wc, 2), np.int16)
        for y in range(hc):
            for x in range(wc):
                fc[y, x] = (rng.integers(-x, wc - x), rng.integers(-y, hc - y))
        flow, cost = o.upsample(fa, fb, fc)
        for y in range(h):
            for x in range(w):
                px, py = min(x // 2, wc - 1), min(y // 2, hc - 1)
                assert flow[y, x].tolist() == (2 * fc[py, px]).tolist()
                assert cost[y, x] == sad_numpy(fa, fb, x, y, *flow[y, x].tolist())


def _tiny_level(seed, h, w):
    img_a = smooth_texture(seed, h, w)
    img_b = shifted(img_a, 2, -1, seed + 1)
    return img_a, img_b


def check_propagation_invariants(o):
    h, w = 11, 13
    ia, ib = _tiny_level(21, h, w)
    fa, fb = o.wht(ia), o.wht(ib)
    rng = np.random.default_rng(22)
    flow0 = np.zeros((h, w, 2), np.int16)
    for y in range(h):
        for x in range(w):
            flow0[y, x] = (rng.integers(-x, w - x), rng.integers(-y, h - y))
    cost0 = o.init_cost(fa, fb, flow0)
    assert np.array_equal(cost0, sad_field(fa, fb, flow0))
    iters, R, seed = 2, 2, 77
    states = [(flow0, cost0)]
    for k in range(1, iters * 8 + 1):
        states.append(o.propagate(fa, fb, flow0, cost0, iters, R, seed, 0, 1, max_halfsweeps=k))
    ys, xs = np.mgrid[0:h, 0:w]
    for k in range(1, len(states)):
        (f0, c0), (f1, c1) = states[k - 1], states[k]
        d, colour = ((k - 1) // 2) % 4, (k - 1) % 2
        assert np.all(c1 <= c0), k  # never worse
        assert np.array_equal(c1, sad_field(fa, fb, f1)), k  # cost is the SAD of the flow
        qx, qy = xs + f1[..., 0], ys + f1[..., 1]
        assert qx.min() >= 0 and qx.max() < w and qy.min() >= 0 and qy.max() < h, k
        changed = np.any(f1 != f0, axis=-1)
        assert not np.any(changed & ((xs + ys) % 2 != colour)), k  # only the active colour moves
        assert np.all(c1[changed] < c0[changed]), k  # a change strictly lowers the cost
        for y in range(h):
            for x in range(w):
                if (x + y) % 2 != colour:
                    continue
                for ox, oy in UPSTREAM[d]:  # no worse than any neighbour's flow
                    nx, ny = x + ox, y + oy
                    if 0 <= nx < w and 0 <= ny < h:
                        c = sad_numpy(fa, fb, x, y, *f0[ny, nx].tolist())
                        if c >= 0:
                            assert c1[y, x] <= c, (k, x, y)
    # the full schedule runs 8 half-sweeps per iteration
    full = o.propagate(fa, fb, flow0, cost0, iters, R, seed, 0, 1)
    assert np.array_equal(full[0], states[-1][0])
    # a constant target frame makes every in-level candidate tie: under strict acceptance nothing may move
    flat = o.wht(np.full((h, w, 3), 90, np.uint8))
    cflat = o.init_cost(fa, flat, flow0)
    f2, c2 = o.propagate(fa, flat, flow0, cflat, iters, R, seed, 0, 1)
    assert np.array_equal(f2, flow0) and np.array_equal(c2, cflat)


def check_propagation_schedule(o):
    """Cross-check against the pure-Python restatement of the schedule (tiny inputs, all steps)."""
    for (h, w, dir, level, seed) in ((7, 9, 0, 0, 5), (6, 5, 1, 2, 0xDEADBEEF)):
        ia, ib = _tiny_level(31 + h, h, w)
        fa, fb = o.wht(ia), o.wht(ib)
        flow0 = np.zeros((h, w, 2), np.int16)
        cost0 = o.init_cost(fa, fb, flow0)
        for k in (1, 3, 8, 16):
            f_o, c_o = o.propagate(fa, fb, flow0, cost0, 2, 2, seed, dir, level, max_halfsweeps=k)
            f_p, c_p = propagate_py(fa, fb, flow0, cost0, 2, 2, seed, dir, level, max_halfsweeps=k)
            assert np.array_equal(f_o, f_p) and np.array_equal(c_o, c_p), (h, w, k)


def hashed_offset(seed, dir, level, t, d, x, y, R):
    """The random-search offset of pixel (x, y) at (level, iteration t, direction step d): each component uniform in
    [-R, R] from the published lowbias32 finaliser keyed as in the reading of Sec. 3.1 (Python integers)."""
    span = 2 * R + 1
    return (hash_py(seed, dir, level, t, d, x, y, 0) % span - R, hash_py(seed, dir, level, t, d, x, y, 1) % span - R)


def _upstream_flows(f, x, y, d):
    h, w, _ = f.shape
    out = []
    for ox, oy in UPSTREAM[d]:
        nx, ny = x + ox, y + oy
        if 0 <= nx < w and 0 <= ny < h:
            out.append((int(f[ny, nx, 0]), int(f[ny, nx, 1])))
    return out


def check_random_search_moves(o):
    """Where every move of a half-sweep comes from (Sec. 3.1: propagation towards the four quadrants, then a random
    search after each of the last three propagation steps of an iteration):
      * d = 0 (the first propagation step): a pixel that changes takes the flow one of its two upstream
        neighbours held when the half-sweep started -- never a random candidate;
      * d >= 1: a changed flow is an upstream neighbour's flow, or a base (the pixel's own flow or a neighbour's)
        plus this pixel's hashed offset for (level, t, d), which lies in [-R, R]^2 and is not (0, 0);
      * a pixel whose random candidate was not taken could not have lowered its cost with it.
    Random initial flows, so that every kind of move happens (the counts are checked)."""
    h, w = 12, 14
    ia = smooth_texture(401, h, w)
    ib = shifted(ia, 2, -1, 402)
    fa, fb = o.wht(ia), o.wht(ib)
    rng = np.random.default_rng(403)
    flow0 = np.zeros((h, w, 2), np.int16)
    for y in range(h):
        for x in range(w):
            flow0[y, x] = (rng.integers(-x, w - x), rng.integers(-y, h - y))
    cost0 = o.init_cost(fa, fb, flow0)
    iters, R, seed, dir, level = 2, 2, 4242, 1, 2
    states = [(flow0, cost0)]
    for k in range(1, iters * 8 + 1):
        states.append(o.propagate(fa, fb, flow0, cost0, iters, R, seed, dir, level, max_halfsweeps=k))
    moves = {"neighbour_d0": 0, "neighbour": 0, "random": [0, 0, 0, 0]}
    for k in range(1, len(states)):
        (f0, c0), (f1, c1) = states[k - 1], states[k]
        t, d, colour = (k - 1) // 8, ((k - 1) // 2) % 4, (k - 1) % 2
        for y in range(h):
            for x in range(w):
                if (x + y) % 2 != colour:
                    continue
                old = (int(f0[y, x, 0]), int(f0[y, x, 1]))
                new = (int(f1[y, x, 0]), int(f1[y, x, 1]))
                nbs = _upstream_flows(f0, x, y, d)
                off = hashed_offset(seed, dir, level, t, d, x, y, R)
                assert -R <= off[0] <= R and -R <= off[1] <= R
                bases = [old] + nbs
                if new != old:
                    if d == 0:
                        assert new in nbs, ("d=0 move that is no neighbour's flow", k, x, y, old, new, nbs)
                        moves["neighbour_d0"] += 1
                    elif new in nbs:
                        moves["neighbour"] += 1
                    else:
                        assert off != (0, 0), (k, x, y)
                        assert (new[0] - off[0], new[1] - off[1]) in bases, \
                            ("move that is neither a neighbour's flow nor a base plus the hashed offset", k, x, y,
                             old, new, nbs, off)
                        moves["random"][d] += 1
                if d >= 1 and off != (0, 0) and new in bases and (new[0] - off[0], new[1] - off[1]) not in bases:
                    # the random candidate was not taken: it must not have been strictly cheaper
                    c = sad_numpy(fa, fb, x, y, new[0] + off[0], new[1] + off[1])
                    assert c < 0 or c >= int(c1[y, x]), ("missed random improvement", k, x, y)
    assert moves["neighbour_d0"] > 0 and moves["neighbour"] > 0, moves
    assert all(moves["random"][d] > 0 for d in (1, 2, 3)), moves


def check_random_search_finds_negative_offset(o):
    """Only the random search can move a pixel whose upstream neighbours hold its own flow (they are skipped):
    from an all-zero field, a target shifted by (-1, -2) -- inside the radius, negative in both components -- is
    recovered exactly (cost 0) on every pixel whose patch lies inside both frames; with R = 0 (no random
    candidate) nothing moves at all.  Offsets drawn from [0, 2R] instead of [-R, R] could never reach it."""
    h, w = 24, 28
    ia = smooth_texture(410, h, w)
    ib = shifted(ia, -1, -2, 411)
    fa, fb = o.wht(ia), o.wht(ib)
    flow0 = np.zeros((h, w, 2), np.int16)
    cost0 = o.init_cost(fa, fb, flow0)
    assert cost0.min() > 0
    f, c = o.propagate(fa, fb, flow0, cost0, 2, 2, 1234, 0, 0)
    inner = np.zeros((h, w), bool)
    inner[4 + 2:h - 4, 4 + 1:w - 4] = True  # patch margin (3 above/left, 4 below/right) plus the shift
    assert np.all(f[inner] == (-1, -2)), "random search did not recover a negative shift"
    assert np.all(c[inner] == 0)
    f0, c0 = o.propagate(fa, fb, flow0, cost0, 2, 0, 1234, 0, 0)
    assert np.array_equal(f0, flow0) and np.array_equal(c0, cost0), "something moved without a random candidate"


def check_stream_keys(o):
    """The level and the matching direction are part of the random-search key of the whole stage (reading of
    Sec. 3.1: one counter-based stream per (direction, level, iteration)).
      * Level: the same content placed at level 1 of a 2-level pyramid and at level 2 of a 3-level one, under
        finer levels whose target frame is constant (every candidate ties there, so nothing moves and the
        level-0 field is the coarse result doubled at each hand-over), must come out different.
      * Direction: the inverse field of (A, B) matches B to A on the inverse stream, so it must differ from the
        forward field of (B, A), which matches the same content on the forward stream."""
    import oracle as _o

    w1, h1 = 12, 10
    xa = o.wht(smooth_texture(500, h1, w1))
    xb = o.wht(smooth_texture(501, h1, w1))  # unrelated content: the random search keeps finding better targets
    flat = lambda hh, ww: o.wht(np.full((hh, ww, 3), 90, np.uint8))

    def prm(L):
        return _o.params(n_scales=L, iters=2, rs_radius=2, eps=1, seed=31)

    f2, _ = o.match_dir([o.wht(smooth_texture(502, 2 * h1, 2 * w1)), xa], [flat(2 * h1, 2 * w1), xb], prm(2), 0)
    f3, _ = o.match_dir([o.wht(smooth_texture(503, 4 * h1, 4 * w1)), o.wht(smooth_texture(504, 2 * h1, 2 * w1)), xa],
                        [flat(4 * h1, 4 * w1), flat(2 * h1, 2 * w1), xb], prm(3), 0)
    r1 = f2[::2, ::2] // 2
    r2 = f3[::4, ::4] // 4
    # the finer levels were frozen: the outputs are the coarse results, doubled per level and repeated
    assert np.array_equal(f2, 2 * np.repeat(np.repeat(r1, 2, 0), 2, 1))
    assert np.array_equal(f3, 4 * np.repeat(np.repeat(r2, 4, 0), 4, 1))
    assert not np.array_equal(r1, r2), "the same content drew the same offsets at levels 1 and 2"
    a = smooth_texture(510, 30, 40)
    b = smooth_texture(511, 30, 40)
    p = _o.params(n_scales=2, iters=2, rs_radius=2, eps=1, seed=32)
    inv_ab = o.match_bidir(a, b, p)[1]
    fwd_ba = o.match_bidir(b, a, p)[0]
    assert not np.array_equal(inv_ab, fwd_ba), "the inverse field drew the forward field's offsets"


def check_sub_scale_handovers(o):
    """Hand-overs of the sub-scale reading (Sec. 3.1 defers sub-scales to Flow Fields+): onto the grid of every
    g-th pixel of a level from the level above, twice the flow of the parent of level pixel (g*u, g*v), always
    inside the level; and from the grid of stride 2g to the grid of stride g of the same level, the parent grid
    pixel's flow unchanged but with its target clamped into the level; the cost is the SAD at (g*u, g*v)."""
    rng = np.random.default_rng(61)
    for (h, w) in ((17, 23), (16, 20), (9, 5)):
        fa = o.wht(rand_img(62, h, w))
        fb = o.wht(rand_img(63, h, w))
        hc, wc = max(1, h // 2), max(1, w // 2)
        fc = np.zeros((hc, wc, 2), np.int16)
        for y in range(hc):
            for x in range(wc):
                fc[y, x] = (rng.integers(-x, wc - x), rng.integers(-y, hc - y))
        for g in (2, 4):
            gw, gh = -(-w // g), -(-h // g)
            flow, cost = o.upsample_grid(fa, fb, g, fc)
            assert flow.shape == (gh, gw, 2)
            for v in range(gh):
                for u in range(gw):
                    x, y = g * u, g * v
                    want = 2 * fc[min(y // 2, hc - 1), min(x // 2, wc - 1)]
                    assert flow[v, u].tolist() == want.tolist(), (g, u, v)
                    assert 0 <= x + want[0] < w and 0 <= y + want[1] < h
                    assert cost[v, u] == sad_numpy(fa, fb, x, y, *want.tolist())
            # the next finer grid of the same level: parent pixel's flow, target clamped into the level
            pw, ph = gw, gh
            fp = np.zeros((ph, pw, 2), np.int16)
            for v in range(ph):
                for u in range(pw):
                    x, y = g * u, g * v
                    fp[v, u] = (rng.integers(-x, w - x), rng.integers(-y, h - y))
            g2 = g // 2
            cw, ch = -(-w // g2), -(-h // g2)
            flow, cost = o.grid_handover(fa, fb, g2, fp)
            assert flow.shape == (ch, cw, 2)
            clamped = 0
            for v in range(ch):
                for u in range(cw):
                    x, y = g2 * u, g2 * v
                    f = fp[min(v // 2, ph - 1), min(u // 2, pw - 1)].astype(int)
                    tx, ty = min(max(x + f[0], 0), w - 1), min(max(y + f[1], 0), h - 1)
                    clamped += (tx, ty) != (x + f[0], y + f[1])
                    assert flow[v, u].tolist() == [tx - x, ty - y], (g2, u, v)
                    assert cost[v, u] == sad_numpy(fa, fb, x, y, tx - x, ty - y)
            assert clamped > 0  # the case the clamp exists for did occur


def check_sub_scale_propagation(o):
    """Propagation on the grid of every second or fourth pixel of a level: the cost of grid pixel (u, v) is the
    SAD at level pixel (g*u, g*v), never rises and only the active colour (u + v parity) moves; at d = 0 a changed
    pixel takes a grid neighbour's snapshot flow; at d >= 1 a changed flow is a grid neighbour's flow or a base
    plus the offset hashed with the level coordinates (g*u, g*v) and the grid's stream id, in [-R, R]^2."""
    h, w = 26, 30
    ia = smooth_texture(420, h, w)
    ib = shifted(ia, 3, -2, 421)
    fa, fb = o.wht(ia), o.wht(ib)
    rng = np.random.default_rng(422)
    for g in (2, 4):
        gw, gh = -(-w // g), -(-h // g)
        flow0 = np.zeros((gh, gw, 2), np.int16)
        for v in range(gh):
            for u in range(gw):
                flow0[v, u] = (rng.integers(-g * u, w - g * u), rng.integers(-g * v, h - g * v))
        cost0 = np.array([[sad_numpy(fa, fb, g * u, g * v, *flow0[v, u].tolist()) for u in range(gw)]
                          for v in range(gh)], np.int64)
        iters, R, seed, dir, stream = 2, 2, 99, 1, 3 + 8 * (g.bit_length() - 1)
        states = [(flow0, cost0)]
        for k in range(1, iters * 8 + 1):
            states.append(o.propagate_grid(fa, fb, g, flow0, cost0, iters, R, seed, dir, stream, max_halfsweeps=k))
        rnd = 0
        for k in range(1, len(states)):
            (f0, c0), (f1, c1) = states[k - 1], states[k]
            t, d, colour = (k - 1) // 8, ((k - 1) // 2) % 4, (k - 1) % 2
            assert np.all(c1 <= c0), (g, k)
            for v in range(gh):
                for u in range(gw):
                    new = (int(f1[v, u, 0]), int(f1[v, u, 1]))
                    assert c1[v, u] == sad_numpy(fa, fb, g * u, g * v, *new), (g, k, u, v)
                    old = (int(f0[v, u, 0]), int(f0[v, u, 1]))
                    if new == old:
                        continue
                    assert (u + v) % 2 == colour, (g, k, u, v)
                    nbs = _upstream_flows(f0, u, v, d)
                    if d == 0:
                        assert new in nbs, (g, k, u, v)
                    elif new not in nbs:
                        off = hashed_offset(seed, dir, stream, t, d, g * u, g * v, R)
                        assert off != (0, 0) and (new[0] - off[0], new[1] - off[1]) in [old] + nbs, (g, k, u, v)
                        rnd += 1
        assert rnd > 0, g


def check_sub_scale_translation(o):
    """With sub-scales (and sub-sub-scales), known integer translations are still recovered exactly (cost 0,
    consistent), and the sub-scales change the schedule (the fields differ from those without them)."""
    import oracle as _o

    for (h, w, L, dx, dy, n_sub) in ((64, 72, 3, 8, -4, 1), (48, 56, 2, -6, 4, 2), (64, 72, 3, -5, 7, 2)):
        ia = smooth_texture(700 + L + n_sub, h, w)
        ib = shifted(ia, dx, dy, 710 + L)
        prm = _o.params(n_scales=L, iters=3, rs_radius=2, eps=0, seed=9, sub_scales=n_sub)
        ff, fb, cf, cb, mask = o.match_bidir(ia, ib, prm)
        m = 4 + 2 ** (L - 1)
        ys, xs = np.mgrid[0:h, 0:w]
        inner = (xs >= m + max(0, -dx)) & (xs < w - m - max(0, dx)) & (ys >= m + max(0, -dy)) & (ys < h - m - max(0, dy))
        assert np.all(ff[inner] == (dx, dy)), (L, n_sub, dx, dy)
        assert np.all(cf[inner] == 0) and np.all(mask[inner] == 1)
    ia = smooth_texture(730, 40, 52)
    ib = smooth_texture(731, 40, 52)
    plain = o.match_bidir(ia, ib, _o.params(n_scales=2, iters=2, seed=4))
    sub = o.match_bidir(ia, ib, _o.params(n_scales=2, iters=2, seed=4, sub_scales=1))
    assert not np.array_equal(plain[0], sub[0])


def check_translation(o):
    """Known integer translations are recovered exactly (cost 0) and pass the consistency check."""
    prm_cls = __import__("oracle").params
    for (h, w, L, dx, dy) in ((40, 48, 1, 3, -2), (64, 72, 3, 8, -4), (48, 56, 2, -6, 4)):
        ia = smooth_texture(100 + L, h, w)
        ib = shifted(ia, dx, dy, 200 + L)
        prm = prm_cls(n_scales=L, iters=3, rs_radius=2, eps=0, seed=9)
        ff, fb, cf, cb, mask = o.match_bidir(ia, ib, prm)
        m = 4 + 2 ** (L - 1)  # margin: patch half-size plus the clamp reach of the coarse levels
        ys, xs = np.mgrid[0:h, 0:w]
        inner = (xs >= m + max(0, -dx)) & (xs < w - m - max(0, dx)) & (ys >= m + max(0, -dy)) & (ys < h - m - max(0, dy))
        assert np.all(ff[inner] == (dx, dy)), (L, dx, dy)
        assert np.all(cf[inner] == 0)
        assert np.all(mask[inner] == 1)
        # the inverse field recovers (-dx, -dy) on frame 2's matching region
        inner2 = (xs >= m + max(0, dx)) & (xs < w - m - max(0, -dx)) & (ys >= m + max(0, dy)) & (ys < h - m - max(0, -dy))
        assert np.all(fb[inner2] == (-dx, -dy))


def check_consistency(o):
    rng = np.random.default_rng(3)
    for (h, w) in ((5, 7), (16, 9), (1, 1)):
        fwd = rng.integers(-3, 4, size=(h, w, 2)).astype(np.int16)
        bwd = rng.integers(-3, 4, size=(h, w, 2)).astype(np.int16)
        for eps in (0, 1, 2, 7):
            assert np.array_equal(o.consistency(fwd, bwd, eps), consistency_numpy(fwd, bwd, eps))
    # f = -b at the target: every in-image match is consistent at eps = 0
    h, w = 6, 8
    fwd = np.zeros((h, w, 2), np.int16)
    fwd[..., 0] = 1
    bwd = np.zeros((h, w, 2), np.int16)
    bwd[..., 0] = -1
    m = o.consistency(fwd, bwd, 0)
    assert np.all(m[:, :-1] == 1) and np.all(m[:, -1] == 0)
    # boundary: error (1, 0) is kept at eps = 1 (not exceeding), error (1, 1) is not
    fwd = np.zeros((1, 2, 2), np.int16)
    bwd = np.zeros((1, 2, 2), np.int16)
    bwd[0, 0] = (1, 0)
    bwd[0, 1] = (1, 1)
    fwd[0, 1] = (0, 0)
    assert o.consistency(fwd, bwd, 1).tolist() == [[1, 0]]


def sparsify_numpy(fwd, bwd, eps, s, keep=None):
    """Brute-force restatement: per 3x3 block, the lowest-error inlier if the block has >= s inliers (an inlier
    passes the consistency check and, when a filter mask `keep` is given, is set in it)."""
    h, w, _ = fwd.shape
    ys, xs = np.mgrid[0:h, 0:w]
    qx = xs + fwd[..., 0].astype(np.int64)
    qy = ys + fwd[..., 1].astype(np.int64)
    inside = (qx >= 0) & (qx < w) & (qy >= 0) & (qy < h)
    qxc, qyc = np.clip(qx, 0, w - 1), np.clip(qy, 0, h - 1)
    e = (fwd[..., 0] + bwd[qyc, qxc, 0].astype(np.int64)) ** 2 + (fwd[..., 1] + bwd[qyc, qxc, 1].astype(np.int64)) ** 2
    ok = inside & (e <= eps * eps)
    if keep is not None:
        ok &= keep.astype(bool)
    out = np.zeros((h, w), np.uint8)
    for by in range(0, h, 3):
        for bx in range(0, w, 3):
            cand = [(int(e[y, x]), y, x) for y in range(by, min(by + 3, h)) for x in range(bx, min(bx + 3, w))
                    if ok[y, x]]
            if len(cand) >= s:
                _, y, x = min(cand)  # smallest error, then row-major first
                out[y, x] = 1
    return out


def check_sparsify(o):
    # hand example: one 3x3 block, errors 0 at (1,1) and 0 at (2,2) -> the first in row-major order wins
    fwd = np.zeros((3, 3, 2), np.int16)
    bwd = np.zeros((3, 3, 2), np.int16)
    bwd[..., 0] = 1  # every pixel has error 1 ...
    bwd[1, 1] = (0, 0)
    bwd[2, 2] = (0, 0)  # ... except (1,1) and (2,2), error 0
    assert o.sparsify(fwd, bwd, 1, 9).tolist() == [[0, 0, 0], [0, 1, 0], [0, 0, 0]]
    assert o.sparsify(fwd, bwd, 0, 2).tolist() == [[0, 0, 0], [0, 1, 0], [0, 0, 0]]  # 2 inliers at eps 0
    assert o.sparsify(fwd, bwd, 0, 3).sum() == 0  # only 2 inliers < s
    # partial edge blocks, random flows, several s and eps: brute force
    rng = np.random.default_rng(17)
    for (h, w) in ((7, 8), (10, 11), (1, 5), (3, 3)):
        fwd = rng.integers(-2, 3, size=(h, w, 2)).astype(np.int16)
        bwd = rng.integers(-2, 3, size=(h, w, 2)).astype(np.int16)
        for eps, s in ((1, 1), (2, 4), (3, 7), (0, 1)):
            got = o.sparsify(fwd, bwd, eps, s)
            assert np.array_equal(got, sparsify_numpy(fwd, bwd, eps, s)), (h, w, eps, s)
            # at most one match per block, and only consistent matches survive
            for by in range(0, h, 3):
                for bx in range(0, w, 3):
                    assert got[by:by + 3, bx:bx + 3].sum() <= 1
            assert np.all(got <= o.consistency(fwd, bwd, eps))
            # a filter mask: all ones changes nothing, all zeros keeps nothing, a random one is brute force
            assert np.array_equal(o.sparsify(fwd, bwd, eps, s, np.ones((h, w), np.uint8)), got)
            assert o.sparsify(fwd, bwd, eps, s, np.zeros((h, w), np.uint8)).sum() == 0
            keep = (rng.random((h, w)) < 0.7).astype(np.uint8)
            got_k = o.sparsify(fwd, bwd, eps, s, keep)
            assert np.array_equal(got_k, sparsify_numpy(fwd, bwd, eps, s, keep)), (h, w, eps, s)
            assert np.all(got_k <= keep)
    # hand example with a mask: the error-0 match (1,1) is filtered out, so (2,2) (error 0) wins
    fwd = np.zeros((3, 3, 2), np.int16)
    bwd = np.zeros((3, 3, 2), np.int16)
    bwd[..., 0] = 1
    bwd[1, 1] = (0, 0)
    bwd[2, 2] = (0, 0)
    keep = np.ones((3, 3), np.uint8)
    keep[1, 1] = 0
    assert o.sparsify(fwd, bwd, 1, 8, keep).tolist() == [[0, 0, 0], [0, 0, 0], [0, 0, 1]]
    assert o.sparsify(fwd, bwd, 1, 9, keep).sum() == 0  # 8 matches left < s


def check_second_consistency(o):
    """Two checks (Sec. 3.1): the first inverse field and forward field equal the single-check stage, the second
    inverse field is the inverse matching with radius rs_radius2 and direction id 2, the mask is the AND."""
    import oracle as _o

    h, w, L, T = 30, 40, 2, 2
    ia = smooth_texture(600, h, w)
    ib = shifted(ia, 2, -1, 601)
    ib[5:15, 10:25] = smooth_texture(602, 10, 15)
    prm = _o.params(n_scales=L, iters=T, rs_radius=2, eps=1, seed=5)
    ff, fb, fb2, mask = o.match_bidir2(ia, ib, prm, 4)
    one = o.match_bidir(ia, ib, prm)
    assert np.array_equal(ff, one[0]) and np.array_equal(fb, one[1])
    fa = [o.wht(x) for x in o.pyramid(ia, L)]
    fbb = [o.wht(x) for x in o.pyramid(ib, L)]
    want2, _ = o.match_dir(fbb, fa, _o.params(n_scales=L, iters=T, rs_radius=4, eps=1, seed=5), 2)
    assert np.array_equal(fb2, want2)
    assert not np.array_equal(fb2, fb)  # different parameters give a different inverse field here
    assert np.array_equal(mask, one[4] & o.consistency(ff, fb2, 1))


def census_numpy(img):
    """Brute-force restatement of the 7x7 Census transform: bit k = k-th neighbour (row-major, centre skipped,
    edge pixels repeated) strictly darker than the centre."""
    h, w, _ = img.shape
    pad = np.pad(img.astype(np.int64), ((3, 3), (3, 3), (0, 0)), mode="edge")
    out = np.zeros((h, w, 3), np.uint64)
    k = 0
    for dy in range(-3, 4):
        for dx in range(-3, 4):
            if dy == 0 and dx == 0:
                continue
            nb = pad[3 + dy:3 + dy + h, 3 + dx:3 + dx + w]
            out |= (nb < img).astype(np.uint64) << np.uint64(k)
            k += 1
    return out


def check_census(o):
    flat = np.full((9, 9, 3), 77, np.uint8)
    assert not o.census(flat).any()  # no neighbour is darker
    spot = np.zeros((9, 9, 3), np.uint8)
    spot[4, 4] = (200, 0, 30)
    c = o.census(spot)
    assert int(c[4, 4, 0]) == (1 << 48) - 1 and int(c[4, 4, 1]) == 0 and int(c[4, 4, 2]) == (1 << 48) - 1
    # bit order: only the top-left neighbour (dy=-3, dx=-3) darker -> bit 0; bottom-right -> bit 47
    one = np.full((7, 7, 3), 100, np.uint8)
    one[0, 0] = 10
    assert int(o.census(one)[3, 3, 0]) == 1
    one = np.full((7, 7, 3), 100, np.uint8)
    one[6, 6] = 10
    assert int(o.census(one)[3, 3, 0]) == 1 << 47
    # equal neighbours do not count (strictly darker)
    eq = np.full((7, 7, 3), 100, np.uint8)
    eq[3, 3] = 100
    assert int(o.census(eq)[3, 3, 0]) == 0
    for seed, (h, w) in enumerate(((9, 13), (1, 5), (6, 1), (17, 11))):
        im = rand_img(40 + seed, h, w)
        assert np.array_equal(o.census(im), census_numpy(im)), (h, w)
    ca = o.census(rand_img(50, 8, 9))
    cb = o.census(rand_img(51, 8, 9))
    for (x, y, fx, fy) in ((0, 0, 0, 0), (3, 4, 2, -1), (8, 7, -8, -7)):
        want = sum(bin(int(ca[y, x, ch]) ^ int(cb[y + fy, x + fx, ch])).count("1") for ch in range(3))
        assert o.hamming(ca, cb, x, y, fx, fy) == want
    assert o.hamming(ca, ca, 2, 2, 0, 0) == 0 and o.hamming(ca, cb, 0, 0, -1, 0) == -1
    assert o.hamming(o.census(spot), o.census(flat), 4, 4, 0, 0) == 96  # 2 x 48 bits differ


def check_census_matching(o):
    """Under the Census cost: propagation never raises a cost, cost = Hamming of the flow, and an integer
    translation is recovered exactly (cost 0) by the whole stage."""
    import oracle as _o

    h, w = 11, 13
    ia, ib = _tiny_level(71, h, w)
    ca, cb = o.census(ia), o.census(ib)
    rng = np.random.default_rng(72)
    flow0 = np.zeros((h, w, 2), np.int16)
    for y in range(h):
        for x in range(w):
            flow0[y, x] = (rng.integers(-x, w - x), rng.integers(-y, h - y))
    cost0 = np.array([[o.hamming(ca, cb, x, y, *flow0[y, x].tolist()) for x in range(w)] for y in range(h)], np.int32)
    prev = cost0
    for k in range(1, 17):
        f, c = o.propagate_census(ca, cb, flow0, cost0, 2, 2, 5, 0, 1, max_halfsweeps=k)
        assert np.all(c <= prev)
        assert all(c[y, x] == o.hamming(ca, cb, x, y, *f[y, x].tolist()) for y in range(h) for x in range(w))
        prev = c
    for (hh, ww, L, dx, dy) in ((40, 48, 1, 3, -2), (48, 56, 2, -4, 2)):
        ia = smooth_texture(800 + L, hh, ww)
        ib = shifted(ia, dx, dy, 801 + L)
        prm = _o.params(n_scales=L, iters=3, rs_radius=2, eps=0, seed=9, cost=_o.COST_CENSUS)
        ff, fb, cf, cb_, mask = o.match_bidir(ia, ib, prm)
        m = 4 + 2 ** (L - 1)
        ys, xs = np.mgrid[0:hh, 0:ww]
        inner = (xs >= m + max(0, -dx)) & (xs < ww - m - max(0, dx)) & (ys >= m + max(0, -dy)) & (ys < hh - m - max(0, dy))
        assert np.all(ff[inner] == (dx, dy)) and np.all(cf[inner] == 0) and np.all(mask[inner] == 1)


def check_pipeline_composition(o):
    """The whole stage equals its steps composed in the order of Sec. 3.1 (pyramid, WHT, seed at the coarsest
    level, per level hand-over + propagation keyed by (direction, level), inverse field with the frames
    swapped, consistency of the forward field)."""
    import oracle as _o

    for (h, w, L, T, eps, seed) in ((24, 30, 3, 2, 1, 123), (17, 21, 2, 1, 2, 77)):
        ia = smooth_texture(300 + h, h, w)
        ib = shifted(ia, 3, 1, 301 + h)
        ib[2:9, 4:12] = smooth_texture(302, 7, 8)  # an occluder so that the fields are not trivial
        prm = _o.params(n_scales=L, iters=T, rs_radius=2, eps=eps, seed=seed)
        got = o.match_bidir(ia, ib, prm)
        pa, pb = o.pyramid(ia, L), o.pyramid(ib, L)
        for lvl, (wl, hl) in enumerate(o.level_dims(w, h, L)):
            assert pa[lvl].shape == (hl, wl, 3)
        fa = [o.wht(x) for x in pa]
        fb = [o.wht(x) for x in pb]
        out = []
        for dir, (A, B) in enumerate(((fa, fb), (fb, fa))):
            flow = None
            for s in range(L - 1, -1, -1):
                if s == L - 1:
                    flow, _ = o.seed(A[s], B[s])
                    cost = o.init_cost(A[s], B[s], flow)
                else:
                    flow, cost = o.upsample(A[s], B[s], flow)
                flow, cost = o.propagate(A[s], B[s], flow, cost, T, 2, seed, dir, s)
            out.append((flow, cost))
        mask = o.consistency(out[0][0], out[1][0], eps)
        assert np.array_equal(got[0], out[0][0]) and np.array_equal(got[2], out[0][1])
        assert np.array_equal(got[1], out[1][0]) and np.array_equal(got[3], out[1][1])
        assert np.array_equal(got[4], mask)


ALL_CHECKS = [
    check_pyramid,
    check_wht,
    check_hash,
    check_sad,
    check_seed,
    check_upsample,
    check_propagation_invariants,
    check_random_search_moves,
    check_random_search_finds_negative_offset,
    check_stream_keys,
    check_sub_scale_handovers,
    check_sub_scale_propagation,
    check_sub_scale_translation,
    check_propagation_schedule,
    check_translation,
    check_consistency,
    check_sparsify,
    check_second_consistency,
    check_census,
    check_census_matching,
    check_pipeline_composition,
]
