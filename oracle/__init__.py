"""CPU oracle of the Flow Fields dense-matching stage of FlowFields++ (arXiv 1805.03517, Sec. 3.1).

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and its binding) never does,
and shares no code with it.

The arithmetic lives in ``ff_oracle.c`` (plain single-threaded C, integer only); this module compiles it
with gcc into ``oracle/_build/libffo.so`` on first use and exposes NumPy-facing wrappers.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ff_oracle.c")
_HDR = os.path.join(_HERE, "ff_oracle.h")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libffo.so")
_lock = threading.Lock()
_lib = None

NF = 48


class Params(ctypes.Structure):
    """Mirror of ``ffo_params`` (the oracle's own parameter block)."""

    _fields_ = [
        ("n_scales", ctypes.c_int),
        ("iters", ctypes.c_int),
        ("rs_radius", ctypes.c_int),
        ("eps", ctypes.c_int),
        ("seed", ctypes.c_uint32),
        ("cost", ctypes.c_int),
        ("sub_scales", ctypes.c_int),
    ]


def compile_library(src: str = _SRC, out: str = _LIB_PATH, extra_flags=()) -> str:
    """Compile the oracle C source into a shared library (also used to build planted-mistake variants)."""
    os.makedirs(os.path.dirname(out), exist_ok=True)
    tmp = f"{out}.{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-I", _HERE, *extra_flags, src, "-o", tmp]
    subprocess.run(cmd, check=True, capture_output=True)
    os.replace(tmp, out)
    return out


def build() -> str:
    """Compile ``libffo.so`` if it is missing or older than its sources."""
    with _lock:
        stale = not os.path.exists(_LIB_PATH) or any(
            os.path.getmtime(p) > os.path.getmtime(_LIB_PATH) for p in (_SRC, _HDR)
        )
        if stale:
            compile_library()
    return _LIB_PATH


def _declare(lib):
    i16p = np.ctypeslib.ndpointer(np.int16, flags="C_CONTIGUOUS")
    i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
    u8p = np.ctypeslib.ndpointer(np.uint8, flags="C_CONTIGUOUS")
    ip = ctypes.POINTER(ctypes.c_int)
    c_int, c_u32, c_long = ctypes.c_int, ctypes.c_uint32, ctypes.c_long
    lib.ffo_level_dims.argtypes = [c_int, c_int, c_int, ip, ip]
    lib.ffo_level_dims.restype = c_int
    lib.ffo_downsample.argtypes = [u8p, c_int, c_int, u8p]
    lib.ffo_downsample.restype = None
    lib.ffo_wht.argtypes = [u8p, c_int, c_int, i16p]
    lib.ffo_wht.restype = None
    lib.ffo_mix32.argtypes = [c_u32]
    lib.ffo_mix32.restype = c_u32
    lib.ffo_hash.argtypes = [c_u32, c_int, c_int, c_int, c_int, c_int, c_int, c_int]
    lib.ffo_hash.restype = c_u32
    lib.ffo_sad.argtypes = [i16p, i16p, c_int, c_int, c_int, c_int, c_int, c_int]
    lib.ffo_sad.restype = ctypes.c_int32
    lib.ffo_seed.argtypes = [i16p, i16p, c_int, c_int, i16p, i32p]
    lib.ffo_seed.restype = None
    lib.ffo_init_cost.argtypes = [i16p, i16p, c_int, c_int, i16p, i32p]
    lib.ffo_init_cost.restype = None
    lib.ffo_upsample.argtypes = [i16p, i16p, c_int, c_int, i16p, c_int, c_int, i16p, i32p]
    lib.ffo_upsample.restype = c_int
    lib.ffo_upsample_grid.argtypes = [i16p, i16p, c_int, c_int, c_int, i16p, c_int, c_int, i16p, i32p]
    lib.ffo_upsample_grid.restype = c_int
    lib.ffo_grid_handover.argtypes = [i16p, i16p, c_int, c_int, c_int, i16p, c_int, c_int, i16p, i32p]
    lib.ffo_grid_handover.restype = None
    lib.ffo_propagate_grid.argtypes = [i16p, i16p, c_int, c_int, c_int, i16p, i32p, c_int, c_int, c_u32, c_int, c_int,
                                       c_long]
    lib.ffo_propagate_grid.restype = c_long
    lib.ffo_propagate.argtypes = [i16p, i16p, c_int, c_int, i16p, i32p, c_int, c_int, c_u32, c_int, c_int, c_long]
    lib.ffo_propagate.restype = c_long
    pp = ctypes.POINTER(ctypes.c_void_p)
    lib.ffo_match_dir.argtypes = [pp, pp, ip, ip, ctypes.POINTER(Params), c_int, i16p, i32p]
    lib.ffo_match_dir.restype = c_int
    lib.ffo_consistency.argtypes = [i16p, i16p, c_int, c_int, c_int, u8p]
    lib.ffo_consistency.restype = None
    lib.ffo_match_bidir2.argtypes = [u8p, u8p, c_int, c_int, ctypes.POINTER(Params), c_int, i16p, i16p, i16p, u8p]
    lib.ffo_match_bidir2.restype = c_int
    u64p = np.ctypeslib.ndpointer(np.uint64, flags="C_CONTIGUOUS")
    lib.ffo_census.argtypes = [u8p, c_int, c_int, u64p]
    lib.ffo_census.restype = None
    lib.ffo_hamming.argtypes = [u64p, u64p, c_int, c_int, c_int, c_int, c_int, c_int]
    lib.ffo_hamming.restype = ctypes.c_int32
    lib.ffo_propagate_census.argtypes = [u64p, u64p, c_int, c_int, i16p, i32p, c_int, c_int, c_u32, c_int, c_int,
                                         c_long]
    lib.ffo_propagate_census.restype = c_long
    lib.ffo_sparsify.argtypes = [i16p, i16p, ctypes.c_void_p, c_int, c_int, c_int, c_int, u8p]
    lib.ffo_sparsify.restype = None
    lib.ffo_match_bidir.argtypes = [u8p, u8p, c_int, c_int, ctypes.POINTER(Params), i16p, i16p, i32p, i32p, u8p]
    lib.ffo_match_bidir.restype = c_int
    return lib


def load_library(path: str):
    """Load and declare an oracle shared library at ``path`` (the real one or a planted-mistake variant)."""
    return _declare(ctypes.CDLL(path))


def lib():
    global _lib
    if _lib is None:
        _lib = load_library(build())
    return _lib


class Oracle:
    """NumPy-facing wrappers around one oracle library instance."""

    def __init__(self, library=None):
        self.L = library if library is not None else lib()

    def level_dims(self, w, h, n_scales):
        ws = (ctypes.c_int * n_scales)()
        hs = (ctypes.c_int * n_scales)()
        if self.L.ffo_level_dims(w, h, n_scales, ws, hs) != 0:
            raise ValueError("bad pyramid size")
        return list(zip(list(ws), list(hs)))

    def downsample(self, img):
        img = np.ascontiguousarray(img, dtype=np.uint8)
        h, w, _ = img.shape
        out = np.empty((max(1, h // 2), max(1, w // 2), 3), np.uint8)
        self.L.ffo_downsample(img, w, h, out)
        return out

    def pyramid(self, img, n_scales):
        levels = [np.ascontiguousarray(img, dtype=np.uint8)]
        for _ in range(1, n_scales):
            levels.append(self.downsample(levels[-1]))
        return levels

    def wht(self, img):
        img = np.ascontiguousarray(img, dtype=np.uint8)
        h, w, _ = img.shape
        out = np.empty((h, w, NF), np.int16)
        self.L.ffo_wht(img, w, h, out)
        return out

    def mix32(self, x):
        return int(self.L.ffo_mix32(int(x) & 0xFFFFFFFF))

    def hash(self, seed, dir, level, t, d, x, y, comp):
        return int(self.L.ffo_hash(seed & 0xFFFFFFFF, dir, level, t, d, x, y, comp))

    def sad(self, fa, fb, x, y, fx, fy):
        h, w, _ = fa.shape
        return int(self.L.ffo_sad(_i16(fa), _i16(fb), w, h, x, y, fx, fy))

    def seed(self, fa, fb):
        h, w, _ = fa.shape
        flow = np.empty((h, w, 2), np.int16)
        dist = np.empty((h, w), np.int32)
        self.L.ffo_seed(_i16(fa), _i16(fb), w, h, flow, dist)
        return flow, dist

    def init_cost(self, fa, fb, flow):
        h, w, _ = fa.shape
        cost = np.empty((h, w), np.int32)
        self.L.ffo_init_cost(_i16(fa), _i16(fb), w, h, _i16(flow), cost)
        return cost

    def upsample(self, fa, fb, flow_coarse):
        h, w, _ = fa.shape
        hc, wc, _ = flow_coarse.shape
        flow = np.empty((h, w, 2), np.int16)
        cost = np.empty((h, w), np.int32)
        rc = self.L.ffo_upsample(_i16(fa), _i16(fb), w, h, _i16(flow_coarse), wc, hc, flow, cost)
        if rc != 0:
            raise RuntimeError(f"ffo_upsample failed: {rc}")
        return flow, cost

    @staticmethod
    def grid_dims(w, h, g):
        return (w + g - 1) // g, (h + g - 1) // g

    def upsample_grid(self, fa, fb, g, flow_coarse):
        """Hand-over from the level above onto the grid of every g-th pixel of this level."""
        h, w, _ = fa.shape
        gw, gh = self.grid_dims(w, h, g)
        hc, wc, _ = flow_coarse.shape
        flow = np.empty((gh, gw, 2), np.int16)
        cost = np.empty((gh, gw), np.int32)
        rc = self.L.ffo_upsample_grid(_i16(fa), _i16(fb), w, h, g, _i16(flow_coarse), wc, hc, flow, cost)
        if rc != 0:
            raise RuntimeError(f"ffo_upsample_grid failed: {rc}")
        return flow, cost

    def grid_handover(self, fa, fb, g, flow_parent):
        """Hand-over from the grid of every 2g-th pixel to the grid of every g-th pixel of the same level."""
        h, w, _ = fa.shape
        gw, gh = self.grid_dims(w, h, g)
        ph, pw, _ = flow_parent.shape
        flow = np.empty((gh, gw, 2), np.int16)
        cost = np.empty((gh, gw), np.int32)
        self.L.ffo_grid_handover(_i16(fa), _i16(fb), w, h, g, _i16(flow_parent), pw, ph, flow, cost)
        return flow, cost

    def propagate_grid(self, fa, fb, g, flow, cost, iters, rs_radius, seed, dir, stream, max_halfsweeps=-1):
        """Propagation with random search on the grid of every g-th pixel (stream = the hash's level id)."""
        h, w, _ = fa.shape
        flow = np.array(flow, dtype=np.int16, order="C", copy=True)
        cost = np.array(cost, dtype=np.int32, order="C", copy=True)
        n = self.L.ffo_propagate_grid(_i16(fa), _i16(fb), w, h, g, flow, cost, iters, rs_radius, seed & 0xFFFFFFFF,
                                      dir, stream, max_halfsweeps)
        if n < 0:
            raise MemoryError("ffo_propagate_grid")
        return flow, cost

    def propagate(self, fa, fb, flow, cost, iters, rs_radius, seed, dir, level, max_halfsweeps=-1):
        """Run (a prefix of) the level schedule; returns updated copies of flow and cost."""
        h, w, _ = fa.shape
        flow = np.array(flow, dtype=np.int16, order="C", copy=True)
        cost = np.array(cost, dtype=np.int32, order="C", copy=True)
        n = self.L.ffo_propagate(_i16(fa), _i16(fb), w, h, flow, cost, iters, rs_radius, seed & 0xFFFFFFFF,
                                 dir, level, max_halfsweeps)
        if n < 0:
            raise MemoryError("ffo_propagate")
        return flow, cost

    def match_dir(self, feats_a, feats_b, params: Params, dir):
        L = params.n_scales
        ws = (ctypes.c_int * L)(*[f.shape[1] for f in feats_a])
        hs = (ctypes.c_int * L)(*[f.shape[0] for f in feats_a])
        fa = [_i16(f) for f in feats_a]
        fb = [_i16(f) for f in feats_b]
        pa = (ctypes.c_void_p * L)(*[f.ctypes.data for f in fa])
        pb = (ctypes.c_void_p * L)(*[f.ctypes.data for f in fb])
        h, w = hs[0], ws[0]
        flow = np.empty((h, w, 2), np.int16)
        cost = np.empty((h, w), np.int32)
        rc = self.L.ffo_match_dir(pa, pb, ws, hs, ctypes.byref(params), dir, flow, cost)
        if rc != 0:
            raise RuntimeError(f"ffo_match_dir failed: {rc}")
        return flow, cost

    def consistency(self, fwd, bwd, eps):
        h, w, _ = fwd.shape
        mask = np.empty((h, w), np.uint8)
        self.L.ffo_consistency(_i16(fwd), _i16(bwd), w, h, eps, mask)
        return mask

    def match_bidir2(self, img_a, img_b, params: Params, rs_radius2):
        """Forward field, both inverse fields and the mask of the two consistency checks."""
        a = np.ascontiguousarray(img_a, dtype=np.uint8)
        b = np.ascontiguousarray(img_b, dtype=np.uint8)
        h, w, _ = a.shape
        ff = np.empty((h, w, 2), np.int16)
        fb = np.empty((h, w, 2), np.int16)
        fb2 = np.empty((h, w, 2), np.int16)
        mask = np.empty((h, w), np.uint8)
        rc = self.L.ffo_match_bidir2(a, b, w, h, ctypes.byref(params), rs_radius2, ff, fb, fb2, mask)
        if rc != 0:
            raise RuntimeError(f"ffo_match_bidir2 failed: {rc}")
        return ff, fb, fb2, mask

    def census(self, img):
        """uint64 [h][w][3]: the 48-bit Census pattern of every pixel and channel."""
        img = np.ascontiguousarray(img, dtype=np.uint8)
        h, w, _ = img.shape
        out = np.empty((h, w, 3), np.uint64)
        self.L.ffo_census(img, w, h, out)
        return out

    def hamming(self, ca, cb, x, y, fx, fy):
        h, w, _ = ca.shape
        return int(self.L.ffo_hamming(_u64(ca), _u64(cb), w, h, x, y, fx, fy))

    def propagate_census(self, ca, cb, flow, cost, iters, rs_radius, seed, dir, level, max_halfsweeps=-1):
        h, w, _ = ca.shape
        flow = np.array(flow, dtype=np.int16, order="C", copy=True)
        cost = np.array(cost, dtype=np.int32, order="C", copy=True)
        n = self.L.ffo_propagate_census(_u64(ca), _u64(cb), w, h, flow, cost, iters, rs_radius, seed & 0xFFFFFFFF,
                                        dir, level, max_halfsweeps)
        if n < 0:
            raise MemoryError("ffo_propagate_census")
        return flow, cost

    def sparsify(self, fwd, bwd, eps, s, keep=None):
        """keep: optional uint8 [h][w] mask of the matches left by the consistency checks (None: all)."""
        h, w, _ = fwd.shape
        out = np.empty((h, w), np.uint8)
        if keep is not None:
            keep = np.ascontiguousarray(keep, dtype=np.uint8)
            assert keep.shape == (h, w)
        self.L.ffo_sparsify(_i16(fwd), _i16(bwd), None if keep is None else keep.ctypes.data, w, h, eps, s, out)
        return out

    def match_bidir(self, img_a, img_b, params: Params):
        """The whole stage for one pair: (flow_fwd, flow_bwd, cost_fwd, cost_bwd, mask)."""
        a = np.ascontiguousarray(img_a, dtype=np.uint8)
        b = np.ascontiguousarray(img_b, dtype=np.uint8)
        h, w, _ = a.shape
        ff = np.empty((h, w, 2), np.int16)
        fb = np.empty((h, w, 2), np.int16)
        cf = np.empty((h, w), np.int32)
        cb = np.empty((h, w), np.int32)
        mask = np.empty((h, w), np.uint8)
        rc = self.L.ffo_match_bidir(a, b, w, h, ctypes.byref(params), ff, fb, cf, cb, mask)
        if rc != 0:
            raise RuntimeError(f"ffo_match_bidir failed: {rc}")
        return ff, fb, cf, cb, mask


def _i16(a):
    return np.ascontiguousarray(a, dtype=np.int16)


def _u64(a):
    return np.ascontiguousarray(a, dtype=np.uint64)


COST_WHT_SAD, COST_CENSUS = 0, 1


def params(n_scales, iters, rs_radius=2, eps=1, seed=0, cost=COST_WHT_SAD, sub_scales=0) -> Params:
    return Params(n_scales, iters, rs_radius, eps, seed & 0xFFFFFFFF, cost, sub_scales)


_default = None


def default() -> Oracle:
    global _default
    if _default is None:
        _default = Oracle()
    return _default
