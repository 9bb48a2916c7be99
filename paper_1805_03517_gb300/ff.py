"""Python binding of libff (include/ff.h): the Flow Fields dense-matching stage of FlowFields++ on GB300.

The functions named ``ff_*`` are one-to-one wrappers of the C-ABI (argument marshalling only; every step of the
matching runs in the library's CUDA kernels).  They take raw device pointers (``tensor.data_ptr()``) and raise
``FFError`` on a non-OK status.  ``Matcher`` is a small convenience layer that allocates outputs as torch
tensors on the context's device and stream.

There is no CPU fallback: if ``libff.so`` has not been built this module raises on first use.
"""
from __future__ import annotations

import ctypes
import os
import re
from dataclasses import dataclass

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_lib", "libff.so")
# FF_LIBRARY selects another build of the same library (the debug-bounds build, _lib/libff_debug.so)
LIB_PATH = os.environ.get("FF_LIBRARY", LIB_PATH)
HEADER = os.path.join(os.path.dirname(_PKG), "include", "ff.h")

FF_OK, FF_ERR_ARG, FF_ERR_OOM, FF_ERR_CUDA, FF_ERR_TIMEOUT, FF_ERR_BUSY = range(6)
FF_OPT_SEED_KERNEL, FF_OPT_WAIT_LIMIT, FF_OPT_TEST_WITHHOLD_COPIES, FF_OPT_TEST_FAIL_ALLOCS, FF_OPT_OVERLAP = 1, 2, 3, 4, 5
FF_SEED_MMA_SYNC, FF_SEED_TCGEN05 = 0, 1
FF_COST_WHT_SAD, FF_COST_CENSUS = 0, 1
STATUS_NAMES = {0: "FF_OK", 1: "FF_ERR_ARG", 2: "FF_ERR_OOM", 3: "FF_ERR_CUDA", 4: "FF_ERR_TIMEOUT", 5: "FF_ERR_BUSY"}
PHASES = ("features", "seed", "handover", "propagate", "consistency")


class FFError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class Params(ctypes.Structure):
    _fields_ = [("n_scales", ctypes.c_int), ("iters", ctypes.c_int), ("patch", ctypes.c_int),
                ("n_coef", ctypes.c_int), ("rs_radius", ctypes.c_int), ("eps", ctypes.c_int),
                ("seed", ctypes.c_uint32), ("rs_radius2", ctypes.c_int), ("cost", ctypes.c_int),
                ("sub_scales", ctypes.c_int)]


class PairJob(ctypes.Structure):
    _fields_ = [("a", ctypes.c_void_p), ("b", ctypes.c_void_p), ("flow_fwd", ctypes.c_void_p),
                ("flow_bwd", ctypes.c_void_p), ("cost_fwd", ctypes.c_void_p), ("cost_bwd", ctypes.c_void_p),
                ("mask", ctypes.c_void_p), ("flow_bwd2", ctypes.c_void_p)]


class Request(ctypes.Structure):
    _fields_ = [("rgb_a", ctypes.c_void_p), ("rgb_b", ctypes.c_void_p), ("w", ctypes.c_int), ("h", ctypes.c_int),
                ("pitch_bytes", ctypes.c_int), ("flow_fwd", ctypes.c_void_p), ("flow_bwd", ctypes.c_void_p),
                ("cost_fwd", ctypes.c_void_p), ("cost_bwd", ctypes.c_void_p), ("mask", ctypes.c_void_p)]


class Frame(ctypes.Structure):
    _fields_ = [("rgb_dev", ctypes.c_void_p), ("w", ctypes.c_int), ("h", ctypes.c_int), ("pitch_bytes", ctypes.c_int)]


class FrameJob(ctypes.Structure):
    _fields_ = [("a", ctypes.c_int), ("b", ctypes.c_int), ("flow_fwd", ctypes.c_void_p),
                ("flow_bwd", ctypes.c_void_p), ("cost_fwd", ctypes.c_void_p), ("cost_bwd", ctypes.c_void_p),
                ("mask", ctypes.c_void_p), ("flow_bwd2", ctypes.c_void_p)]


class Tuning(ctypes.Structure):
    _fields_ = [("tile_w", ctypes.c_int), ("tile_h", ctypes.c_int), ("iters_per_launch", ctypes.c_int),
                ("threads", ctypes.c_int), ("speculate", ctypes.c_int), ("cluster", ctypes.c_int),
                ("dataflow", ctypes.c_int)]


class Stats(ctypes.Structure):
    _fields_ = [("kernel_launches", ctypes.c_int64), ("graph_replays", ctypes.c_int64),
                ("plans_built", ctypes.c_int64), ("scratch_bytes", ctypes.c_int64),
                ("cluster_launches", ctypes.c_int64)]


_lib = None


def header_functions(path: str = HEADER):
    """Names of the functions include/ff.h declares."""
    with open(path) as f:
        return re.findall(r"^FF_API [^(]*?\b(ff_\w+)\(", f.read(), flags=re.M)


def lib():
    """Load libff.so (built by ``paper_1805_03517_gb300.build``); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libff.so is not built ({LIB_PATH}); run `python -m paper_1805_03517_gb300.build`")
    L = ctypes.CDLL(LIB_PATH)
    vp, i, i64p = ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int64)
    S = ctypes.c_int
    sig = {
        "ff_default_params": (None, [ctypes.POINTER(Params)]),
        "ff_create": (S, [ctypes.POINTER(vp), ctypes.POINTER(Params), i, vp]),
        "ff_features": (S, [vp, vp, i, i, i, ctypes.POINTER(vp)]),
        "ff_features_batch": (S, [vp, i, ctypes.POINTER(Frame), ctypes.POINTER(vp)]),
        "ff_match_pair": (S, [vp, vp, vp, i, vp, vp]),
        "ff_match_batch": (S, [vp, i, ctypes.POINTER(PairJob)]),
        "ff_match_frames": (S, [vp, i, ctypes.POINTER(Frame), i, ctypes.POINTER(FrameJob), ctypes.POINTER(vp)]),
        "ff_autotune": (S, [vp, i, ctypes.POINTER(PairJob), i]),
        "ff_set_tuning": (S, [vp, i, ctypes.POINTER(Tuning)]),
        "ff_get_tuning": (S, [vp, i, ctypes.POINTER(Tuning)]),
        "ff_consistency": (S, [vp, vp, vp, i, i, i, vp]),
        "ff_sparsify": (S, [vp, vp, vp, vp, i, i, i, i, vp]),
        "ff_pyr_release": (S, [vp, vp]),
        "ff_pyr_level_dims": (S, [vp, i, ctypes.POINTER(i), ctypes.POINTER(i)]),
        "ff_pyr_features": (vp, [vp, i]),
        "ff_pyr_census": (vp, [vp, i]),
        "ff_last_error": (ctypes.c_char_p, [vp]),
        "ff_sync": (S, [vp]),
        "ff_get_stats": (S, [vp, ctypes.POINTER(Stats)]),
        "ff_profile_enable": (S, [vp, i]),
        "ff_profile_read": (S, [vp, ctypes.POINTER(ctypes.c_double), i64p]),
        "ff_profile_read_passes": (S, [vp, ctypes.POINTER(ctypes.c_double), i64p]),
        "ff_work_counts": (S, [vp, i, i, i64p, i64p]),
        "ff_match_pair_noalloc": (S, [vp, vp, vp, i, vp, vp]),
        "ff_server_create": (S, [vp, ctypes.c_int64, i, ctypes.POINTER(vp)]),
        "ff_server_submit": (S, [vp, ctypes.c_uint64, ctypes.POINTER(Request)]),
        "ff_server_step": (S, [vp, ctypes.POINTER(i), ctypes.POINTER(i)]),
        "ff_server_poll": (S, [vp, i, ctypes.POINTER(ctypes.c_uint64), i, ctypes.POINTER(i)]),
        "ff_server_stats": (S, [vp, i64p, i64p, i64p]),
        "ff_server_cancel": (S, [vp, ctypes.c_uint64]),
        "ff_server_destroy": (S, [vp]),
        "ff_set_option": (S, [vp, i, ctypes.c_int64]),
        "ff_destroy": (S, [vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def _check(ctx, status):
    if status != FF_OK:
        msg = lib().ff_last_error(ctx).decode() if ctx else ""
        raise FFError(status, msg)


# ------------------------------------------------------------------------------------------------------------
# one-to-one wrappers of the C-ABI


def ff_default_params() -> Params:
    p = Params()
    lib().ff_default_params(ctypes.byref(p))
    return p


def ff_create(params: Params, device: int = 0, stream: int | None = 0):
    ctx = ctypes.c_void_p()
    _check(None, lib().ff_create(ctypes.byref(ctx), ctypes.byref(params), device, stream or None))
    return ctx


def ff_features(ctx, rgb_dev: int, w: int, h: int, pitch_bytes: int):
    pyr = ctypes.c_void_p()
    _check(ctx, lib().ff_features(ctx, rgb_dev, w, h, pitch_bytes, ctypes.byref(pyr)))
    return pyr


def ff_features_batch(ctx, frames):
    """frames: list of (rgb_dev, w, h, pitch_bytes); returns the list of pyramid handles."""
    arr = (Frame * len(frames))(*[Frame(*f) for f in frames])
    out = (ctypes.c_void_p * len(frames))()
    _check(ctx, lib().ff_features_batch(ctx, len(frames), arr, out))
    return [ctypes.c_void_p(p) for p in out]


def ff_match_pair(ctx, a, b, dir: int, flow_dev: int, cost_dev: int | None):
    _check(ctx, lib().ff_match_pair(ctx, a, b, dir, flow_dev, cost_dev or None))


def ff_match_batch(ctx, jobs):
    arr = (PairJob * len(jobs))(*jobs)
    _check(ctx, lib().ff_match_batch(ctx, len(jobs), arr))


def ff_match_frames(ctx, frames, jobs, keep: bool = False):
    """frames: list of (rgb_dev, w, h, pitch_bytes); jobs: list of FrameJob.  Returns the pyramid handles with
    keep, else None (the pyramids are released by the call)."""
    arr = (Frame * len(frames))(*[Frame(*f) for f in frames])
    jarr = (FrameJob * len(jobs))(*jobs)
    out = (ctypes.c_void_p * len(frames))() if keep else None
    _check(ctx, lib().ff_match_frames(ctx, len(frames), arr, len(jobs), jarr, out))
    return [ctypes.c_void_p(p) for p in out] if keep else None


def ff_autotune(ctx, jobs, reps: int = 3):
    arr = (PairJob * len(jobs))(*jobs)
    _check(ctx, lib().ff_autotune(ctx, len(jobs), arr, reps))


def ff_set_tuning(ctx, level: int, cfg):
    """cfg: (tile_w, tile_h, iters_per_launch[, threads[, speculate[, cluster[, dataflow]]]]) (threads 256, the
    others 0 by default) or None to remove the override.  `level` is a pass index (s, or s + 8k for the sub-scale
    grid of stride 2^k of level s)."""
    if cfg is None:
        _check(ctx, lib().ff_set_tuning(ctx, level, None))
        return
    t = Tuning(*cfg, *((256, 0, 0, 0)[len(cfg) - 3:]))
    _check(ctx, lib().ff_set_tuning(ctx, level, ctypes.byref(t)))


def ff_get_tuning(ctx, level: int):
    """(tile_w, tile_h, iters_per_launch, threads, speculate[, cluster[, dataflow]]) in force for pass `level`:
    the optional entries are present up to the last non-zero one."""
    t = Tuning()
    _check(ctx, lib().ff_get_tuning(ctx, level, ctypes.byref(t)))
    cfg = (t.tile_w, t.tile_h, t.iters_per_launch, t.threads, t.speculate, t.cluster, t.dataflow)
    n = 7 if t.dataflow else 6 if t.cluster else 5
    return cfg[:n]


def ff_consistency(ctx, fwd: int, bwd: int, w: int, h: int, eps: int, mask_dev: int):
    _check(ctx, lib().ff_consistency(ctx, fwd, bwd, w, h, eps, mask_dev))


def ff_sparsify(ctx, fwd: int, bwd: int, keep, w: int, h: int, eps: int, min_matches: int, sparse_dev: int):
    _check(ctx, lib().ff_sparsify(ctx, fwd, bwd, keep, w, h, eps, min_matches, sparse_dev))


def ff_pyr_release(ctx, pyr):
    _check(ctx, lib().ff_pyr_release(ctx, pyr))


def ff_pyr_level_dims(pyr, level: int):
    w, h = ctypes.c_int(), ctypes.c_int()
    _check(None, lib().ff_pyr_level_dims(pyr, level, ctypes.byref(w), ctypes.byref(h)))
    return w.value, h.value


def ff_pyr_features(pyr, level: int) -> int:
    return lib().ff_pyr_features(pyr, level) or 0


def ff_pyr_census(pyr, level: int) -> int:
    return lib().ff_pyr_census(pyr, level) or 0


def ff_last_error(ctx) -> str:
    return lib().ff_last_error(ctx).decode()


def ff_sync(ctx):
    _check(ctx, lib().ff_sync(ctx))


def ff_get_stats(ctx) -> dict:
    s = Stats()
    _check(ctx, lib().ff_get_stats(ctx, ctypes.byref(s)))
    return {k: getattr(s, k) for k, _ in Stats._fields_}


def ff_profile_enable(ctx, on: bool):
    _check(ctx, lib().ff_profile_enable(ctx, 1 if on else 0))


def ff_profile_read(ctx):
    ms = (ctypes.c_double * len(PHASES))()
    n = (ctypes.c_int64 * len(PHASES))()
    _check(ctx, lib().ff_profile_read(ctx, ms, n))
    return {p: (ms[i], n[i]) for i, p in enumerate(PHASES)}


N_PASSES = 24


def ff_profile_read_passes(ctx):
    """Propagation time per pass: {pass index: (ms, launches)} for the passes that ran (level s, grid s + 8k)."""
    ms = (ctypes.c_double * N_PASSES)()
    n = (ctypes.c_int64 * N_PASSES)()
    _check(ctx, lib().ff_profile_read_passes(ctx, ms, n))
    return {i: (ms[i], n[i]) for i in range(N_PASSES) if n[i]}


def ff_work_counts(ctx, w: int, h: int):
    a, b = ctypes.c_int64(), ctypes.c_int64()
    _check(ctx, lib().ff_work_counts(ctx, w, h, ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def ff_match_pair_noalloc(ctx, a, b, dir: int, flow_dev: int, cost_dev: int | None):
    """ff_match_pair for callers that must not allocate device memory (fixed file-scope scratch)."""
    _check(ctx, lib().ff_match_pair_noalloc(ctx, a, b, dir, flow_dev, cost_dev or None))


def ff_server_create(ctx, mem_budget_bytes: int, max_active: int):
    srv = ctypes.c_void_p()
    _check(ctx, lib().ff_server_create(ctx, mem_budget_bytes, max_active, ctypes.byref(srv)))
    return srv


def ff_server_submit(ctx, srv, rid: int, req: Request):
    _check(ctx, lib().ff_server_submit(srv, rid, ctypes.byref(req)))


def ff_server_step(ctx, srv):
    a, q = ctypes.c_int(), ctypes.c_int()
    _check(ctx, lib().ff_server_step(srv, ctypes.byref(a), ctypes.byref(q)))
    return a.value, q.value


def ff_server_poll(ctx, srv, wait: bool = False, max_ids: int = 256):
    ids = (ctypes.c_uint64 * max_ids)()
    n = ctypes.c_int()
    _check(ctx, lib().ff_server_poll(srv, 1 if wait else 0, ids, max_ids, ctypes.byref(n)))
    return list(ids[: n.value])


def ff_server_cancel(ctx, srv, rid: int):
    _check(ctx, lib().ff_server_cancel(srv, rid))


def ff_server_stats(ctx, srv):
    t, l, b = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    _check(ctx, lib().ff_server_stats(srv, ctypes.byref(t), ctypes.byref(l), ctypes.byref(b)))
    return {"ticks": t.value, "launches": l.value, "bytes_in_use": b.value}


def ff_server_destroy(srv):
    _check(None, lib().ff_server_destroy(srv))


def ff_set_option(ctx, option: int, value: int):
    _check(ctx, lib().ff_set_option(ctx, option, value))


def ff_destroy(ctx):
    _check(None, lib().ff_destroy(ctx))


# ------------------------------------------------------------------------------------------------------------
# torch-facing convenience layer


def to_params(p) -> Params:
    """Accept a Params, a configs.MatchParams or any object with the same fields."""
    if isinstance(p, Params):
        return p
    return Params(p.n_scales, p.iters, getattr(p, "patch", 8), getattr(p, "n_coef", 16), p.rs_radius, p.eps,
                  p.seed & 0xFFFFFFFF, getattr(p, "rs_radius2", 4), getattr(p, "cost", FF_COST_WHT_SAD),
                  getattr(p, "sub_scales", 0))


@dataclass
class Pyramid:
    handle: ctypes.c_void_p
    w: int
    h: int


class Matcher:
    """One matching context on one device and stream; outputs are torch tensors on that device."""

    def __init__(self, params, device: int = 0, stream=None):
        import torch

        self.torch = torch
        self.device = torch.device("cuda", device)
        self.stream = stream if stream is not None else torch.cuda.Stream(device=self.device)
        self.params = to_params(params)
        self.ctx = ff_create(self.params, device, self.stream.cuda_stream)

    def close(self):
        if self.ctx:
            ff_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # interpreter shutdown: the library or CUDA may already be gone
            pass

    def _empty(self, shape, dtype):
        with self.torch.cuda.stream(self.stream):
            return self.torch.empty(shape, dtype=dtype, device=self.device)

    def _uses(self, *tensors):
        """The library reads these tensors on its stream: order that after the work already queued on the
        caller's current stream, and keep torch's allocator from reusing their memory before it has run (the
        call returns before the kernels do, so a temporary argument may be freed right away)."""
        cur = self.torch.cuda.current_stream(self.device)
        if cur != self.stream:
            self.stream.wait_stream(cur)
        for t in tensors:
            t.record_stream(self.stream)

    def features(self, img) -> Pyramid:
        """img: uint8 [h][w][3] CUDA tensor (rows may be strided)."""
        assert img.dtype == self.torch.uint8 and img.is_cuda and img.dim() == 3 and img.shape[2] == 3
        assert img.stride(2) == 1 and img.stride(1) == 3
        h, w = int(img.shape[0]), int(img.shape[1])
        self._uses(img)
        return Pyramid(ff_features(self.ctx, img.data_ptr(), w, h, img.stride(0)), w, h)

    def _frames(self, imgs):
        frames = []
        for img in imgs:
            assert img.dtype == self.torch.uint8 and img.is_cuda and img.dim() == 3 and img.shape[2] == 3
            assert img.stride(2) == 1 and img.stride(1) == 3
            frames.append((img.data_ptr(), int(img.shape[1]), int(img.shape[0]), img.stride(0)))
        self._uses(*imgs)
        return frames

    def features_batch(self, imgs) -> list:
        """Pyramids of many frames (uint8 [h][w][3] CUDA tensors of any sizes) in one launch per kernel."""
        frames = self._frames(imgs)
        hs = ff_features_batch(self.ctx, frames)
        return [Pyramid(hd, f[1], f[2]) for hd, f in zip(hs, frames)]

    def release(self, pyr: Pyramid):
        ff_pyr_release(self.ctx, pyr.handle)

    def level_features(self, pyr: Pyramid, level: int):
        """Copy of the features of one level as int16 [h][w][48] coefficients in plain row order (the library
        stores rows colour-split -- even x first, then odd x -- and coefficients in offset binary)."""
        w, h = ff_pyr_level_dims(pyr.handle, level)
        ptr = ff_pyr_features(pyr.handle, level)
        split = self._empty((h, w, 48), self.torch.int16)
        self.torch.cuda.current_stream(self.device).wait_stream(self.stream)
        src = _DevView(ptr, h * w * 96)
        split.view(-1).view(self.torch.uint8).copy_(self.torch.as_tensor(src, device=self.device))
        split.bitwise_xor_(-32768)
        return self._unsplit(split)

    def level_census(self, pyr: Pyramid, level: int):
        """Copy of the Census patterns of one level as uint64 [h][w][3] (48 bits per channel) in plain row order,
        or None when the context does not match with the Census cost."""
        w, h = ff_pyr_level_dims(pyr.handle, level)
        ptr = ff_pyr_census(pyr.handle, level)
        if not ptr:
            return None
        split = self._empty((h, w, 4), self.torch.int64)
        self.torch.cuda.current_stream(self.device).wait_stream(self.stream)
        src = _DevView(ptr, h * w * 32)
        split.view(-1).view(self.torch.uint8).copy_(self.torch.as_tensor(src, device=self.device))
        return self._unsplit(split)[:, :, :3]

    def _unsplit(self, split):
        w = split.shape[1]
        out = self.torch.empty_like(split)
        ne = (w + 1) // 2
        out[:, 0::2] = split[:, :ne]
        out[:, 1::2] = split[:, ne:]
        return out

    def match_pair(self, a: Pyramid, b: Pyramid, dir: int = 0, with_cost: bool = True):
        flow = self._empty((a.h, a.w, 2), self.torch.int16)
        cost = self._empty((a.h, a.w), self.torch.int32) if with_cost else None
        ff_match_pair(self.ctx, a.handle, b.handle, dir, flow.data_ptr(), cost.data_ptr() if cost is not None else None)
        return flow, cost

    def alloc_outputs(self, pairs, with_cost=True, second_check=False):
        outs = []
        for a, _ in pairs:
            o = {"flow_fwd": self._empty((a.h, a.w, 2), self.torch.int16),
                 "flow_bwd": self._empty((a.h, a.w, 2), self.torch.int16),
                 "mask": self._empty((a.h, a.w), self.torch.uint8)}
            if second_check:
                o["flow_bwd2"] = self._empty((a.h, a.w, 2), self.torch.int16)
            if with_cost:
                o["cost_fwd"] = self._empty((a.h, a.w), self.torch.int32)
                o["cost_bwd"] = self._empty((a.h, a.w), self.torch.int32)
            outs.append(o)
        return outs

    @staticmethod
    def _jobs(pairs, outs):
        jobs = []
        for (a, b), o in zip(pairs, outs):
            jobs.append(PairJob(a.handle, b.handle, o["flow_fwd"].data_ptr(), o["flow_bwd"].data_ptr(),
                                o["cost_fwd"].data_ptr() if "cost_fwd" in o else None,
                                o["cost_bwd"].data_ptr() if "cost_bwd" in o else None, o["mask"].data_ptr(),
                                o["flow_bwd2"].data_ptr() if "flow_bwd2" in o else None))
        return jobs

    def match_batch(self, pairs, outs=None, with_cost=True, second_check=False):
        """pairs: list of (Pyramid a, Pyramid b).  Returns (or fills) one dict of outputs per pair; with
        second_check, also the second inverse field 'flow_bwd2', and the mask applies both checks."""
        if outs is None:
            outs = self.alloc_outputs(pairs, with_cost, second_check)
        ff_match_batch(self.ctx, self._jobs(pairs, outs))
        return outs

    def match_frames(self, img_pairs, outs=None, with_cost=True, second_check=False, keep_pyramids=False):
        """Features and matching of image pairs [(a, b), ...] (uint8 [h][w][3] CUDA tensors) in one call, the fine
        levels' descriptors written beside the coarse levels' matching.  Returns (or fills) the outputs of
        match_batch; with keep_pyramids, (outputs, [(Pyramid a, Pyramid b), ...]), released by the caller."""
        frames = self._frames([x for pr in img_pairs for x in pr])
        if outs is None:
            outs = self.alloc_outputs([(Pyramid(None, f[1], f[2]), None) for f in frames[0::2]], with_cost,
                                      second_check)
        jobs = [FrameJob(2 * k, 2 * k + 1, o["flow_fwd"].data_ptr(), o["flow_bwd"].data_ptr(),
                         o["cost_fwd"].data_ptr() if "cost_fwd" in o else None,
                         o["cost_bwd"].data_ptr() if "cost_bwd" in o else None, o["mask"].data_ptr(),
                         o["flow_bwd2"].data_ptr() if "flow_bwd2" in o else None) for k, o in enumerate(outs)]
        hs = ff_match_frames(self.ctx, frames, jobs, keep_pyramids)
        if not keep_pyramids:
            return outs
        pyrs = [Pyramid(hd, f[1], f[2]) for hd, f in zip(hs, frames)]
        return outs, list(zip(pyrs[0::2], pyrs[1::2]))

    def autotune(self, pairs, outs=None, reps=3):
        """Tune the per-level propagation configuration for batches shaped like `pairs` (outputs overwritten)."""
        if outs is None:
            outs = self.alloc_outputs(pairs, with_cost=False)
        ff_autotune(self.ctx, self._jobs(pairs, outs), reps)
        return [ff_get_tuning(self.ctx, s) for s in range(self.params.n_scales)]

    def consistency(self, fwd, bwd, eps: int):
        h, w = int(fwd.shape[0]), int(fwd.shape[1])
        mask = self._empty((h, w), self.torch.uint8)
        self._uses(fwd, bwd)
        ff_consistency(self.ctx, fwd.data_ptr(), bwd.data_ptr(), w, h, eps, mask.data_ptr())
        return mask

    def sparsify(self, fwd, bwd, eps: int, min_matches: int, keep=None):
        """keep: optional uint8 [h][w] CUDA mask of the matches the consistency checks left (e.g. the 'mask' of
        match_batch with second_check); None counts every match that passes the check against bwd."""
        h, w = int(fwd.shape[0]), int(fwd.shape[1])
        out = self._empty((h, w), self.torch.uint8)
        if keep is not None:
            assert keep.dtype == self.torch.uint8 and keep.is_cuda and keep.is_contiguous() and keep.numel() == h * w
            self._uses(fwd, bwd, keep)
        else:
            self._uses(fwd, bwd)
        ff_sparsify(self.ctx, fwd.data_ptr(), bwd.data_ptr(), keep.data_ptr() if keep is not None else None, w, h, eps,
                    min_matches, out.data_ptr())
        return out

    def sync(self):
        ff_sync(self.ctx)

    def stats(self):
        return ff_get_stats(self.ctx)


class _DevView:
    """Minimal __cuda_array_interface__ over a device pointer owned by the library (read-only bytes)."""

    def __init__(self, ptr: int, nbytes: int):
        self.__cuda_array_interface__ = {"shape": (nbytes,), "typestr": "|u1", "data": (ptr, False), "version": 3,
                                         "strides": None}


class Server:
    """Continuous-batching server on a Matcher's context (requests reference caller-owned device tensors)."""

    def __init__(self, matcher: Matcher, mem_budget_bytes: int = 60 << 30, max_active: int = 256):
        self.m = matcher
        self.srv = ff_server_create(matcher.ctx, mem_budget_bytes, max_active)
        self.keep = {}

    def submit(self, rid: int, img_a, img_b, out: dict):
        """img_a/img_b: uint8 [h][w][3] CUDA tensors; out: dict with flow_fwd, flow_bwd, mask (and optionally
        cost_fwd, cost_bwd) CUDA tensors.  All must stay alive until `rid` is reported by poll()."""
        h, w = int(img_a.shape[0]), int(img_a.shape[1])
        req = Request(img_a.data_ptr(), img_b.data_ptr(), w, h, img_a.stride(0), out["flow_fwd"].data_ptr(),
                      out["flow_bwd"].data_ptr(), out["cost_fwd"].data_ptr() if "cost_fwd" in out else None,
                      out["cost_bwd"].data_ptr() if "cost_bwd" in out else None, out["mask"].data_ptr())
        ff_server_submit(self.m.ctx, self.srv, rid, req)
        self.keep[rid] = (img_a, img_b, out)

    def step(self):
        return ff_server_step(self.m.ctx, self.srv)

    def poll(self, wait=False):
        ids = ff_server_poll(self.m.ctx, self.srv, wait)
        for i in ids:
            self.keep.pop(i, None)
        return ids

    def stats(self):
        return ff_server_stats(self.m.ctx, self.srv)

    def cancel(self, rid: int):
        """Withdraw a request that has not been admitted yet (FFError FF_ERR_BUSY once it has)."""
        ff_server_cancel(self.m.ctx, self.srv, rid)
        self.keep.pop(rid, None)

    def close(self):
        if self.srv:
            ff_server_destroy(self.srv)
            self.srv = None
