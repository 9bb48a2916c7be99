"""Helpers of the GPU tests: run the CUDA path through the C-ABI and the oracle on the same seeded inputs."""
from __future__ import annotations

import numpy as np

import oracle


def oracle_params(p):
    return oracle.params(p.n_scales, p.iters, p.rs_radius, p.eps, p.seed, getattr(p, "cost", 0),
                         getattr(p, "sub_scales", 0))


def gpu_bidir(M, img_a, img_b, torch):
    """Features of both frames + one batched job (fwd, bwd, consistency) through the C-ABI; numpy results."""
    ta = torch.from_numpy(np.ascontiguousarray(img_a)).to(M.device)
    tb = torch.from_numpy(np.ascontiguousarray(img_b)).to(M.device)
    torch.cuda.current_stream(M.device).synchronize()
    pa, pb = M.features(ta), M.features(tb)
    out = M.match_batch([(pa, pb)])[0]
    M.sync()
    res = tuple(out[k].cpu().numpy() for k in ("flow_fwd", "flow_bwd", "cost_fwd", "cost_bwd", "mask"))
    M.release(pa)
    M.release(pb)
    return res


def assert_same(got, want, names=("flow_fwd", "flow_bwd", "cost_fwd", "cost_bwd", "mask")):
    for g, w, n in zip(got, want, names):
        assert g.shape == w.shape, (n, g.shape, w.shape)
        if not np.array_equal(g, w):
            bad = np.argwhere(g != w)
            raise AssertionError(f"{n}: {len(bad)} mismatches, first at {bad[0].tolist()}: "
                                 f"gpu {g[tuple(bad[0])]} oracle {w[tuple(bad[0])]}")


def _oracle_bidir_task(args):
    img_a, img_b, prm = args
    return oracle.default().match_bidir(img_a, img_b, oracle.params(*prm))


def oracle_bidir_many(pairs, p):
    """The oracle's whole stage for many pairs on the host cores (one single-threaded oracle per process).  The
    pool is started with 'spawn': a process forked after CUDA has been initialised can hang."""
    import multiprocessing as mp
    import os

    oracle.build()
    prm = (p.n_scales, p.iters, p.rs_radius, p.eps, p.seed, getattr(p, "cost", 0), getattr(p, "sub_scales", 0))
    tasks = [(np.ascontiguousarray(a), np.ascontiguousarray(b), prm) for a, b in pairs]
    n = max(1, min(len(tasks), os.cpu_count() or 1))
    with mp.get_context("spawn").Pool(n) as pool:
        return pool.map(_oracle_bidir_task, tasks, chunksize=1)
