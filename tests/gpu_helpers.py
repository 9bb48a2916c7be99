"""Helpers of the GPU tests: run the CUDA path through the C-ABI and the oracle on the same seeded inputs."""
from __future__ import annotations

import numpy as np

import oracle


def oracle_params(p):
    return oracle.params(p.n_scales, p.iters, p.rs_radius, p.eps, p.seed, getattr(p, "cost", 0))


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
