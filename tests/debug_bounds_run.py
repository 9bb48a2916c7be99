"""Run by tests/test_gpu_failures.py in a child process whose FF_LIBRARY points at the debug-bounds build of
libff: small parity cases against the oracle (plain, sub-scale grids, Census cost, the cluster and dataflow
forms of the propagation on levels and grids, two consistency checks and sparsification, a 1x1 and a
1-pixel-high frame), each followed by ff_sync, which fails if any index check of the propagation, hand-over or
filter kernels recorded a violation.  Prints "debug-bounds ok" at the end."""
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import torch  # noqa: E402

from paper_1805_03517_gb300 import configs, ff, synth  # noqa: E402
from tests import gpu_helpers as G  # noqa: E402
from tests import oracle_pins as P  # noqa: E402

import oracle  # noqa: E402

assert ff.LIB_PATH.endswith("libff_debug.so"), ff.LIB_PATH
o = oracle.default()
cases = [(configs.SMALL, synth.make_pair("rects", 1000, 128, 96)[:2])]
a = P.smooth_texture(77, 61, 45)
b = P.shifted(a, 3, -2, 78)
cases.append((configs.MatchParams(n_scales=3, iters=3, sub_scales=2), (a, b)))
cases.append((configs.MatchParams(n_scales=3, iters=2, cost=1), (a, b)))
cases.append((configs.MatchParams(n_scales=1, iters=2), (P.rand_img(5, 1, 1), P.rand_img(6, 1, 1))))
cases.append((configs.MatchParams(n_scales=2, iters=2), (P.rand_img(7, 1, 37), P.rand_img(8, 1, 37))))
# the cluster form on every level and grid pass (16, 6 and 1 CTAs per problem: 4x4, 3x2 / 2x3 and 1x1 blocks)
CLUSTER = {0: (0, 0, 3, 256, 0, 16), 1: (0, 0, 2, 512, 0, 6), 2: (0, 0, 3, 256, 0, 1), 8: (0, 0, 3, 512, 0, 6),
           16: (0, 0, 1, 256, 0, 16), 9: (0, 0, 3, 256, 0, 16), 17: (0, 0, 3, 512, 0, 4)}
cases.append((configs.MatchParams(n_scales=3, iters=3, sub_scales=2), (a, b), CLUSTER))
cases.append((configs.MatchParams(n_scales=3, iters=2, cost=1), (a, b), CLUSTER))
# the dataflow form on every level and grid pass (ragged tiles, 128 to 512 threads)
DATAFLOW = {p_: ((7, 5), (16, 8), (4, 4))[i % 3] + (1, (128, 256, 512)[i % 3], 0, 0, 1)
            for i, p_ in enumerate((0, 1, 2, 8, 9, 16, 17))}
cases.append((configs.MatchParams(n_scales=3, iters=3, sub_scales=2), (a, b), DATAFLOW))
for prm, (img_a, img_b), *tuning in cases:
    M = ff.Matcher(prm, 0)
    for p_, cfg in (tuning[0] if tuning else {}).items():
        ff.ff_set_tuning(M.ctx, p_, cfg)
    c0 = M.stats()["cluster_launches"]
    got = G.gpu_bidir(M, img_a, img_b, torch)  # ends with ff_sync: raises on a recorded violation
    assert (M.stats()["cluster_launches"] > c0) == (bool(tuning) and tuning[0] is CLUSTER)
    G.assert_same(got, o.match_bidir(img_a, img_b, G.oracle_params(prm)))
    M.close()
# two consistency checks and sparsification (Table 3, KITTI s)
prm = configs.MatchParams(n_scales=3, iters=2, eps=1)
M = ff.Matcher(prm, 0)
ta, tb = torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()
torch.cuda.synchronize()
pa, pb = M.features(ta), M.features(tb)
out = M.match_batch([(pa, pb)], second_check=True)[0]
sp = M.sparsify(out["flow_fwd"], out["flow_bwd"], 1, 7, keep=out["mask"])
M.sync()
ff_, fb_, fb2_, mask_ = o.match_bidir2(a, b, G.oracle_params(prm), prm.rs_radius2)
assert np.array_equal(out["mask"].cpu().numpy(), mask_)
assert np.array_equal(sp.cpu().numpy(), o.sparsify(ff_, fb_, 1, 7, mask_))
M.close()
print("debug-bounds ok")
