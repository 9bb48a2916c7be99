"""The initial matches on the tcgen05 tensor cores (TMA-fed, f32 accumulators in tensor memory) and on mma.sync
give the exact nearest neighbour of the oracle, ties included, at coarsest-level sizes on both sides of the
128-row and 256-column tile edges; and the tensor-core kernel's bounded waits report an expiry instead of
hanging, leaving the context usable."""
import numpy as np
import pytest

import oracle
from paper_1805_03517_gb300 import configs
from tests import gpu_helpers as G
from tests import oracle_pins as P

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

SIZES = [(1, 1), (1, 7), (10, 10), (127, 1), (8, 16), (3, 43), (15, 17), (16, 16), (1, 257), (20, 30), (23, 77)]


@pytest.fixture(scope="module")
def ffm():
    from paper_1805_03517_gb300 import build, ff

    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return ff


def _run(ffm, kernel, a, b, prm):
    M = ffm.Matcher(prm, 0)
    ffm.ff_set_option(M.ctx, ffm.FF_OPT_SEED_KERNEL, kernel)
    got = G.gpu_bidir(M, a, b, torch)
    M.close()
    return got


@pytest.mark.parametrize("h,w", SIZES)
def test_seed_kernels_equal_oracle(ffm, h, w):
    prm = configs.MatchParams(n_scales=1, iters=1, eps=1)
    a = P.rand_img(700 + h * 31 + w, h, w)
    b = P.rand_img(800 + h * 37 + w, h, w)
    want = oracle.default().match_bidir(a, b, G.oracle_params(prm))
    for kernel in (ffm.FF_SEED_TCGEN05, ffm.FF_SEED_MMA_SYNC):
        G.assert_same(_run(ffm, kernel, a, b, prm), want)


def test_seed_ties_take_the_first_index(ffm):
    prm = configs.MatchParams(n_scales=1, iters=1, eps=1)
    a = np.full((23, 77, 3), 60, np.uint8)
    b = np.full((23, 77, 3), 60, np.uint8)
    b[:, 40:] = P.rand_img(5, 23, 37)  # the flat left part of frame 2 ties for every flat source pixel
    want = oracle.default().match_bidir(a, b, G.oracle_params(prm))
    for kernel in (ffm.FF_SEED_TCGEN05, ffm.FF_SEED_MMA_SYNC):
        G.assert_same(_run(ffm, kernel, a, b, prm), want)


def test_bounded_wait_reports_expiry_and_context_recovers(ffm):
    prm = configs.MatchParams(n_scales=2, iters=1, eps=1)
    a = P.smooth_texture(11, 40, 56)
    b = P.shifted(a, 2, 1, 12)
    M = ffm.Matcher(prm, 0)
    ffm.ff_set_option(M.ctx, ffm.FF_OPT_WAIT_LIMIT, 2000)
    ffm.ff_set_option(M.ctx, ffm.FF_OPT_TEST_WITHHOLD_COPIES, 1)  # nothing will ever complete the load barrier
    ta, tb = torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()
    torch.cuda.synchronize()
    pa, pb = M.features(ta), M.features(tb)
    M.match_batch([(pa, pb)])
    with pytest.raises(ffm.FFError) as e:
        M.sync()
    assert e.value.status == ffm.FF_ERR_TIMEOUT
    M.release(pa)
    M.release(pb)
    ffm.ff_set_option(M.ctx, ffm.FF_OPT_TEST_WITHHOLD_COPIES, 0)
    ffm.ff_set_option(M.ctx, ffm.FF_OPT_WAIT_LIMIT, 1 << 22)
    got = G.gpu_bidir(M, a, b, torch)  # the same context still works and is exact
    G.assert_same(got, oracle.default().match_bidir(a, b, G.oracle_params(prm)))
    M.close()
