"""Failure paths, exercised on the host side only (nothing faults, traps or hangs the GPU):
  * out of memory: FF_OPT_TEST_FAIL_ALLOCS makes the next device allocations of a context fail as on an
    exhausted device; ff_features, ff_match_batch and the server's admission report FF_ERR_OOM, launch nothing,
    and the same context afterwards matches bit for bit as if nothing had happened;
  * withdrawal: ff_server_cancel removes a queued request (never reported), refuses an admitted one;
  * the debug-bounds build (every gather and shared-memory index of the propagation, hand-over and filter kernels
    checked, the first violation recorded, nothing trapped) runs parity cases with its record clear.
The bounded device-side waits are tested in tests/test_gpu_seed.py."""
import os
import subprocess
import sys

import pytest

from paper_1805_03517_gb300 import configs
from tests import gpu_helpers as G
from tests import oracle_pins as P

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

NAMES = ("flow_fwd", "flow_bwd", "cost_fwd", "cost_bwd", "mask")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def ffm():
    from paper_1805_03517_gb300 import build, ff

    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return ff


def _pair(seed, h, w):
    a = P.smooth_texture(seed, h, w)
    b = P.shifted(a, 4, -3, seed + 1)
    return a, b


def test_forced_allocation_failures_report_oom_and_the_context_recovers(ffm, orc):
    prm = configs.MatchParams(n_scales=3, iters=2, eps=1)
    M = ffm.Matcher(prm, 0)
    a, b = _pair(1400, 70, 90)
    ta, tb = torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()
    torch.cuda.synchronize()
    held = M.stats()["scratch_bytes"]
    ffm.ff_set_option(M.ctx, ffm.FF_OPT_TEST_FAIL_ALLOCS, 1)
    with pytest.raises(ffm.FFError) as e:  # a new pyramid size needs an allocation
        M.features(ta)
    assert e.value.status == ffm.FF_ERR_OOM
    assert M.stats()["scratch_bytes"] == held
    pa, pb = M.features(ta), M.features(tb)  # the failure count is used up
    ffm.ff_set_option(M.ctx, ffm.FF_OPT_TEST_FAIL_ALLOCS, 1)
    with pytest.raises(ffm.FFError) as e:  # a new plan needs its scratch
        M.match_batch([(pa, pb)])
    assert e.value.status == ffm.FF_ERR_OOM
    out = M.match_batch([(pa, pb)])[0]
    M.sync()
    G.assert_same(tuple(out[k].cpu().numpy() for k in NAMES), orc.match_bidir(a, b, G.oracle_params(prm)))
    M.release(pa)
    M.release(pb)
    M.close()


def _outputs(M, h, w):
    with torch.cuda.stream(M.stream):
        return {"flow_fwd": torch.full((h, w, 2), -9, dtype=torch.int16, device="cuda"),
                "flow_bwd": torch.full((h, w, 2), -9, dtype=torch.int16, device="cuda"),
                "cost_fwd": torch.full((h, w), -9, dtype=torch.int32, device="cuda"),
                "cost_bwd": torch.full((h, w), -9, dtype=torch.int32, device="cuda"),
                "mask": torch.full((h, w), 9, dtype=torch.uint8, device="cuda")}


def test_server_admission_out_of_memory_and_cancel(ffm, orc):
    prm = configs.MatchParams(n_scales=3, iters=2, eps=1)
    M = ffm.Matcher(prm, 0)
    sizes = [(64, 80), (52, 70), (64, 80)]
    pairs = [_pair(1500 + i, h, w) for i, (h, w) in enumerate(sizes)]
    dev = [(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()) for a, b in pairs]
    torch.cuda.synchronize()
    S = ffm.Server(M, mem_budget_bytes=1 << 30, max_active=1)
    outs = {i: _outputs(M, h, w) for i, (h, w) in enumerate(sizes)}
    for i in range(3):
        S.submit(i, dev[i][0], dev[i][1], outs[i])
    ffm.ff_set_option(M.ctx, ffm.FF_OPT_TEST_FAIL_ALLOCS, 1)
    with pytest.raises(ffm.FFError) as e:  # admitting request 0 needs its pyramids
        S.step()
    assert e.value.status == ffm.FF_ERR_OOM
    n_active, n_queued = S.step()  # the request stayed queued and is admitted now
    assert (n_active, n_queued) == (1, 2)
    S.cancel(1)  # still queued: withdrawn
    with pytest.raises(ffm.FFError) as e:
        S.cancel(0)  # admitted
    assert e.value.status == ffm.FF_ERR_BUSY
    with pytest.raises(ffm.FFError) as e:
        S.cancel(99)
    assert e.value.status == ffm.FF_ERR_ARG
    done = []
    for _ in range(1000):
        S.step()
        done += S.poll(wait=True)
        if len(done) == 2:
            break
    assert sorted(done) == [0, 2]
    assert S.stats()["bytes_in_use"] == 0
    M.sync()
    for i in (0, 2):
        a, b = pairs[i]
        G.assert_same(tuple(outs[i][k].cpu().numpy() for k in NAMES), orc.match_bidir(a, b, G.oracle_params(prm)))
    assert int(outs[1]["mask"].max().item()) == 9  # the withdrawn request's outputs were never written
    S.close()
    M.close()


def test_debug_bounds_build_runs_clean(ffm):
    from paper_1805_03517_gb300 import build as B

    lib = B.build(extra_flags=["-DFF_DEBUG_BOUNDS=1"], lib_path=os.path.join(B.LIBDIR, "libff_debug.so"),
                  build_dir=os.path.join(B.PKG, "_build_debug"))
    env = dict(os.environ, FF_LIBRARY=lib)
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "debug_bounds_run.py")], env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert "debug-bounds ok" in r.stdout
