"""The batched workload (48 pairs of three sizes in merged launches, replayed from a graph): every pair's
output equals matching it alone and equals the oracle, bit for bit (the oracle runs on the host cores)."""
import pytest

from paper_1805_03517_gb300 import configs, synth
from tests import gpu_helpers as G

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

NAMES = ("flow_fwd", "flow_bwd", "cost_fwd", "cost_bwd", "mask")


@pytest.fixture(scope="module")
def ffm():
    from paper_1805_03517_gb300 import build, ff

    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return ff


def test_batch48_equals_alone_and_oracle(ffm):
    wl = configs.workload("batch48_mixed")
    prm = wl.pairs[0].params
    assert all(p.params == prm for p in wl.pairs)
    imgs = [synth.make_pair(p.kind, p.seed, p.w, p.h)[:2] for p in wl.pairs]
    M = ffm.Matcher(prm, 0)
    dev = [(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()) for a, b in imgs]
    torch.cuda.synchronize()
    pyrs = [(M.features(a), M.features(b)) for a, b in dev]
    M.autotune(pyrs, reps=1)  # the launch configuration the benchmark uses
    outs = M.match_batch(pyrs)
    outs = M.match_batch(pyrs, outs=outs)  # replayed from the captured graph
    M.sync()
    got = [tuple(o[k].cpu().numpy() for k in NAMES) for o in outs]
    for i, pp in enumerate(pyrs):
        alone = M.match_batch([pp])[0]
        M.sync()
        G.assert_same(got[i], tuple(alone[k].cpu().numpy() for k in NAMES))
    want = G.oracle_bidir_many(imgs, prm)
    for i in range(len(imgs)):
        try:
            G.assert_same(got[i], want[i])
        except AssertionError as e:
            raise AssertionError(f"pair {i} ({wl.pairs[i].w}x{wl.pairs[i].h}): {e}") from None
    for pa, pb in pyrs:
        M.release(pa)
        M.release(pb)
    M.close()
