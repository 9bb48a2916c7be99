"""Continuous batching: requests of different sizes are admitted while others are on the GPU, share merged
launches with them, and each result is bit-identical to matching that pair alone (tolerance zero: the whole
stage is integer).  One request of each size is also checked against the oracle."""
import numpy as np
import pytest

import oracle
from paper_1805_03517_gb300 import configs
from tests import gpu_helpers as G
from tests import oracle_pins as P

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


def _pair(i, h, w):
    a = P.smooth_texture(1000 + i, h, w)
    b = P.shifted(a, (i % 7) - 3, (i % 5) - 2, 2000 + i)
    b[h // 3:h // 2, w // 4:w // 2] = P.smooth_texture(3000 + i, h // 2 - h // 3, w // 2 - w // 4)
    return a, b


def _outputs(M, h, w):
    with torch.cuda.stream(M.stream):
        return {"flow_fwd": torch.full((h, w, 2), -9, dtype=torch.int16, device="cuda"),
                "flow_bwd": torch.full((h, w, 2), -9, dtype=torch.int16, device="cuda"),
                "cost_fwd": torch.full((h, w), -9, dtype=torch.int32, device="cuda"),
                "cost_bwd": torch.full((h, w), -9, dtype=torch.int32, device="cuda"),
                "mask": torch.full((h, w), 9, dtype=torch.uint8, device="cuda")}


def test_served_mix_equals_alone(ffm):
    prm = configs.MatchParams(n_scales=4, iters=3, eps=1)
    M = ffm.Matcher(prm, 0)
    sizes = [(96, 128), (60, 90), (120, 200), (96, 128), (33, 47), (120, 200), (60, 90), (80, 80)]
    pairs = [_pair(i, h, w) for i, (h, w) in enumerate(sizes)]
    dev = [(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()) for a, b in pairs]
    torch.cuda.synchronize()
    # alone: each pair through ff_match_batch by itself
    alone = []
    for da, db in dev:
        pa, pb = M.features(da), M.features(db)
        o = M.match_batch([(pa, pb)])[0]
        M.sync()
        alone.append(tuple(o[k].cpu().numpy() for k in NAMES))
        M.release(pa)
        M.release(pb)
    # served: staggered arrivals, later requests join while earlier ones are mid-flight
    S = ffm.Server(M, mem_budget_bytes=1 << 30, max_active=5)
    outs, done, order = {}, [], []
    nxt = 0
    for step in range(400):
        if nxt < len(dev) and step % 3 == 0:
            h, w = sizes[nxt]
            outs[nxt] = _outputs(M, h, w)
            S.submit(nxt, dev[nxt][0], dev[nxt][1], outs[nxt])
            nxt += 1
        n_active, n_queued = S.step()
        done += S.poll()
        if nxt == len(dev) and len(done) == len(dev):
            break
    while len(done) < len(dev):
        S.step()
        done += S.poll(wait=True)
    assert sorted(done) == list(range(len(dev)))
    st = S.stats()
    assert st["ticks"] > 0 and st["bytes_in_use"] == 0
    M.sync()
    for i in range(len(dev)):
        G.assert_same(tuple(outs[i][k].cpu().numpy() for k in NAMES), alone[i])
    o = oracle.default()
    for i in (0, 1, 2, 4):
        a, b = pairs[i]
        G.assert_same(alone[i], o.match_bidir(a, b, G.oracle_params(prm)))
    S.close()
    M.close()


def test_server_rejects_and_bounds(ffm):
    prm = configs.MatchParams(n_scales=3, iters=2, eps=1)
    M = ffm.Matcher(prm, 0)
    S = ffm.Server(M, mem_budget_bytes=4 << 20, max_active=2)
    big = torch.zeros((600, 800, 3), dtype=torch.uint8, device="cuda")
    out = _outputs(M, 600, 800)
    with pytest.raises(ffm.FFError) as e:  # can never fit the 4 MiB budget
        S.submit(1, big, big, out)
    assert e.value.status == ffm.FF_ERR_ARG
    small = [_pair(50 + i, 40, 48) for i in range(4)]
    dev = [(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()) for a, b in small]
    outs = [_outputs(M, 40, 48) for _ in dev]
    for i, (da, db) in enumerate(dev):
        S.submit(10 + i, da, db, outs[i])
    n_active, n_queued = S.step()
    assert n_active <= 2 and n_active + n_queued == 4
    done = []
    while len(done) < 4:
        S.step()
        done += S.poll(wait=True)
    assert sorted(done) == [10, 11, 12, 13]
    S.close()
    M.close()


def test_many_in_flight_one_chunk_per_tick(ffm):
    """More requests in flight than the whole-level threshold: ticks advance one chunk per request (and switch
    to whole levels once few are left); every result equals matching the pair alone."""
    prm = configs.MatchParams(n_scales=3, iters=3, eps=1)
    M = ffm.Matcher(prm, 0)
    sizes = [(40 + 4 * i, 56 + 6 * i) for i in range(14)]
    pairs = [_pair(600 + i, h, w) for i, (h, w) in enumerate(sizes)]
    dev = [(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()) for a, b in pairs]
    torch.cuda.synchronize()
    alone = []
    for da, db in dev:
        pa, pb = M.features(da), M.features(db)
        o = M.match_batch([(pa, pb)])[0]
        M.sync()
        alone.append(tuple(o[k].cpu().numpy() for k in NAMES))
        M.release(pa)
        M.release(pb)
    S = ffm.Server(M, mem_budget_bytes=1 << 30, max_active=14)
    outs = {i: _outputs(M, h, w) for i, (h, w) in enumerate(sizes)}
    for i in range(len(sizes)):
        S.submit(i, dev[i][0], dev[i][1], outs[i])
    done = []
    while len(done) < len(sizes):
        S.step()
        done += S.poll(wait=True)
    M.sync()
    for i in range(len(sizes)):
        G.assert_same(tuple(outs[i][k].cpu().numpy() for k in NAMES), alone[i])
    S.close()
    M.close()


def test_served_workload_sizes_against_the_oracle(ffm):
    """Requests of every size of the served workload (320x240, 640x480, 1024x436, 1242x375; L=5, T=6, eps=1)
    through the server, twelve in flight at once, so that ticks advance one chunk per request with the launch
    configurations tuned for eight pairs per launch; every result equals the oracle's."""
    from paper_1805_03517_gb300 import synth

    prm = configs.KITTI
    M = ffm.Matcher(prm, 0)
    specs = [(w, h, kind, 7000 + 10 * k + j) for k, (w, h, kind) in enumerate(configs.SERVE_SIZES) for j in range(3)]
    pairs = [synth.make_pair(kind, seed, w, h)[:2] for (w, h, kind, seed) in specs]
    dev = [(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()) for a, b in pairs]
    torch.cuda.synchronize()
    for k in range(len(configs.SERVE_SIZES)):  # launch configurations for many pairs per launch, per size
        group = dev[3 * k:3 * k + 3] * 3  # eight or more pairs of one size
        pyrs = [(M.features(a), M.features(b)) for a, b in group[:8]]
        M.autotune(pyrs, reps=1)
        for pa, pb in pyrs:
            M.release(pa)
            M.release(pb)
    S = ffm.Server(M, mem_budget_bytes=60 << 30, max_active=len(dev))
    outs = {i: _outputs(M, h, w) for i, (w, h, _, _) in enumerate(specs)}
    for i in range(len(dev)):
        S.submit(i, dev[i][0], dev[i][1], outs[i])
    n_active, _ = S.step()
    assert n_active > 8
    done = []
    while len(done) < len(dev):
        S.step()
        done += S.poll(wait=True)
    M.sync()
    want = G.oracle_bidir_many(pairs, prm)
    for i, (w, h, _, _) in enumerate(specs):
        try:
            G.assert_same(tuple(outs[i][k].cpu().numpy() for k in NAMES), want[i])
        except AssertionError as e:
            raise AssertionError(f"request {i} ({w}x{h}): {e}") from None
    S.close()
    M.close()


def test_served_mix_in_the_dataflow_form_equals_the_oracle(ffm):
    """Passes configured in the dataflow form (levels and sub-scale grids) run through the server as one chunk
    each, their problems merged across requests; each pair equals the oracle."""
    import dataclasses

    prm = dataclasses.replace(configs.MatchParams(n_scales=3, iters=3, eps=1), sub_scales=1)
    sizes = [(60, 90), (97, 131), (33, 47), (60, 90), (80, 80), (45, 70)]
    pairs = [_pair(2100 + i, h, w) for i, (h, w) in enumerate(sizes)]
    M = ffm.Matcher(prm, 0)
    for p in (0, 1, 2, 8, 9):  # the dataflow form, its affine variant at levels 1 and 2
        ffm.ff_set_tuning(M.ctx, p, (16, 8, 1, 256, 0, 0, 2 if p in (1, 2) else 1))
    dev = [(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()) for a, b in pairs]
    torch.cuda.synchronize()
    S = ffm.Server(M, mem_budget_bytes=1 << 30, max_active=12)
    outs = {i: _outputs(M, h, w) for i, (h, w) in enumerate(sizes)}
    done, nxt = [], 0
    for step in range(2000):
        if nxt < len(dev):
            S.submit(nxt, dev[nxt][0], dev[nxt][1], outs[nxt])
            nxt += 1
        S.step()
        done += S.poll()
        if len(done) == len(dev):
            break
    while len(done) < len(dev):
        S.step()
        done += S.poll(wait=True)
    M.sync()  # also reports an expired wait
    got = [tuple(outs[i][k].cpu().numpy() for k in NAMES) for i in range(len(dev))]
    want = G.oracle_bidir_many(pairs, prm)
    for i in range(len(dev)):
        G.assert_same(got[i], want[i])
    S.close()
    M.close()
