"""The C-ABI library builds, loads without a GPU and exports every function include/ff.h declares.

No compute call is made here: only parameter validation, which returns before any CUDA work.
"""
import ctypes
import os

import pytest

from paper_1805_03517_gb300 import build as B
from paper_1805_03517_gb300 import ff


@pytest.fixture(scope="module")
def L():
    B.build()
    return ff.lib()


def test_exports_every_declared_symbol(L):
    names = ff.header_functions()
    assert len(names) >= 16
    for n in ("ff_create", "ff_features", "ff_match_pair", "ff_match_batch", "ff_consistency", "ff_destroy"):
        assert n in names
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


def test_binding_wraps_every_declared_symbol():
    for n in ff.header_functions():
        assert callable(getattr(ff, n, None)), n


def test_default_params(L):
    p = ff.ff_default_params()
    assert (p.n_scales, p.iters, p.patch, p.n_coef, p.rs_radius, p.eps, p.seed, p.rs_radius2, p.cost) == \
        (5, 6, 8, 16, 2, 1, 0x20180503, 4, ff.FF_COST_WHT_SAD)


@pytest.mark.parametrize("field,value", [("n_scales", 0), ("n_scales", 9), ("iters", 0), ("iters", 256),
                                         ("patch", 7), ("n_coef", 12), ("rs_radius", -1), ("rs_radius", 17),
                                         ("eps", -1), ("rs_radius2", -1), ("rs_radius2", 17), ("cost", -1),
                                         ("cost", 2)])
def test_create_rejects_bad_params(L, field, value):
    p = ff.ff_default_params()
    setattr(p, field, value)
    ctx = ctypes.c_void_p()
    assert L.ff_create(ctypes.byref(ctx), ctypes.byref(p), 0, None) == ff.FF_ERR_ARG
    assert not ctx.value


def test_null_arguments(L):
    assert L.ff_create(None, None, 0, None) == ff.FF_ERR_ARG
    assert L.ff_sync(None) == ff.FF_ERR_ARG
    assert L.ff_destroy(None) == ff.FF_ERR_ARG
    assert L.ff_pyr_level_dims(None, 0, None, None) == ff.FF_ERR_ARG
    assert not L.ff_pyr_features(None, 0)


def test_library_is_in_tree():
    assert os.path.commonpath([ff.LIB_PATH, os.path.dirname(ff.__file__)]) == os.path.dirname(ff.__file__)


def test_tuned_table_is_well_formed():
    """The package table of tuned launch configurations: one valid [tile_w, tile_h, iterations per launch,
    threads, speculate[, cluster[, dataflow]]] per level of each listed workload, in the tile, cluster or
    dataflow form."""
    import json

    from paper_1805_03517_gb300 import configs

    table = json.load(open(os.path.join(os.path.dirname(ff.__file__), "tuned.json")))
    names = [k for k in table if k != "note"]
    assert names and all(k in configs.WORKLOADS for k in names)
    for name in names:
        prm = configs.workload(name).pairs[0].params
        assert len(table[name]) == prm.n_scales
        for cfg in table[name]:
            tw, th, k, threads, spec, cluster, dataflow = list(cfg) + [0] * (7 - len(cfg))
            assert 5 <= len(cfg) <= 7 and 1 <= k <= prm.iters and threads in (128, 256, 512) and spec in (0, 1)
            if cluster:  # the cluster form: no tiles, no speculation
                assert tw == th == 0 and 1 <= cluster <= 16 and threads in (256, 512) and spec == 0 and not dataflow
            elif dataflow:  # the dataflow form: one iteration per tile task, tiles of at least 4 x 4
                assert dataflow in (1, 2) and k == 1 and tw >= 4 and th >= 4 and spec == 0
            else:
                assert tw >= 1 and th >= 1
