"""CPU-side checks of the C ABI: the library builds, loads without a GPU and
exports every entry point declared in include/dscreen.h; host-side argument
checks reject bad input before touching the GPU."""
import ctypes

import numpy as np

import paper_1412_4080_gb300 as ds


def test_library_exports_every_declared_symbol():
    L = ds.lib()
    names = ds.declared_functions()
    assert "ds_solve" in names and "ds_dict_create" in names and "ds_lambda_max" in names
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


def test_status_strings():
    for code, name in enumerate(["DS_OK", "DS_ERR_INVALID", "DS_ERR_OOM", "DS_ERR_CUDA", "DS_ERR_TIMEOUT",
                                 "DS_ERR_NOT_CONVERGED", "DS_ERR_UNSUPPORTED"]):
        assert ds.ds_status_str(code) == name


def test_options_default_and_null_checks():
    o = ds.ds_options_default()
    assert o.alg == ds.DS_FISTA and o.test == ds.DS_DST3 and o.dynamic == 1 and o.max_iter > 0
    L = ds.lib()
    assert L.ds_options_default(None) == ds.DS_ERR_INVALID
    assert L.ds_create(0, None, None) == ds.DS_ERR_INVALID
    assert L.ds_destroy(None) == ds.DS_OK
    assert L.ds_dict_destroy(None) == ds.DS_OK
    assert L.ds_set_history(None, None, 0) == ds.DS_ERR_INVALID
    r = ds.ds_result()
    o = ds.ds_options_default()
    assert L.ds_solve(None, None, None, ctypes.c_double(1.0), ctypes.byref(o), None, None, ctypes.byref(r)) \
        == ds.DS_ERR_INVALID
    v = ctypes.c_double()
    assert L.ds_dict_lipschitz(None, ctypes.byref(v)) == ds.DS_ERR_INVALID
    assert L.ds_lambda_max(None, None, None, ctypes.byref(v)) == ds.DS_ERR_INVALID


def test_dict_create_rejects_bad_shapes_without_gpu_work():
    L = ds.lib()
    h = ctypes.c_void_p()
    D = np.zeros((4, 6), order="F")
    # null context, bad N/K/ld and bad dtype are rejected before any CUDA call
    assert L.ds_dict_create(None, D.ctypes.data, 4, 6, 4, ds.DS_FP64, None, None, 0, ds.DS_FP64,
                            ctypes.byref(h)) == ds.DS_ERR_INVALID


def test_selftest_rejects_null_outputs_without_gpu_work():
    L = ds.lib()
    v = ctypes.c_double()
    st = ctypes.c_int()
    assert L.ds_selftest_wait_timeout(0, None, ctypes.byref(v)) == ds.DS_ERR_INVALID
    assert L.ds_selftest_wait_timeout(0, ctypes.byref(st), None) == ds.DS_ERR_INVALID
