"""CPU-side checks of the C ABI: the library builds, loads without a GPU and
exports every entry point declared in include/dscreen.h; host-side argument
checks reject bad input before touching the GPU."""
import ctypes

import numpy as np
import pytest

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


_DESTROY = {"ds_destroy", "ds_dict_destroy", "ds_batch_destroy", "ds_server_destroy"}


def _zero_args(f):
    scalars = (ctypes.c_int, ctypes.c_int64, ctypes.c_size_t, ctypes.c_uint64, ctypes.c_double, ctypes.c_float)
    return [t(0) if t in scalars else None for t in f.argtypes]


@pytest.mark.parametrize("name", [n for n in ds.declared_functions() if n != "ds_status_str"])
def test_every_entry_point_rejects_null_handles(name):
    """With every pointer null and every size zero, each call returns
    DS_ERR_INVALID (destroy calls: DS_OK) before any CUDA call."""
    f = getattr(ds.lib(), name)
    assert f.argtypes is not None, f"{name}: the binding declares no argument types"
    want = ds.DS_OK if name in _DESTROY else ds.DS_ERR_INVALID
    assert f(*_zero_args(f)) == want


def _noalloc(N=8, K=16, ld=8, lam=0.5, D_offset=0, **opt_fields):
    """Call ds_solve_lasso_noalloc on host buffers: every case here must be
    rejected by the argument checks, which run before the first CUDA call."""
    D = np.zeros(ld * K + 4, dtype=np.float32)
    y = np.zeros(N, dtype=np.float32)
    x = np.zeros(K, dtype=np.float32)
    o = ds.ds_options_default()
    o.L = 1.0
    for k, v in opt_fields.items():
        setattr(o, k, v)
    r = ds.ds_result()
    return ds.lib().ds_solve_lasso_noalloc(0, None, D.ctypes.data + D_offset, N, K, ld, y.ctypes.data,
                                           ctypes.c_double(lam), ctypes.byref(o), x.ctypes.data, ctypes.byref(r))


@pytest.mark.parametrize("case", [
    dict(N=0), dict(K=0), dict(ld=4), dict(lam=0.0), dict(lam=-1.0), dict(lam=float("nan")),
    dict(L=0.0), dict(max_iter=0), dict(tol_gap_rel=-1.0), dict(tol_gap_rel=float("nan")),
    dict(alg=7), dict(test=9), dict(ld=10, N=10), dict(D_offset=4),
])
def test_noalloc_rejects_bad_arguments_without_gpu_work(case):
    assert _noalloc(**case) == ds.DS_ERR_INVALID


def test_noalloc_reports_sizes_beyond_its_fixed_scratch():
    assert _noalloc(N=4097, ld=4100) == ds.DS_ERR_UNSUPPORTED
    assert _noalloc(K=16385) == ds.DS_ERR_UNSUPPORTED


def test_noalloc_bounds_the_leading_dimension_by_the_correlation_chunk():
    # the kernel's shared staging vectors hold N rounded up to 512 rows: a taller
    # column stride is rejected before any CUDA call, a stride within it passes
    # the size checks (and fails later only because these buffers are host memory)
    assert _noalloc(N=700, ld=1028) == ds.DS_ERR_UNSUPPORTED
    assert _noalloc(N=8, ld=516) == ds.DS_ERR_UNSUPPORTED
    assert _noalloc(N=700, ld=1024) != ds.DS_ERR_UNSUPPORTED


_C_USER = r"""
#include <stdio.h>
#include <string.h>
#include "dscreen.h"

int main(void)
{
    ds_options o;
    ds_result r;
    if (ds_options_default(&o) != DS_OK) return 1;
    if (o.alg != DS_FISTA || o.test != DS_DST3 || o.max_iter <= 0) return 2;
    if (strcmp(ds_status_str(DS_ERR_TIMEOUT), "DS_ERR_TIMEOUT") != 0) return 3;
    if (ds_solve(NULL, NULL, NULL, 1.0, &o, NULL, NULL, &r) != DS_ERR_INVALID) return 4;
    if (ds_solve_lasso_noalloc(0, NULL, NULL, 0, 0, 0, NULL, 1.0, &o, NULL, &r) != DS_ERR_INVALID) return 5;
    if (ds_destroy(NULL) != DS_OK) return 6;
    puts("ok");
    return 0;
}
"""


def test_header_is_c99_and_a_c_program_links_the_library(tmp_path):
    """The boundary is a C ABI: include/dscreen.h compiles as strict C99 and a
    plain C program (no Python, no PyTorch) links and calls the library."""
    import os
    import subprocess

    so = ds.build()
    src = tmp_path / "user.c"
    src.write_text(_C_USER)
    exe = tmp_path / "user"
    inc = os.path.dirname(ds.HEADER)
    subprocess.check_call(["gcc", "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", inc, str(src),
                           so, f"-Wl,-rpath,{os.path.dirname(so)}", "-o", str(exe)])
    p = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert p.returncode == 0 and p.stdout.strip() == "ok", (p.returncode, p.stdout, p.stderr)


def test_readme_c_example_compiles(tmp_path):
    """The C example in README.md stays in step with the header."""
    import os
    import re
    import subprocess

    root = os.path.dirname(os.path.dirname(ds.HEADER))
    with open(os.path.join(root, "README.md")) as f:
        blocks = re.findall(r"```c\n(.*?)```", f.read(), re.S)
    assert blocks, "README.md has no C example"
    src = tmp_path / "readme.c"
    src.write_text(blocks[-1])
    subprocess.check_call(["gcc", "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I",
                           os.path.dirname(ds.HEADER), "-c", str(src), "-o", str(tmp_path / "readme.o")])


def _c_layout(tmp_path, include, header, structs):
    """sizeof and offsetof of every field of the given C structs, as compiled by gcc."""
    import subprocess

    lines = ["#include <stddef.h>", "#include <stdio.h>", f'#include "{header}"', "int main(void) {"]
    for cname, fields in structs.items():
        lines.append(f'    printf("{cname} %zu\\n", sizeof({cname}));')
        for f in fields:
            lines.append(f'    printf("{cname}.{f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-std=c99", "-I", include, str(src), "-o", str(exe), "-lm"])
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    return {k: int(v) for k, v in (line.split() for line in out if line)}


def _check(layout, cname, cstruct, rename=None):
    rename = rename or {}
    assert layout[cname] == ctypes.sizeof(cstruct), cname
    for name, _ in cstruct._fields_:
        cfield = rename.get(name, name)
        assert layout[f"{cname}.{cfield}"] == getattr(cstruct, name).offset, (cname, cfield)


def test_binding_structs_match_the_c_layout(tmp_path):
    """ds_options and ds_result of the ctypes binding have the header's layout."""
    import os

    structs = {"ds_options": [n for n, _ in ds.ds_options._fields_],
               "ds_result": ["lambda" if n == "lambda_" else n for n, _ in ds.ds_result._fields_]}
    lay = _c_layout(tmp_path, os.path.dirname(ds.HEADER), "dscreen.h", structs)
    _check(lay, "ds_options", ds.ds_options)
    _check(lay, "ds_result", ds.ds_result, {"lambda_": "lambda"})


def test_oracle_structs_match_the_c_layout(tmp_path):
    """The oracle's ctypes option and result structures have its C layout."""
    import os

    import oracle

    src = os.path.abspath(oracle._SRC)
    structs = {"or_options": [n for n, _ in oracle._Options._fields_],
               "or_result": [n for n, _ in oracle._Result._fields_]}
    lay = _c_layout(tmp_path, os.path.dirname(src), os.path.basename(src), structs)
    _check(lay, "or_options", oracle._Options)
    _check(lay, "or_result", oracle._Result)


def test_binding_rejects_short_or_mistyped_buffers_before_the_call():
    """The library reads y and writes x_out through raw pointers, so the binding checks
    their element type, contiguity and length against the registered dictionary first
    (a short buffer would be an out-of-bounds device access)."""
    from paper_1412_4080_gb300 import _binding as B

    h = B._DictHandle()
    h.N, h.K, h.esize = 5, 7, 4
    o = ds.ds_options_default()
    f32 = np.float32
    bad = [((np.zeros(4, f32), np.zeros(7, f32)), ValueError),          # y too short
           ((np.zeros(5, np.float64), np.zeros(7, f32)), TypeError),   # y of another type
           ((np.zeros(5, f32), np.zeros(6, f32)), ValueError),          # x_out too short
           ((np.zeros(5, f32), np.zeros((7, 2), f32)[:, 0]), ValueError)]  # x_out strided
    for (y, x), exc in bad:
        with pytest.raises(exc):
            ds.ds_solve(None, h, y, 1.0, o, x)
    with pytest.raises(ValueError):
        ds.ds_solve_path(None, h, np.zeros(5, f32), [0.5, 0.3], o, np.zeros(7, f32))
    with pytest.raises(ValueError):
        ds.ds_solve(None, h, np.zeros(5, f32), 1.0, o, np.zeros(7, f32), x0=np.zeros(3, f32))
    # well-formed buffers reach the library, which rejects the null context
    with pytest.raises(ds.DscreenError):
        ds.ds_solve(None, h, np.zeros(5, f32), 1.0, o, np.zeros(7, f32))
    with pytest.raises(ds.DscreenError):
        ds.ds_solve_path(None, h, np.zeros(5, f32), [0.5, 0.3], o, np.zeros((2, 7), f32))


def test_server_and_allocation_free_calls_check_their_buffers():
    from paper_1412_4080_gb300 import _binding as B

    h = B._DictHandle()
    h.N, h.K, h.esize = 5, 7, 4
    f32 = np.float32
    o = ds.ds_options_default(L=1.0)
    with pytest.raises(ValueError):
        ds.ds_server_submit(None, h, np.zeros(5, f32), 0.5, o, np.zeros(6, f32))
    D = np.zeros((8, 16), dtype=f32, order="F")
    with pytest.raises(TypeError):
        ds.ds_solve_lasso_noalloc(0, None, D.astype(np.float64), np.zeros(8, f32), 0.5, o, np.zeros(16, f32))
    with pytest.raises(ValueError):
        ds.ds_solve_lasso_noalloc(0, None, D, np.zeros(7, f32), 0.5, o, np.zeros(16, f32))
    with pytest.raises(ValueError):
        ds.ds_solve_lasso_noalloc(0, None, D, np.zeros(8, f32), 0.5, o, np.zeros(15, f32))
    # well-formed host buffers reach the library, which rejects host pointers (no GPU work)
    with pytest.raises(ds.DscreenError):
        ds.ds_server_submit(None, h, np.zeros(5, f32), 0.5, o, np.zeros(7, f32))


def test_batch_arguments_are_checked_per_instance():
    from paper_1412_4080_gb300 import _binding as B

    h = B._DictHandle()
    h.N, h.K, h.esize = 5, 7, 4
    f32 = np.float32
    o = ds.ds_options_default()
    Y = np.zeros((3, 5), f32)
    X = np.zeros((3, 7), f32)
    with pytest.raises(ValueError):     # right-hand sides stored column-major
        ds.ds_solve_batch(None, [h], [np.asfortranarray(Y)[:, :]], [np.ones(3)], o, [X])
    with pytest.raises(ValueError):     # too few solutions
        ds.ds_solve_batch(None, [h], [Y], [np.ones(3)], o, [np.zeros((2, 7), f32)])
    with pytest.raises(ValueError):     # too few lambdas
        ds.ds_solve_batch(None, [h], [Y], [np.ones(2)], o, [X])
    with pytest.raises(ValueError):     # lists of different lengths
        ds.ds_solve_batch(None, [h, h], [Y], [np.ones(3)], o, [X])
    with pytest.raises(ds.DscreenError):  # well-formed: the library rejects the null context
        ds.ds_solve_batch(None, [h], [Y], [np.ones(3)], o, [X])


def test_history_buffer_is_checked():
    with pytest.raises(ValueError):
        ds.ds_set_history(None, np.zeros((10, 5)))
    with pytest.raises(TypeError):
        ds.ds_set_history(None, np.zeros((10, 6), np.float32))
    with pytest.raises(ValueError):
        ds.ds_set_history(None, np.asfortranarray(np.zeros((10, 6))))
    with pytest.raises(ds.DscreenError):  # well-formed: the library rejects the null context
        ds.ds_set_history(None, np.zeros((10, 6)))


def test_group_weights_are_checked_against_the_offsets():
    D = np.zeros((4, 6), order="F")
    goff = np.array([0, 2, 6])
    with pytest.raises(ValueError):
        ds.ds_dict_create(None, D, goff, np.ones(3))
    with pytest.raises(ValueError):
        ds.ds_dict_create(None, D, None, np.ones(2))
    with pytest.raises(ds.DscreenError):  # well-formed: the library rejects the null context
        ds.ds_dict_create(None, D, goff, np.ones(2))


def test_oracle_compiles_without_warnings(tmp_path):
    """The oracle's C source is warning-free under -Wall -Wextra -Wpedantic -Wshadow."""
    import os
    import subprocess

    import oracle

    subprocess.check_call(["gcc", "-std=c99", "-O2", "-Wall", "-Wextra", "-Wpedantic", "-Wshadow", "-Werror",
                           "-fsyntax-only", os.path.abspath(oracle._SRC)])


def test_header_compiles_as_cpp17(tmp_path):
    """C++ callers include the same header (its declarations sit in extern "C")."""
    import os
    import subprocess

    src = tmp_path / "user.cpp"
    src.write_text('#include "dscreen.h"\nint main() { ds_options o; return ds_options_default(&o) == DS_OK ? 0 : 1; }\n')
    subprocess.check_call(["g++", "-std=c++17", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I",
                           os.path.dirname(ds.HEADER), "-c", str(src), "-o", str(tmp_path / "user.o")])
