"""Host-side checks of the C ABI: the library loads, exports every entry point
that include/sg.h declares, the binding's struct layouts match the header,
and argument validation answers before any device work."""

import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sg.h")


def header_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sg_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def sg():
    import paper_2306_05332_gb300 as sg
    if not os.path.exists(sg.LIB_PATH):
        from paper_2306_05332_gb300 import build
        build.build()
    sg.lib()
    return sg


def test_library_exports_every_header_function(sg):
    names = header_functions()
    assert len(names) >= 18
    L = sg.lib()
    for n in names:
        assert hasattr(L, n), n
    assert sorted(sg.exported_symbols()) == names


def test_struct_layouts_match_header(sg, tmp_path):
    src = tmp_path / "sizes.c"
    src.write_text('#include "sg.h"\n#include <stdio.h>\n#include <stddef.h>\n'
                   'int main(void){printf("%zu %zu %zu %zu %zu\\n", sizeof(sg_options), sizeof(sg_solve_info),'
                   ' offsetof(sg_solve_info, history), offsetof(sg_solve_info, elapsed_ms),'
                   ' sizeof(sg_tune_entry));return 0;}\n')
    exe = tmp_path / "sizes"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    assert int(out[0]) == ctypes.sizeof(sg.Options)
    assert int(out[1]) == ctypes.sizeof(sg.SolveInfo)
    assert int(out[2]) == sg.SolveInfo.history.offset
    assert int(out[3]) == sg.SolveInfo.elapsed_ms.offset
    assert int(out[4]) == ctypes.sizeof(sg.TuneEntry)


def test_status_codes_match_header(sg):
    text = open(HEADER).read()
    for code, name in sg.STATUS.items():
        assert re.search(rf"{name}\s*=\s*{code}\b", text), name


def test_default_options(sg):
    o = sg.default_options()
    assert (o.rkl_order, o.s_smooth, o.n_pre, o.n_post) == (2, 3, 2, 1)
    assert o.tau_frac == 1.0 and o.use_graph == 1 and o.coarse_tol == 1e-2
    assert (o.smoother, o.omega, o.max_residual_tol) == (0, 1.0, 0.0)
    assert (o.staging, o.host_copy) == (sg.STAGINGS["cp_async"], sg.HOST_COPIES["engine"])


def test_option_enums_match_header(sg):
    text = open(HEADER).read()
    for names in ({"cp_async": "SG_STAGE_CP_ASYNC", "tma": "SG_STAGE_TMA"},
                  {"engine": "SG_HOST_COPY_ENGINE", "kernel": "SG_HOST_COPY_KERNEL"}):
        table = sg.STAGINGS if "tma" in names else sg.HOST_COPIES
        for key, name in names.items():
            assert re.search(rf"{name}\s*=\s*{table[key]}\b", text), name


@pytest.mark.parametrize("shape,lo,hi,bc,prec", [
    ((1, 8, 8), (0, 0, 0), (1, 1, 1), (0, 0, 0), 1),
    ((8, 8, 5000), (0, 0, 0), (1, 1, 1), (0, 0, 0), 1),
    ((8, 8, 8), (0, 0, 0), (0, 1, 1), (0, 0, 0), 1),
    ((8, 8, 8), (0, 0, 0), (1, 1, 1), (0, 3, 0), 1),
    ((8, 8, 8), (0, 0, 0), (1, 1, 1), (0, 0, 0), 7),
])
def test_create_rejects_bad_arguments_before_device_work(sg, shape, lo, hi, bc, prec):
    nz, ny, nx = shape
    D, I = ctypes.c_double, ctypes.c_int
    h = ctypes.c_void_p()
    st = sg.lib().sg_create_grid(nx, ny, nz, (D * 3)(*lo), (D * 3)(*hi), (I * 3)(*bc), prec, None,
                                 ctypes.byref(h))
    assert st == 1
    assert h.value is None
    assert sg.lib().sg_last_error()


def test_null_arguments_rejected(sg):
    L = sg.lib()
    assert L.sg_default_options(None) == 1
    assert L.sg_solve(None, 1e-8, 0, 0, None) == 1
    assert L.sg_set_density(None, None, 0, 1.0) == 1
    assert L.sg_gravity(None, None, None, 0) == 1
    assert L.sg_op_gsrb_sweep(None, 0, 0, 0, 1.0, None, None) == 1
    assert L.sg_op_residual_exact(None, 0, None, None, None, None, None) == 1
    L.sg_destroy(None)


def test_product_path_fails_loudly_without_library(sg, monkeypatch, tmp_path):
    import paper_2306_05332_gb300 as pkg
    monkeypatch.setattr(pkg, "_LIB", None)
    monkeypatch.setattr(pkg, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError):
        pkg.lib()
