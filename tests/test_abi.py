"""Host-side checks of the C ABI: the library loads without a GPU, exports
every function include/kzk.h declares, and rejects bad arguments before any
device work (status codes, no exception across the boundary)."""
import ctypes
import os
import re

import pytest

from paper_2103_06080_b300 import _lib as L

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    src = open(os.path.join(ROOT, "include", "kzk.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(kzk_[a-z_]+)\s*\(", src)))


def test_library_exports_every_declared_function():
    lib = L.lib()
    names = header_functions()
    assert len(names) >= 12
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(L.exported_names()) == names


def test_status_strings():
    lib = L.lib()
    for s in range(9):
        assert lib.kzk_status_string(s)


def _create(nx=64, ny=32, prec=0, dt=0.01, B=0.05, A=7e-6, M=1.0, batch=1, relax=None):
    g = L.KzkGrid(nx=nx, ny=ny, tau_min=-4, tau_max=4, y_min=-8, y_max=8, prec=prec)
    c = L.KzkCoeffs(B=B, A=A, lf_umax=M)
    if relax is not None:
        n, C, theta = relax
        c.n_relax = n
        c.relax_C = (ctypes.c_double * 2)(*C)
        c.relax_theta = (ctypes.c_double * 2)(*theta)
    h = ctypes.c_void_p()
    st = L.lib().kzk_plan_create(ctypes.byref(g), ctypes.byref(c), dt, batch, ctypes.byref(h))
    return st, h


@pytest.mark.parametrize("kw,code", [
    (dict(nx=44), L.KZK_ERR_SIZE), (dict(nx=4), L.KZK_ERR_SIZE), (dict(nx=16384), L.KZK_ERR_SIZE),
    (dict(ny=1), L.KZK_ERR_SIZE), (dict(ny=3002), L.KZK_ERR_SIZE), (dict(ny=8192), L.KZK_ERR_SIZE),
    (dict(nx=45), L.KZK_ERR_SIZE), (dict(ny=25), L.KZK_ERR_SIZE), (dict(nx=7 * 2 ** 12), L.KZK_ERR_SIZE),
    (dict(nx=2 * 13, ny=50), L.KZK_ERR_SIZE), (dict(nx=56, ny=2 * 11), L.KZK_ERR_SIZE),
    (dict(prec=7), L.KZK_ERR_ARG), (dict(dt=0.0), L.KZK_ERR_ARG), (dict(dt=float("nan")), L.KZK_ERR_ARG),
    (dict(B=0.0), L.KZK_ERR_ARG), (dict(A=-1.0), L.KZK_ERR_ARG), (dict(M=0.0), L.KZK_ERR_ARG),
    (dict(batch=0), L.KZK_ERR_ARG),
    (dict(relax=(3, (1e-3, 1e-3), (0.1, 0.1))), L.KZK_ERR_ARG),
    (dict(relax=(-1, (0.0, 0.0), (1.0, 1.0))), L.KZK_ERR_ARG),
    (dict(relax=(1, (-1e-3, 0.0), (0.1, 1.0))), L.KZK_ERR_ARG),
    (dict(relax=(2, (1e-3, 1e-3), (0.1, 0.0))), L.KZK_ERR_ARG),
    (dict(relax=(1, (float("inf"), 0.0), (0.1, 1.0))), L.KZK_ERR_ARG),
])
def test_plan_create_rejects_bad_arguments(kw, code):
    st, h = _create(**kw)
    assert st == code and not h.value
    assert L.lib().kzk_last_error()


def test_null_arguments_are_rejected():
    lib = L.lib()
    assert lib.kzk_plan_create(None, None, 0.1, 1, None) == L.KZK_ERR_ARG
    assert lib.kzk_advance(None, None, 1, 0.0, None, None) == L.KZK_ERR_ARG
    assert lib.kzk_rhs(None, None, None, 0.0, None) == L.KZK_ERR_ARG
    assert lib.kzk_tau_fft(None, None, None, 1, None) == L.KZK_ERR_ARG
    assert lib.kzk_adjoint(None, None, None, None, 1, 0.0, 1, None) == L.KZK_ERR_ARG
    assert lib.kzk_plan_destroy(None) == L.KZK_OK
    m = L.KzkMedium(n_modes=0)
    assert lib.kzk_plan_set_medium(None, ctypes.byref(m)) == L.KZK_ERR_ARG
    assert lib.kzk_medium_eval(None, 0.0, None, None, None) == L.KZK_ERR_ARG


@pytest.mark.parametrize("field,value,code", [
    ("row_kernel", 3, L.KZK_ERR_ARG), ("col_kernel", 4, L.KZK_ERR_ARG), ("fp32_state", -1, L.KZK_ERR_ARG),
    ("transforms", 2, L.KZK_ERR_ARG), ("graph", 3, L.KZK_ERR_ARG), ("graph", -1, L.KZK_ERR_ARG)])
def test_unknown_option_values_are_rejected(field, value, code):
    # refused before any device work
    g = L.KzkGrid(nx=64, ny=32, tau_min=-4, tau_max=4, y_min=-8, y_max=8, prec=L.KZK_FP32)
    c = L.KzkCoeffs(B=0.05, A=7e-6, lf_umax=1.0)
    o = L.KzkOptions()
    setattr(o, field, value)
    h = ctypes.c_void_p()
    assert L.lib().kzk_plan_create_ex(ctypes.byref(g), ctypes.byref(c), 0.01, 1, ctypes.byref(o), ctypes.byref(h)) == code
    assert not h.value


def test_mixed_radix_plans_refuse_pair_kernels():
    g = L.KzkGrid(nx=56, ny=50, tau_min=-4, tau_max=4, y_min=-8, y_max=8, prec=L.KZK_FP32)
    c = L.KzkCoeffs(B=0.05, A=7e-6, lf_umax=1.0)
    h = ctypes.c_void_p()
    for field, value in (("row_kernel", 1), ("col_kernel", 1), ("col_kernel", 3)):
        o = L.KzkOptions()
        setattr(o, field, value)
        st = L.lib().kzk_plan_create_ex(ctypes.byref(g), ctypes.byref(c), 0.01, 1, ctypes.byref(o), ctypes.byref(h))
        assert st == L.KZK_ERR_SIZE and not h.value


def test_batched_mode_flags_are_exclusive():
    g = (L.KzkGrid * 1)(L.KzkGrid(nx=64, ny=32, tau_min=-4, tau_max=4, y_min=-8, y_max=8, prec=L.KZK_FP32))
    c = (L.KzkCoeffs * 1)(L.KzkCoeffs(B=0.05, A=7e-6, lf_umax=1.0))
    dts = (ctypes.c_double * 1)(0.01)
    h = ctypes.c_void_p()
    st = L.lib().kzk_plan_create_batched(g, c, dts, 1, L.KZK_BATCH_STREAMS | L.KZK_BATCH_PERSISTENT, ctypes.byref(h))
    assert st == L.KZK_ERR_ARG and not h.value
    assert L.lib().kzk_plan_create_batched(g, c, dts, 1, 64, ctypes.byref(h)) == L.KZK_ERR_ARG


def test_binding_structs_match_the_header(tmp_path):
    """The ctypes mirrors have the sizes and field offsets the C compiler gives
    the structs of include/kzk.h."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"kzk_grid": L.KzkGrid, "kzk_coeffs": L.KzkCoeffs, "kzk_diag": L.KzkDiag, "kzk_medium": L.KzkMedium,
               "kzk_options": L.KzkOptions}
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "kzk.h"', "int main(void) {"]
    for cname, cls in structs.items():
        lines.append(f'printf("{cname} sizeof %zu\\n", sizeof({cname}));')
        for f, _ in cls._fields_:
            lines.append(f'printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    out = subprocess.check_output([str(exe)], text=True).split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for cname, cls in structs.items():
        assert got[(cname, "sizeof")] == ctypes.sizeof(cls), cname
        for f, _ in cls._fields_:
            assert got[(cname, f)] == getattr(cls, f).offset, (cname, f)


def test_tile_copy_rate_rejects_bad_arguments():
    # refused before any device work
    lib = L.lib()
    out = ctypes.c_double()
    assert lib.kzk_tile_copy_rate(2048, 2048, L.KZK_COPY_STRIP, None, None) == L.KZK_ERR_ARG
    assert lib.kzk_tile_copy_rate(2048, 2048, 2, None, ctypes.byref(out)) == L.KZK_ERR_ARG
    for n, ny in ((2047, 2048), (0, 2048), (2048, 128), (2048, 8192), (2048, 3000), (1 << 18, 2048)):
        assert lib.kzk_tile_copy_rate(n, ny, L.KZK_COPY_STRIP, None, ctypes.byref(out)) == L.KZK_ERR_SIZE
