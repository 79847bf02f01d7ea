"""Host-side checks of the C ABI (no GPU needed): the library builds, loads and
exports every function include/pnoeom.h declares; the host subspace
eigensolver agrees with LAPACK."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def pkg():
    import paper_1802_06738_gb300 as p
    p.build()
    return p


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b([a-z_][a-z0-9_]*)\s*\([^;{]*\)\s*;", txt))
    return sorted(names)


def test_every_declared_symbol_is_exported(pkg):
    lib = ctypes.CDLL(pkg.LIB_PATH)
    names = _declared()
    assert "sigma" in names and "pno_build" in names and "davidson_solve" in names
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) <= set(pkg.EXPORTS) | {"pnoeom_create"}


def test_struct_layouts_match_the_header(pkg, tmp_path):
    """The ctypes mirrors of pnoeom_system and pnoeom_opts have the C layout: size and
    every field's offset, from a C program compiled against include/pnoeom.h."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"pnoeom_system": pkg.System, "pnoeom_opts": pkg.Opts}
    lines = ['#include "pnoeom.h"', "#include <stddef.h>", "#include <stdio.h>", "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'  printf("{cname} sizeof %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'  printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(ln.split()[:2]): int(ln.split()[2]) for ln in out if ln.strip()}
    for cname, py in structs.items():
        assert got[(cname, "sizeof")] == ctypes.sizeof(py), cname
        for fname, _ in py._fields_:
            assert got[(cname, fname)] == getattr(py, fname).offset, (cname, fname)


def test_binding_declares_argument_types_of_every_export(pkg):
    # without argtypes ctypes passes Python ints as C int, truncating 64-bit handles
    L = pkg.lib()
    for n in set(pkg.EXPORTS) | {"pnoeom_create"}:
        assert getattr(L, n).argtypes is not None, n


@pytest.mark.parametrize("n", [1, 2, 3, 8, 24, 48])
def test_small_eig_real_spectrum(pkg, n):
    rng = np.random.default_rng(n)
    A = np.diag(np.linspace(0.3, 3.0, n)) + (0.05 / n) * rng.standard_normal((n, n))
    w, V = pkg.pnoeom_small_eig(A)
    ref = np.sort(np.linalg.eigvals(A).real)
    assert np.abs(np.sort(w.real) - ref).max() < 1e-12
    assert np.abs(w.imag).max() < 1e-12
    assert np.abs(A @ V - V * w.real).max() < 1e-11
    assert np.allclose(np.linalg.norm(V, axis=0), 1.0)


def test_small_eig_complex_pairs(pkg):
    rng = np.random.default_rng(3)
    A = rng.standard_normal((9, 9))
    w, _ = pkg.pnoeom_small_eig(A)
    ref = np.linalg.eigvals(A)
    # every eigenvalue matches one of LAPACK's (conjugate pairs may come in either order)
    d = np.abs(w[:, None] - ref[None, :])
    assert d.min(axis=1).max() < 1e-11 and d.min(axis=0).max() < 1e-11


def test_errors_are_codes_not_aborts(pkg):
    L = pkg.lib()
    rc = L.pnoeom_small_eig(0, None, None, None, None)
    assert rc == pkg.ERR_INVALID_ARG
    assert b"bad arguments" in L.pnoeom_last_error()
    rc = L.pno_query(None, None, None, None, None, None)
    assert rc == pkg.ERR_INVALID_ARG
