"""The C ABI library builds for sm_103a, loads without a GPU, and exports
every function that include/mlba.h declares (no compute calls here)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mlba.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(mlba_[a-z_0-9]+)\s*\(", text)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1504_07234_gb300.build import build
    import paper_1504_07234_gb300 as M
    build()
    return M.load_library()


def test_header_declares_api():
    names = declared_functions()
    for must in ("mlba_create", "mlba_iterate", "mlba_result", "mlba_batch_create",
                 "mlba_op_blur", "mlba_op_precond", "mlba_op_frame"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_declares_every_symbol():
    import paper_1504_07234_gb300 as M
    assert set(declared_functions()) == set(M.SIGNATURES)


def test_strerror_and_defaults_without_gpu(lib):
    import ctypes
    import paper_1504_07234_gb300 as M
    assert lib.mlba_strerror(0) == b"ok"
    assert lib.mlba_strerror(-7).startswith(b"unsupported")
    o = M.Opts()
    lib.mlba_opts_default(ctypes.byref(o))
    assert abs(o.mu - 10 / 255) < 1e-15 and o.levels == 1 and o.pcg_max == 5 and o.stop == 1


def test_invalid_arguments_rejected_before_device_work(lib):
    """Validation happens on the host: even p, p > n, Algorithm 4 with the
    rectangular operator (Section 5) return MLBA_E_INVAL without a GPU."""
    import ctypes
    import numpy as np
    import paper_1504_07234_gb300 as M
    o = M.Opts()
    lib.mlba_opts_default(ctypes.byref(o))
    h = ctypes.c_void_p()
    psf = np.full((4, 4), 1 / 16.0)
    assert lib.mlba_create(psf.ctypes.data_as(ctypes.c_void_p), 4, 16, 1, 1, ctypes.byref(o), ctypes.byref(h)) == -1
    psf = np.full((5, 5), 1 / 25.0)
    assert lib.mlba_create(psf.ctypes.data_as(ctypes.c_void_p), 5, 4, 1, 1, ctypes.byref(o), ctypes.byref(h)) == -1
    assert lib.mlba_create(psf.ctypes.data_as(ctypes.c_void_p), 5, 16, 3, 4, ctypes.byref(o), ctypes.byref(h)) == -1
    assert lib.mlba_create(psf.ctypes.data_as(ctypes.c_void_p), 5, 16, 3, 5, ctypes.byref(o), ctypes.byref(h)) == -1
    # batch-wide copies without a batch or without arrays
    assert lib.mlba_batch_set_data_all(None, None, 0, None) == -1
    assert lib.mlba_batch_result_all(None, None, 0) == -1
    # a PSF wider than the stencil tile supports is refused, also before any device work
    big = np.full((67, 67), 1 / 67.0 ** 2)
    assert lib.mlba_create(big.ctypes.data_as(ctypes.c_void_p), 67, 128, 1, 1, ctypes.byref(o), ctypes.byref(h)) == -7


def test_binding_structs_match_header_layout(tmp_path):
    """The ctypes mirrors of mlba_opts, mlba_stats and mlba_problem have the
    C layout of include/mlba.h: every field offset and the struct sizes, as a
    host C compiler lays the header out (no GPU)."""
    import ctypes
    import shutil
    import subprocess
    import paper_1504_07234_gb300 as M
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    mirrors = {"mlba_opts": M.Opts, "mlba_stats": M.Stats, "mlba_problem": M.ProblemDesc}
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "mlba.h"', "int main(void) {"]
    for cname, cls in mirrors.items():
        lines.append(f'  printf("{cname} . %zu\\n", sizeof({cname}));')
        for fname, _ in cls._fields_:
            lines.append(f'  printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    c_layout = {}
    for line in out:
        if line.strip():
            cname, fname, v = line.split()
            c_layout[(cname, fname)] = int(v)
    for cname, cls in mirrors.items():
        assert c_layout[(cname, ".")] == ctypes.sizeof(cls), cname
        for fname, _ in cls._fields_:
            assert c_layout[(cname, fname)] == getattr(cls, fname).offset, (cname, fname)
