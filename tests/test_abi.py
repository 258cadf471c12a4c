"""The C-ABI library builds, loads and exports every entry point of include/mpcg.h (CPU)."""
import ctypes
import os
import re

import pytest

from conftest import ROOT


def declared_functions():
    src = open(os.path.join(ROOT, "include", "mpcg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mpcg_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib_path():
    from paper_2412_08059_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("mpcg_features", "mpcg_choose_eps1", "mpcg_solve", "mpcg_solve_batch",
                     "mpcg_workspace_bytes", "mpcg_options_default"):
        assert required in names


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_declares_every_symbol():
    from paper_2412_08059_gb300 import mpcg
    assert sorted(mpcg.SYMBOLS) == declared_functions()


def test_host_only_entry_points(lib_path):
    """Calls that do no device work: defaults, status strings, workspace sizes."""
    from paper_2412_08059_gb300 import mpcg
    mpcg.load(lib_path)
    o = mpcg.options()
    assert (o.eps1, o.eps2, o.k0, o.knn_k, o.weighted, o.tol_relative) == (-1.0, 1e-10, 10, 5, 1, 1)
    assert mpcg.status_string(0) == "ok"
    assert "workspace" in mpcg.status_string(-2)
    assert mpcg.workspace_bytes(0, 10) == 0
    n, nnz = 2_097_152, 14_581_760
    wb = mpcg.workspace_bytes(n, nnz)
    # sliced arrays (<= 32 * wcap per slice, 16 B per entry) + vectors: < 1 GB at 128^3
    assert 16 * nnz < wb < 1_000_000_000
    assert mpcg.load().mpcg_batch_step_launches(None) == -1


def test_oracle_and_library_share_no_code():
    """The oracle and the CUDA sources do not include or import each other."""
    csrc = os.path.join(ROOT, "paper_2412_08059_gb300", "csrc")
    for f in os.listdir(csrc):
        txt = open(os.path.join(csrc, f)).read()
        assert "oracle" not in txt.lower(), f          # no include, no shared helper
    for f in ("mpcg.py", "build.py", "__init__.py"):
        txt = open(os.path.join(ROOT, "paper_2412_08059_gb300", f)).read()
        assert "import oracle" not in txt and "from oracle" not in txt
    for f in os.listdir(os.path.join(ROOT, "oracle")):
        if f.endswith((".c", ".h", ".py")):
            txt = open(os.path.join(ROOT, "oracle", f)).read()
            assert "import paper_2412_08059_gb300" not in txt
            assert "from paper_2412_08059_gb300" not in txt
            assert "mpcg.h" not in txt and "libmpcg.so" not in txt


def test_binding_structs_match_the_header_layout(tmp_path):
    """Every ctypes structure of the binding has the size and field offsets
    that a C compiler gives the header's struct (gcc on the host)."""
    import shutil
    import subprocess

    from paper_2412_08059_gb300 import mpcg
    if shutil.which("gcc") is None:
        pytest.skip("no gcc")
    pairs = {"mpcg_csr_t": mpcg.CsrDesc, "mpcg_features_t": mpcg.Features,
             "mpcg_sample_t": mpcg.SampleDesc, "mpcg_options_t": mpcg.Options,
             "mpcg_result_t": mpcg.Result}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "mpcg.h"', "int main(void) {"]
    for cname, py in pairs.items():
        lines.append(f'  printf("{cname} sizeof %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'  printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), "-o", str(exe),
                    str(src)], check=True)
    got = {}
    for line in subprocess.run([str(exe)], check=True, capture_output=True,
                               text=True).stdout.splitlines():
        cname, field, val = line.split()
        got[(cname, field)] = int(val)
    for cname, py in pairs.items():
        assert got[(cname, "sizeof")] == ctypes.sizeof(py), cname
        for f, _ in py._fields_:
            assert got[(cname, f)] == getattr(py, f).offset, (cname, f)


def test_static_variant_checks_options_before_the_size(lib_path):
    """mpcg_solve_static validates its arguments and options the way
    mpcg_solve does before it looks at the size: an invalid option on a
    system too large for the fixed array is an invalid argument, and a valid
    one is refused for its size.  Both answers come from host checks alone
    (the descriptor's pointers are never dereferenced), so no GPU is needed."""
    import ctypes as C

    from paper_2412_08059_gb300 import mpcg
    L = mpcg.load(lib_path)
    n, nnz = 4_000_000, 28_000_000
    assert mpcg.workspace_bytes(n, nnz) > mpcg.STATIC_WS_BYTES
    fake = C.c_void_p(256)  # stands in for device memory; no call reaches it
    A = mpcg.CsrDesc(n, nnz, fake, fake, fake)
    res = C.c_void_p(512)
    bad = mpcg.options(knn_k=0)
    good = mpcg.options(eps1=1e-4)
    f = L.mpcg_solve_static
    assert f(C.byref(A), fake, fake, None, C.byref(bad), res, None) == mpcg.ERR_INVALID_ARG
    assert f(C.byref(A), fake, fake, None, C.byref(good), res, None) == mpcg.ERR_WORKSPACE
    assert f(C.byref(A), fake, fake, None, None, res, None) == mpcg.ERR_INVALID_ARG
