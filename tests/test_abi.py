"""The C-ABI library builds, loads and exports every symbol include/tls.h declares.

CPU only: no compute call is made.  tls_create on a machine without a GPU must
return an error status instead of crashing.
"""

import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "tls.h")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(tls_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2301_05518_gb300 import build
    return build.build()


def test_header_declares_expected_entry_points():
    names = _declared()
    for need in ("tls_create", "tls_load_gauge", "tls_build_twolink", "tls_smear",
                 "tls_serve_submit", "tls_serve_wait"):
        assert need in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\sT\s(tls_[a-z_0-9]+)", out))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing


def test_binding_covers_header(libpath):
    from paper_2301_05518_gb300 import tls
    assert sorted(tls.EXPORTS) == _declared()
    for n in tls.EXPORTS:
        assert hasattr(tls, n)
        assert hasattr(tls.lib, n)
    assert tls.tls_version() >= 10000


def test_create_without_gpu_reports_error(libpath):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2301_05518_gb300 import tls
    h = ctypes.c_void_p()
    st = tls.lib.tls_create(ctypes.byref(h), 0, 0)
    assert st != tls.TLS_OK
    assert h.value is None
    assert len(tls.tls_last_error()) > 0


def test_struct_sizes_match_header(libpath):
    """ctypes mirrors of the public structs have the C sizes (checked with gcc)."""
    from paper_2301_05518_gb300 import tls
    src = ('#include "tls.h"\n#include <stdio.h>\nint main(){printf("%zu %zu %zu %zu %zu\\n",'
           'sizeof(tls_profile),sizeof(tls_serve_opts),sizeof(tls_job),sizeof(tls_job_result),'
           'sizeof(tls_tune_entry));}\n')
    import tempfile
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "s.c")
        exe = os.path.join(d, "s")
        open(c, "w").write(src)
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        sizes = [int(x) for x in subprocess.run([exe], capture_output=True, text=True).stdout.split()]
    assert sizes == [ctypes.sizeof(tls.tls_profile), ctypes.sizeof(tls.tls_serve_opts),
                     ctypes.sizeof(tls.tls_job), ctypes.sizeof(tls.tls_job_result),
                     ctypes.sizeof(tls.tls_tune_entry)]


def test_binding_argument_counts_match_header(libpath):
    """Every ctypes prototype has as many arguments as its declaration in tls.h."""
    from paper_2301_05518_gb300 import tls
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    decls = re.findall(r"\b(tls_[a-z_0-9]+)\s*\(([^;{]*?)\)\s*;", text, flags=re.S)
    assert decls
    checked = 0
    for name, params in decls:
        params = params.strip()
        n = 0 if params in ("", "void") else len([p for p in params.split(",") if p.strip()])
        fn = getattr(tls.lib, name)
        assert fn.argtypes is not None, name
        assert len(fn.argtypes) == n, (name, len(fn.argtypes), n)
        checked += 1
    assert checked == len(_declared())


def test_binding_without_library_fails_loudly(tmp_path):
    """No CPU fallback: a package copy without libtls.so refuses to import."""
    import shutil
    import sys
    pkg = os.path.join(ROOT, "paper_2301_05518_gb300")
    dst = tmp_path / "paper_2301_05518_gb300"
    shutil.copytree(pkg, dst, ignore=shutil.ignore_patterns("*.so", "_build", "__pycache__"))
    code = ("import sys; sys.path.insert(0, %r)\n"
            "try:\n    import paper_2301_05518_gb300.tls\nexcept ImportError as e:\n    print('refused:', e)\n"
            "else:\n    print('imported')\n") % str(tmp_path)
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, cwd=str(tmp_path)).stdout
    assert out.startswith("refused:"), out
