"""The C-ABI library builds, loads and exports every entry point include/hsweep.h
declares (no GPU needed: nothing here calls into the device)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "hsweep.h")).read()
    return sorted(set(re.findall(r"HSWEEP_API\s+(?:int|void)\s+(hsweep_\w+)\s*\(", txt)))


def _lib_path():
    import __graft_entry__ as g
    b = g._build_module()
    if not os.path.exists(b.LIB):
        b.build()
    return b.LIB


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("hsweep_setup", "hsweep_apply", "hsweep_solve", "hsweep_grad",
                     "hsweep_status", "hsweep_free"):
        assert required in names


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(_lib_path())
    for name in _declared():
        assert hasattr(lib, name), name


def test_python_binding_lists_the_same_names():
    _lib_path()
    import paper_1007_4290_gb300 as hs
    assert sorted(hs.EXPORTED) == _declared()


def test_default_opts_and_argument_checks_without_gpu():
    _lib_path()
    import paper_1007_4290_gb300 as hs
    o = hs.default_opts()
    assert (o.leaf, o.r_max, o.precision, o.pml_form) == (8, 48, hs.MIXED, 0)
    assert abs(o.pml_C - 2 * 3.141592653589793) < 1e-15
    # argument errors are reported before any device work
    raw = ctypes.c_void_p()
    rc = hs._lib.hsweep_setup(None, 1.0, 64, 8, 1e-6, None, None, ctypes.byref(raw))
    assert rc == hs.ERR_ARG and not raw.value
    bad = hs.default_opts(leaf=9)
    rc = hs._lib.hsweep_setup(ctypes.c_void_p(16), 1.0, 64, 8, 1e-6, ctypes.byref(bad), None, ctypes.byref(raw))
    assert rc == hs.ERR_ARG
    rc = hs._lib.hsweep_setup(ctypes.c_void_p(16), 1.0, 64, 40, 1e-6, None, None, ctypes.byref(raw))
    assert rc == hs.ERR_ARG
    assert hs._lib.hsweep_apply(None, None, None, 1) == hs.ERR_ARG
    assert hs._lib.hsweep_set_stream(None, None) == hs.ERR_ARG
    hs._lib.hsweep_free(None)


def test_philox_generator_matches_the_published_known_answers():
    # the counter-based generator of the randomized SVD's test vectors (strong admissibility)
    _lib_path()
    import paper_1007_4290_gb300 as hs
    rows = [l.split() for l in open(os.path.join(ROOT, "tests", "golden", "philox4x32_10_kat.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        assert hs.philox4x32_10(v[0:4], v[4:6]) == v[6:10]


def test_strong_rank_argument_checks_without_gpu():
    _lib_path()
    import paper_1007_4290_gb300 as hs
    raw = ctypes.c_void_p()
    for bad in (hs.default_opts(strong_rank=9), hs.default_opts(strong_rank=-1)):
        rc = hs._lib.hsweep_setup(ctypes.c_void_p(16), 1.0, 64, 8, 1e-6, ctypes.byref(bad), None, ctypes.byref(raw))
        assert rc == hs.ERR_ARG and not raw.value
    # n = 2047, leaf 8: depth 8, the expanded strong form of rank 3 needs 3*3*7 + 8 = 71 > 56 columns
    o = hs.default_opts(strong_rank=3)
    rc = hs._lib.hsweep_setup(ctypes.c_void_p(16), 1.0, 2047, 16, 1e-6, ctypes.byref(o), None, ctypes.byref(raw))
    assert rc == hs.ERR_ARG and not raw.value


def test_binding_fails_loudly_without_the_library(tmp_path):
    # no CPU fallback: a missing libhsweep.so is an import-time error
    _lib_path()
    import pytest
    import paper_1007_4290_gb300 as hs
    with pytest.raises(ImportError):
        hs.load_library(str(tmp_path / "libhsweep.so"))


def test_plain_c_program_compiles_links_and_calls_the_library(tmp_path):
    """The header is plain C (C99) and the library links from C: a program that takes the
    default options and makes calls the library must refuse before any device work."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        import pytest
        pytest.skip("no C compiler")
    lib = _lib_path()
    src = tmp_path / "abi.c"
    src.write_text(
        '#include "hsweep.h"\n'
        "int main(void) {\n"
        "  hsweep_opts o;\n"
        "  hsweep_t h = 0;\n"
        "  if (hsweep_default_opts(&o) != HSWEEP_OK || o.leaf != 8) return 1;\n"
        "  if (hsweep_setup(0, 1.0, 64, 8, 1e-6, &o, 0, &h) != HSWEEP_ERR_ARG || h) return 2;\n"
        "  if (hsweep_apply(0, 0, 0, 1) != HSWEEP_ERR_ARG) return 3;\n"
        "  if (hsweep_set_stream(0, 0) != HSWEEP_ERR_ARG) return 4;\n"
        "  hsweep_free(0);\n"
        "  return 0;\n"
        "}\n")
    exe = tmp_path / "abi"
    libdir = os.path.dirname(lib)
    out = subprocess.run([cc, "-std=c99", "-Wall", "-Werror", "-I" + os.path.join(ROOT, "include"), str(src),
                          "-L" + libdir, "-lhsweep", "-Wl,-rpath," + libdir, "-o", str(exe)],
                         capture_output=True, text=True)
    assert out.returncode == 0, out.stderr
    run = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert run.returncode == 0, (run.returncode, run.stderr)
