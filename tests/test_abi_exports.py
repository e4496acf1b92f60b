"""The C-ABI library builds, loads and exports every entry point that
include/gbchol.h declares; the binding declares each one; the library and
the oracle share no symbols.  No GPU is needed (no compute call is made)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gbchol.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(gb_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1812_02056_gb300 import _build, binding
    _build.build()
    return binding.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["gb_create", "gb_destroy", "gb_chol_factor", "gb_lu_factor",
                     "gb_chol_solve", "gb_lu_solve", "gb_chol_factor_batched"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    from paper_1812_02056_gb300 import binding
    out = subprocess.run(["nm", "-D", "--defined-only", binding.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (gb_\w+)", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    for n in declared_functions():
        assert n in binding.SIGNATURES, f"binding lacks {n}"
        getattr(lib, n)


def test_status_strings(lib):
    from paper_1812_02056_gb300 import binding
    assert binding.status_string(0) == "success"
    assert "tolerance" in binding.status_string(binding.GB_ERR_NOT_CONVERGED)
    assert binding.status_string(-3) == "invalid argument"


def test_argument_checks_need_no_gpu(lib):
    import ctypes
    # NULL handle is argument 1 for every call
    assert lib.gb_chol_factor(None, 4, 2, 0, None, 4, None, 4, None, None) == -1
    assert lib.gb_lu_factor(None, 4, 2, 0, None, 4, None, 4, None, None) == -1
    assert lib.gb_set_option(None, 1, 8) == -1
    h = ctypes.c_void_p()
    assert lib.gb_create(None, 0) == -1


def test_library_and_oracle_are_independent(lib):
    """No symbol of one appears in the other, and neither links the other."""
    import oracle
    from paper_1812_02056_gb300 import binding
    orc = oracle.build()
    lib_syms = subprocess.run(["nm", "-D", binding.LIB_PATH], capture_output=True, text=True).stdout
    orc_syms = subprocess.run(["nm", "-D", orc], capture_output=True, text=True).stdout
    assert "orc_" not in lib_syms
    assert "gb_" not in orc_syms
    ldd = subprocess.run(["ldd", binding.LIB_PATH], capture_output=True, text=True).stdout
    assert "oracle" not in ldd
    src = os.path.join(ROOT, "paper_1812_02056_gb300")
    for dirpath, _, files in os.walk(src):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "oracle.c" not in text, f


def header_constants():
    """Every `GB_NAME = value` enumerator and `#define GB_NAME (value)` of the
    header, comments removed."""
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    consts = {k: int(v) for k, v in re.findall(r"\b(GB_[A-Z0-9_]+)\s*=\s*(-?\d+)", text)}
    consts.update({k: int(v) for k, v in
                   re.findall(r"#define\s+(GB_[A-Z0-9_]+)\s+\(?(-?\d+)\)?", text)})
    return consts


def test_binding_constants_match_the_header():
    from paper_1812_02056_gb300 import binding
    consts = header_constants()
    opts = {k: v for k, v in consts.items() if k.startswith(("GB_OPT_", "GB_ERR_"))}
    assert len([k for k in opts if k.startswith("GB_OPT_")]) >= 15
    for k, v in opts.items():
        assert getattr(binding, k) == v, k
    for name in ("GB_F64", "GB_F32", "GB_MIX_BF16", "GB_MIX_F16", "GB_MIX_BF16X3"):
        assert getattr(binding, name) == consts[name], name
    peaks = {k: v for k, v in consts.items() if k.startswith("GB_PEAK_")}
    assert sorted(binding.PEAKS.values()) == sorted(peaks.values())
    for kind, v in binding.PEAKS.items():
        assert consts["GB_PEAK_" + kind.upper()] == v, kind
