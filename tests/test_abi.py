"""The C-ABI library builds for sm_103a, loads, and exports every symbol the header declares.

No compute call is made here (no GPU on this host).
"""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_symbols():
    text = open(os.path.join(ROOT, "include", "pb_spgemm.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pb_[a-z_0-9]+)\s*\(", text)) - {"pb_alloc_fn", "pb_free_fn"})


def test_library_exports_every_declared_symbol():
    from paper_2002_11302_gb300 import binding
    lib = binding.load_library()
    syms = header_symbols()
    assert len(syms) >= 12
    for s in syms:
        assert hasattr(lib, s), f"{s} declared in the header but not exported"
    assert set(syms) == set(binding.SIGNATURES), "binding signatures out of step with the header"
    assert lib.pb_version() == 10000


def test_library_targets_sm103a():
    from paper_2002_11302_gb300 import build
    assert "arch=compute_103a,code=sm_103a" in " ".join(build.ARCH)
    assert os.path.exists(build.LIB)


def test_status_codes_match_header():
    from paper_2002_11302_gb300 import binding
    text = open(os.path.join(ROOT, "include", "pb_spgemm.h")).read()
    codes = dict((name, int(v)) for name, v in re.findall(r"(PB_(?:OK|ERR_[A-Z_]+))\s*=\s*(\d+)", text))
    assert {v: k for k, v in codes.items()} == binding.STATUS_NAMES
    dts = dict((name, int(v)) for name, v in re.findall(r"(PB_F[0-9A-Z_]+)\s*=\s*(\d+)", text))
    assert dts == {"PB_F64": binding.PB_F64, "PB_F32": binding.PB_F32, "PB_F64_F32TUPLE": binding.PB_F64_F32TUPLE}


def test_product_path_has_no_cpu_fallback():
    """The binding never imports the oracle; the package has no CPU compute path."""
    pkg = os.path.join(ROOT, "paper_2002_11302_gb300")
    for f in os.listdir(pkg):
        if f.endswith(".py"):
            src = open(os.path.join(pkg, f)).read()
            assert "import oracle" not in src and "from oracle" not in src, f


def test_null_handle_calls_are_rejected_without_gpu():
    from paper_2002_11302_gb300 import binding
    lib = binding.load_library()
    assert lib.pb_plan_query(None, None, None, None, None, None) == 1
    assert lib.pb_plan_destroy(None) == 0
    assert lib.pb_destroy(None) == 0
