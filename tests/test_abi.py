"""The C-ABI library: it builds for sm_103a, loads, and exports every function include/mrc.h declares.

CPU only: no compute call is made (there may be no GPU here).
"""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mrc.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*([a-z_][a-z0-9_]*)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib_path():
    from paper_1810_03099_gb300 import build
    return build.build()


def test_header_declares_the_five_entry_points():
    names = declared_functions()
    for n in ["mrc_build_index", "mrc_signature", "mrc_match", "cosine_allpairs", "simhash_match"]:
        assert n in names


def test_library_exports_every_declared_symbol(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True, check=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if " T " in ln}
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing


def test_binding_covers_every_declared_symbol(lib_path):
    from paper_1810_03099_gb300 import mrc
    assert set(declared_functions()) == set(mrc.exported_symbols())
    lib = ctypes.CDLL(lib_path)  # loads without a GPU (no CUDA call at load time)
    for n in declared_functions():
        assert hasattr(lib, n)


def test_struct_layouts_match_header(lib_path):
    from paper_1810_03099_gb300 import mrc
    assert ctypes.sizeof(mrc.Pair) == 12
    assert ctypes.sizeof(mrc.Docs) == 24
    assert ctypes.sizeof(mrc.Params) == 48
    assert ctypes.sizeof(mrc.IndexInfo) == 40
    assert mrc.Params.feature_hash.offset == 36 and mrc.Params.seed.offset == 40


def test_params_default_is_pure_host(lib_path):
    from paper_1810_03099_gb300 import mrc
    p = mrc.params_default()
    assert p.k == 8 and p.L == -1 and p.select_mode == mrc.SELECT_REGION and p.weighting == mrc.WEIGHT_TFIDF
    assert abs(p.tau - 0.9) < 1e-7 and p.hamming_max == 3 and p.precision == mrc.PREC_FP32
    assert p.feature_hash == mrc.HASH_SPLITMIX64 and p.seed == 0x1810030990


def test_product_package_never_imports_the_oracle():
    pkg = os.path.join(ROOT, "paper_1810_03099_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".c", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "mrc_oracle" not in text and "orc_" not in text, f
