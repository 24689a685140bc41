"""CPU-only checks of the C-ABI library: it builds, loads and exports every
entry point declared in include/ddm.h; the oracle and the CUDA path share no
code.  No compute call is made (there is no GPU here)."""
import ctypes
import glob
import os
import re

import pytest

import paper_1703_06680_gb300 as ddm
from paper_1703_06680_gb300 import build as pkg_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?\w+\s*\**\s*(ddm_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib_path():
    return pkg_build.build()


def test_header_declares_entry_points():
    names = declared_functions()
    for must in ("ddm_create", "ddm_destroy", "ddm_count", "ddm_match"):
        assert must in names


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert missing == []


def test_binding_covers_every_declared_symbol():
    assert sorted(ddm.SIGNATURES) == declared_functions()


def test_binding_fails_loudly_without_library(tmp_path):
    with pytest.raises(ImportError):
        ddm.load_library(str(tmp_path / "missing.so"))


def _imports(path):
    src = open(path).read()
    return set(re.findall(r"^\s*(?:from|import)\s+([\w.]+)", src, flags=re.M))


def test_oracle_and_cuda_path_share_no_code():
    pkg_files = glob.glob(os.path.join(ROOT, "paper_1703_06680_gb300", "**", "*.*"), recursive=True)
    for f in pkg_files:
        if f.endswith(".py"):
            assert not any(m.split(".")[0] == "oracle" for m in _imports(f)), f
        if f.endswith((".cu", ".cuh", ".h", ".cpp")):
            assert "oracle" not in open(f).read().lower(), f
    for f in glob.glob(os.path.join(ROOT, "oracle", "*.*")):
        if f.endswith(".py"):
            assert not any(m.startswith("paper_1703_06680_gb300") for m in _imports(f)), f
        if f.endswith(".c"):
            assert "#include \"" not in open(f).read(), f
    # the generators hold no matching arithmetic and import neither side
    for f in glob.glob(os.path.join(ROOT, "synth", "*.py")):
        mods = _imports(f)
        assert not any(m.startswith(("oracle", "paper_1703_06680_gb300")) for m in mods), f


def test_cuda_sources_are_sm103a_only():
    assert "arch=compute_103a,code=sm_103a" in " ".join(pkg_build.NVCC_FLAGS)
    for f in glob.glob(os.path.join(ROOT, "paper_1703_06680_gb300", "csrc", "*")):
        text = open(f).read()
        assert "wgmma" not in text and "triton" not in text.lower(), f
