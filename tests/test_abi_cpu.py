"""CPU-side checks of the boundary: the library builds, loads, and exports every entry point
that include/vbx.h declares (no compute call is made without a GPU)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "vbx.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(vbx_[a-z_]+)\s*\(", src)))


def test_library_builds_and_exports_every_declared_symbol():
    import __graft_entry__

    __graft_entry__.build()
    from paper_1611_03631_gb300 import build, vbx

    lib = ctypes.CDLL(build.LIB)
    declared = _declared()
    assert len(declared) >= 15
    for name in declared:
        assert hasattr(lib, name), f"{name} declared in vbx.h but not exported"
    # the Python binding marshals exactly the declared entry points
    assert sorted(vbx.exported_symbols()) == declared
    out = subprocess.run(["nm", "-D", "--defined-only", build.LIB], capture_output=True, text=True).stdout
    for name in declared:
        assert re.search(rf"\bT {name}\b", out), name


def test_library_is_built_for_sm_103a():
    from paper_1611_03631_gb300 import build

    assert "arch=compute_103a,code=sm_103a" in " ".join(build.ARCH)


def test_binding_fails_loudly_without_library(tmp_path):
    from paper_1611_03631_gb300 import vbx

    saved = vbx._lib
    vbx._lib = None
    try:
        with pytest.raises(ImportError):
            vbx.load_library(str(tmp_path / "missing.so"))
    finally:
        vbx._lib = saved


def test_oracle_builds_without_contraction():
    import oracle

    oracle.build()
    src = open(os.path.join(ROOT, "oracle", "__init__.py")).read()
    assert "-ffp-contract=off" in src


def test_product_package_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_1611_03631_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                txt = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle\b", txt, re.M), f
                assert "vbx_oracle" not in txt, f


def test_map_bytes_without_a_device():
    """vbx_map_bytes needs no GPU (the queue ring is sized for 152 SMs when no device answers):
    it grows with the block pool and the point capacity, and shrinks with fewer scratch
    blocks; invalid block edges are refused."""
    import __graft_entry__

    __graft_entry__.build()
    from paper_1611_03631_gb300 import vbx

    vbx.load_library()
    small = vbx.map_bytes(16, 1024, 1 << 16)
    assert vbx.map_bytes(16, 4096, 1 << 16) > small
    assert vbx.map_bytes(16, 1024, 1 << 18) > small
    assert vbx.map_bytes(16, 1024, 1 << 16, scratch_blocks=64) < small
    # a pool voxel costs at least its TSDF and ESDF words (16 B) plus the queue ring per tile
    assert small > 1024 * 16 ** 3 * 16 + 1024 * 8 * 16
    with pytest.raises(vbx.VbxError):
        vbx.map_bytes(12, 1024, 1 << 16)
