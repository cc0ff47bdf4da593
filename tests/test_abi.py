"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
entry point that include/roam.h declares.  CPU only (no compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "roam.h")


def declared_entry_points():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(roam_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib_path():
    from paper_2208_02705_gb300 import build
    return build.build()


def test_header_lists_the_boundary():
    names = declared_entry_points()
    for required in ("roam_create", "roam_destroy", "roam_load_grid", "roam_load_fields", "roam_load_weights",
                     "roam_render", "roam_march", "roam_bucket", "roam_mlp_eval", "roam_composite",
                     "roam_train_forward", "roam_train_backward", "roam_adam_step"):
        assert required in names


def test_library_exports_every_declared_symbol(lib_path):
    L = ctypes.CDLL(lib_path)
    for name in declared_entry_points():
        assert hasattr(L, name), name


def test_binding_lists_every_declared_symbol():
    import paper_2208_02705_gb300 as roam
    assert sorted(roam.ENTRY_POINTS) == declared_entry_points()


def test_binding_structs_match_header_sizes():
    import paper_2208_02705_gb300 as roam
    assert ctypes.sizeof(roam.roam_camera) == 64
    assert ctypes.sizeof(roam.roam_render_opts) == 36
    assert ctypes.sizeof(roam.roam_grid_desc) == 28
    assert ctypes.sizeof(roam.roam_mlp_desc) == 16


def test_library_built_for_sm103a_only(lib_path):
    """The fatbinary holds sm_103a code (checked through the toolkit's own
    listing of the embedded ELF names, no disassembly)."""
    import shutil
    import subprocess
    tool = shutil.which("cuobjdump") or "/usr/local/cuda/bin/cuobjdump"
    if not os.path.exists(tool):
        pytest.skip("cuobjdump not available")
    out = subprocess.run([tool, "--list-elf", lib_path], capture_output=True, text=True).stdout
    archs = set(re.findall(r"sm_(\d+a?)", out))
    assert archs == {"103a"}, archs


def test_missing_library_fails_loudly(tmp_path):
    import paper_2208_02705_gb300 as roam
    saved = roam._lib
    roam._lib = None
    try:
        with pytest.raises(roam.RoamError):
            roam.load_library(str(tmp_path / "nope.so"))
    finally:
        roam._lib = saved
