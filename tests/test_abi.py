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


def test_binding_structs_match_header_layouts(tmp_path):
    """Every ctypes structure of the binding has the size and field offsets
    that a C compiler gives the header's struct (gcc on include/roam.h)."""
    import shutil
    import subprocess
    import paper_2208_02705_gb300 as roam
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not available")
    structs = ["roam_grid_desc", "roam_mlp_desc", "roam_camera", "roam_render_opts", "roam_stats",
               "roam_kernel_time", "roam_adam_cfg", "roam_occ_params"]
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "roam.h"', "int main(void) {"]
    for name in structs:
        lines.append(f'printf("{name} size %zu\\n", sizeof({name}));')
        for fname, _ in getattr(roam, name)._fields_:
            lines.append(f'printf("{name} {fname} %zu\\n", offsetof({name}, {fname}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call([gcc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    for row in out:
        if not row:
            continue
        name, what, val = row.split()
        cls = getattr(roam, name)
        got = ctypes.sizeof(cls) if what == "size" else getattr(cls, what).offset
        assert got == int(val), (name, what, got, val)


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
