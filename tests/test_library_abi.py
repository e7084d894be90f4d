"""CPU checks of the C ABI: the library builds for sm_103a, loads, exports every
symbol include/chemgpu.h declares, and its structs have the layout the Python
binding assumes.  No compute calls (no GPU here)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "chemgpu.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(chem_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2501_00011_gb300 import build, chemgpu
    build.build()
    return chemgpu.load()


def test_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert len(names) >= 15
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    from paper_2501_00011_gb300 import chemgpu
    assert sorted(chemgpu.EXPORTS) == names


def test_struct_layouts_match_header(tmp_path):
    from paper_2501_00011_gb300 import chemgpu
    prog = tmp_path / "layout.c"
    prog.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "chemgpu.h"\n'
                    'int main(void){printf("%zu %zu %zu %zu %zu %zu %zu\\n", sizeof(chem_reaction), '
                    'offsetof(chem_reaction, yield), offsetof(chem_reaction, J), sizeof(chem_opts), '
                    'sizeof(chem_mech_info), offsetof(chem_mech_info, flops_f), sizeof(chem_cell_stats));return 0;}\n')
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)], check=True)
    vals = list(map(int, subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()))
    R = chemgpu.Reaction
    assert vals == [ctypes.sizeof(R), R.yld.offset, R.J.offset, ctypes.sizeof(chemgpu.Opts),
                    ctypes.sizeof(chemgpu.MechInfo), chemgpu.MechInfo.flops_f.offset,
                    chemgpu.STATS_DTYPE.itemsize]


def test_binding_refuses_without_library(tmp_path):
    from paper_2501_00011_gb300 import chemgpu
    saved = chemgpu._lib
    chemgpu._lib = None
    try:
        with pytest.raises(chemgpu.ChemError):
            chemgpu.load(str(tmp_path / "missing.so"))
    finally:
        chemgpu._lib = saved


def test_pipeline_host_arrays_are_checked_without_copies():
    # the pipeline reads and writes the caller's host arrays in place, so the binding
    # must refuse anything it would have to copy
    import numpy as np
    from paper_2501_00011_gb300 import chemgpu
    a = np.zeros((4, 6))
    assert chemgpu._host_ptr(a, "y").value == a.ctypes.data
    for bad in (np.zeros((4, 6), np.float32), np.asfortranarray(np.zeros((4, 6))), np.zeros((4, 12))[:, ::2]):
        with pytest.raises(chemgpu.ChemError):
            chemgpu._host_ptr(bad, "y")
    ro = np.zeros(3)
    ro.flags.writeable = False
    with pytest.raises(chemgpu.ChemError):
        chemgpu._host_ptr(ro, "T")
    torch = pytest.importorskip("torch")
    t = torch.zeros(5, dtype=torch.float64)
    assert chemgpu._host_ptr(t, "T").value == t.data_ptr()
    with pytest.raises(chemgpu.ChemError):
        chemgpu._host_ptr(torch.zeros(5, dtype=torch.float32), "T")
