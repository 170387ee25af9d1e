"""The C-ABI library builds for sm_103a, loads, and exports every symbol that
include/dem.h declares (no compute call: this runs without a GPU)."""
import ctypes
import os
import re

from paper_2309_15417_gb300 import build as B
from paper_2309_15417_gb300 import dem as D

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    """Function names declared by every header under include/."""
    names = set()
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(dem_[a-z_0-9]+)\s*\(", src))
    return sorted(names)


def test_header_declarations_match_binding():
    assert _declared() == sorted(D.EXPORTS)


def test_library_builds_and_exports_every_symbol():
    path = B.build()
    assert os.path.exists(path)
    lib = ctypes.CDLL(path)
    for name in _declared():
        assert hasattr(lib, name), name


def test_struct_layouts_match_header(tmp_path):
    """Every field of the Python mirrors sits at the offset the C compiler
    gives it for include/dem.h, and the structs have the same sizes."""
    import subprocess
    structs = [D.dem_config, D.dem_particles, D.dem_narrow_out, D.dem_stats, D.dem_lts_params, D.dem_lts_out,
               D.dem_tuning]
    lines = ['#include <stdio.h>', '#include "dem.h"', 'int main(void) {']
    for S in structs:
        name = S.__name__
        lines.append(f'  printf("{name} %zu\\n", sizeof({name}));')
        for f, _ in S._fields_:
            lines.append(f'  printf("{name}.{f} %zu\\n", offsetof({name}, {f}));')
    lines += ['  return 0;', '}']
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = dict(l.split() for l in subprocess.check_output([str(exe)], text=True).splitlines())
    for S in structs:
        name = S.__name__
        assert int(got[name]) == ctypes.sizeof(S), name
        for f, _ in S._fields_:
            assert int(got[f"{name}.{f}"]) == getattr(S, f).offset, f"{name}.{f}"