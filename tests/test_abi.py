"""The C-ABI library builds for sm_103a, loads, and exports every symbol that
include/dem.h declares (no compute call: this runs without a GPU)."""
import ctypes
import os
import re

from paper_2309_15417_gb300 import build as B
from paper_2309_15417_gb300 import dem as D

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "dem.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dem_[a-z_0-9]+)\s*\(", src)))


def test_header_declarations_match_binding():
    assert _declared() == sorted(D.EXPORTS)


def test_library_builds_and_exports_every_symbol():
    path = B.build()
    assert os.path.exists(path)
    lib = ctypes.CDLL(path)
    for name in _declared():
        assert hasattr(lib, name), name


def test_struct_sizes_match_header():
    # dem_stats: 16 int64; dem_config: 48 bytes with natural alignment
    assert ctypes.sizeof(D.dem_stats) == 16 * 8
    assert ctypes.sizeof(D.dem_config) == 48
    assert ctypes.sizeof(D.dem_particles) == 48
    assert ctypes.sizeof(D.dem_narrow_out) == 80
