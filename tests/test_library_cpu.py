"""Library checks that need no GPU: it builds, loads and exports every entry
point declared in include/*.h, and host-only paths behave."""
import ctypes
import glob
import math
import os
import re

import pytest

from oracle import operator as op
from paper_1803_06237_gb300 import build, vie

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?\w+\s*\*?\s*(vie_\w+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    build.build_library()
    return vie.load()


def test_header_declares_entry_points():
    names = _declared_functions()
    for required in ("vie_plan_create", "vie_plan_destroy", "vie_set_contrast", "vie_matvec", "vie_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    missing = [n for n in _declared_functions() if not hasattr(vie, n)]
    assert not missing, missing


def test_invalid_arguments_rejected_before_any_device_call(lib):
    with pytest.raises(vie.VieError) as ei:
        vie.vie_plan_create((0, 3, 3), 0.02, 4.0, 2.085)
    assert ei.value.status == 1 and "grid" in str(ei.value)
    with pytest.raises(vie.VieError):
        vie.vie_plan_create((3, 3, 3), -1.0, 4.0, 2.085)
    with pytest.raises(vie.VieError):
        vie.vie_eps2_from_round_trip(1.5, 2, 4.0, 4.05, 12.11)


def test_round_trip_helper_matches_oracle(lib):
    k0 = 2 * math.pi / 1.55
    for d in range(4):
        a = vie.vie_eps2_from_round_trip(1e-10, d, 4.0, k0, 12.11)
        b = op.eps2_max_from_rrt(1e-10, d, 4.0, k0, 12.11)
        assert abs(a - b) <= 1e-14 * abs(b)


def test_binding_structs_match_the_header(tmp_path):
    """Size and field offsets of every struct the binding mirrors, from a C
    program compiled against include/vie.h, equal those of the ctypes
    structures."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"vie_plan_info": vie.vie_plan_info, "vie_absorber": vie.vie_absorber,
               "vie_solve_opts": vie.vie_solve_opts, "vie_solve_info": vie.vie_solve_info}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "vie.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'  printf("{name} size %zu\\n", sizeof({name}));')
        for fname, _ in cls._fields_:
            lines.append(f'  printf("{name} {fname} %zu\\n", offsetof({name}, {fname}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {}
    for line in out:
        if line:
            parts = line.split()
            got[(parts[0], parts[1])] = int(parts[2])
    for name, cls in structs.items():
        assert got[(name, "size")] == ctypes.sizeof(cls), name
        for fname, _ in cls._fields_:
            assert got[(name, fname)] == getattr(cls, fname).offset, (name, fname)
