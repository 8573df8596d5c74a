"""The ctypes mirrors of the C-ABI structs (paper_1905_05515_b300/abi.py)
against the declarations in include/: each struct's size and every field's
offset, printed by a small C program compiled with gcc.  Host only: a field
added on one side and not the other, or in another place, fails here before
any device call reads the wrong word."""
import ctypes as C
import os
import subprocess

import pytest

from paper_1905_05515_b300 import abi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
INCLUDE = os.path.join(ROOT, "include")

PAIRS = [(abi.TpcParams, "tpc_params"), (abi.TpcGeometry, "tpc_geometry"), (abi.TpcClusters, "tpc_clusters"),
         (abi.TpcTracks, "tpc_tracks"), (abi.TpcCalibTracks, "tpc_calib_tracks"),
         (abi.TpcCompressIn, "tpc_compress_in"), (abi.TpcCalibFitOpts, "tpc_calib_fit_opts"),
         (abi.TpcCalibFitReport, "tpc_calib_fit_report")]


def _c_layout(tmp_path):
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "tpc_track.h"', '#include "tpc_calib.h"',
             '#include "tpc_compress.h"', "int main(void) {"]
    for cls, cname in PAIRS:
        lines.append(f'printf("{cname} sizeof %zu\\n", sizeof({cname}));')
        for f in cls._fields_:
            lines.append(f'printf("{cname} {f[0]} %zu\\n", offsetof({cname}, {f[0]}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", INCLUDE, str(src), "-o", str(exe)], check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    got = {}
    for line in out.splitlines():
        cname, field, value = line.split()
        got[(cname, field)] = int(value)
    return got


@pytest.mark.parametrize("cls,cname", PAIRS, ids=[c for _, c in PAIRS])
def test_struct_layout_matches_header(tmp_path, cls, cname):
    got = _c_layout(tmp_path)
    assert got[(cname, "sizeof")] == C.sizeof(cls), f"{cname}: size"
    for f in cls._fields_:
        assert got[(cname, f[0])] == getattr(cls, f[0]).offset, f"{cname}.{f[0]}: offset"
