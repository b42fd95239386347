"""The Python binding's ctypes structures against the C header: a small C
program built with the host compiler prints sizeof and offsetof of every
public struct, and each must equal the ctypes layout (a field added to one side
only would otherwise shift every later field silently)."""
import ctypes
import os
import shutil
import subprocess

import pytest

from paper_2609_09322_gb300 import gbdart

INCLUDE = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")

# C typedef name -> ctypes structure of the binding
STRUCTS = {
    "gbd_grid": gbdart.Grid,
    "gbd_fields": gbdart.Fields,
    "gbd_view": gbdart.CView,
    "gbd_image_spec": gbdart.ImageSpec,
    "gbd_launch": gbdart.Launch,
    "gbd_volume_desc": gbdart.VolumeDesc,
    "gbd_stream_info": gbdart.StreamInfo,
    "gbd_request": gbdart.Request,
    "gbd_stats": gbdart.Stats,
    "gbd_serve_config": gbdart.ServeConfig,
    "gbd_serve_summary": gbdart.ServeSummary,
    "gbd_tune_result": gbdart.TuneResult,
}


def c_layouts(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no host C compiler")
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "gbdart.h"', "int main(void) {"]
    for cname, cls in STRUCTS.items():
        lines.append(f'  printf("{cname} sizeof %zu\\n", sizeof({cname}));')
        for field, _ in cls._fields_:
            lines.append(f'  printf("{cname} {field} %zu\\n", offsetof({cname}, {field}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", INCLUDE, str(src), "-o", str(exe)], check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    got = {}
    for line in out.splitlines():
        cname, key, value = line.split()
        got[(cname, key)] = int(value)
    return got


def test_ctypes_structs_match_the_header(tmp_path):
    got = c_layouts(tmp_path)
    for cname, cls in STRUCTS.items():
        assert got[(cname, "sizeof")] == ctypes.sizeof(cls), f"{cname}: sizeof differs"
        for field, _ in cls._fields_:
            assert got[(cname, field)] == getattr(cls, field).offset, f"{cname}.{field}: offset differs"
