"""The binding's ctypes structures match the C structs of include/minjoin.h
field for field: a small C program compiled against the header prints every
struct's size and field offsets (CPU only; gcc)."""
import ctypes
import os
import shutil
import subprocess
import sys
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

PAIRS = {   # C struct -> binding class
    "mj_params": "Params",
    "mj_derived": "Derived",
    "mj_band_train_params": "BandTrainParams",
    "mj_verify_config": "VerifyConfig",
    "mj_autotune_report": "AutotuneReport",
    "mj_stats": "Stats",
    "mj_band_calibration": "BandCalibration",
}


def _c_layout():
    import paper_1810_08833_gb300 as mj
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "minjoin.h"', "int main(void) {"]
    for cname, pyname in PAIRS.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in getattr(mj, pyname)._fields_:
            lines.append(f'  printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines.append("  return 0;\n}")
    d = tempfile.mkdtemp()
    try:
        src, exe = os.path.join(d, "layout.c"), os.path.join(d, "layout")
        open(src, "w").write("\n".join(lines) + "\n")
        subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), src, "-o", exe], check=True,
                       capture_output=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    finally:
        shutil.rmtree(d, ignore_errors=True)
    res = {}
    for line in out.splitlines():
        c, k, v = line.split()
        res[(c, k)] = int(v)
    return res


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
def test_ctypes_structs_match_the_header():
    import paper_1810_08833_gb300 as mj
    lay = _c_layout()
    for cname, pyname in PAIRS.items():
        cls = getattr(mj, pyname)
        assert ctypes.sizeof(cls) == lay[(cname, "size")], cname
        for f, _ in cls._fields_:
            assert getattr(cls, f).offset == lay[(cname, f)], (cname, f)
