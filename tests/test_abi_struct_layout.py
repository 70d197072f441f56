"""The ctypes mirrors in the Python binding match the C structs of
include/smc.h field by field: a small C program compiled against the header
prints sizeof and every field's offsetof, compared with ctypes."""
import ctypes as C
import os
import shutil
import subprocess

import pytest

from paper_2504_02627_gb300 import _binding as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PAIRS = [(B.SmcModel, "smc_model"), (B.SmcConfig, "smc_config"), (B.SmcFlowConfig, "smc_flow_config"),
         (B.SmcStats, "smc_stats"), (B.SmcSummary, "smc_summary")]


def test_struct_layouts_match_the_header(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "smc.h"', "int main(void) {"]
    for cls, cname in PAIRS:
        lines.append(f'    printf("{cname} sizeof %zu\\n", sizeof({cname}));')
        for f, _ in cls._fields_:
            lines.append(f'    printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(ln.split()[:2]): int(ln.split()[2]) for ln in out if ln.strip()}
    for cls, cname in PAIRS:
        assert got[(cname, "sizeof")] == C.sizeof(cls), cname
        for f, _ in cls._fields_:
            assert got[(cname, f)] == getattr(cls, f).offset, (cname, f)


def test_oracle_struct_layouts_match_its_header(tmp_path):
    import oracle
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    pairs = [(oracle.Target, "oracle_target"), (oracle.Config, "oracle_config"), (oracle.Stats, "oracle_stats"),
             (oracle.CheesState, "oracle_chees_state"), (oracle.IterIO, "oracle_iter_io"),
             (oracle.Flow, "oracle_flow")]
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "oracle.h"', "int main(void) {"]
    for cls, cname in pairs:
        lines.append(f'    printf("{cname} sizeof %zu\\n", sizeof({cname}));')
        for f, _ in cls._fields_:
            lines.append(f'    printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["    return 0;", "}"]
    src = tmp_path / "olayout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "olayout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "oracle"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(ln.split()[:2]): int(ln.split()[2]) for ln in out if ln.strip()}
    for cls, cname in pairs:
        assert got[(cname, "sizeof")] == C.sizeof(cls), cname
        for f, _ in cls._fields_:
            assert got[(cname, f)] == getattr(cls, f).offset, (cname, f)
