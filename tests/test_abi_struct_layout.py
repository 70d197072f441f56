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


def test_enum_values_match_the_header(tmp_path):
    """The binding's status codes, model kinds, precisions and buffer ids are
    the values of the header's enums."""
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    names = {"SMC_OK": B.SMC_OK, "SMC_E_INVAL": B.SMC_E_INVAL, "SMC_E_NOMEM": B.SMC_E_NOMEM,
             "SMC_E_CUDA": B.SMC_E_CUDA, "SMC_E_DEGENERATE": B.SMC_E_DEGENERATE, "SMC_E_TIMEOUT": B.SMC_E_TIMEOUT,
             "SMC_E_STATE": B.SMC_E_STATE}
    for k in ("GAUSS_DENSE", "LOGISTIC", "HIER_NORMAL", "BANANA", "LINEAR_GAUSS"):
        names["SMC_MODEL_" + k] = getattr(B, k)
    for k in ("FP32", "BF16X3", "BF16", "BF16X2", "BF16C"):
        names["SMC_PREC_" + k] = getattr(B, "PREC_" + k)
    for k in ("THETA", "GRAD", "LOGPI", "LOGW", "W", "ANCESTORS", "STEPS", "P_FINAL", "DH", "ALPHA", "THETA_PREV",
              "RUNSTATE", "Z0", "Z1", "ORDER"):
        names["SMC_BUF_" + k] = getattr(B, "BUF_" + k)
    lines = ['#include <stdio.h>', '#include "smc.h"', "int main(void) {"]
    lines += [f'    printf("{n} %d\\n", (int){n});' for n in names]
    lines += ["    return 0;", "}"]
    src = tmp_path / "enums.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "enums"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {ln.split()[0]: int(ln.split()[1]) for ln in out if ln.strip()}
    assert got == names
