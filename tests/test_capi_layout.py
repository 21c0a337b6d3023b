"""The Python binding's ctypes structs and constants match include/stm.h as a C compiler lays them
out: every struct's size and every field's offset, and the values of the status, precision,
smoother and kernel-class enums. A field added on one side only would shift every later argument."""
import ctypes as C
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

STRUCTS = {
    "stm_params": "StmParams",
    "stm_gmres_opts": "GmresOpts",
    "stm_solve_info": "SolveInfo",
    "stm_newton_opts": "NewtonOpts",
    "stm_newton_info": "NewtonInfo",
}
ENUMS = ["STM_OK", "STM_ERR_INVALID_ARG", "STM_ERR_CUDA", "STM_ERR_OOM", "STM_ERR_SINGULAR_CELL",
         "STM_ERR_NOT_CONVERGED", "STM_ERR_NONFINITE", "STM_ERR_STATE", "STM_F64", "STM_F32", "STM_BF16",
         "STM_VANKA_ADDITIVE", "STM_VANKA_COLOURED", "STM_VANKA_PAPER_OVERWRITE", "STM_KCLASS_VANKA_LOCAL",
         "STM_KCLASS_JACOBIAN_SPMV", "STM_KCLASS_VANKA_COMBINE", "STM_KCLASS_TRANSFER", "STM_KCLASS_COARSE",
         "STM_KCLASS_KRYLOV", "STM_KCLASS_DEFECT_F32", "STM_KCLASS_ROUND_F32", "STM_NEWTON_MAX_STEPS"]


@pytest.fixture(scope="module")
def c_layout(tmp_path_factory):
    """sizeof/offsetof of every struct field and the enum values, printed by a C program built with
    the host compiler against the header."""
    from paper_2107_10561_gb300 import _lib
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "stm.h"', "int main(void) {"]
    for cname, pyname in STRUCTS.items():
        lines.append(f'  printf("size {cname} %zu\\n", sizeof({cname}));')
        for field, _ in getattr(_lib, pyname)._fields_:
            lines.append(f'  printf("off {cname} {field} %zu\\n", offsetof({cname}, {field}));')
    for e in ENUMS:
        lines.append(f'  printf("enum {e} %d\\n", (int){e});')
    lines += ["  return 0;", "}"]
    d = tmp_path_factory.mktemp("abi")
    src, exe = d / "abi.c", d / "abi"
    src.write_text("\n".join(lines) + "\n")
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    sizes, offsets, enums = {}, {}, {}
    for line in out.splitlines():
        kind, *rest = line.split()
        if kind == "size":
            sizes[rest[0]] = int(rest[1])
        elif kind == "off":
            offsets[(rest[0], rest[1])] = int(rest[2])
        else:
            enums[rest[0]] = int(rest[1])
    return sizes, offsets, enums


@pytest.mark.parametrize("cname", list(STRUCTS))
def test_struct_layout_matches_header(c_layout, cname):
    from paper_2107_10561_gb300 import _lib
    sizes, offsets, _ = c_layout
    cls = getattr(_lib, STRUCTS[cname])
    assert C.sizeof(cls) == sizes[cname], cname
    for field, _ in cls._fields_:
        assert getattr(cls, field).offset == offsets[(cname, field)], (cname, field)


def test_constants_match_header(c_layout):
    from paper_2107_10561_gb300 import _lib
    _, _, enums = c_layout
    for value, name in _lib.STATUS_NAMES.items():
        assert enums[name] == value, name
    for key, name in (("f64", "STM_F64"), ("f32", "STM_F32"), ("bf16", "STM_BF16")):
        assert _lib.PRECISION[key] == enums[name]
    for key, name in (("additive", "STM_VANKA_ADDITIVE"), ("coloured", "STM_VANKA_COLOURED"),
                      ("overwrite", "STM_VANKA_PAPER_OVERWRITE")):
        assert _lib.SMOOTHER[key] == enums[name]
    for key, value in _lib.KCLASS.items():
        assert enums["STM_KCLASS_" + key.upper()] == value, key
    assert _lib.NEWTON_MAX_STEPS == enums["STM_NEWTON_MAX_STEPS"]
