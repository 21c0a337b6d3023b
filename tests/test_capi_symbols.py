"""The C-ABI library builds for sm_103a, loads without a GPU and exports every declared symbol."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "stm.h")).read()
    return re.findall(r"^\s*(?:stm_status|void|const char\*|long long)\s+(stm_\w+)\(", text, re.M)


def test_header_declares_the_boundary():
    names = set(declared_symbols())
    for required in ("stm_build_hierarchy", "stm_assemble_jacobian", "stm_factor_cells", "stm_vcycle",
                     "stm_gmres_solve", "stm_vanka_sweep", "stm_spmv", "stm_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_2107_10561_gb300 import build, _lib
    if not os.path.exists(_lib.LIB_PATH):
        build.build()
    lib = _lib.load()
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing
    assert set(declared_symbols()) == set(_lib.SIGNATURES)


def test_missing_library_fails_loudly(tmp_path):
    from paper_2107_10561_gb300 import _lib
    with pytest.raises(RuntimeError):
        _lib.CDLL_path_check = None
        saved = _lib._lib
        _lib._lib = None
        try:
            _lib.load(str(tmp_path / "nope.so"))
        finally:
            _lib._lib = saved
