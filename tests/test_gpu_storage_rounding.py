"""Storage rounding of the cell inverses (Sec. 4.3 inverses, stored in FP32 / BF16): the stored
value is the FP64 inverse rounded once to the nearest FP32 / BF16 value (ties to even), bit for bit.
The FP64 inverse is the one the same device computes for the same cell matrix (FP64 hierarchy)."""
import numpy as np
import pytest

import synth
from helpers import gpu_hierarchy, round_bf16

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = {
    "3d_k1": synth.small_workload(3, 1, (3, 2, 2), 2, obstacle=True, seed=71),
    "2d_k2": synth.small_workload(2, 2, (6, 3), 2, obstacle=True, seed=72),
}


@pytest.mark.parametrize("name", list(CASES))
def test_stored_inverses_are_rounded_once(name):
    wl = CASES[name]
    h64 = gpu_hierarchy(wl, "f64")
    g = h64.finest
    inv64 = h64.copy_cell_inverses(g)
    h64.close()
    for prec in ("f32", "bf16"):
        h = gpu_hierarchy(wl, prec)
        got = h.copy_cell_inverses(g)
        expect = inv64.astype(np.float32).astype(np.float64) if prec == "f32" else round_bf16(inv64)
        np.testing.assert_array_equal(got, expect)
        h.close()
