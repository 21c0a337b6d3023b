"""Failure detection without a GPU fault: the bounded mbarrier wait of the pipelined kernels (the
tensor-core smoother) gives up on a barrier that nothing completes, reports it in the error word and
leaves the context usable. The wait is the same helper the tcgen05 pipeline runs; the barrier is one
that no thread arrives on, so the wait can only run out."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_wait_on_a_barrier_nothing_completes_times_out_and_reports():
    from paper_2107_10561_gb300 import Hierarchy
    timed_out, ms = Hierarchy.selftest_bounded_wait()
    assert timed_out
    # one second of wall time, then an orderly return (generous upper bound for a shared machine)
    assert 900.0 <= ms <= 10000.0, ms
    # the context is still usable: a device computation afterwards gives the right answer
    a = torch.arange(1000, dtype=torch.float64, device="cuda")
    assert float((a * 2).sum()) == float(np.arange(1000).sum() * 2)
