"""Failure paths of the bounded waits, on the GPU without a fault: a wait that runs out returns an
error status the host reads, and the device context stays usable.

The staged kernels (Gram-Schmidt sweeps, the V-cycle tail) wait on mbarriers for bulk
asynchronous copies.  sbm_async_wait_selftest runs one such wait with a copy that is announced but
never issued (a phase that nothing completes): the wait gives up after a bounded number of polls,
sets the library's fault flag, and the call returns SBM_ERR_CUDA.  A solve afterwards must still
converge and report no fault.
"""
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_bounded_wait_succeeds_when_the_copy_arrives():
    import paper_2506_12899_gb300 as S
    S.async_wait_selftest(False)


def test_bounded_wait_runs_out_and_reports():
    import paper_2506_12899_gb300 as S
    with pytest.raises(S.SbmError) as ei:
        S.async_wait_selftest(True)
    assert "mbarrier wait gave up" in str(ei.value)
    # the flag was cleared by the failing call: the next good wait and a full solve are clean
    S.async_wait_selftest(False)
    g = S.Solver(W.disk2d_p1(16, 0), "f32")
    b = g.rhs()
    x = torch.zeros_like(b)
    info = g.solve(b, x)
    assert info.converged and info.true_rel_residual <= 1e-8
