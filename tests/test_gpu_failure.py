"""Failure handling that a test can drive without faulting the GPU.

The dataflow Jacobi sweep of the preconditioner (min(m, n) > 1024) lets each
pair of rows wait for its two rows to finish the previous round.  Every wait is
bounded by elapsed time on the GPU's global timer; when one runs out the CTA
raises a flag, every CTA leaves at its next poll and lsrn_precond returns
LSRN_ERR_TIMEOUT.  The kernel's own ordering never lets a wait run out, so the
test uses the library's test knobs: the sweep starts after the first round
(every later pair then waits on rows nobody publishes) with a 2 ms limit.  The
kernel polls global counters only and has no copies in flight, so giving up is
safe.  Afterwards the same plan must solve correctly (it sketches again: the
QR overwrote the sketch)."""
import time

import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
L = pytest.importorskip("paper_1109_5981_gb300")


@pytest.mark.parametrize("svd_mode", ["df", "f64"])
def test_dataflow_jacobi_wait_runs_out_then_the_plan_recovers(svd_mode):
    # df: the double-float pre-sweep kernel is the one that gives up;
    # f64: the FP64 sweep kernel
    P = W.dense_haar(2600, 1100, 1000, 1e4, 1e-3, seed=5)     # q = 1100: dataflow sweep
    A = torch.from_numpy(P.A).cuda()
    b = torch.from_numpy(P.b).cuda()
    mode = L.LSRN_SVD_DF if svd_mode == "df" else L.LSRN_SVD_F64
    plan = L.lsrn_plan(A, L.default_options(seed=2, svd_mode=mode))
    try:
        L.lsrn_sketch(plan)
        L.lsrn_set_test_knob(L.LSRN_KNOB_JACOBI_WAIT_NS, 2_000_000)
        L.lsrn_set_test_knob(L.LSRN_KNOB_JACOBI_SKIP_FIRST_ROUND, 1)
        t0 = time.perf_counter()
        try:
            with pytest.raises(L.LsrnError) as e:
                L.lsrn_precond(plan)
        finally:
            L.lsrn_set_test_knob(L.LSRN_KNOB_JACOBI_WAIT_NS, 0)
            L.lsrn_set_test_knob(L.LSRN_KNOB_JACOBI_SKIP_FIRST_ROUND, 0)
        assert e.value.status == L.LSRN_ERR_TIMEOUT
        assert time.perf_counter() - t0 < 10.0
        # the context and the plan stay usable: the solve sketches again
        x, info = L.lsrn_solve_lsqr(plan, b)
    finally:
        plan.close()
    assert info["rank"] == 1000
    assert (info["jacobi_sweeps_df"] > 0) == (svd_mode == "df")
    xs, _ = O.minlen_refined(P.A, P.b)
    assert O.rel_err(x.cpu().numpy(), xs) <= 1e-10


def test_test_knobs_reject_bad_arguments():
    with pytest.raises(L.LsrnError) as e:
        L.lsrn_set_test_knob(7, 1)
    assert e.value.status == L.LSRN_ERR_INVALID_ARG
    with pytest.raises(L.LsrnError) as e:
        L.lsrn_set_test_knob(L.LSRN_KNOB_JACOBI_WAIT_NS, -5)
    assert e.value.status == L.LSRN_ERR_INVALID_ARG


def test_cooperative_qr_barrier_wait_runs_out_then_the_plan_recovers():
    # one CTA of the cooperative QR leaves before the first grid barrier; the
    # others wait 2 ms of global time, raise the flag and return
    P = W.dense_haar(3000, 400, 380, 1e4, 1e-3, seed=6)
    A = torch.from_numpy(P.A).cuda()
    b = torch.from_numpy(P.b).cuda()
    plan = L.lsrn_plan(A, L.default_options(seed=4))
    try:
        L.lsrn_sketch(plan)
        L.lsrn_set_test_knob(L.LSRN_KNOB_JACOBI_WAIT_NS, 2_000_000)
        L.lsrn_set_test_knob(L.LSRN_KNOB_QR_ABSENT_CTA, 1)
        t0 = time.perf_counter()
        try:
            with pytest.raises(L.LsrnError) as e:
                L.lsrn_precond(plan)
        finally:
            L.lsrn_set_test_knob(L.LSRN_KNOB_JACOBI_WAIT_NS, 0)
            L.lsrn_set_test_knob(L.LSRN_KNOB_QR_ABSENT_CTA, 0)
        assert e.value.status == L.LSRN_ERR_TIMEOUT
        assert time.perf_counter() - t0 < 10.0
        x, info = L.lsrn_solve_lsqr(plan, b)
    finally:
        plan.close()
    assert info["rank"] == 380
    xs, _ = O.minlen_refined(P.A, P.b)
    assert O.rel_err(x.cpu().numpy(), xs) <= 1e-10
