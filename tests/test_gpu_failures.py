"""Failure detection, injected on the host: bad values in the caller's data and a forced
wait timeout in the A pass.  Nothing here faults, traps or hangs the GPU: the NaN / Inf
cases only feed arithmetic (every device loop has a fixed bound), and the timeout case
makes one CTA's bounded mbarrier wait run out because its load was never posted (no
transaction is left pending).  After each failure the handle is destroyed and a fresh solve
on the same device must still match the oracle.
"""
import numpy as np
import pytest

from oracle import bicadmm_ref as ref
from paper_2405_16267_b300 import bicadmm as bc
from paper_2405_16267_b300 import synth

from gpu_util import compare_state, run_gpu, run_oracle

pytestmark = pytest.mark.gpu

ERR_NUMERIC, ERR_TIMEOUT = -5, -6


def _healthy_after():
    P = synth.small_problem(ref.LOSS_SQUARED, m=600, n=40, nnz=4, N=3, M=2, kappa=4, seed=4)
    st, _ = run_gpu(P, 20)
    compare_state(st, run_oracle(P, 20), 1e-9)


def _solver(P, A=None, b=None, precision=bc.PREC_FP64):
    import torch
    return bc.Solver(P.A if A is None else A, P.b if b is None else b, loss=P.loss, N=P.N,
                     M=P.M, kappa=P.kappa, gamma=P.gamma, rho_c=P.rho, precision=precision,
                     stream=torch.cuda.current_stream())


def test_nan_in_A_is_numeric_error():
    """A NaN in A reaches the block Gram matrices: setup reports a non-positive pivot."""
    P = synth.small_problem(ref.LOSS_SQUARED, m=600, n=40, nnz=4, N=3, M=2, kappa=4, seed=4)
    A = P.A.copy()
    A[123, 17] = np.nan
    with pytest.raises(bc.BicadmmError) as e:
        with _solver(P, A=A) as s:
            s.step(2)
    assert e.value.code == ERR_NUMERIC
    _healthy_after()


@pytest.mark.parametrize("loss,bad,precision", [
    (ref.LOSS_SQUARED, np.inf, bc.PREC_FP64),
    (ref.LOSS_LOGISTIC, np.nan, bc.PREC_FP32),
    (ref.LOSS_SQHINGE, -np.inf, bc.PREC_BF16),
])
def test_nonfinite_target_is_numeric_error_from_step(loss, bad, precision):
    """A non-finite target passes setup (b is not in the factors) and makes the residual of
    the first iteration non-finite: bicadmm_step with info reports ERR_NUMERIC."""
    P = synth.small_problem(loss, m=900, n=50, nnz=5, N=3, M=2, kappa=5, seed=6)
    b = P.b.copy()
    b[400] = bad
    A = P.A if precision == bc.PREC_FP64 else np.asarray(P.A, dtype=np.float32)
    s = _solver(P, A=A, b=b, precision=precision)
    try:
        with pytest.raises(bc.BicadmmError) as e:
            s.step(3)
        assert e.value.code == ERR_NUMERIC
        assert "non-finite" in str(e.value)
    finally:
        s.close()
    _healthy_after()


@pytest.mark.parametrize("panel", ["first", "last"])
def test_forced_pass_timeout(panel):
    """One panel's load is never posted: its CTA's bounded wait (2e6 cycles, about 1 ms)
    runs out, the pass records the timeout and step reports ERR_TIMEOUT; destroy is clean."""
    P = synth.small_problem(ref.LOSS_LOGISTIC, m=4000, n=96, nnz=6, N=4, M=2, kappa=6, seed=8)
    s = _solver(P, A=np.asarray(P.A, dtype=np.float32), precision=bc.PREC_FP32)
    try:
        s.step(2)   # healthy iterations first
        if panel == "first":
            bc.inject_pass_stall(s.h, 0, 2_000_000)
        else:
            # the largest panel index the handle accepts
            lo, hi = 0, P.m
            while lo + 1 < hi:
                mid = (lo + hi) // 2
                try:
                    bc.inject_pass_stall(s.h, mid, 2_000_000)
                    lo = mid
                except bc.BicadmmError:
                    hi = mid
            bc.inject_pass_stall(s.h, lo, 2_000_000)
        with pytest.raises(bc.BicadmmError) as e:
            s.step(1)
        assert e.value.code == ERR_TIMEOUT
    finally:
        s.close()
    _healthy_after()


def test_stall_hook_rejects_bad_arguments():
    P = synth.small_problem(ref.LOSS_SQUARED, m=600, n=40, nnz=4, N=3, M=2, kappa=4, seed=4)
    with _solver(P) as s:
        for panel, limit in ((10 ** 9, 2_000_000), (0, 10)):
            with pytest.raises(bc.BicadmmError) as e:
                bc.inject_pass_stall(s.h, panel, limit)
            assert e.value.code == -1
        bc.inject_pass_stall(s.h, -1, 0)   # disarm: always accepted
        s.step(2)
