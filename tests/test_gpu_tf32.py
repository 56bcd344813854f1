"""TF32 storage (BICADMM_PREC_TF32): A rounded to TF32 at setup, the Gram matrices on the
tensor cores in kind::tf32, everything else as in FP32 mode.  Parity is stated against the
oracle run on the TF32-rounded A (and the FP32-rounded targets), at the mixed-precision
tolerance 1e-4; the run must also be measurably closer to that than to the oracle on the
unrounded FP32 A, which shows the rounding took place."""
import numpy as np
import pytest

from oracle import bicadmm_ref as ref
from paper_2405_16267_b300 import bicadmm as bc
from paper_2405_16267_b300 import synth

from gpu_util import compare_state, rel_err, run_gpu, run_oracle

pytestmark = pytest.mark.gpu

TOL = 1e-4


def _b32(P):
    return np.asarray(P.b, dtype=np.float32).astype(np.float64)


@pytest.mark.parametrize("loss,m,n,N,M,kappa,iters", [
    (ref.LOSS_SQUARED, 2003, 131, 3, 2, 6, 40),
    (ref.LOSS_LOGISTIC, 3001, 517, 3, 4, 6, 25),     # blocks starting off any alignment grid
    (ref.LOSS_SQHINGE, 1500, 300, 4, 1, 5, 25),      # a 300-column block: two chunk widths
])
def test_tf32_vs_oracle_on_rounded_A(loss, m, n, N, M, kappa, iters):
    P = synth.small_problem(loss, m=m, n=n, nnz=kappa, N=N, M=M, kappa=kappa, seed=m)
    At = synth.round_to_tf32(P.A)
    st, _ = run_gpu(P, iters, precision=bc.PREC_TF32)
    o = run_oracle(P, iters, A=At, b=_b32(P))
    compare_state(st, o, TOL)
    # the GPU saw the TF32 values, not the FP32 ones
    o32 = run_oracle(P, iters, A=P.A.astype(np.float32).astype(np.float64), b=_b32(P))
    assert rel_err(st["x"], o.x) < 0.1 * rel_err(st["x"], o32.x)


def test_tf32_softmax_vs_oracle_on_rounded_A():
    P = synth.sparse_softmax(m=2400, n=150, K=3, nnz=8, N=3, M=2, kappa=8, seed=12)
    st, _ = run_gpu(P, 20, precision=bc.PREC_TF32)
    o = run_oracle(P, 20, A=synth.round_to_tf32(P.A))
    compare_state(st, o, TOL)


def test_tf32_device_input():
    import torch
    P = synth.small_problem(ref.LOSS_LOGISTIC, m=1800, n=200, nnz=5, N=3, M=2, kappa=5, seed=3)
    A = torch.tensor(P.A.astype(np.float32), device="cuda")
    b = torch.tensor(P.b, device="cuda")
    st, _ = run_gpu(P, 20, precision=bc.PREC_TF32, A=A, b=b)
    o = run_oracle(P, 20, A=synth.round_to_tf32(P.A), b=_b32(P))
    compare_state(st, o, TOL)
