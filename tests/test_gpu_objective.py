"""info.objective: F(z) = sum_r l(a_r z; b_r) + ||z||^2 / (2 gamma) of problem (p:SML)
(Sec. 2) at the GPU's consensus iterate z, computed on the device in FP64, against the
oracle's objective evaluated on that same z with the stored (rounded) A and b.

The zero start (no nonzero feature), a dense z (the l1 constraint inactive) and a
thresholded, sparse z (after many iterations) take different paths through the feature
compaction; every loss and storage precision is covered.
"""
import numpy as np
import pytest

from oracle import bicadmm_ref as ref
from paper_2405_16267_b300 import bicadmm as bc
from paper_2405_16267_b300 import synth

pytestmark = pytest.mark.gpu

TOL = 1e-11  # FP64 sums in a different order, over up to a few thousand rows


def _stored(A, precision):
    if precision == bc.PREC_FP32:
        return np.asarray(A, dtype=np.float32).astype(np.float64)
    if precision == bc.PREC_BF16:
        return synth.round_to_bf16(A)
    return np.asarray(A, dtype=np.float64)


def _check(P, precision, iters_list, K=1, **extra):
    import torch
    A = P.A if precision == bc.PREC_FP64 else np.asarray(P.A, dtype=np.float32)
    As = _stored(P.A, precision)
    # b is stored in the arithmetic type too (FP32 unless FP64): targets are rounded,
    # labels and class indices are exact
    bs = P.b if precision == bc.PREC_FP64 else np.asarray(P.b, dtype=np.float32).astype(np.float64)
    seen_nnz = []
    with bc.Solver(A, P.b, loss=P.loss, N=P.N, M=P.M, kappa=P.kappa, gamma=P.gamma,
                   rho_c=P.rho, precision=precision, K=K, stream=torch.cuda.current_stream(),
                   **extra) as s:
        done = 0
        for it in iters_list:
            info = s.step(it - done)
            done = it
            z = s.state()["z"]
            want = ref.objective(P.loss, As, bs, z, P.gamma, K=K)
            nnz = int(np.count_nonzero(z))
            seen_nnz.append(nnz)
            assert abs(info.objective - want) <= TOL * max(abs(want), 1.0), \
                (it, nnz, info.objective, want)
    return seen_nnz


def test_objective_linear_2000x200_fp64():
    P = synth.sparse_linear()
    nnz = _check(P, bc.PREC_FP64, [0, 1, 3, 60, 200])
    assert nnz[0] == 0 and 0 < nnz[-1] < P.n  # zero and thresholded z


def test_objective_dense_z_at_kappa_n():
    """kappa = n (the ridge limit): z = w is dense, every feature is compacted."""
    P = synth.small_problem(ref.LOSS_SQUARED, m=500, n=40, nnz=40, N=4, M=3, kappa=40, seed=2)
    nnz = _check(P, bc.PREC_FP64, [0, 5, 50])
    assert nnz[-1] == P.n


@pytest.mark.parametrize("loss,precision", [
    (ref.LOSS_LOGISTIC, bc.PREC_FP32),
    (ref.LOSS_SQHINGE, bc.PREC_BF16),
    (ref.LOSS_SQUARED, bc.PREC_FP32),
    (ref.LOSS_LOGISTIC, bc.PREC_FP64),
])
def test_objective_ragged(loss, precision):
    P = synth.small_problem(loss, m=1501, n=77, nnz=5, N=3, M=2, kappa=5, seed=21)
    _check(P, precision, [0, 1, 2, 40])


@pytest.mark.parametrize("precision,K,extra", [
    (bc.PREC_FP64, 3, {}),
    (bc.PREC_BF16, 4, {"pass_rows": 64}),   # tensor-core pass
])
def test_objective_softmax(precision, K, extra):
    P = synth.sparse_softmax(m=2000, n=96, K=K, nnz=10, N=3, M=2, kappa=10, seed=5)
    _check(P, precision, [0, 1, 30], K=K, **extra)


def test_objective_after_solve():
    import torch
    P = synth.sparse_linear()
    with bc.Solver(P.A, P.b, loss=P.loss, N=P.N, M=P.M, kappa=P.kappa, gamma=P.gamma,
                   rho_c=P.rho, stream=torch.cuda.current_stream()) as s:
        info = s.solve()
        z = s.state()["z"]
    want = ref.objective(P.loss, P.A, P.b, z, P.gamma)
    assert abs(info.objective - want) <= TOL * abs(want)
