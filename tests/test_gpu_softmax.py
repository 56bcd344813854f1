"""Softmax (K classes) and BF16-storage paths of the CUDA library against the FP64 oracle.

FP64 mode: every state array within 1e-9 relative after a fixed iteration count, and the
entrywise top-kappa support identical.  FP32 and BF16 modes: within 1e-4 relative of the
oracle run on the same rounded A (FP32-rounded, resp. BF16-rounded), so the comparison
isolates the arithmetic.
"""
import numpy as np
import pytest

from oracle import bicadmm_ref as ref
from paper_2405_16267_b300 import bicadmm as bc
from paper_2405_16267_b300 import synth

from gpu_util import compare_state, run_gpu, run_oracle

pytestmark = pytest.mark.gpu

TOL64 = 1e-9
TOL32 = 1e-4


@pytest.mark.parametrize("case", [
    # (m, n, K, N, M, kappa, iters, J)
    (1003, 77, 3, 3, 2, 8, 40, 1),     # ragged shards, blocks, panels; K -> 4-class tiles
    (900, 60, 10, 4, 3, 25, 30, 1),    # the 10-class tiles
    (640, 40, 16, 2, 2, 30, 25, 1),    # 16 classes
    (500, 33, 2, 2, 1, 4, 30, 1),      # K = 2, one block
    (800, 50, 5, 3, 2, 12, 20, 2),     # J = 2 inner sweeps
    (37, 5, 3, 2, 2, 1, 20, 1),        # tiny, kappa = 1
])
def test_softmax_fp64_vs_oracle(case):
    m, n, K, N, M, kappa, iters, J = case
    P = synth.sparse_softmax(m=m, n=n, K=K, nnz=min(kappa, n * K), N=N, M=M, kappa=kappa,
                             seed=21, dtype=np.float64)
    st, _ = run_gpu(P, iters, J=J)
    o = run_oracle(P, iters, J=J)
    compare_state(st, o, TOL64)


def test_softmax_kappa_full():
    """kappa = n K: the l0 constraint is void."""
    P = synth.sparse_softmax(m=400, n=12, K=4, nnz=10, N=2, M=2, kappa=48, seed=2, dtype=np.float64)
    st, _ = run_gpu(P, 30)
    compare_state(st, run_oracle(P, 30), TOL64)


def test_softmax_fp32_vs_oracle_on_rounded_A():
    P = synth.sparse_softmax(m=6000, n=200, K=10, nnz=40, N=4, M=4, kappa=40, seed=5)
    A32 = synth.round_to_f32(P.A)
    st, _ = run_gpu(P, 25, precision=bc.PREC_FP32, A=A32)
    compare_state(st, run_oracle(P, 25, A=A32), TOL32)


@pytest.mark.parametrize("pass_rows", [8, 0])
def test_softmax_bf16_vs_oracle_on_rounded_A(pass_rows):
    """pass_rows 8: CUDA-core pass; 0: the tensor-core pass (64-row panels)."""
    P = synth.sparse_softmax(m=6000, n=200, K=10, nnz=40, N=4, M=4, kappa=40, seed=6)
    Ab = synth.round_to_bf16(P.A)
    st, _ = run_gpu(P, 25, precision=bc.PREC_BF16, A=P.A, pass_rows=pass_rows)
    compare_state(st, run_oracle(P, 25, A=Ab), TOL32)


@pytest.mark.parametrize("case", [
    # (m, n, K, N, M, kappa, iters)
    (20000, 2000, 10, 4, 4, 100, 6),    # 16 slabs, the last 64-column box partly outside A
    (60000, 300, 10, 16, 2, 40, 8),     # several shards per CTA, ragged panels
    (9000, 2048, 3, 3, 4, 30, 6),       # full 2048-column rows, 4-class tiles
    (5000, 130, 16, 5, 2, 50, 10),      # 16 classes, one partial slab
    (3000, 200, 10, 40, 2, 20, 6),      # 75-row shards: a full and an 11-row panel each
])
@pytest.mark.parametrize("pass_rows", [64, 128])
def test_softmax_bf16_tensor_core_pass(case, pass_rows):
    """64: single-SM kernel (64-row panels); 128: the pair kernel (two-CTA clusters split the
    columns: 16 slabs 8 / 8, 3 slabs 2 / 1, 2 slabs of which the second is mostly padding)."""
    m, n, K, N, M, kappa, iters = case
    P = synth.sparse_softmax(m=m, n=n, K=K, nnz=kappa, N=N, M=M, kappa=kappa, seed=13)
    Ab = synth.round_to_bf16(P.A)
    st, _ = run_gpu(P, iters, precision=bc.PREC_BF16, A=P.A, pass_rows=pass_rows)
    compare_state(st, run_oracle(P, iters, A=Ab), TOL32)


def test_pair_pass_needs_two_slabs():
    """128-row panels split the row's 128-column slabs between two CTAs: rows of at most 128
    columns are refused (auto takes the single-SM kernel there)."""
    P = synth.sparse_softmax(m=500, n=100, K=4, nnz=10, N=2, M=2, kappa=10, seed=3)
    with pytest.raises(bc.BicadmmError) as e:
        run_gpu(P, 2, precision=bc.PREC_BF16, A=P.A, pass_rows=128)
    assert e.value.code == -7
    st, _ = run_gpu(P, 6, precision=bc.PREC_BF16, A=P.A)
    compare_state(st, run_oracle(P, 6, A=synth.round_to_bf16(P.A)), TOL32)


@pytest.mark.parametrize("loss", [ref.LOSS_SQUARED, ref.LOSS_LOGISTIC, ref.LOSS_SQHINGE])
def test_bf16_storage_k1_vs_oracle_on_rounded_A(loss):
    P = synth.small_problem(loss, m=4000, n=300, nnz=8, N=4, M=3, kappa=8, seed=7)
    Ab = synth.round_to_bf16(P.A)
    b = P.b.astype(np.float32).astype(np.float64)
    st, _ = run_gpu(P, 30, precision=bc.PREC_BF16, A=P.A, b=b)
    compare_state(st, run_oracle(P, 30, A=Ab, b=b), TOL32)


def test_bf16_device_input():
    import torch
    P = synth.sparse_softmax(m=3000, n=128, K=10, nnz=20, N=2, M=2, kappa=20, seed=8)
    A = torch.tensor(P.A, dtype=torch.float32, device="cuda").to(torch.bfloat16)
    Ab = A.double().cpu().numpy()
    st, _ = run_gpu(P, 15, precision=bc.PREC_BF16, A=A, b=torch.tensor(P.b, device="cuda"))
    compare_state(st, run_oracle(P, 15, A=Ab), TOL32)


def test_softmax_deterministic_and_model_layout():
    import torch
    P = synth.sparse_softmax(m=2000, n=64, K=10, nnz=16, N=4, M=2, kappa=16, seed=9, dtype=np.float64)
    a, _ = run_gpu(P, 20)
    b, _ = run_gpu(P, 20)
    for k in ("z", "x", "u", "omega", "nu", "s"):
        assert np.array_equal(a[k], b[k]), k
    with bc.Solver(P.A, P.b, loss=P.loss, N=P.N, M=P.M, kappa=P.kappa, gamma=P.gamma,
                   rho_c=P.rho, K=P.K, stream=torch.cuda.current_stream()) as s:
        s.step(20)
        x, sup = bc.get_x(s.h, P.n * P.K, with_support=True, kappa=P.kappa)
        assert np.array_equal(x, a["z"])
        assert list(sup) == list(ref.top_kappa(a["z"], P.kappa))


def test_softmax_rejects_bad_labels_and_params():
    import torch
    P = synth.sparse_softmax(m=300, n=20, K=3, nnz=4, N=2, M=2, kappa=4, seed=1, dtype=np.float64)
    bad = P.b.copy()
    bad[7] = 3.0  # class index out of range
    with pytest.raises(bc.BicadmmError) as e:
        bc.Solver(P.A, bad, loss=P.loss, N=2, M=2, kappa=4, K=3, stream=torch.cuda.current_stream())
    assert e.value.code == -1
    bad[7] = 0.5  # not integral
    with pytest.raises(bc.BicadmmError):
        bc.Solver(P.A, bad, loss=P.loss, N=2, M=2, kappa=4, K=3, stream=torch.cuda.current_stream())
    with pytest.raises(bc.BicadmmError):  # K = 1 with softmax
        bc.Solver(P.A, P.b, loss=P.loss, N=2, M=2, kappa=4, K=1, stream=torch.cuda.current_stream())


@pytest.mark.parametrize("precision", [bc.PREC_FP64, bc.PREC_BF16])
def test_softmax_polish_vs_oracle(precision):
    """FP64 polish on the entrywise support: the restricted softmax problem solved by damped
    Newton on the device equals the oracle's polish on the same support (and the same data:
    the BF16-rounded A for BF16 storage)."""
    import torch
    P = synth.sparse_softmax(m=3000, n=40, K=4, nnz=8, N=3, M=2, kappa=8, seed=17, dtype=np.float64,
                             scale=1.5)
    A_used = P.A if precision == bc.PREC_FP64 else synth.round_to_bf16(P.A)
    A_in = P.A if precision == bc.PREC_FP64 else P.A.astype(np.float32)
    with bc.Solver(A_in, P.b, loss=P.loss, N=P.N, M=P.M, kappa=P.kappa, gamma=P.gamma, rho_c=P.rho,
                   K=P.K, precision=precision, stream=torch.cuda.current_stream()) as s:
        s.step(60)
        x, sup = bc.get_x(s.h, P.n * P.K, polished=True, with_support=True, kappa=P.kappa)
    want = ref.polish(A_used, P.b, ref.LOSS_SOFTMAX, P.gamma, np.array(sup), K=P.K)
    assert np.count_nonzero(x) <= P.kappa
    np.testing.assert_allclose(x, want, rtol=0, atol=1e-9 * np.abs(want).max())
