"""The setup's block inverses (rho_l A_ij'A_ij + c0 I)^-1 of the x_ij solve (eq. p:GPU;x)
against the oracle's factorisation of the same matrices, in every storage precision: FP64
Gram matrices on the CUDA cores, FP32 (TF32 hi/lo pairs) and TF32 on the tensor cores in
kind::tf32 (blocks of any width and column offset), BF16 on the tensor cores (column windows that
start off the 64-column grid, blocks wider than one 256-column chunk, shards whose length
is not a multiple of the 64-row stage, a shard shorter than one stage), and blocks wide
enough for the narrower Cholesky panels and for the column-by-column fallback."""
import numpy as np
import pytest
import scipy.linalg

from oracle import bicadmm_ref as ref
from paper_2405_16267_b300 import bicadmm as bc
from paper_2405_16267_b300 import synth

pytestmark = pytest.mark.gpu

CASES = [  # (m, n, N, M, K)
    (3001, 517, 3, 4, 1),     # blocks of 130/129 columns starting off the 64-grid
    (2100, 700, 2, 2, 1),     # 350-column blocks: several strips and chunks
    (1000, 90, 5, 1, 1),      # 200-row shards (3 stages + a 8-row tail)
    (220, 64, 4, 1, 1),       # 55-row shards: one partial stage
    (1500, 150, 3, 2, 3),     # softmax, three classes (same block matrices)
    (2000, 900, 2, 1, 1),     # a 900-column block: 16-column Cholesky panels
    (4000, 640, 2, 1, 1),     # a 640-column block: ten 64-row chunks per Cholesky panel
    (5000, 1300, 2, 1, 1),    # 1300 columns: 16-column panels, twenty chunks per panel
    (3600, 3500, 1, 1, 1),    # a 3500-column block: too wide for a panel in shared memory,
                              # the column-by-column kernels
]
# relative error per unit condition number of the block matrix: FP64 arithmetic; FP32
# storage of P (and FP32 partial sums of the products: CUDA cores flush to FP64 every 256
# rows, the tensor cores accumulate a shard in FP32)
TOL = {bc.PREC_FP64: 1e-13, bc.PREC_FP32: 3e-6, bc.PREC_BF16: 3e-6, bc.PREC_TF32: 3e-6}


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("precision", [bc.PREC_FP64, bc.PREC_FP32, bc.PREC_BF16, bc.PREC_TF32])
def test_block_inverses_match_oracle(case, precision):
    m, n, N, M, K = case
    if K == 1:
        P = synth.small_problem(ref.LOSS_SQUARED, m=m, n=n, nnz=3, N=N, M=M, kappa=3, seed=m + n)
    else:
        P = synth.sparse_softmax(m=m, n=n, K=K, nnz=6, N=N, M=M, kappa=6, seed=m + n)
    A = P.A
    if precision == bc.PREC_FP32:
        A = A.astype(np.float32).astype(np.float64)
    elif precision == bc.PREC_BF16:
        A = synth.round_to_bf16(P.A)
    elif precision == bc.PREC_TF32:
        A = synth.round_to_tf32(P.A)
    o = ref.BiCADMM(A, P.b, P.loss, P.N, P.M, P.kappa, gamma=P.gamma, rho_c=P.rho, K=K)
    A_in = P.A if precision == bc.PREC_FP64 else P.A.astype(np.float32)
    with bc.Solver(A_in, P.b, loss=P.loss, N=P.N, M=P.M, kappa=P.kappa, gamma=P.gamma,
                   rho_c=P.rho, precision=precision, K=K) as s:
        got = s.block_inverses(o.blocks)
    for i in range(N):
        for j in range(M):
            nj = o.blocks[j][1] - o.blocks[j][0]
            want = scipy.linalg.cho_solve(o.factors[i][j], np.eye(nj))
            kappa = np.linalg.cond(want)
            err = np.max(np.abs(got[i][j] - want)) / np.max(np.abs(want))
            assert err <= TOL[precision] * max(kappa, 10.0), (i, j, err, kappa)


@pytest.mark.parametrize("K", [1, 4])
def test_host_bf16_input_equals_rounded_fp32_input(K):
    """BF16 storage from a host BF16 matrix (copied shard by shard, the Gram matrices of a
    shard overlapping the later copies) and from an FP32 matrix rounded at setup: the same
    block inverses and, after a few iterations, the same state bit for bit."""
    import torch
    if K == 1:
        P = synth.small_problem(ref.LOSS_LOGISTIC, m=2500, n=300, nnz=5, N=5, M=2, kappa=5, seed=9)
    else:
        P = synth.sparse_softmax(m=2500, n=200, K=K, nnz=8, N=5, M=2, kappa=8, seed=9)
    o = ref.BiCADMM(P.A, P.b, P.loss, P.N, P.M, P.kappa, K=K)
    A32 = torch.from_numpy(P.A.astype(np.float32))
    states = []
    for A_in in (A32.to(torch.bfloat16).pin_memory(), A32.numpy()):
        with bc.Solver(A_in, P.b, loss=P.loss, N=P.N, M=P.M, kappa=P.kappa, gamma=P.gamma,
                       rho_c=P.rho, precision=bc.PREC_BF16, K=K) as s:
            inv = s.block_inverses(o.blocks)
            s.step(6)
            states.append((inv, s.state()))
    (inv_a, st_a), (inv_b, st_b) = states
    for i in range(P.N):
        for j in range(P.M):
            assert np.array_equal(inv_a[i][j], inv_b[i][j])
    for key in ("x", "z", "omega", "nu"):
        assert np.array_equal(st_a[key], st_b[key]), key
