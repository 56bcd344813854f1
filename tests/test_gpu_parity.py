"""CUDA path vs the FP64 oracle, element by element, on the same seeded inputs.

FP64 mode: every state array within 1e-9 relative after a fixed iteration count and the
selected support identical.  FP32 mode: within 1e-4 relative of the oracle run on the
FP32-rounded A.
"""
import numpy as np
import pytest

from oracle import bicadmm_ref as ref
from paper_2405_16267_b300 import bicadmm as bc
from paper_2405_16267_b300 import synth

from gpu_util import compare_state, rel_err, run_gpu, run_oracle

pytestmark = pytest.mark.gpu

TOL64 = 1e-9
TOL32 = 1e-4


def test_linear_2000x200_fp64_200_iterations():
    """The 2000 x 200 sparse-regression workload: N=4, M=2, kappa=10, rho=1, 200 iters."""
    P = synth.sparse_linear()
    st, info = run_gpu(P, 200)
    o = run_oracle(P, 200)
    compare_state(st, o, TOL64)
    h = o.history[-1]
    for k in ("p_r", "d_r", "b_r", "i_r"):
        assert abs(getattr(info, k) - h[k]) <= 1e-8 * max(abs(h[k]), 1e-6), k
    assert info.iters == 200


@pytest.mark.parametrize("case", [
    # (loss, m, n, N, M, kappa, iters, J)
    (ref.LOSS_SQUARED, 1003, 77, 3, 4, 5, 60, 1),     # ragged shards, blocks, panels
    (ref.LOSS_SQUARED, 37, 5, 2, 2, 1, 40, 1),        # tiny, kappa = 1
    (ref.LOSS_SQUARED, 500, 40, 4, 3, 40, 80, 1),     # kappa = n (ridge limit)
    (ref.LOSS_SQUARED, 640, 64, 1, 1, 6, 50, 1),      # one shard, one block
    (ref.LOSS_SQUARED, 800, 96, 5, 3, 8, 30, 3),      # J = 3 inner sweeps
    (ref.LOSS_LOGISTIC, 1500, 60, 4, 2, 6, 40, 1),
    (ref.LOSS_SQHINGE, 1200, 50, 3, 2, 5, 40, 1),
    (ref.LOSS_SQUARED, 3000, 300, 7, 5, 12, 25, 2),   # several tiles wide
])
def test_small_cases_fp64(case):
    loss, m, n, N, M, kappa, iters, J = case
    P = synth.small_problem(loss, m=m, n=n, nnz=min(kappa, n), N=N, M=M, kappa=kappa, seed=11)
    st, _ = run_gpu(P, iters, J=J)
    o = run_oracle(P, iters, J=J)
    compare_state(st, o, TOL64)


def test_unit_columns_converges_like_oracle():
    """Paper's data recipe (unit-norm columns): both reach the planted support."""
    P = synth.sparse_linear(unit_columns=True)
    st, info = run_gpu(P, 120)
    o = run_oracle(P, 120)
    compare_state(st, o, TOL64)
    assert set(ref.top_kappa(st["z"], P.kappa)) == set(np.flatnonzero(P.x_star))


def test_fp32_logistic_vs_oracle_on_rounded_A():
    P = synth.sparse_logistic(m=20000, n=300, nnz=8, N=4, M=3, kappa=8, rho=0.5, dtype=np.float64)
    A32 = synth.round_to_f32(P.A)
    st, _ = run_gpu(P, 30, precision=bc.PREC_FP32, A=A32)
    o = run_oracle(P, 30, A=A32)
    compare_state(st, o, TOL32)


def test_fp32_linear_vs_oracle_on_rounded_A():
    P = synth.sparse_linear(m=6000, n=400, nnz=12, N=4, M=4, kappa=12, unit_columns=True)
    A32 = synth.round_to_f32(P.A)
    b32 = P.b.astype(np.float32).astype(np.float64)
    st, _ = run_gpu(P, 40, precision=bc.PREC_FP32, A=A32, b=b32)
    o = run_oracle(P, 40, A=A32, b=b32)
    compare_state(st, o, TOL32)


def test_runs_are_bitwise_deterministic():
    P = synth.small_problem(ref.LOSS_LOGISTIC, m=3000, n=120, nnz=6, N=4, M=2, kappa=6, seed=3)
    a, _ = run_gpu(P, 25)
    b, _ = run_gpu(P, 25)
    for k in ("z", "x", "u", "omega", "nu", "s"):
        assert np.array_equal(a[k], b[k]), k


def test_step_in_pieces_equals_one_call():
    import torch
    P = synth.sparse_linear(m=900, n=90, nnz=5, N=3, M=2, kappa=5)
    with bc.Solver(P.A, P.b, loss=P.loss, N=P.N, M=P.M, kappa=P.kappa, gamma=P.gamma,
                   rho_c=P.rho, stream=torch.cuda.current_stream()) as s:
        s.step(7); s.step(0); s.step(13)
        z1 = s.x()
    st, _ = run_gpu(P, 20)
    assert np.array_equal(z1, st["z"])


@pytest.mark.parametrize("rows,stages", [(1, 1), (2, 3), (4, 2), (8, 4)])
def test_pass_tiling_choices_agree(rows, stages):
    """Every panel height / stage count gives the oracle's iterates."""
    P = synth.small_problem(ref.LOSS_LOGISTIC, m=2001, n=130, nnz=6, N=3, M=2, kappa=6, seed=4)
    st, _ = run_gpu(P, 20, pass_rows=rows, pass_stages=stages)
    o = run_oracle(P, 20)
    compare_state(st, o, TOL64)


@pytest.mark.parametrize("rows,stages", [(8, 1), (4, 1), (2, 1), (0, 0)])
def test_pass_tiling_choices_fp32(rows, stages):
    """FP32 storage, one-stage panels (the panel held in registers while its stage reloads)
    and the automatic choice: the oracle's iterates on the FP32-rounded A."""
    P = synth.small_problem(ref.LOSS_LOGISTIC, m=3001, n=700, nnz=6, N=3, M=2, kappa=6, seed=8)
    A32 = P.A.astype(np.float32).astype(np.float64)
    st, _ = run_gpu(P, 20, precision=bc.PREC_FP32, pass_rows=rows, pass_stages=stages)
    o = run_oracle(P, 20, A=A32, b=P.b)
    compare_state(st, o, 1e-4)


def test_solve_stops_at_tolerance():
    import torch
    P = synth.sparse_linear(unit_columns=True)
    with bc.Solver(P.A, P.b, loss=P.loss, N=P.N, M=P.M, kappa=P.kappa, gamma=P.gamma,
                   rho_c=P.rho, tol_rel=1e-6, check_every=1, max_iters=2000,
                   stream=torch.cuda.current_stream()) as s:
        info = s.solve()
    assert info.converged == 1
    o = ref.BiCADMM(P.A, P.b, P.loss, P.N, P.M, P.kappa, gamma=P.gamma, rho_c=P.rho)
    assert o.solve(tol_rel=1e-6, max_iters=2000)
    assert info.iters == o.iters
    assert max(info.p_rel, info.d_rel, info.b_rel, info.i_rel) <= 1e-6


def test_device_input_buffers():
    import torch
    P = synth.sparse_linear(m=1000, n=100, nnz=5, N=2, M=2, kappa=5)
    A = torch.tensor(P.A, device="cuda")
    b = torch.tensor(P.b, device="cuda")
    st, _ = run_gpu(P, 15, A=A, b=b)
    o = run_oracle(P, 15)
    compare_state(st, o, TOL64)


def test_errors_are_reported_not_raised_across_abi():
    import torch
    P = synth.sparse_linear(m=100, n=20, nnz=3, N=2, M=2, kappa=3)
    p = bc.default_params(m=100, n=20, N_shards=2, M_blocks=2, kappa=3)
    h = bc.create(p, torch.cuda.current_stream())
    try:
        with pytest.raises(bc.BicadmmError) as e:
            bc.step(h, 1)  # before setup
        assert e.value.code == -4
        bc.setup(h, P.A, P.b)
        bc.step(h, 2)
        with pytest.raises(bc.BicadmmError):
            bc.get_state(h, bc.FIELD_Z, 19)
    finally:
        bc.destroy(h)
