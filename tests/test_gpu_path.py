"""A sparsity path (bicadmm_create_path): several instances of one problem that differ only
in kappa, solved together on one copy of A.  Each instance's iterates must be those of the
oracle run alone at its kappa (Sec. 3 iterations block, every step per instance): the
multi-column pass forms A X and A'D for all columns, each column has its own omega prox
(eq. p:GPU;omega), its own block solve right-hand side (eq. p:GPU;x) and its own consensus
step (eqs. global-z-t-updae, s-update-final, v-update).  FP64 on the CUDA-core
multi-column pass (1e-9); BF16 storage on the tensor-core pass (1e-4 against the oracle on
the BF16-rounded A)."""
import numpy as np
import pytest

from oracle import bicadmm_ref as ref
from paper_2405_16267_b300 import bicadmm as bc
from paper_2405_16267_b300 import synth

from gpu_util import rel_err

pytestmark = pytest.mark.gpu


def _oracles(P, kappas, iters, A=None):
    A = P.A if A is None else A
    out = []
    for k in kappas:
        o = ref.BiCADMM(A, P.b, P.loss, P.N, P.M, k, gamma=P.gamma, rho_c=P.rho)
        o.iterate(iters)
        out.append(o)
    return out


def _check_instances(ps, P, kappas, orcs, tol):
    for q, (k, o) in enumerate(zip(kappas, orcs)):
        st = ps.state(q)
        for key in ("x", "u", "z", "s"):
            want = getattr(o, key)
            assert rel_err(st[key], want) <= tol, (q, key, rel_err(st[key], want))
        z, sup = ps.x(q, with_support=True)
        assert np.array_equal(z, st["z"])
        assert list(sup) == list(ref.top_kappa(o.z, k)), q
        assert np.array_equal(st["s"] != 0, o.s != 0), q
        inf = ps.info(q)
        h = o.history[-1]
        if tol <= 1e-8:
            for f in ("d_r", "b_r"):
                assert abs(getattr(inf, f) - h[f]) <= 1e-8 * max(abs(h[f]), 1e-6), (q, f)
        assert abs(inf.t - o.t) <= tol * max(abs(o.t), 1e-12), q


@pytest.mark.parametrize("loss", [ref.LOSS_SQUARED, ref.LOSS_LOGISTIC, ref.LOSS_SQHINGE])
def test_path_fp64_matches_each_oracle(loss):
    import torch
    P = synth.small_problem(loss, m=1501, n=97, nnz=8, N=3, M=2, kappa=8, seed=31)
    kappas = [3, 8, 20]
    iters = 25
    with bc.PathSolver(P.A, P.b, loss=P.loss, N=P.N, M=P.M, kappas=kappas, gamma=P.gamma,
                       rho_c=P.rho, stream=torch.cuda.current_stream()) as ps:
        info = ps.step(iters)
        assert info.iters == iters
        _check_instances(ps, P, kappas, _oracles(P, kappas, iters), 1e-9)


def test_path_objective_per_instance():
    import torch
    P = synth.small_problem(ref.LOSS_LOGISTIC, m=1200, n=64, nnz=5, N=2, M=2, kappa=5, seed=8)
    kappas = [2, 5, 9, 30]
    with bc.PathSolver(P.A, P.b, loss=P.loss, N=P.N, M=P.M, kappas=kappas, gamma=P.gamma,
                       rho_c=P.rho, stream=torch.cuda.current_stream()) as ps:
        ps.step(20)
        for q in range(len(kappas)):
            z = ps.x(q)
            want = ref.objective(P.loss, P.A, P.b, z, P.gamma)
            assert abs(ps.info(q).objective - want) <= 1e-11 * abs(want), q


@pytest.mark.parametrize("pass_rows", [64, 128])
def test_path_bf16_tensor_core_pass(pass_rows):
    """BF16 storage, n <= 2048: the multi-column pass runs on the tensor cores (A X and A'D
    as skinny GEMMs over the instances' columns), on single SMs (64) or SM pairs (128)."""
    import torch
    P = synth.small_problem(ref.LOSS_LOGISTIC, m=4000, n=192, nnz=10, N=3, M=2, kappa=10, seed=12)
    kappas = [4, 10, 16, 40]
    iters = 15
    with bc.PathSolver(P.A.astype(np.float32), P.b, loss=P.loss, N=P.N, M=P.M, kappas=kappas,
                       gamma=P.gamma, rho_c=P.rho, precision=bc.PREC_BF16, pass_rows=pass_rows,
                       stream=torch.cuda.current_stream()) as ps:
        ps.step(iters)
        orcs = _oracles(P, kappas, iters, A=synth.round_to_bf16(P.A))
        for q, o in enumerate(orcs):
            st = ps.state(q)
            for key in ("x", "u", "z"):
                assert rel_err(st[key], getattr(o, key)) <= 1e-4, (q, key)


def test_path_solve_stops_when_every_instance_converges():
    import torch
    P = synth.sparse_linear(unit_columns=True)
    kappas = [5, 10, 15]
    with bc.PathSolver(P.A, P.b, loss=P.loss, N=P.N, M=P.M, kappas=kappas, gamma=P.gamma,
                       rho_c=P.rho, tol_rel=1e-6, check_every=1, max_iters=3000,
                       stream=torch.cuda.current_stream()) as ps:
        info = ps.solve()
        assert info.converged == 1 and info.iters < 3000
        for q in range(len(kappas)):
            iq = ps.info(q)
            assert max(iq.p_rel, iq.d_rel, iq.b_rel, iq.i_rel) <= 1e-6, q
            z, sup = ps.x(q, with_support=True)
            assert len(sup) == kappas[q] and list(sup) == list(ref.top_kappa(z, kappas[q]))
            assert iq.iters == info.iters


def test_path_rejects_bad_arguments():
    p = bc.default_params(m=100, n=20, N_shards=2, M_blocks=2, kappa=3)
    for kappas in ([3], [3] * 17, [0, 3], [3, 21]):
        with pytest.raises(bc.BicadmmError) as e:
            bc.create_path(p, kappas)
        assert e.value.code == -1
    ps = bc.default_params(m=100, n=20, N_shards=2, M_blocks=2, kappa=3, loss=bc.LOSS_SOFTMAX, K=3)
    with pytest.raises(bc.BicadmmError):
        bc.create_path(ps, [3, 4])
