"""FP64 polish on the selected support (bicadmm_get_x with polished = 1) against the
oracle's restricted solve, and the support output."""
import numpy as np
import pytest

from oracle import bicadmm_ref as ref
from paper_2405_16267_b300 import bicadmm as bc
from paper_2405_16267_b300 import synth

from gpu_util import rel_err, run_oracle

pytestmark = pytest.mark.gpu

TOL64 = 1e-9


def _gpu_polish(P, iters, precision=bc.PREC_FP64, A=None, b=None):
    import torch
    A = P.A if A is None else A
    b = P.b if b is None else b
    if precision == bc.PREC_FP32:
        A = np.asarray(A, dtype=np.float32)
    with bc.Solver(A, b, loss=P.loss, N=P.N, M=P.M, kappa=P.kappa, gamma=P.gamma, rho_c=P.rho,
                   precision=precision, stream=torch.cuda.current_stream()) as s:
        s.step(iters)
        z, supp0 = bc.get_x(s.h, P.n, polished=False, with_support=True, kappa=P.kappa)
        xp, supp = bc.get_x(s.h, P.n, polished=True, with_support=True, kappa=P.kappa)
    return z, supp0, xp, supp


def test_polish_linear_2000x200():
    P = synth.sparse_linear()
    z, supp0, xp, supp = _gpu_polish(P, 200)
    o = run_oracle(P, 200)
    assert list(supp0) == list(o.support()) and list(supp) == list(o.support())
    want = ref.polish(P.A, P.b, P.loss, P.gamma, o.support())
    assert rel_err(xp, want) <= TOL64
    assert np.count_nonzero(xp) <= P.kappa


@pytest.mark.parametrize("loss", [ref.LOSS_LOGISTIC, ref.LOSS_SQHINGE])
def test_polish_classification(loss):
    P = synth.small_problem(loss, m=4000, n=90, nnz=6, N=4, M=3, kappa=6, seed=12)
    z, supp0, xp, supp = _gpu_polish(P, 60)
    o = run_oracle(P, 60)
    assert list(supp) == list(o.support())
    want = ref.polish(P.A, P.b, loss, P.gamma, o.support())
    assert rel_err(xp, want) <= TOL64


def test_polish_fp32_mode_is_fp64_on_the_rounded_matrix():
    P = synth.sparse_logistic(m=20000, n=300, nnz=8, N=4, M=3, kappa=8, rho=0.5, dtype=np.float64)
    A32 = synth.round_to_f32(P.A)
    z, supp0, xp, supp = _gpu_polish(P, 40, precision=bc.PREC_FP32, A=A32)
    want = ref.polish(A32, P.b, P.loss, P.gamma, np.asarray(supp))
    assert list(supp) == list(ref.top_kappa(z, P.kappa))
    assert rel_err(xp, want) <= TOL64


def test_polish_large_kappa_tiles():
    """kappa spanning several 32-wide Hessian tiles with a ragged last tile."""
    P = synth.sparse_linear(m=3000, n=120, nnz=70, N=3, M=2, kappa=70, unit_columns=True, seed=5)
    z, supp0, xp, supp = _gpu_polish(P, 30)
    want = ref.polish(P.A, P.b, P.loss, P.gamma, np.asarray(supp))
    assert list(supp) == list(ref.top_kappa(z, P.kappa))
    assert rel_err(xp, want) <= TOL64
