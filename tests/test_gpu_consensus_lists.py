"""The consensus CTA's warm-started step on the entry lists of the all-SM prep kernel (K > 1:
softmax and sparsity paths).  With the previous root tau_prev > 0, only the entries of
U = {r : tau_r > tau_prev or z_r != 0 or s_r != 0} can change or add to a sum of the global
step (eqs. global-z-t-updae, s-update-final, v-update of Sec. 3); the step visits only them.
Checked: the trace says the list form ran, and the states still equal the oracle's."""
import numpy as np
import pytest

from oracle import bicadmm_ref as ref
from paper_2405_16267_b300 import bicadmm as bc
from paper_2405_16267_b300 import synth

from gpu_util import compare_state, run_oracle, rel_err

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("case", [
    # (m, n, K, N, M, kappa, iters)
    (1003, 77, 3, 3, 2, 8, 40),
    (900, 60, 10, 4, 3, 25, 30),
    (640, 40, 16, 2, 2, 30, 25),
])
def test_softmax_lists_match_oracle(case):
    import torch
    m, n, K, N, M, kappa, iters = case
    P = synth.sparse_softmax(m=m, n=n, K=K, nnz=min(kappa, n * K), N=N, M=M, kappa=kappa,
                             seed=21, dtype=np.float64)
    with bc.Solver(P.A, P.b, loss=P.loss, N=P.N, M=P.M, kappa=P.kappa, gamma=P.gamma,
                   rho_c=P.rho, K=P.K, stream=torch.cuda.current_stream()) as s:
        s.step(iters)
        st = s.state()
        tr = bc.get_trace(s.h)
    compare_state(st, run_oracle(P, iters), 1e-9)
    used = tr["zt_lists"][5:]
    assert used.size and used.mean() >= 0.5, tr["zt_lists"]
    # the first step (tau_prev = 0) visits every entry
    assert tr["zt_lists"][0] == 0


@pytest.mark.parametrize("loss", [ref.LOSS_LOGISTIC, ref.LOSS_SQUARED])
def test_path_lists_match_each_oracle(loss):
    """Each instance's consensus CTA works on its own slice of the lists (indices within the
    instance, counts per instance)."""
    import torch
    P = synth.small_problem(loss, m=1501, n=97, nnz=8, N=3, M=2, kappa=8, seed=31)
    kappas = [3, 8, 20]
    iters = 30
    with bc.PathSolver(P.A, P.b, loss=P.loss, N=P.N, M=P.M, kappas=kappas, gamma=P.gamma,
                       rho_c=P.rho, stream=torch.cuda.current_stream()) as ps:
        ps.step(iters)
        tr = bc.get_trace(ps.h)
        for q, k in enumerate(kappas):
            o = ref.BiCADMM(P.A, P.b, P.loss, P.N, P.M, k, gamma=P.gamma, rho_c=P.rho)
            o.iterate(iters)
            st = ps.state(q)
            for key in ("x", "u", "z", "s"):
                assert rel_err(st[key], getattr(o, key)) <= 1e-9, (q, key)
            assert np.array_equal(st["s"] != 0, o.s != 0), q
    assert tr["zt_lists"][5:].mean() >= 0.5, tr["zt_lists"]
