"""Residual traces for the paper's bi-linear penalty sweep (Sec. 4, empirical convergence,
Fig. 1: n = 4000, m = 10000, s_l = 0.8, rho_b in {2, 4, 8, 16} with rho_b <= alpha rho_c,
alpha = 0.5).  The figure's data are not in the paper, so this checks its stated shape:
rho_b barely changes the primal and dual residuals but changes how fast the bi-linear
residual converges.  rho_c = 32 (the smallest with rho_b = 16 <= 0.5 rho_c), N = 4 nodes,
unit-norm columns per node, squared loss."""
import numpy as np
import pytest

from paper_2405_16267_b300 import bicadmm as bc
from paper_2405_16267_b300 import synth

pytestmark = pytest.mark.gpu


def test_rho_b_sweep_shape():
    import torch
    P = synth.sparse_linear(m=10000, n=4000, nnz=800, noise=0.01, N=4, M=4, kappa=800,
                            unit_columns="shard", seed=0)
    A = torch.tensor(P.A, device="cuda")
    b = torch.tensor(P.b, device="cuda")
    traces = {}
    for rho_b in (2.0, 4.0, 8.0, 16.0):
        with bc.Solver(A, b, loss=bc.LOSS_SQUARED, N=4, M=4, kappa=800, gamma=10.0, rho_c=32.0,
                       rho_b=rho_b, stream=torch.cuda.current_stream()) as s:
            s.step(250)
            traces[rho_b] = bc.get_trace(s.h)
    for k, tr in traces.items():
        assert len(tr["iter"]) == 250 and tr["iter"][-1] == 250
        assert np.all(np.isfinite(tr["p_r"]))
    def spread(key):
        # median over iterations 20..80 of log10(max / min across rho_b), values floored at 1e-16
        v = np.maximum(np.array([traces[r][key][19:80] for r in traces]), 1e-16)
        return float(np.median(np.log10(v.max(axis=0) / v.min(axis=0))))

    sp, sd, sb = spread("p_rel"), spread("d_rel"), spread("b_rel")
    assert sp < 0.3 and sd < 0.3, (sp, sd)   # within a factor of 2 across rho_b
    assert sb > 1.0 and sb > 5 * max(sp, sd), (sb, sp, sd)   # at least a decade apart
    # the bi-linear residual settles to rounding within the run for every rho_b
    last = np.array([int(np.flatnonzero(traces[r]["b_rel"] > 1e-12).max()) + 1 for r in traces])
    assert np.all(last > 1) and np.all(last < 250), last
