"""CUDA-graph replay of outer iterations (bicadmm_set_graph): the iterates, the residual
record and the launch count equal those of eager stepping, bit for bit, for every loss and
any split of the iterations into step calls."""
import numpy as np
import pytest

from paper_2405_16267_b300 import bicadmm as bc
from paper_2405_16267_b300 import synth

pytestmark = pytest.mark.gpu


def _solver(P, stream, precision=bc.PREC_FP64, **kw):
    return bc.Solver(P.A, P.b, loss=P.loss, N=P.N, M=P.M, kappa=P.kappa, gamma=P.gamma,
                     rho_c=P.rho, precision=precision, stream=stream, **kw)


@pytest.mark.parametrize("loss", [bc.LOSS_SQUARED, bc.LOSS_LOGISTIC, bc.LOSS_SQHINGE])
@pytest.mark.parametrize("precision", [bc.PREC_FP64, bc.PREC_FP32])
def test_graph_replay_equals_eager(loss, precision):
    import torch
    P = synth.small_problem(loss, m=2000, n=200, nnz=10, N=4, M=2, kappa=10, seed=11)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        with _solver(P, stream, precision) as eager, _solver(P, stream, precision) as g:
            g.set_graph(5)
            eager.step(37)
            for k in (1, 10, 26):      # capture on the first call, replays plus remainders
                g.step(k)
            a, b = eager.state(), g.state()
            for key in ("x", "u", "z", "s", "omega", "nu"):
                assert np.array_equal(a[key], b[key]), key
            assert (a["t"], a["v"]) == (b["t"], b["v"])
            ta, tb = bc.get_trace(eager.h), bc.get_trace(g.h)
            assert ta.keys() == tb.keys() and len(ta["p_r"]) == 37
            for key in ta:
                assert np.array_equal(ta[key], tb[key]), key
            assert bc.step(eager.h, 0).kernel_launches == bc.step(g.h, 0).kernel_launches


def test_graph_solve_matches_eager_and_off_switch():
    import torch
    P = synth.small_problem(bc.LOSS_SQUARED, m=2000, n=200, nnz=10, N=4, M=2, kappa=10, seed=3)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        with _solver(P, stream, max_iters=400, check_every=10) as eager, \
                _solver(P, stream, max_iters=400, check_every=10) as g:
            g.set_graph(10)
            ia, ib = eager.solve(), g.solve()
            assert ia.iters == ib.iters and ia.converged == ib.converged
            assert np.array_equal(eager.x(polished=True), g.x(polished=True))
            g.set_graph(0)             # back to eager launches on the same handle
            eager.step(7)
            g.step(7)
            assert np.array_equal(eager.state()["z"], g.state()["z"])


def test_graph_needs_a_stream_and_yields_to_profiling():
    import torch
    P = synth.small_problem(bc.LOSS_SQUARED, m=600, n=50, nnz=4, N=2, M=1, kappa=4, seed=5)
    with _solver(P, None) as s:
        with pytest.raises(bc.BicadmmError):
            s.set_graph(4)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        with _solver(P, stream) as eager, _solver(P, stream) as g:
            g.set_graph(4)
            bc.set_profiling(g.h, 2)   # profiling needs eager launches: replay is skipped
            eager.step(9)
            g.step(9)
            kt = bc.get_kernel_times(g.h)
            assert kt["pass"][1] == 9
            assert np.array_equal(eager.state()["x"], g.state()["x"])
