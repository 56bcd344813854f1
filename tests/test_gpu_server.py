"""Serving loop: requests of mixed loss and size arriving over time are admitted while
others are on the GPU, batched together, and each result equals solving it alone."""
import numpy as np
import pytest

from oracle import bicadmm_ref as ref
from paper_2405_16267_b300 import bicadmm as bc
from paper_2405_16267_b300 import synth

from gpu_util import rel_err

pytestmark = pytest.mark.gpu


def _requests(seed=0):
    specs = [(ref.LOSS_SQUARED, 1500, 90, 3, 2, 6, 30), (ref.LOSS_LOGISTIC, 2300, 150, 4, 3, 7, 45),
             (ref.LOSS_SQHINGE, 900, 61, 2, 2, 4, 20), (ref.LOSS_SQUARED, 4100, 333, 5, 4, 12, 60),
             (ref.LOSS_LOGISTIC, 700, 40, 1, 1, 3, 35), (ref.LOSS_SQHINGE, 3000, 210, 6, 3, 9, 50),
             (ref.LOSS_SQUARED, 2000, 200, 4, 2, 10, 40)]
    out = []
    for k, (loss, m, n, N, M, kappa, iters) in enumerate(specs):
        P = synth.small_problem(loss, m=m, n=n, nnz=kappa, N=N, M=M, kappa=kappa, seed=300 + k + seed)
        out.append((P, iters))
    return out


def _alone(P, iters, precision):
    import torch
    A = P.A if precision == bc.PREC_FP64 else P.A.astype(np.float32)
    with bc.Solver(A, P.b, loss=P.loss, N=P.N, M=P.M, kappa=P.kappa, gamma=P.gamma, rho_c=P.rho,
                   precision=precision, stream=torch.cuda.current_stream()) as s:
        s.step(iters)
        return bc.get_x(s.h, P.n, polished=True, with_support=True, kappa=P.kappa)


@pytest.mark.parametrize("precision,tol", [(bc.PREC_FP64, 1e-9), (bc.PREC_FP32, 1e-4), (bc.PREC_BF16, 1e-4)])
def test_results_same_alone_and_in_the_mix(precision, tol):
    reqs = _requests()
    with bc.Server(hbm_budget_bytes=8 << 30, max_active=16, iters_per_round=7,
                   precision=precision, use_graph=True) as srv:
        t0 = srv.clock()
        ids = []
        for k, (P, iters) in enumerate(reqs):
            A = P.A if precision == bc.PREC_FP64 else P.A.astype(np.float32)
            ids.append(srv.submit(A, P.b, arrival=t0 + 0.004 * k, loss=P.loss, precision=precision,
                                  N_shards=P.N, M_blocks=P.M, kappa=P.kappa, gamma=P.gamma,
                                  rho_c=P.rho, max_iters=iters, tol_rel=0.0))
        srv.run()
        res = [srv.result(i) for i in ids]
        st = srv.stats()
    assert st["finished"] == len(reqs) and st["rounds"] >= 2
    # continuous batching: some request was admitted while another was still running
    overlap = any(r2["admitted"] > r1["admitted"] and r2["admitted"] < r1["done"]
                  for r1 in res for r2 in res)
    assert overlap
    for (P, iters), r in zip(reqs, res):
        assert r["status"] == 0 and r["info"].iters == iters
        x_alone, supp_alone = _alone(P, iters, precision)
        assert list(r["support"]) == list(supp_alone)
        assert rel_err(r["x"], x_alone) <= tol


def test_budget_serialises_and_rejects_oversized():
    # four requests of one shape: the budget holds exactly one of them
    reqs = [(synth.small_problem(ref.LOSS_LOGISTIC, m=2500, n=120, nnz=5, N=3, M=2, kappa=5,
                                 seed=400 + k), 15 + 5 * k) for k in range(4)]
    need = [bc.estimate_bytes(bc.default_params(m=P.m, n=P.n, N_shards=P.N, M_blocks=P.M,
                                                kappa=P.kappa, loss=P.loss, precision=bc.PREC_FP64))
            for P, _ in reqs]
    budget = max(a + b for a, b in need) + 1024  # one request at a time
    with bc.Server(hbm_budget_bytes=budget, max_active=8, iters_per_round=5,
                   precision=bc.PREC_FP64, use_graph=False) as srv:
        ids = [srv.submit(P.A, P.b, arrival=0.0, loss=P.loss, precision=bc.PREC_FP64,
                          N_shards=P.N, M_blocks=P.M, kappa=P.kappa, gamma=P.gamma, rho_c=P.rho,
                          max_iters=iters, tol_rel=0.0) for P, iters in reqs]
        big = synth.small_problem(ref.LOSS_SQUARED, m=20000, n=400, nnz=5, N=4, M=2, kappa=5, seed=9)
        bid = srv.submit(big.A, big.b, arrival=0.0, loss=0, precision=bc.PREC_FP64, N_shards=4,
                         M_blocks=2, kappa=5, max_iters=10, tol_rel=0.0)
        srv.run()
        res = [srv.result(i) for i in ids]
        rb = srv.result(bid)
        st = srv.stats()
    assert rb["status"] == -2  # BICADMM_ERR_OOM: can never fit the budget
    assert all(r["status"] == 0 for r in res)
    spans = sorted((r["admitted"], r["done"]) for r in res)
    for (a0, d0), (a1, d1) in zip(spans, spans[1:]):
        assert a1 >= d0 - 1e-9  # never two at once under this budget
    assert st["peak_bytes"] <= budget


def test_tolerance_stop_in_server():
    P = synth.table1_sls(m=20000, n=400, N=4, M=2)
    with bc.Server(hbm_budget_bytes=4 << 30, iters_per_round=5, precision=bc.PREC_FP64) as srv:
        rid = srv.submit(P.A, P.b, arrival=0.0, loss=0, precision=bc.PREC_FP64, N_shards=4,
                         M_blocks=2, kappa=P.kappa, gamma=P.gamma, rho_c=P.rho, max_iters=2000,
                         tol_rel=1e-6)
        srv.run()
        r = srv.result(rid)
    assert r["status"] == 0 and r["info"].converged == 1 and r["info"].iters < 2000
    assert set(r["support"].tolist()) == set(np.flatnonzero(P.x_star).tolist())


def test_submissions_from_another_thread_while_running():
    """Requests submitted by another host thread while run() loops are admitted into the
    running batch; each result equals the same request solved alone; the per-request time
    breakdown is ordered and the server reports its rebuilds and rounds."""
    import threading
    import time
    reqs = _requests(seed=7)[:5]
    reqs[0] = (reqs[0][0], 1000)  # long enough to still be running when the others arrive
    kw = lambda P, iters: dict(loss=P.loss, precision=bc.PREC_FP64, N_shards=P.N, M_blocks=P.M,
                               kappa=P.kappa, gamma=P.gamma, rho_c=P.rho, max_iters=iters,
                               tol_rel=0.0)
    with bc.Server(hbm_budget_bytes=8 << 30, max_active=16, iters_per_round=5,
                   precision=bc.PREC_FP64, use_graph=True) as srv:
        srv.set_open(True)
        P0, it0 = reqs[0]
        ids = [srv.submit(P0.A, P0.b, arrival=srv.clock(), **kw(P0, it0))]
        done = []
        runner = threading.Thread(target=lambda: done.append(srv.run(until=srv.clock() + 120)))
        runner.start()
        for P, iters in reqs[1:]:
            time.sleep(0.002)
            ids.append(srv.submit(P.A, P.b, arrival=srv.clock(), **kw(P, iters)))
        deadline = time.time() + 120
        while time.time() < deadline and any(srv.result(i)["status"] == -4 for i in ids):
            time.sleep(0.005)
        srv.set_open(False)
        runner.join(timeout=120)
        assert not runner.is_alive() and done == [len(ids)]
        res = [srv.result(i) for i in ids]
        times = [srv.timing(i) for i in ids]
        prof = srv.timing(-1)
    for (P, iters), r, t in zip(reqs, res, times):
        assert r["status"] == 0 and r["info"].iters == iters
        x_alone, supp_alone = _alone(P, iters, bc.PREC_FP64)
        assert list(r["support"]) == list(supp_alone)
        assert rel_err(r["x"], x_alone) <= 1e-9
        assert t["arrival"] <= t["admitted"] <= t["setup_done"] <= t["retiring"] <= t["done"]
        assert t["iters"] == iters and t["rounds"] >= 1
    # a request submitted while the loop ran shared it with an earlier one
    assert any(b["admitted"] > a["admitted"] and b["admitted"] < a["done"] for a in times for b in times)
    assert prof["rebuilds"] >= 1 and prof["rounds"] >= 2 and prof["admit_s"] > 0
