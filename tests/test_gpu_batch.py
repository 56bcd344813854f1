"""Batched execution: uneven instances advanced together by one launch per kernel kind per
iteration must give each instance the iterates it gets alone (same handle API), up to the
rounding of the regrouped A'd partial sums, and the oracle's iterates."""
import numpy as np
import pytest

from oracle import bicadmm_ref as ref
from paper_2405_16267_b300 import bicadmm as bc
from paper_2405_16267_b300 import synth

from gpu_util import compare_state, rel_err, run_oracle

pytestmark = pytest.mark.gpu

TOL64 = 1e-9


def _instances(seed=0):
    rng = np.random.default_rng(seed)
    probs = []
    specs = [(bc.LOSS_SQUARED, 1500, 90, 3, 2, 6), (bc.LOSS_SQHINGE, 2300, 150, 4, 3, 7),
             (bc.LOSS_LOGISTIC, 900, 61, 2, 2, 4), (bc.LOSS_SQUARED, 4100, 333, 5, 4, 12),
             (bc.LOSS_SQHINGE, 700, 40, 1, 1, 3), (bc.LOSS_LOGISTIC, 3000, 210, 6, 3, 9)]
    for k, (loss, m, n, N, M, kappa) in enumerate(specs):
        probs.append(synth.small_problem(loss, m=m, n=n, nnz=kappa, N=N, M=M, kappa=kappa,
                                         seed=100 + k + seed))
    return probs


def _solvers(probs, precision=bc.PREC_FP64):
    import torch
    out = []
    for P in probs:
        A = P.A if precision == bc.PREC_FP64 else P.A.astype(np.float32)  # BF16: rounded at setup
        out.append(bc.Solver(A, P.b, loss=P.loss, N=P.N, M=P.M, kappa=P.kappa, gamma=P.gamma,
                             rho_c=P.rho, precision=precision, stream=torch.cuda.current_stream()))
    return out


@pytest.mark.parametrize("flags", [0, 1, 2, 3])
def test_batch_equals_alone(flags):
    import torch
    probs = _instances()
    iters = 25
    alone = []
    for s in _solvers(probs):
        s.step(iters)
        alone.append(s.state())
        s.close()
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        sol = _solvers(probs)
        b = bc.batch_create(sol, stream=stream, flags=flags)
        try:
            launches = bc.batch_step(b, 10)
            launches = bc.batch_step(b, iters - 10)
            rows, stages = bc.batch_tiling(b)
        finally:
            stream.synchronize()
            bc.batch_destroy(b)
        states = [s.state() for s in sol]
        for s in sol:
            s.close()
    assert 16 <= rows <= 96 and 1 <= stages <= 4  # stage KB, stage count
    # graph replays count one iteration's launches; eager: 4 or 5 per iteration (one pass
    # launch for the wide and one for the narrow instances)
    assert launches in (4 * iters, 5 * iters) or (flags & 1)
    for st, want, P in zip(states, alone, probs):
        for k in ("z", "x", "u", "s", "omega", "nu"):
            assert rel_err(st[k], want[k]) <= TOL64, (P.name, k)
        assert abs(st["t"] - want["t"]) <= TOL64 * max(1.0, abs(want["t"]))
        assert list(ref.top_kappa(st["z"], P.kappa)) == list(ref.top_kappa(want["z"], P.kappa))


def test_batch_matches_oracle():
    import torch
    probs = _instances(seed=7)[:3]
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        sol = _solvers(probs)
        b = bc.batch_create(sol, stream=stream, flags=bc.BATCH_GRAPH)
        bc.batch_step(b, 20)
        stream.synchronize()
        bc.batch_destroy(b)
        states = [s.state() for s in sol]
        for s in sol:
            s.close()
    for st, P in zip(states, probs):
        o = run_oracle(P, 20)
        compare_state(st, o, TOL64)


def test_batch_fp32_close_to_alone():
    import torch
    probs = _instances(seed=3)
    alone = []
    for s in _solvers(probs, bc.PREC_FP32):
        s.step(15)
        alone.append(s.state())
        s.close()
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        sol = _solvers(probs, bc.PREC_FP32)
        b = bc.batch_create(sol, stream=stream, flags=0)
        bc.batch_step(b, 15)
        stream.synchronize()
        bc.batch_destroy(b)
        states = [s.state() for s in sol]
        for s in sol:
            s.close()
    for st, want in zip(states, alone):
        for k in ("z", "x", "omega", "nu"):
            assert rel_err(st[k], want[k]) <= 1e-4, k


@pytest.mark.parametrize("flags", [0, 1])
def test_batch_bf16_close_to_alone_and_oracle(flags):
    """BF16 storage in a batch: each instance within 1e-4 of itself stepped alone and of the
    oracle run on its BF16-rounded A."""
    import torch
    probs = _instances(seed=5)
    iters = 15
    alone = []
    for s in _solvers(probs, bc.PREC_BF16):
        s.step(iters)
        alone.append(s.state())
        s.close()
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        sol = _solvers(probs, bc.PREC_BF16)
        b = bc.batch_create(sol, stream=stream, flags=flags)
        bc.batch_step(b, iters)
        stream.synchronize()
        bc.batch_destroy(b)
        states = [s.state() for s in sol]
        for s in sol:
            s.close()
    for st, want, P in zip(states, alone, probs):
        for k in ("z", "x", "omega", "nu"):
            assert rel_err(st[k], want[k]) <= 1e-4, k
        b32 = P.b.astype(np.float32).astype(np.float64)
        compare_state(st, run_oracle(P, iters, A=synth.round_to_bf16(P.A), b=b32), 1e-4)


def _mixed_instances(seed=0):
    """Row widths across both batched pass kernels: row groups of 8, 16, 32 and 128 threads
    (narrow pass) and one or more vectors per thread (wide pass); shards shorter than a
    panel."""
    specs = [(bc.LOSS_SQUARED, 900, 20, 3, 1, 3), (bc.LOSS_LOGISTIC, 70, 30, 3, 1, 2),
             (bc.LOSS_SQHINGE, 1200, 100, 2, 1, 5), (bc.LOSS_SQUARED, 1500, 240, 4, 2, 8),
             (bc.LOSS_LOGISTIC, 1100, 300, 3, 2, 6), (bc.LOSS_SQUARED, 1300, 520, 2, 2, 9),
             (bc.LOSS_SQHINGE, 2000, 1100, 4, 3, 11)]
    return [synth.small_problem(loss, m=m, n=n, nnz=kappa, N=N, M=M, kappa=kappa,
                                seed=300 + k + seed)
            for k, (loss, m, n, N, M, kappa) in enumerate(specs)]


@pytest.mark.parametrize("precision", [bc.PREC_FP64, bc.PREC_FP32, bc.PREC_BF16])
def test_batch_mixed_widths(precision):
    """Instances of every row-group size and of the wide pass in one batch: each within the
    precision's tolerance of itself stepped alone and of the oracle (on the rounded A)."""
    import torch
    probs = _mixed_instances()
    iters = 12
    tol = TOL64 if precision == bc.PREC_FP64 else 1e-4
    alone = []
    for s in _solvers(probs, precision):
        s.step(iters)
        alone.append(s.state())
        s.close()
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        sol = _solvers(probs, precision)
        b = bc.batch_create(sol, stream=stream, flags=bc.BATCH_AUTOTUNE)
        launches = bc.batch_step(b, iters)
        stream.synchronize()
        bc.batch_destroy(b)
        states = [s.state() for s in sol]
        for s in sol:
            s.close()
    assert launches == 5 * iters
    for st, want, P in zip(states, alone, probs):
        for k in ("z", "x", "omega", "nu"):
            assert rel_err(st[k], want[k]) <= tol, (P.name, k)
        if precision == bc.PREC_FP64:
            o = run_oracle(P, iters)
        else:
            A = P.A.astype(np.float32).astype(np.float64)
            if precision == bc.PREC_BF16:
                A = synth.round_to_bf16(P.A)
            o = run_oracle(P, iters, A=A, b=P.b.astype(np.float32).astype(np.float64))
        compare_state(st, o, tol, support_exact=precision == bc.PREC_FP64)


def test_batch_rejects_bad_requests():
    import torch
    probs = _instances()[:2]
    sol = _solvers(probs)
    try:
        with pytest.raises(bc.BicadmmError):
            bc.batch_create([sol[0], sol[0]])
        with pytest.raises(bc.BicadmmError):
            bc.batch_create(sol, stream=None, flags=bc.BATCH_GRAPH)
    finally:
        for s in sol:
            s.close()


def test_batch_ring_mixed_panel_sizes():
    """Wide-row instances whose panels span 19 to 96 KB in the default one-ring tiling (96 KB
    in FP32), tall enough that each CTA of the pass streams a few dozen panels of several
    instances through its ring (placement next to the newest panel, wrapping to the start):
    each instance within 1e-4 of itself stepped alone."""
    import torch
    specs = [(bc.LOSS_SQUARED, 12000, 600, 3, 2, 8), (bc.LOSS_SQHINGE, 12000, 1500, 4, 3, 20),
             (bc.LOSS_LOGISTIC, 12000, 2500, 3, 5, 30), (bc.LOSS_SQUARED, 12000, 4000, 4, 8, 40)]
    probs = [synth.small_problem(loss, m=m, n=n, nnz=kappa, N=N, M=M, kappa=kappa, seed=500 + k)
             for k, (loss, m, n, N, M, kappa) in enumerate(specs)]
    iters = 8
    alone = []
    for s in _solvers(probs, bc.PREC_FP32):
        s.step(iters)
        alone.append(s.state())
        s.close()
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        sol = _solvers(probs, bc.PREC_FP32)
        b = bc.batch_create(sol, stream=stream, flags=0)
        assert bc.batch_tiling(b) == (96, 1)
        launches = bc.batch_step(b, iters)
        stream.synchronize()
        bc.batch_destroy(b)
        states = [s.state() for s in sol]
        for s in sol:
            s.close()
    assert launches == 4 * iters  # no narrow instance: x-update, pass, consensus, dual
    for st, want, P in zip(states, alone, probs):
        for k in ("z", "x", "omega", "nu"):
            assert rel_err(st[k], want[k]) <= 1e-4, (P.name, k)
