"""The allocation-free consensus update against the handle-based solver.

bicadmm_consensus_step_noalloc is for callers that cannot allocate device memory when
they call in (graph capture, pool-owned memory, latency-bound loops); its scratch lives in
a file-scope device array of the library.  These tests drive the ordinary handle API
(bicadmm_step) for a few iterations, rebuild each iteration's consensus inputs from its
state, and check that two consecutive allocation-free calls reproduce the handle path's
z, s, t and v within the FP64 parity tolerance.  This file is collected last on purpose.
"""
import numpy as np
import pytest

from oracle import bicadmm_ref as ref
from paper_2405_16267_b300 import bicadmm as bc
from paper_2405_16267_b300 import synth

pytestmark = pytest.mark.gpu

TOL64 = 1e-9


def _rel(a, b):
    return float(np.max(np.abs(a - b))) / max(float(np.max(np.abs(b))), 1e-12)


def _handle_states(P, k):
    import torch
    with bc.Solver(P.A, P.b, loss=P.loss, N=P.N, M=P.M, kappa=P.kappa, gamma=P.gamma,
                   rho_c=P.rho, stream=torch.cuda.current_stream()) as s:
        s.step(k)
        states = [s.state()]
        for _ in range(2):
            s.step(1)
            states.append(s.state())
    return states


@pytest.mark.parametrize("workload", ["linear_2000x200", "logistic_ragged"])
def test_noalloc_consensus_matches_handle_path_two_calls(workload):
    import torch
    if workload == "linear_2000x200":
        P = synth.sparse_linear()
        k = 40
    else:
        P = synth.small_problem(ref.LOSS_LOGISTIC, m=3001, n=317, nnz=7, N=5, M=3, kappa=7, seed=9)
        k = 15
    st = _handle_states(P, k)
    dev = torch.device("cuda")
    stream = torch.cuda.current_stream()
    z = torch.tensor(st[0]["z"], device=dev)
    s = torch.tensor(st[0]["s"], device=dev)
    tvt = torch.tensor([0.0, st[0]["v"], 0.0, 0.0], device=dev)
    rho_b = 0.5 * P.rho
    for call in (1, 2):
        want = st[call]
        # w^{k+1} = mean_i(x_i^{k+1} + u_i^k) = mean_i(u_i^{k+1}) + z^{k+1}  (eq. u-update)
        w = torch.tensor(want["u"].mean(axis=0) + want["z"], device=dev)
        bc.consensus_step_noalloc(w, z, s, tvt, P.kappa, P.N, P.rho, rho_b, stream)
        torch.cuda.synchronize()
        zg, sg, tv = z.cpu().numpy(), s.cpu().numpy(), tvt.cpu().numpy()
        assert tv[3] == 0.0
        assert _rel(zg, want["z"]) <= TOL64, call
        assert _rel(sg, want["s"]) <= TOL64, call
        assert abs(tv[0] - want["t"]) <= TOL64 * max(abs(want["t"]), 1e-12), call
        assert abs(tv[1] - want["v"]) <= TOL64 * max(abs(want["v"]), abs(want["t"]), 1e-12), call
        assert list(ref.top_kappa(zg, P.kappa)) == list(ref.top_kappa(want["z"], P.kappa))
        assert np.array_equal(sg != 0, want["s"] != 0)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    n = 32769
    w = torch.zeros(n, dtype=torch.float64, device="cuda")
    z, s = torch.zeros_like(w), torch.zeros_like(w)
    tvt = torch.zeros(4, dtype=torch.float64, device="cuda")
    with pytest.raises(bc.BicadmmError) as e:
        bc.consensus_step_noalloc(w, z, s, tvt, 5, 2, 1.0, 0.5)
    assert e.value.code == -1
