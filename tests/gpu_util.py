"""Helpers shared by the GPU tests: run the CUDA path and the oracle on the same input."""
import numpy as np

from oracle import bicadmm_ref as ref
from paper_2405_16267_b300 import bicadmm as bc


def run_gpu(P, iters, precision=bc.PREC_FP64, J=1, A=None, b=None, rho_c=None, **extra):
    """Run `iters` outer iterations through the C ABI; return the full state and info."""
    import torch
    A = P.A if A is None else A
    b = P.b if b is None else b
    if precision in (bc.PREC_FP32, bc.PREC_BF16, bc.PREC_TF32) and not isinstance(A, torch.Tensor):
        A = np.asarray(A, dtype=np.float32)
    stream = torch.cuda.current_stream()
    with bc.Solver(A, b, loss=P.loss, N=P.N, M=P.M, kappa=P.kappa, gamma=P.gamma,
                   rho_c=P.rho if rho_c is None else rho_c, inner_iters=J, precision=precision,
                   stream=stream, K=P.K, **extra) as s:
        info = s.step(iters)
        st = s.state()
    return st, info


def run_oracle(P, iters, J=1, A=None, b=None, rho_c=None):
    A = P.A if A is None else A
    b = P.b if b is None else b
    o = ref.BiCADMM(A, b, P.loss, P.N, P.M, P.kappa, gamma=P.gamma,
                    rho_c=P.rho if rho_c is None else rho_c, inner_iters=J, K=P.K)
    o.iterate(iters)
    return o


def rel_err(got, want, floor=1e-12):
    got = np.asarray(got, dtype=np.float64)
    want = np.asarray(want, dtype=np.float64)
    scale = max(float(np.max(np.abs(want))) if want.size else 0.0, floor)
    return float(np.max(np.abs(got - want))) / scale if want.size else 0.0


def compare_state(st, o, tol, support_exact=True):
    """Element-wise comparison of the GPU state with the oracle's; returns a dict of errors."""
    errs = {
        "z": rel_err(st["z"], o.z),
        "x": rel_err(st["x"], o.x),
        "u": rel_err(st["u"], o.u),
        "s": rel_err(st["s"], o.s),
        "omega": rel_err(st["omega"], o.omega),
        "nu": rel_err(st["nu"], o.nu),
        "t": abs(st["t"] - o.t) / max(abs(o.t), 1e-12),
        "v": abs(st["v"] - o.v) / max(abs(o.v), abs(o.t), 1e-12),
    }
    bad = {k: e for k, e in errs.items() if not (e <= tol)}
    assert not bad, "parity failed (tol %g): %s" % (tol, bad)
    if support_exact:
        assert list(ref.top_kappa(st["z"], o.kappa)) == list(o.support())
        # the nonzero pattern of s (the selected top-kappa set) matches exactly
        assert np.array_equal(st["s"] != 0, o.s != 0)
    return errs


def consensus_state(solver):
    """The n-space part of a Solver's state (x, u, z, s and the scalars t, v, tau); leaves
    out the m-space omega/nu, which are large at full size."""
    N, n = solver.N, solver.n * solver.K
    sc = bc.get_state(solver.h, bc.FIELD_SCALARS, 3)
    return dict(x=bc.get_state(solver.h, bc.FIELD_X, N * n).reshape(N, n),
                u=bc.get_state(solver.h, bc.FIELD_U, N * n).reshape(N, n),
                z=bc.get_state(solver.h, bc.FIELD_Z, n), s=bc.get_state(solver.h, bc.FIELD_S, n),
                t=sc[0], v=sc[1], tau=sc[2])


def check_consensus_step(prev, cur, N, rho_c, rho_b, kappa, tol=1e-9):
    """One outer iteration's global step against the oracle, element by element: the GPU's
    own w = mean_i(x_i^{k+1} + u_i^k), s^k and v^k go through ref.zt_step (eq.
    global-z-t-updae) and its z^{k+1}, t^{k+1} through ref.s_step (eq. s-update-final); z, t,
    tau, s and v (eq. v-update) must agree, and s must select the same entries.  Returns tau."""
    w = (cur["x"] + prev["u"]).mean(axis=0)
    z, t, tau = ref.zt_step(w, prev["s"], prev["v"], N, rho_c, rho_b)
    zs = max(float(np.max(np.abs(z))), 1e-300)
    assert float(np.max(np.abs(cur["z"] - z))) <= tol * zs, "z"
    assert abs(cur["t"] - t) <= tol * max(abs(t), zs), ("t", cur["t"], t)
    assert abs(cur["tau"] - tau) <= tol * max(abs(tau), 1e-12), ("tau", cur["tau"], tau)
    s = ref.s_step(cur["z"], cur["t"], prev["v"], kappa)
    assert np.array_equal(s != 0, cur["s"] != 0), "selected entries of s"
    assert float(np.max(np.abs(cur["s"] - s))) <= 1e-12, "s"
    v = prev["v"] + float(cur["z"] @ cur["s"]) - cur["t"]
    assert abs(cur["v"] - v) <= tol * max(abs(v), abs(cur["t"]), 1e-12), ("v", cur["v"], v)
    np.testing.assert_allclose(cur["u"], prev["u"] + cur["x"] - cur["z"][None, :], rtol=0,
                               atol=1e-12 * max(1.0, float(np.max(np.abs(cur["x"])))))
    return tau
