"""Helpers shared by the GPU tests: run the CUDA path and the oracle on the same input."""
import numpy as np

from oracle import bicadmm_ref as ref
from paper_2405_16267_b300 import bicadmm as bc


def run_gpu(P, iters, precision=bc.PREC_FP64, J=1, A=None, b=None, rho_c=None, **extra):
    """Run `iters` outer iterations through the C ABI; return the full state and info."""
    import torch
    A = P.A if A is None else A
    b = P.b if b is None else b
    if precision in (bc.PREC_FP32, bc.PREC_BF16) and not isinstance(A, torch.Tensor):
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
