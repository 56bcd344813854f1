"""Planted mistakes in the FP64 oracle, used to show that its pins catch them.

Each mutant replaces one snippet of one oracle function's source with a wrong variant
(a dropped term, a flipped sign, a wrong index rule, a wrong denominator) and re-defines
that function in the oracle module (or class).  `apply(name)` is called only inside a child
pytest process (tests/conftest.py reads BICADMM_ORACLE_MUTANT); the oracle on disk and in
every other process is untouched.  Every snippet must occur exactly once in its function,
so a mutant that no longer matches the oracle fails loudly instead of silently planting
nothing.
"""
import inspect
import textwrap

# name -> (function or "Class.method", original snippet, mutated snippet, what it breaks)
MUTANTS = {
    "zt_drop_v": ("zt_step", "h0 = v + c.sum()", "h0 = c.sum()",
                  "eq. (global-z-t-updae): the scaled dual v left out of h(0)"),
    "zt_beta_without_N": ("zt_step", "beta = N * rho_c / rho_b", "beta = rho_c / rho_b",
                          "eq. (global-z-t-updae): the z-penalty weight N rho_c"),
    "zt_shift_sign": ("zt_step", "y = w + tau * s", "y = w - tau * s",
                      "eq. (global-z-t-updae): sign of the s-shift in z(tau)"),
    "topk_ties_highest": ("top_kappa", "np.lexsort((np.arange(z.size), -np.abs(z)))",
                          "np.lexsort((-np.arange(z.size), -np.abs(z)))",
                          "tie rule of the s step (lowest index)"),
    "s_no_clamp": ("s_step", "return min(1.0, max(-1.0, theta / T)) * s_top", "return s_top",
                   "eq. (s-update-final): the minimiser when theta < T"),
    "s_theta_sign": ("s_step", "theta = t - v", "theta = t + v",
                     "eq. (s-update-final): the target t - v"),
    "prox_squared_no_M": ("omega_prox",
                          "# d/dw: 2M(Mw - b) + M rho_l (w - a) = 0\n"
                          "        return (2.0 * b + rho_l * a) / (2.0 * M + rho_l)",
                          "# d/dw: 2M(Mw - b) + M rho_l (w - a) = 0\n"
                          "        return (2.0 * b + rho_l * a) / (2.0 + rho_l)",
                          "eq. (p:GPU;omega): the factor M of the squared loss"),
    "prox_logistic_sign": ("omega_prox", "return -b * M * expit(-b * M * w) + M * rho_l * (w - a)",
                           "return b * M * expit(-b * M * w) + M * rho_l * (w - a)",
                           "eq. (p:GPU;omega): sign of the logistic gradient"),
    "prox_softmax_grad_no_M": ("softmax_prox",
                               "return M * (softmax_rows(M * w) - onehot) + M * rho_l * (w - a)",
                               "return (softmax_rows(M * w) - onehot) + M * rho_l * (w - a)",
                               "eq. (p:GPU;omega), softmax: the chain-rule factor M"),
    "x_rhs_u_sign": ("BiCADMM.x_step_shard", "self.rho_c * (Z[c0_:c1_] - U[c0_:c1_])",
                     "self.rho_c * (Z[c0_:c1_] + U[c0_:c1_])",
                     "eq. (p:GPU;x): the prox centre z - u"),
    "x_c0_without_N": ("BiCADMM.__init__", "self.c0 = 1.0 / (N_all * self.gamma) + self.rho_c",
                       "self.c0 = 1.0 / self.gamma + self.rho_c",
                       "eq. (p:bi-convex): the per-shard ridge 1/(N gamma)"),
    "nu_sign": ("BiCADMM.x_step_shard", "nu_v[r0:r1] = nu + Axbar_new - omega_new",
                "nu_v[r0:r1] = nu - Axbar_new + omega_new", "eq. (p:GPU;nu)"),
    "u_sign": ("BiCADMM.iterate", "self.u = self.u + self.x - self.z[None, :]",
               "self.u = self.u - self.x + self.z[None, :]", "eq. (u-update)"),
    "v_sign": ("BiCADMM.iterate", "self.v = self.v + g", "self.v = self.v - g", "eq. (v-update)"),
    "res_d_without_sqrtN": ("BiCADMM.residuals", "d_r = math.sqrt(N) * self.rho_c * dz",
                            "d_r = self.rho_c * dz", "Termination: d_r = sqrt(N) rho_c ||dz||"),
    "res_p_rel_without_N": ("BiCADMM.residuals", "p_rel=p_r / max(nx, N * nz, 1e-30)",
                            "p_rel=p_r / max(nx, nz, 1e-30)", "relative primal residual"),
    "res_i_den_omega_only": ("BiCADMM.residuals",
                             "i_den = max(float(np.linalg.norm(self.omega)), float(np.linalg.norm(self.Axbar)), 1e-30)",
                             "i_den = max(float(np.linalg.norm(self.omega)), 1e-30)",
                             "relative inner residual"),
    "res_b_signed": ("BiCADMM.residuals", "b_r = abs(g)", "b_r = g",
                     "Termination: b_r = |z's - t|"),
    "polish_no_ridge": ("polish", "H = 2.0 * AS.T @ AS + np.eye(k) / gamma", "H = 2.0 * AS.T @ AS",
                        "restricted problem: the ridge term"),
    "polish_softmax_no_ridge_grad": ("_polish_softmax", "grad = G[cols, cls] + w / gamma",
                                     "grad = G[cols, cls]", "restricted softmax problem: ridge gradient"),
}


def _target(ref, where):
    if "." in where:
        cls_name, meth = where.split(".")
        return getattr(getattr(ref, cls_name), meth), getattr(ref, cls_name), meth
    return getattr(ref, where), ref, where


def mutated_source(ref, name):
    where, old, new, _ = MUTANTS[name]
    fn, _, _ = _target(ref, where)
    src = textwrap.dedent(inspect.getsource(fn))
    count = src.count(old)
    if count != 1:
        raise RuntimeError("mutant %s: snippet found %d times in %s" % (name, count, where))
    return src.replace(old, new)


def apply(ref, name):
    """Re-define the mutated function in the oracle module (module functions are looked up
    through the module's globals, so the solver's own calls see the mutant too)."""
    where = MUTANTS[name][0]
    src = mutated_source(ref, name)
    _, owner, attr = _target(ref, where)
    scope = {}
    exec(compile(src, "<mutant %s>" % name, "exec"), ref.__dict__, scope)
    setattr(owner, attr, scope[attr])
