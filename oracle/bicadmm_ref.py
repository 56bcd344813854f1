"""Bi-cADMM oracle: a plain, slow, FP64 CPU restatement of the method.

TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the CPU-baseline leg
of the benchmark may import this module.  The CUDA product path never imports, links or
calls it, and this module imports nothing from the product package.

Paper: "A GPU-Accelerated Bi-linear ADMM Algorithm for Distributed Sparse Machine
Learning" (Olama et al., arXiv 2405.16267).  Equation names below are the paper's LaTeX
labels.  The oracle follows the paper's own decomposition step by step, with no blocking,
fusion or reordering:

  outer iteration (iterations block, Sec. 3, eqs. x-min-step .. global-lambda-updae,
  in the scaled form of eqs. u-update and v-update):
    1. x_i = prox of f_i at z - u_i (eq. p:x-subp), evaluated by Algorithm 2: J sweeps of
       the feature-split sharing ADMM of Sec. 3.1 (eqs. p:GPU;x, p:GPU;omega, p:GPU;nu),
       warm-started across outer iterations;
    2. (z, t) = argmin over ||z||_1 <= t (eq. global-z-t-updae);
    3. s = argmin over S^kappa (eq. s-update-final);
    4. u_i += x_i - z (eq. u-update);  v += z's - t (eq. v-update);
    5. residuals p_r, d_r, b_r (Termination paragraph).

Readings where the paper is silent or inconsistent (each also pinned by a test):
  * Scaled duals follow the standard form: the prox is taken at z - u_i and u_i += x_i - z
    (eqs. x-min-step rewritten, p:x-subp, u-update); the sign of y_i in eq. eq:al is read
    the same way.
  * Losses take the label as a second argument: squared (q-b)^2 (no 1/2, as eq. p:sls),
    logistic log(1+exp(-b q)), squared hinge max(0, 1-b q)^2, with b in {-1,+1}; softmax
    (Sec. 2's sparse softmax regression) is the cross-entropy logsumexp(q) - q_y of the
    K-vector q = a_r W, label y in {0..K-1}.
  * Softmax: the decision variable is the n x K matrix W; every n-space vector (x_i, u_i,
    z, s) holds it flattened feature-major (entry (c, k) at c*K + k), so the sparsity
    budget kappa, the (z,t) step, the s step and the lowest-index tie rule apply entrywise
    to that vector.  The block solve of eq. (p:GPU;x) takes the K columns of W_ij at once
    (the same block matrix for every class); omega, nu and the block products are m x K.
  * All state starts at zero; the inner count J is a parameter.
  * Uneven shards/blocks: contiguous ranges, the first (total mod parts) one longer.
  * The (z,t) problem is solved exactly: z = soft-threshold(w + tau s, tau) with tau the
    root of a strictly increasing piecewise-linear function (derived from the KKT system;
    the paper only says it is a convex QP).
  * The s problem picks sign(z) on the kappa largest |z_r| (ties: lowest index) scaled by
    clamp((t - v)/T, -1, 1), T = sum of those |z_r|; s = 0 when T = 0.
  * Relative residuals: p_r / max(sum_i ||x_i||, N ||z||), ||z - z_prev|| / ||z||,
    b_r / t (denominators floored at 1e-30).  Because the local prox is solved inexactly
    (J sweeps), the stop rule also requires the inner sharing residual
    i_rel = ||Axbar - omega|| / max(||omega||, ||Axbar||) to be small; without it the
    all-zero state after the first iteration would read as converged.
  * After the loop, a restricted problem on the top-kappa support of z is solved in FP64
    ("polish"; not part of the paper's algorithm).
"""
from __future__ import annotations

import math

import numpy as np
import scipy.linalg
from scipy.special import expit

LOSS_SQUARED, LOSS_LOGISTIC, LOSS_SOFTMAX, LOSS_SQHINGE = 0, 1, 2, 3


def split_ranges(total, parts):
    """Contiguous index ranges, the first (total mod parts) ranges one element longer."""
    base, rem = divmod(int(total), int(parts))
    out, start = [], 0
    for k in range(parts):
        size = base + (1 if k < rem else 0)
        out.append((start, start + size))
        start += size
    return out


# --------------------------------------------------------------------------- losses

def logsumexp_rows(q):
    """log sum_k exp(q_rk) per row, shifted by the row maximum."""
    qm = q.max(axis=1)
    return qm + np.log(np.exp(q - qm[:, None]).sum(axis=1))


def softmax_rows(q):
    e = np.exp(q - q.max(axis=1)[:, None])
    return e / e.sum(axis=1)[:, None]


def loss_rows(loss, q, b):
    """Per-row loss l(q; b) of problem (p:SML) for each supported model (Sec. 2).
    Softmax: q is m x K and b holds the class index of each row."""
    if loss == LOSS_SOFTMAX:
        y = np.asarray(b).astype(np.int64)
        return logsumexp_rows(q) - q[np.arange(q.shape[0]), y]
    if loss == LOSS_SQUARED:
        return (q - b) ** 2
    if loss == LOSS_LOGISTIC:
        return np.logaddexp(0.0, -b * q)
    if loss == LOSS_SQHINGE:
        return np.maximum(0.0, 1.0 - b * q) ** 2
    raise ValueError("loss %r" % loss)


def objective(loss, A, b, x, gamma, K=1):
    """F(x) = sum_r l(a_r x; b_r) + ||x||^2 / (2 gamma)   (problem p:SML); for softmax x is
    the flattened n x K matrix."""
    X = np.asarray(x, dtype=np.float64).reshape(A.shape[1], K) if K > 1 else x
    return float(np.sum(loss_rows(loss, A @ X, b)) + np.sum(X * X) / (2.0 * gamma))


def omega_prox(loss, a, b, M, rho_l):
    """omega-bar step of eq. (p:GPU;omega), one scalar problem per row (the loss is separable):

        omega_r = argmin_w  l(M w; b_r) + (M rho_l / 2) (w - a_r)^2,

    with a = (mean of the block products) + nu.
    """
    a = np.asarray(a, dtype=np.float64)
    if loss == LOSS_SOFTMAX:
        return softmax_prox(a, b, M, rho_l)
    if loss == LOSS_SQUARED:
        # d/dw: 2M(Mw - b) + M rho_l (w - a) = 0
        return (2.0 * b + rho_l * a) / (2.0 * M + rho_l)
    if loss == LOSS_SQHINGE:
        # Loss inactive at a (1 - b M a <= 0): the quadratic's minimiser a is optimal.
        # Otherwise the active branch has the squared-loss form with target b (b^2 = 1).
        active = (1.0 - b * M * a) > 0.0
        return np.where(active, (2.0 * b + rho_l * a) / (2.0 * M + rho_l), a)
    if loss == LOSS_LOGISTIC:
        # phi'(w) = -b M sigma(-b M w) + M rho_l (w - a) is increasing; its root lies between
        # a and a + b / rho_l.  Plain bisection to the last bit.
        lo = np.minimum(a, a + b / rho_l)
        hi = np.maximum(a, a + b / rho_l)

        def dphi(w):
            return -b * M * expit(-b * M * w) + M * rho_l * (w - a)

        for _ in range(200):
            mid = 0.5 * (lo + hi)
            pos = dphi(mid) > 0.0
            hi = np.where(pos, mid, hi)
            lo = np.where(pos, lo, mid)
        return 0.5 * (lo + hi)
    raise ValueError("loss %r" % loss)


def softmax_prox(a, y, M, rho_l, max_iters=200):
    """Softmax omega-bar step of eq. (p:GPU;omega), one K-vector problem per row:

        omega_r = argmin_w  CE(M w; y_r) + (M rho_l / 2) ||w - a_r||^2,
        CE(q; y) = logsumexp(q) - q_y.

    phi is strongly convex; gradient g = M (softmax(M w) - e_y) + M rho_l (w - a), Hessian
    H = M^2 (diag p - p p') + M rho_l I.  Newton from w = a, all rows at once, damped by
    backtracking on ||g|| (the Newton direction decreases ||g||^2 at rate 2||g||^2; unlike
    phi itself, ||g|| has no cancellation near the minimum), until every row's step is
    within a few ulps of w.
    """
    a = np.asarray(a, dtype=np.float64)
    y = np.asarray(y).astype(np.int64)
    m, K = a.shape
    onehot = np.zeros((m, K))
    onehot[np.arange(m), y] = 1.0
    eye = np.eye(K)[None]

    def grad(w):
        return M * (softmax_rows(M * w) - onehot) + M * rho_l * (w - a)

    eps = np.finfo(np.float64).eps
    w = a.copy()
    g = grad(w)
    for _ in range(max_iters):
        p = softmax_rows(M * w)
        H = (M * M) * (p[:, :, None] * eye - p[:, :, None] * p[:, None, :]) + M * rho_l * eye
        step = np.linalg.solve(H, g[:, :, None])[:, :, 0]
        done = np.all(np.abs(step) <= 4.0 * eps * np.maximum(1.0, np.abs(w)), axis=1)
        if done.all():
            break
        gn = np.linalg.norm(g, axis=1)
        alpha = np.where(done, 0.0, 1.0)
        for _ in range(60):
            g_try = grad(w - alpha[:, None] * step)
            bad = (np.linalg.norm(g_try, axis=1) > (1.0 - 1e-4 * alpha) * gn) & ~done
            if not bad.any():
                break
            alpha = np.where(bad, 0.5 * alpha, alpha)
        w = w - alpha[:, None] * step
        g = grad(w)
    return w


# --------------------------------------------------------------------------- (z,t) step

def zt_step(w, s, v, N, rho_c, rho_b):
    """(z, t) update of eq. (global-z-t-updae) in scaled form:

        min_{||z||_1 <= t}  (N rho_c / 2) ||z - w||^2 + (rho_b / 2) (s'z - t + v)^2,
        w = (1/N) sum_i (x_i + u_i).

    KKT with multiplier mu = N rho_c tau >= 0 gives z(tau) = S_tau(w + tau s) (soft
    threshold) and, when the l1 constraint is active, t = ||z||_1 and h(tau) = 0 with

        h(tau) = s'z(tau) - ||z(tau)||_1 + v + beta tau,     beta = N rho_c / rho_b.

    h is continuous, piecewise linear and strictly increasing.  Coordinate r contributes
    c_r + e_r tau while z_r != 0, with c_r = s_r w_r - |w_r|, e_r = (s_r - sign w_r)^2, and
    0 from its breakpoint tau_r = |w_r| / (1 - sign(w_r) s_r) on.  The root is found exactly
    by sorting the breakpoints.  Returns (z, t, tau).
    """
    w = np.asarray(w, dtype=np.float64)
    s = np.asarray(s, dtype=np.float64)
    beta = N * rho_c / rho_b
    sig = np.sign(w)
    c = s * w - np.abs(w)
    e = (s - sig) ** 2
    h0 = v + c.sum()
    if h0 >= 0.0:  # l1 constraint inactive: z = w, t makes the bilinear term vanish
        return w.copy(), float(s @ w + v), 0.0
    finite = (w != 0.0) & (sig * s < 1.0)
    tau_r = np.abs(w[finite]) / (1.0 - sig[finite] * s[finite])
    order = np.argsort(tau_r, kind="stable")
    bp = tau_r[order]
    cs = c[finite][order]
    es = e[finite][order]
    # segment k = [bp[k-1], bp[k]) has active coordinates order[k:]
    C = np.concatenate([np.cumsum(cs[::-1])[::-1], [0.0]])
    E = np.concatenate([np.cumsum(es[::-1])[::-1], [0.0]])
    right = np.concatenate([bp, [np.inf]])
    tau = None
    for k in range(len(right)):
        if np.isinf(right[k]) or v + C[k] + (beta + E[k]) * right[k] >= 0.0:
            tau = -(v + C[k]) / (beta + E[k])
            break
    y = w + tau * s
    z = np.sign(y) * np.maximum(np.abs(y) - tau, 0.0)
    return z, float(np.abs(z).sum()), float(tau)


# --------------------------------------------------------------------------- s step

def top_kappa(z, kappa):
    """Indices of the kappa largest |z_r|; ties go to the lowest index.  Sorted ascending."""
    z = np.asarray(z)
    order = np.lexsort((np.arange(z.size), -np.abs(z)))
    return np.sort(order[:kappa])


def s_step(z, t, v, kappa):
    """s update of eq. (s-update-final): argmin over S^kappa of (z's - t + v)^2.

    Over S^kappa = {||s||_inf <= 1, ||s||_1 <= kappa} the achievable values of z's fill
    [-T, T], T = sum of the kappa largest |z_r|, the extremes attained by +/- sign(z) on
    those coordinates.  The minimiser taken is clamp((t - v)/T, -1, 1) times that vector.
    """
    z = np.asarray(z, dtype=np.float64)
    theta = t - v
    S = top_kappa(z, kappa)
    s_top = np.zeros_like(z)
    s_top[S] = np.sign(z[S])
    T = float(np.abs(z[S]).sum())
    if T == 0.0:
        return np.zeros_like(z)
    return min(1.0, max(-1.0, theta / T)) * s_top


# --------------------------------------------------------------------------- solver state

class BiCADMM:
    """Bi-cADMM over N sample shards, each with M feature blocks (Algorithms 1 and 2).

    A: (m, n) FP64, b: (m,) targets (squared), labels in {-1,+1}, or class indices
    0..K-1 (softmax, K classes).  n-space vectors have length n*K (feature-major).
    """

    def __init__(self, A, b, loss, N, M, kappa, gamma=10.0, rho_c=1.0, rho_b=None,
                 rho_l=None, inner_iters=1, n_shards_total=None, K=1):
        self.A = np.asarray(A, dtype=np.float64)
        self.b = np.asarray(b, dtype=np.float64)
        self.m, self.n = self.A.shape
        self.loss, self.N, self.M, self.kappa = int(loss), int(N), int(M), int(kappa)
        self.K = int(K)
        if (self.loss == LOSS_SOFTMAX) != (self.K > 1):
            raise ValueError("K > 1 exactly for the softmax loss")
        self.gamma, self.rho_c = float(gamma), float(rho_c)
        self.rho_b = 0.5 * self.rho_c if rho_b is None else float(rho_b)
        self.rho_l = self.rho_c if rho_l is None else float(rho_l)
        self.J = int(inner_iters)
        self.shards = split_ranges(self.m, self.N)
        self.blocks = split_ranges(self.n, self.M)
        # coefficient of x_ij in r_j (eq. before the sharing problem): 1/(N gamma) + rho_c.
        # n_shards_total lets an instance hold a subset of the shards of a larger problem
        # (its x-steps are then those of the full problem; its z-step is not).
        N_all = self.N if n_shards_total is None else int(n_shards_total)
        self.c0 = 1.0 / (N_all * self.gamma) + self.rho_c
        # Block factors for the x_ij solve of eq. (p:GPU;x): setting its gradient to zero
        # gives (rho_l A_ij'A_ij + c0 I) x_ij = rho_l A_ij' c_ij + rho_c (z_j - u_ij).
        self.factors = []
        for (r0, r1) in self.shards:
            row = []
            for (c0_, c1_) in self.blocks:
                Aij = self.A[r0:r1, c0_:c1_]
                K = self.rho_l * (Aij.T @ Aij) + self.c0 * np.eye(c1_ - c0_)
                row.append(scipy.linalg.cho_factor(K, lower=True))
            self.factors.append(row)
        n, N, K = self.n, self.N, self.K
        self.x = np.zeros((N, n * K))
        self.u = np.zeros((N, n * K))
        self.z = np.zeros(n * K)
        self.s = np.zeros(n * K)
        self.t = 0.0
        self.v = 0.0
        self.tau = 0.0
        mshape = (self.m,) if K == 1 else (self.m, K)
        self.omega = np.zeros(mshape)   # omega-bar, per shard row range
        self.nu = np.zeros(mshape)
        self.Axbar = np.zeros(mshape)   # (1/M) sum_j A_ij x_ij
        self.p = [[np.zeros((r1 - r0, K)) for _ in self.blocks] for (r0, r1) in self.shards]
        self.iters = 0
        self.history = []

    # ---- Algorithm 2: node-level sharing ADMM for the local prox (eq. p:x-subp)
    def x_step_shard(self, i):
        r0, r1 = self.shards[i]
        b_i = self.b[r0:r1]
        K = self.K
        # (rows, K) views of the m-space state and (n, K) views of the n-space state
        omega_v = self.omega.reshape(self.m, K)
        nu_v = self.nu.reshape(self.m, K)
        Axbar_v = self.Axbar.reshape(self.m, K)
        X, U, Z = self.x[i].reshape(self.n, K), self.u[i].reshape(self.n, K), self.z.reshape(self.n, K)
        for _ in range(self.J):
            omega, Axbar, nu = omega_v[r0:r1], Axbar_v[r0:r1], nu_v[r0:r1]
            new_x = []
            for j, (c0_, c1_) in enumerate(self.blocks):
                Aij = self.A[r0:r1, c0_:c1_]
                # eq. (p:GPU;x): target A_ij x_ij ~ A_ij x_ij^k + omega^k - Axbar^k - nu^k
                c_ij = self.p[i][j] + omega - Axbar - nu
                rhs = self.rho_l * (Aij.T @ c_ij) + self.rho_c * (Z[c0_:c1_] - U[c0_:c1_])
                new_x.append(scipy.linalg.cho_solve(self.factors[i][j], rhs))
            for j, (c0_, c1_) in enumerate(self.blocks):
                X[c0_:c1_] = new_x[j]
                self.p[i][j] = self.A[r0:r1, c0_:c1_] @ new_x[j]
            Axbar_new = sum(self.p[i]) / self.M                      # "Allreduce", Alg. 2
            if K == 1:                                               # (p:GPU;omega)
                omega_new = omega_prox(self.loss, (Axbar_new + nu)[:, 0], b_i, self.M, self.rho_l)[:, None]
            else:
                omega_new = omega_prox(self.loss, Axbar_new + nu, b_i, self.M, self.rho_l)
            nu_v[r0:r1] = nu + Axbar_new - omega_new                 # (p:GPU;nu)
            omega_v[r0:r1] = omega_new
            Axbar_v[r0:r1] = Axbar_new

    # ---- one outer iteration (iterations block, scaled form)
    def iterate(self, n_iters=1):
        for _ in range(n_iters):
            for i in range(self.N):
                self.x_step_shard(i)
            w = (self.x + self.u).mean(axis=0)
            z_prev = self.z
            self.z, self.t, self.tau = zt_step(w, self.s, self.v, self.N, self.rho_c, self.rho_b)
            self.s = s_step(self.z, self.t, self.v, self.kappa)
            self.u = self.u + self.x - self.z[None, :]
            g = float(self.z @ self.s) - self.t
            self.v = self.v + g
            self.iters += 1
            self.history.append(self.residuals(z_prev, g))
        return self.history[-1]

    def residuals(self, z_prev, g):
        """Termination residuals p_r, d_r, b_r (Sec. 3, Termination) and relative forms."""
        N = self.N
        p_r = float(sum(np.linalg.norm(self.x[i] - self.z) for i in range(N)))
        dz = float(np.linalg.norm(self.z - z_prev))
        d_r = math.sqrt(N) * self.rho_c * dz
        b_r = abs(g)
        nz = float(np.linalg.norm(self.z))
        nx = float(sum(np.linalg.norm(self.x[i]) for i in range(N)))
        i_r = float(np.linalg.norm(self.Axbar - self.omega))
        i_den = max(float(np.linalg.norm(self.omega)), float(np.linalg.norm(self.Axbar)), 1e-30)
        return dict(p_r=p_r, d_r=d_r, b_r=b_r, i_r=i_r,
                    p_rel=p_r / max(nx, N * nz, 1e-30),
                    d_rel=dz / max(nz, 1e-30),
                    b_rel=b_r / max(self.t, 1e-30),
                    i_rel=i_r / i_den)

    def solve(self, tol_rel=1e-6, max_iters=10000):
        for _ in range(max_iters):
            r = self.iterate(1)
            if max(r["p_rel"], r["d_rel"], r["b_rel"], r["i_rel"]) <= tol_rel:
                return True
        return False

    def support(self):
        return top_kappa(self.z, self.kappa)

    def polished(self):
        return polish(self.A, self.b, self.loss, self.gamma, self.support(), K=self.K)


# --------------------------------------------------------------------------- polish

def polish(A, b, loss, gamma, S, tol=1e-13, max_newton=100, K=1):
    """Restricted problem on a fixed support S (not part of the paper's algorithm):

        min_{supp x in S}  sum_r l(a_r x; b_r) + ||x||^2 / (2 gamma),  solved in FP64.
    Softmax: S indexes the flattened n x K matrix (entry (c, k) at c*K + k).
    """
    A = np.asarray(A, dtype=np.float64)
    if loss == LOSS_SOFTMAX:
        return _polish_softmax(A, b, gamma, S, K, tol, max_newton)
    n = A.shape[1]
    AS = A[:, S]
    x = np.zeros(n)
    k = len(S)
    if loss == LOSS_SQUARED:
        H = 2.0 * AS.T @ AS + np.eye(k) / gamma
        x[S] = np.linalg.solve(H, 2.0 * AS.T @ b)
        return x
    xs = np.zeros(k)
    F = lambda v: float(np.sum(loss_rows(loss, AS @ v, b)) + v @ v / (2.0 * gamma))
    for _ in range(max_newton):
        q = AS @ xs
        if loss == LOSS_LOGISTIC:
            sg = expit(-b * q)
            grad = AS.T @ (-b * sg) + xs / gamma
            wts = sg * (1.0 - sg)
        elif loss == LOSS_SQHINGE:
            act = (1.0 - b * q) > 0.0
            grad = AS.T @ np.where(act, -2.0 * b * (1.0 - b * q), 0.0) + xs / gamma
            wts = np.where(act, 2.0, 0.0)
        else:
            raise ValueError(loss)
        H = AS.T @ (AS * wts[:, None]) + np.eye(k) / gamma
        step = np.linalg.solve(H, grad)
        f0, alpha = F(xs), 1.0
        while F(xs - alpha * step) > f0 + 1e-16 * abs(f0) and alpha > 1e-12:
            alpha *= 0.5
        xs = xs - alpha * step
        if np.linalg.norm(alpha * step) <= tol * max(1.0, np.linalg.norm(xs)):
            break
    x[S] = xs
    return x


def _polish_softmax(A, b, gamma, S, K, tol, max_newton):
    """Damped Newton on the entries in S of the n x K matrix W (the rest held at zero).
    With Q = A W and P = softmax rows: gradient A'(P - Y) + W/gamma; Hessian of entries
    (c, k), (c', k'): sum_r a_rc a_rc' p_rk (delta_kk' - p_rk') + delta / gamma."""
    m, n = A.shape
    y = np.asarray(b).astype(np.int64)
    S = np.asarray(S, dtype=np.int64)
    cols, cls = S // K, S % K
    Y = np.zeros((m, K))
    Y[np.arange(m), y] = 1.0
    w = np.zeros(len(S))

    def full(wv):
        W = np.zeros(n * K)
        W[S] = wv
        return W.reshape(n, K)

    def F(wv):
        Q = A @ full(wv)
        return float(np.sum(logsumexp_rows(Q) - Q[np.arange(m), y]) + wv @ wv / (2.0 * gamma))

    AS = A[:, cols]                      # column of A for each support entry
    for _ in range(max_newton):
        P = softmax_rows(A @ full(w))
        G = A.T @ (P - Y)
        grad = G[cols, cls] + w / gamma
        Pk = P[:, cls]                   # p_{r, k(e)} for each support entry e
        same = (cls[:, None] == cls[None, :]).astype(np.float64)
        H = (AS * Pk).T @ AS * same - (AS * Pk).T @ (AS * Pk) + np.eye(len(S)) / gamma
        step = np.linalg.solve(H, grad)
        f0, alpha = F(w), 1.0
        while F(w - alpha * step) > f0 + 1e-16 * abs(f0) and alpha > 1e-12:
            alpha *= 0.5
        w = w - alpha * step
        if np.linalg.norm(alpha * step) <= tol * max(1.0, np.linalg.norm(w)):
            break
    return full(w).reshape(-1)
