"""Pins for the FP64 CPU oracle against facts fixed by the paper and by mathematics.

None of these compare the oracle with itself: each check uses a hand derivation, a
closed form, an independent numerical method (scipy's generic optimisers, brute-force
enumeration, bisection) or an optimality condition stated on the original problem.
"""
import itertools
import math
import json
import os

import numpy as np
import pytest
import scipy.optimize

from oracle import bicadmm_ref as ref
from paper_2405_16267_b300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "worked_examples.json")


def golden():
    with open(GOLDEN) as f:
        return json.load(f)


# ----------------------------------------------------------------- (z,t) step

@pytest.mark.parametrize("case", range(3))
def test_zt_step_worked_examples(case):
    g = golden()["zt_step"][case]
    inp = g["inputs"]
    z, t, _ = ref.zt_step(np.array(inp["w"]), np.array(inp["s"]), inp["v"], inp["N"],
                          inp["rho_c"], inp["rho_b"])
    np.testing.assert_allclose(z, g["expected"]["z"], atol=1e-14)
    assert abs(t - g["expected"]["t"]) < 1e-14


# ----------------------------------------------------------------- residuals

@pytest.mark.parametrize("case", range(3))
def test_residuals_worked_examples(case):
    """Termination residuals (Sec. 3) and their relative forms on hand-derived states: the
    oracle's solver object is given the state directly (one row per shard, M = 1)."""
    g = golden()["residuals"][case]
    inp = g["inputs"]
    N = inp["N"]
    x = np.array(inp["x"], dtype=np.float64)
    n = x.shape[1]
    o = ref.BiCADMM(np.eye(N, n) + 1.0, np.zeros(N), ref.LOSS_SQUARED, N, 1, 1,
                    rho_c=inp["rho_c"])
    o.x = x
    o.z = np.array(inp["z"], dtype=np.float64)
    o.t = inp["t"]
    o.Axbar = np.array(inp["Axbar"], dtype=np.float64)
    o.omega = np.array(inp["omega"], dtype=np.float64)
    r = o.residuals(np.array(inp["z_prev"], dtype=np.float64), inp["g"])
    for key, want in g["expected"].items():
        assert abs(r[key] - want) <= 1e-15 * max(1.0, abs(want)), (key, r[key], want)


def _zt_objective(z, t, w, s, v, N, rho_c, rho_b):
    return 0.5 * N * rho_c * np.sum((z - w) ** 2) + 0.5 * rho_b * (s @ z - t + v) ** 2


def _zt_kkt_violation(z, t, w, s, v, N, rho_c, rho_b):
    """KKT of min (N rho_c/2)||z-w||^2 + (rho_b/2)(s'z - t + v)^2 s.t. ||z||_1 - t <= 0,
    written on the original problem (not on the tau parametrisation)."""
    g = s @ z - t + v
    mu = -rho_b * g                       # stationarity in t:  -rho_b g - mu = 0
    viol = max(0.0, -mu)                  # mu >= 0
    viol = max(viol, np.abs(z).sum() - t)  # primal feasibility
    viol = max(viol, abs(mu * (np.abs(z).sum() - t)))  # complementarity
    grad = N * rho_c * (z - w) + rho_b * g * s   # + mu * xi, xi in d||z||_1
    nz = z != 0
    viol = max(viol, np.max(np.abs(grad[nz] + mu * np.sign(z[nz])), initial=0.0))
    if np.any(~nz):
        if mu > 0:
            xi = -grad[~nz] / mu
            viol = max(viol, np.max(np.abs(xi)) - 1.0)
        else:
            viol = max(viol, np.max(np.abs(grad[~nz])))
    return viol


@pytest.mark.parametrize("seed", range(20))
def test_zt_step_kkt_random(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 60))
    w = rng.standard_normal(n) * rng.choice([0.1, 1.0, 10.0])
    w[rng.random(n) < 0.2] = 0.0
    s = np.clip(rng.standard_normal(n), -1, 1)
    # some coordinates with s_r = sign(w_r) exactly (never-zeroed coordinates)
    idx = rng.random(n) < 0.2
    s[idx] = np.sign(w[idx])
    v = float(rng.standard_normal() * 5)
    N, rho_c, rho_b = int(rng.integers(1, 9)), float(rng.uniform(0.1, 3)), float(rng.uniform(0.1, 3))
    z, t, tau = ref.zt_step(w, s, v, N, rho_c, rho_b)
    scale = 1.0 + np.abs(w).sum() + abs(v)
    assert _zt_kkt_violation(z, t, w, s, v, N, rho_c, rho_b) <= 1e-10 * scale * max(1, N * rho_c, rho_b)
    assert tau >= 0.0


@pytest.mark.parametrize("seed", range(6))
def test_zt_step_vs_generic_solver(seed):
    """Independent check with scipy's SLSQP on the split form z = zp - zm, zp, zm >= 0."""
    rng = np.random.default_rng(100 + seed)
    n = 5
    w = rng.standard_normal(n) * 2
    s = np.clip(rng.standard_normal(n), -1, 1)
    v = float(rng.standard_normal() * 3 - 2)
    N, rho_c, rho_b = 3, 1.0, 0.5
    z, t, _ = ref.zt_step(w, s, v, N, rho_c, rho_b)
    f_oracle = _zt_objective(z, t, w, s, v, N, rho_c, rho_b)

    def f(y):
        zz = y[:n] - y[n:2 * n]
        return _zt_objective(zz, y[-1], w, s, v, N, rho_c, rho_b)

    cons = [{"type": "ineq", "fun": lambda y: y[-1] - y[:2 * n].sum()}]
    best = np.inf
    for start in range(5):
        y0 = np.abs(rng.standard_normal(2 * n + 1)) * 2
        y0[-1] = y0[:2 * n].sum() + 1
        res = scipy.optimize.minimize(f, y0, constraints=cons, bounds=[(0, None)] * (2 * n) + [(None, None)],
                                      method="SLSQP", options=dict(ftol=1e-14, maxiter=2000))
        best = min(best, res.fun)
    assert f_oracle <= best + 1e-7 * (1 + abs(best))


def test_zt_step_root_by_bisection():
    """tau from the sorted-breakpoint solve agrees with plain bisection on h(tau)."""
    rng = np.random.default_rng(7)
    for _ in range(20):
        n = 40
        w = rng.standard_normal(n) * 3
        s = np.clip(rng.standard_normal(n), -1, 1)
        v = -abs(rng.standard_normal()) * 20
        N, rho_c, rho_b = 4, 1.0, 0.5
        beta = N * rho_c / rho_b

        def h(tau):
            y = w + tau * s
            zz = np.sign(y) * np.maximum(np.abs(y) - tau, 0)
            return s @ zz - np.abs(zz).sum() + v + beta * tau

        if h(0.0) >= 0:
            continue
        lo, hi = 0.0, 1.0
        while h(hi) < 0:
            hi *= 2
        for _ in range(200):
            mid = 0.5 * (lo + hi)
            lo, hi = (mid, hi) if h(mid) < 0 else (lo, mid)
        _, _, tau = ref.zt_step(w, s, v, N, rho_c, rho_b)
        assert abs(tau - 0.5 * (lo + hi)) <= 1e-12 * max(1.0, tau)


# ----------------------------------------------------------------- s step

@pytest.mark.parametrize("case", range(2))
def test_s_step_worked_examples(case):
    g = golden()["s_step"][case]
    inp = g["inputs"]
    s = ref.s_step(np.array(inp["z"]), inp["t"], inp["v"], inp["kappa"])
    np.testing.assert_allclose(s, g["expected"]["s"], atol=1e-15)


def _vertices(n, kappa):
    for supp in itertools.combinations(range(n), kappa):
        for signs in itertools.product([-1.0, 1.0], repeat=kappa):
            s = np.zeros(n)
            s[list(supp)] = signs
            yield s


@pytest.mark.parametrize("seed", range(10))
def test_s_step_vertex_enumeration(seed):
    """min over S^kappa of (z's - theta)^2 equals dist(theta, [-T, T])^2 where T is the
    maximum of z's over the vertices of S^kappa (an LP attains it at a vertex)."""
    rng = np.random.default_rng(seed)
    n = int(rng.integers(2, 9))
    kappa = int(rng.integers(1, n + 1))
    z = rng.standard_normal(n)
    z[rng.random(n) < 0.2] = 0.0
    t, v = float(rng.standard_normal() * 4), float(rng.standard_normal())
    theta = t - v
    T = max(float(z @ s) for s in _vertices(n, kappa))
    best = (max(0.0, abs(theta) - T)) ** 2
    s = ref.s_step(z, t, v, kappa)
    assert np.max(np.abs(s)) <= 1.0 + 1e-15 and np.abs(s).sum() <= kappa + 1e-12
    assert (z @ s - theta) ** 2 <= best + 1e-12


def test_top_kappa_ties_lowest_index():
    z = np.array([0.0, 5.0, -5.0, 5.0, 1.0, -5.0])
    assert list(ref.top_kappa(z, 2)) == [1, 2]
    assert list(ref.top_kappa(z, 3)) == [1, 2, 3]
    assert list(ref.top_kappa(np.zeros(4), 2)) == [0, 1]


# ----------------------------------------------------------------- omega-bar prox

@pytest.mark.parametrize("case", range(2))
def test_omega_prox_worked_examples(case):
    g = golden()["omega_prox"][case]
    inp = g["inputs"]
    w = ref.omega_prox(inp["loss"], np.array(inp["a"]), np.array(inp["b"]), inp["M"], inp["rho_l"])
    np.testing.assert_allclose(w, g["expected"], atol=1e-15)


@pytest.mark.parametrize("loss", [ref.LOSS_SQUARED, ref.LOSS_LOGISTIC, ref.LOSS_SQHINGE])
def test_omega_prox_vs_scalar_minimiser(loss):
    rng = np.random.default_rng(3)
    for _ in range(40):
        M = int(rng.integers(1, 9))
        rho_l = float(rng.uniform(0.1, 4))
        a = float(rng.standard_normal() * 3)
        b = float(rng.standard_normal() * 2) if loss == ref.LOSS_SQUARED else float(rng.choice([-1.0, 1.0]))
        phi = lambda w: float(ref.loss_rows(loss, np.array([M * w]), np.array([b]))[0]) + 0.5 * M * rho_l * (w - a) ** 2
        res = scipy.optimize.minimize_scalar(phi, bracket=(a - 10, a + 10), method="brent",
                                             options=dict(xtol=1e-14))
        w = float(ref.omega_prox(loss, np.array([a]), np.array([b]), M, rho_l)[0])
        assert phi(w) <= res.fun + 1e-12 * (1 + abs(res.fun))
        assert abs(w - res.x) <= 1e-6 * (1 + abs(w))


# ----------------------------------------------------------------- inner loop = exact prox

def _exact_prox_squared(A, b, z, u, N, gamma, rho_c):
    n = A.shape[1]
    c0 = 1.0 / (N * gamma) + rho_c
    return np.linalg.solve(2 * A.T @ A + c0 * np.eye(n), 2 * A.T @ b + rho_c * (z - u))


def test_inner_sharing_admm_reaches_exact_prox_squared():
    """Sec. 3.1: the feature-split sharing ADMM computes the local prox of eq. (p:localprox).
    For the squared loss that prox is one linear solve."""
    P = synth.small_problem(ref.LOSS_SQUARED, m=90, n=13, nnz=3, N=1, M=3, kappa=13, seed=5)
    o = ref.BiCADMM(P.A, P.b, P.loss, 1, 3, 13, gamma=2.0, rho_c=0.7, rho_l=2.0, inner_iters=3000)
    rng = np.random.default_rng(0)
    o.z = rng.standard_normal(13)
    o.u[0] = rng.standard_normal(13) * 0.3
    o.x_step_shard(0)
    x_exact = _exact_prox_squared(P.A, P.b, o.z, o.u[0], 1, 2.0, 0.7)
    np.testing.assert_allclose(o.x[0], x_exact, rtol=0, atol=1e-8 * np.abs(x_exact).max())


@pytest.mark.parametrize("loss", [ref.LOSS_LOGISTIC, ref.LOSS_SQHINGE])
def test_inner_sharing_admm_reaches_exact_prox_classification(loss):
    P = synth.small_problem(loss, m=80, n=10, nnz=3, N=2, M=2, kappa=10, seed=6)
    N, gamma, rho_c = 2, 3.0, 0.8
    o = ref.BiCADMM(P.A, P.b, loss, N, 2, 10, gamma=gamma, rho_c=rho_c, rho_l=1.5, inner_iters=4000)
    rng = np.random.default_rng(1)
    o.z = rng.standard_normal(10) * 0.5
    o.u[1] = rng.standard_normal(10) * 0.2
    o.x_step_shard(1)
    r0, r1 = o.shards[1]
    A1, b1 = P.A[r0:r1], P.b[r0:r1]

    def f(x):
        return (np.sum(ref.loss_rows(loss, A1 @ x, b1)) + x @ x / (2 * N * gamma)
                + 0.5 * rho_c * np.sum((x - o.z + o.u[1]) ** 2))

    res = scipy.optimize.minimize(f, np.zeros(10), method="BFGS", options=dict(gtol=1e-11, maxiter=10000))
    np.testing.assert_allclose(o.x[1], res.x, atol=1e-6)


# ----------------------------------------------------------------- whole loop

def test_kappa_equals_n_gives_ridge():
    """With kappa = n the l0 constraint is void and problem (p:SML) with the squared loss
    of (p:sls) is ridge regression: (2 A'A + I/gamma) x = 2 A'b."""
    P = synth.sparse_linear(m=240, n=12, nnz=4, N=3, M=2, kappa=12, unit_columns=True, seed=2)
    o = ref.BiCADMM(P.A, P.b, P.loss, P.N, P.M, P.n, gamma=5.0, rho_c=1.0, inner_iters=2)
    assert o.solve(tol_rel=1e-10, max_iters=20000)
    x_ridge = np.linalg.solve(2 * P.A.T @ P.A + np.eye(P.n) / 5.0, 2 * P.A.T @ P.b)
    np.testing.assert_allclose(o.z, x_ridge, rtol=0, atol=1e-6 * np.abs(x_ridge).max())


def _brute_force(A, b, kappa, gamma):
    n = A.shape[1]
    best = (np.inf, None)
    for S in itertools.combinations(range(n), kappa):
        S = list(S)
        AS = A[:, S]
        xs = np.linalg.solve(2 * AS.T @ AS + np.eye(kappa) / gamma, 2 * AS.T @ b)
        x = np.zeros(n)
        x[S] = xs
        f = float(np.sum((A @ x - b) ** 2) + x @ x / (2 * gamma))
        if f < best[0]:
            best = (f, x)
    return best


@pytest.mark.parametrize("seed,n,kappa", [(0, 12, 3), (1, 14, 4), (2, 16, 2)])
def test_brute_force_support_clear_margin(seed, n, kappa):
    """Clear-margin instances (planted +/-U[1,2], noise 0.1, m >> n): the Bi-cADMM support
    and its polished solution equal the global optimum over all C(n, kappa) supports."""
    P = synth.sparse_linear(m=200, n=n, nnz=kappa, N=2, M=2, kappa=kappa, unit_columns=True, seed=seed)
    o = ref.BiCADMM(P.A, P.b, P.loss, P.N, P.M, kappa, gamma=10.0, rho_c=1.0)
    o.solve(tol_rel=1e-8, max_iters=5000)
    f_best, x_best = _brute_force(P.A, P.b, kappa, 10.0)
    assert set(o.support()) == set(np.flatnonzero(x_best))
    np.testing.assert_allclose(o.polished(), x_best, atol=1e-10)


def test_fixed_point_conditions():
    """At convergence: x_i = z, ||z||_0 <= kappa, z's = t = ||z||_1 (Theorem of Sec. 2.1),
    and the gradient of F restricted to the support vanishes (restricted KKT)."""
    P = synth.sparse_linear(m=400, n=40, nnz=5, N=4, M=3, kappa=5, unit_columns=True, seed=4)
    gamma = 10.0
    o = ref.BiCADMM(P.A, P.b, P.loss, P.N, P.M, P.kappa, gamma=gamma, rho_c=1.0)
    assert o.solve(tol_rel=1e-9, max_iters=20000)
    z = o.z
    S = np.flatnonzero(np.abs(z) > 1e-8 * np.abs(z).max())
    assert len(S) <= P.kappa
    assert np.abs(o.x - z[None]).max() <= 1e-6 * np.abs(z).max()
    assert abs(z @ o.s - o.t) <= 1e-8 * o.t and abs(np.abs(z).sum() - o.t) <= 1e-8 * o.t
    grad = 2 * P.A.T @ (P.A @ z - P.b) + z / gamma
    assert np.abs(grad[S]).max() <= 1e-5 * np.abs(grad).max()


def test_polish_logistic_vs_generic():
    P = synth.small_problem(ref.LOSS_LOGISTIC, m=300, n=20, nnz=4, N=2, M=2, kappa=4, seed=8)
    S = np.flatnonzero(P.x_star)
    x = ref.polish(P.A, P.b, ref.LOSS_LOGISTIC, 10.0, S)
    f = lambda xs: ref.objective(ref.LOSS_LOGISTIC, P.A[:, S], P.b, xs, 10.0)
    res = scipy.optimize.minimize(f, np.zeros(len(S)), method="BFGS", options=dict(gtol=1e-12))
    np.testing.assert_allclose(x[S], res.x, atol=1e-6)
    assert np.count_nonzero(x) <= len(S)


def test_polish_sqhinge_vs_generic():
    P = synth.small_problem(ref.LOSS_SQHINGE, m=300, n=20, nnz=4, N=2, M=2, kappa=4, seed=9)
    S = np.flatnonzero(P.x_star)
    x = ref.polish(P.A, P.b, ref.LOSS_SQHINGE, 10.0, S)
    f = lambda xs: ref.objective(ref.LOSS_SQHINGE, P.A[:, S], P.b, xs, 10.0)
    res = scipy.optimize.minimize(f, np.zeros(len(S)), method="BFGS", options=dict(gtol=1e-12))
    assert f(x[S]) <= res.fun + 1e-9 * abs(res.fun)


def test_split_ranges():
    assert ref.split_ranges(10, 3) == [(0, 4), (4, 7), (7, 10)]
    assert ref.split_ranges(5, 5) == [(0, 1), (1, 2), (2, 3), (3, 4), (4, 5)]
    assert synth.split_ranges(10, 3) == ref.split_ranges(10, 3)


# ----------------------------------------------------------------- softmax (K classes)

def test_softmax_loss_closed_forms():
    """Cross-entropy of Sec. 2's sparse softmax regression: logsumexp(q) - q_y."""
    q = np.array([[0.0, 0.0, 0.0], [1.0, 2.0, 0.0], [-3.0, 5.0, 5.0]])
    y = np.array([1, 0, 2])
    want = [math.log(3.0), math.log(math.e + math.e ** 2 + 1.0) - 1.0,
            math.log(math.exp(-3.0) + 2.0 * math.exp(5.0)) - 5.0]
    np.testing.assert_allclose(ref.loss_rows(ref.LOSS_SOFTMAX, q, y), want, rtol=1e-15)


def test_softmax_prox_two_classes_is_logistic_prox():
    """K = 2: with delta = w_1 - w_0 and sigma = w_0 + w_1 the softmax prox separates into
    sigma = a_0 + a_1 and a logistic prox of eq. (p:GPU;omega) for delta at a_1 - a_0 with
    label +1 (class 1) or -1 (class 0) and penalty rho_l / 2 (||w - a||^2 is half the sum
    of the squared sigma and delta offsets).  The logistic prox is a bisection."""
    rng = np.random.default_rng(11)
    for M, rho_l in [(1, 1.0), (4, 0.5), (8, 2.0), (2, 0.05)]:
        a = rng.standard_normal((200, 2)) * 3
        y = rng.integers(0, 2, 200)
        w = ref.softmax_prox(a, y, M, rho_l)
        delta = ref.omega_prox(ref.LOSS_LOGISTIC, a[:, 1] - a[:, 0], np.where(y == 1, 1.0, -1.0),
                               M, rho_l / 2)
        np.testing.assert_allclose(w[:, 1] - w[:, 0], delta, rtol=0, atol=1e-12 * (1 + np.abs(delta).max()))
        np.testing.assert_allclose(w.sum(axis=1), a.sum(axis=1), rtol=0, atol=1e-12 * (1 + np.abs(a).max()))


def test_softmax_prox_vs_generic_minimiser():
    rng = np.random.default_rng(12)
    K = 5
    for _ in range(25):
        M = int(rng.integers(1, 9))
        rho_l = float(rng.uniform(0.05, 4))
        a = rng.standard_normal(K) * 2
        y = int(rng.integers(0, K))
        phi = lambda w: float(ref.loss_rows(ref.LOSS_SOFTMAX, (M * w)[None], np.array([y]))[0]
                              + 0.5 * M * rho_l * np.sum((w - a) ** 2))
        res = scipy.optimize.minimize(phi, a, method="BFGS", options=dict(gtol=1e-12))
        w = ref.softmax_prox(a[None], np.array([y]), M, rho_l)[0]
        assert phi(w) <= res.fun + 1e-12 * (1 + abs(res.fun))
        np.testing.assert_allclose(w, res.x, atol=1e-6)


def test_inner_sharing_admm_reaches_exact_prox_softmax():
    """Sec. 3.1 with K = 3 classes: J sweeps of the sharing ADMM give the exact local prox
    argmin_W sum_r CE(a_r W; y_r) + ||W||^2/(2 N gamma) + rho_c/2 ||W - Z + U||^2."""
    K, n, N, gamma, rho_c = 3, 8, 2, 3.0, 0.8
    P = synth.sparse_softmax(m=160, n=n, K=K, nnz=5, N=N, M=2, kappa=5, seed=3, dtype=np.float64)
    o = ref.BiCADMM(P.A, P.b, ref.LOSS_SOFTMAX, N, 2, 5, gamma=gamma, rho_c=rho_c, rho_l=1.5,
                    inner_iters=4000, K=K)
    rng = np.random.default_rng(2)
    o.z = rng.standard_normal(n * K) * 0.5
    o.u[1] = rng.standard_normal(n * K) * 0.2
    o.x_step_shard(1)
    r0, r1 = o.shards[1]
    A1, b1 = P.A[r0:r1], P.b[r0:r1]

    def f(x):
        W = x.reshape(n, K)
        return (np.sum(ref.loss_rows(ref.LOSS_SOFTMAX, A1 @ W, b1)) + x @ x / (2 * N * gamma)
                + 0.5 * rho_c * np.sum((x - o.z + o.u[1]) ** 2))

    res = scipy.optimize.minimize(f, np.zeros(n * K), method="BFGS", options=dict(gtol=1e-11, maxiter=20000))
    np.testing.assert_allclose(o.x[1], res.x, atol=1e-6)


def test_softmax_kappa_full_gives_ridge_softmax():
    """kappa = n K: the l0 constraint is void and problem (p:SML) is ridge-regularised
    multinomial logistic regression, whose minimiser a generic method finds."""
    K, n = 3, 5
    P = synth.sparse_softmax(m=150, n=n, K=K, nnz=6, N=3, M=2, kappa=n * K, seed=4, dtype=np.float64)
    o = ref.BiCADMM(P.A, P.b, ref.LOSS_SOFTMAX, 3, 2, n * K, gamma=2.0, rho_c=1.0, inner_iters=2, K=K)
    assert o.solve(tol_rel=1e-8, max_iters=3000)
    f = lambda x: ref.objective(ref.LOSS_SOFTMAX, P.A, P.b, x, 2.0, K=K)
    res = scipy.optimize.minimize(f, np.zeros(n * K), method="BFGS", options=dict(gtol=1e-11))
    np.testing.assert_allclose(o.z, res.x, atol=1e-5 * np.abs(res.x).max())


def _brute_force_softmax(A, b, K, kappa, gamma):
    n = A.shape[1]
    best = (np.inf, None)
    for S in itertools.combinations(range(n * K), kappa):
        S = np.array(S)

        def f(ws):
            x = np.zeros(n * K)
            x[S] = ws
            return ref.objective(ref.LOSS_SOFTMAX, A, b, x, gamma, K=K)

        res = scipy.optimize.minimize(f, np.zeros(kappa), method="BFGS", options=dict(gtol=1e-10))
        if res.fun < best[0]:
            x = np.zeros(n * K)
            x[S] = res.x
            best = (res.fun, x)
    return best


def test_softmax_brute_force_support_clear_margin():
    """n = 4 features, K = 3 classes, entrywise kappa = 2 on a planted W* with two large
    entries: after 200 iterations the Bi-cADMM support (entries (c, k) at c*K + k) and its
    polished solution equal the optimum over all C(12, 2) supports.  (Bi-cADMM on the
    classification losses converges slowly in the residuals; the support settles early.)"""
    K, n, kappa = 3, 4, 2
    P = synth.sparse_softmax(m=600, n=n, K=K, nnz=kappa, N=2, M=2, kappa=kappa, seed=7,
                             dtype=np.float64, scale=2.0)
    o = ref.BiCADMM(P.A, P.b, ref.LOSS_SOFTMAX, 2, 2, kappa, gamma=10.0, rho_c=1.0, K=K)
    o.iterate(200)
    f_best, x_best = _brute_force_softmax(P.A, P.b, K, kappa, 10.0)
    assert set(o.support()) == set(np.flatnonzero(x_best))
    np.testing.assert_allclose(o.polished(), x_best, atol=1e-6)


def test_polish_softmax_vs_generic():
    K, n = 3, 8
    P = synth.sparse_softmax(m=300, n=n, K=K, nnz=5, N=2, M=2, kappa=5, seed=9, dtype=np.float64)
    S = np.flatnonzero(P.x_star)
    x = ref.polish(P.A, P.b, ref.LOSS_SOFTMAX, 10.0, S, K=K)

    def f(ws):
        v = np.zeros(n * K)
        v[S] = ws
        return ref.objective(ref.LOSS_SOFTMAX, P.A, P.b, v, 10.0, K=K)

    res = scipy.optimize.minimize(f, np.zeros(len(S)), method="BFGS", options=dict(gtol=1e-12))
    np.testing.assert_allclose(x[S], res.x, atol=1e-6)
    assert np.count_nonzero(x) <= len(S)
