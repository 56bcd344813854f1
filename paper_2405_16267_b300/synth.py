"""Seeded synthetic inputs for Bi-cADMM workloads.

This module only draws random problem data (A, b, the planted sparse model).  It holds
none of the solver's arithmetic, so the FP64 CPU oracle and the CUDA path can both be
fed from it without sharing any code of the method.

Every generator is deterministic in ``seed``.  Large matrices are generated in row chunks,
each from its own ``numpy.random.SeedSequence([seed, stream, chunk])`` child, so a single
shard of a large workload can be regenerated alone, bit-identically, without building the
whole matrix (the CPU baseline times the oracle on one such shard).

The data model follows the paper's experiments (Sec. 4, "Hardware and Software": dense
Gaussian local feature matrices, a planted sparse ground truth, noisy labels), with the
shapes and distributions of each named workload below.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

try:  # scipy's IIR filter gives the AR(1) column recursion at C speed
    from scipy.signal import lfilter as _lfilter
except Exception:  # pragma: no cover - scipy is present in this image
    _lfilter = None

LOSS_SQUARED, LOSS_LOGISTIC, LOSS_SOFTMAX, LOSS_SQHINGE = 0, 1, 2, 3


def split_ranges(total: int, parts: int):
    """Contiguous ranges; the first ``total % parts`` ranges get one extra element.

    Used for both sample shards (rows) and feature blocks (columns); the paper does not
    say how uneven sizes are split, this is the convention both sides follow.
    """
    base, rem = divmod(int(total), int(parts))
    out, start = [], 0
    for k in range(parts):
        size = base + (1 if k < rem else 0)
        out.append((start, start + size))
        start += size
    return out


@dataclasses.dataclass
class Problem:
    """One synthetic instance: A (m x n, row-major), labels/targets b (m,), planted x_star
    (n, or the flattened n x K matrix W* for softmax: entry (c, k) at c*K + k)."""
    name: str
    A: np.ndarray
    b: np.ndarray
    x_star: np.ndarray
    loss: int
    N: int
    M: int
    kappa: int
    rho: float
    gamma: float = 10.0
    iters: int = 200
    K: int = 1

    @property
    def m(self):
        return self.A.shape[0]

    @property
    def n(self):
        return self.A.shape[1]


def _rng(seed: int, stream: int, chunk: int = 0) -> np.random.Generator:
    return np.random.default_rng(np.random.SeedSequence([int(seed), int(stream), int(chunk)]))


def planted_support(n: int, nnz: int, seed: int, values: str = "pm_uniform12") -> np.ndarray:
    """Sparse ground truth with ``nnz`` nonzeros at uniformly random positions.

    values: 'pm_uniform12' -> +/-U[1,2] (clear margin), 'normal' -> N(0,1).
    """
    g = _rng(seed, 1)
    x = np.zeros(n)
    idx = g.choice(n, size=nnz, replace=False)
    if values == "pm_uniform12":
        x[idx] = g.choice([-1.0, 1.0], size=nnz) * g.uniform(1.0, 2.0, size=nnz)
    elif values == "normal":
        x[idx] = g.standard_normal(nnz)
    else:
        raise ValueError(values)
    return x


def gaussian_rows(m: int, n: int, seed: int, row0: int = 0, chunk_rows: int = 4096,
                  dtype=np.float64) -> np.ndarray:
    """Rows [row0, row0+m) of an i.i.d. N(0,1) matrix with n columns.

    Row r is drawn from chunk r // chunk_rows, so any row range can be regenerated alone.
    """
    out = np.empty((m, n), dtype=dtype)
    r = row0
    while r < row0 + m:
        c = r // chunk_rows
        c0, c1 = c * chunk_rows, (c + 1) * chunk_rows
        block = _rng(seed, 2, c).standard_normal((chunk_rows, n))
        lo, hi = max(r, c0), min(row0 + m, c1)
        out[lo - row0:hi - row0] = block[lo - c0:hi - c0]
        r = hi
    return out


def toeplitz_rows(m: int, n: int, seed: int, corr: float = 0.3, row0: int = 0,
                  chunk_rows: int = 4096, dtype=np.float64) -> np.ndarray:
    """Rows of a Gaussian matrix whose columns have correlation corr^|i-j| (unit variance).

    Each row is a stationary AR(1) sequence across columns:
    a_0 = g_0, a_j = corr * a_{j-1} + sqrt(1 - corr^2) * g_j.
    """
    g = gaussian_rows(m, n, seed, row0=row0, chunk_rows=chunk_rows, dtype=np.float64)
    c = math.sqrt(1.0 - corr * corr)
    if _lfilter is not None:
        zi = ((1.0 - c) * g[:, :1])
        a = _lfilter([c], [1.0, -corr], g, axis=1, zi=zi)[0]
    else:  # plain recursion
        a = np.empty_like(g)
        a[:, 0] = g[:, 0]
        for j in range(1, n):
            a[:, j] = corr * a[:, j - 1] + c * g[:, j]
    return a.astype(dtype, copy=False)


def _noise(m: int, seed: int, row0: int = 0, chunk_rows: int = 4096) -> np.ndarray:
    out = np.empty(m)
    r = row0
    while r < row0 + m:
        c = r // chunk_rows
        c0, c1 = c * chunk_rows, (c + 1) * chunk_rows
        block = _rng(seed, 3, c).standard_normal(chunk_rows)
        lo, hi = max(r, c0), min(row0 + m, c1)
        out[lo - row0:hi - row0] = block[lo - c0:hi - c0]
        r = hi
    return out


def _sign_pm1(v: np.ndarray) -> np.ndarray:
    return np.where(v >= 0.0, 1.0, -1.0)


# ----------------------------------------------------------------------------- workloads

def sparse_linear(m=2000, n=200, nnz=10, noise=0.1, N=4, M=2, kappa=10, rho=1.0,
                  gamma=10.0, iters=200, seed=0, unit_columns=False) -> Problem:
    """Sparse linear regression: A i.i.d. N(0,1), x* with nnz entries +/-U[1,2] at random
    indices, b = A x* + N(0, noise^2).  Defaults are the 2000 x 200 FP64 workload
    (N=4 shards of 500 rows, M=2 blocks of 100 columns, kappa=10, rho=1, 200 iterations).

    unit_columns=True normalises the columns of A to unit l2 norm; unit_columns="shard"
    normalises the columns of each shard's rows A_i separately, as the paper's experiments
    do (Sec. 4, "Hardware and Software").
    """
    A = gaussian_rows(m, n, seed)
    if unit_columns == "shard":
        for (r0, r1) in split_ranges(m, N):
            A[r0:r1] /= np.linalg.norm(A[r0:r1], axis=0, keepdims=True)
    elif unit_columns:
        A /= np.linalg.norm(A, axis=0, keepdims=True)
    x_star = planted_support(n, nnz, seed, "pm_uniform12")
    b = A @ x_star + noise * _noise(m, seed)
    return Problem("sparse_linear_%dx%d" % (m, n), A, b, x_star, LOSS_SQUARED, N, M, kappa,
                   rho, gamma, iters)


def sparse_logistic(m=200000, n=5000, nnz=50, corr=0.3, noise=0.5, N=16, M=8, kappa=50,
                    rho=0.5, gamma=10.0, iters=200, seed=0, dtype=np.float32,
                    rows=None) -> Problem:
    """Sparse logistic regression: A with Toeplitz column correlation corr^|i-j|, x* with
    nnz N(0,1) entries, labels y = sign(A x* + N(0, noise^2)) in {-1,+1}.  Defaults are the
    200000 x 5000 FP32 workload (N=16 shards, M=8 blocks, kappa=50, rho=0.5).

    rows=(r0, r1) generates only that row range (e.g. one shard) of the same matrix.
    A is returned in ``dtype`` (the labels are computed from the FP64 rows before rounding).
    """
    r0, r1 = (0, m) if rows is None else rows
    x_star = planted_support(n, nnz, seed, "normal")
    chunk = 2500
    A = np.empty((r1 - r0, n), dtype=dtype)
    b = np.empty(r1 - r0)
    supp = np.flatnonzero(x_star)
    r = r0
    while r < r1:
        c = min(r1, (r // chunk + 1) * chunk)
        blk = toeplitz_rows(c - r, n, seed, corr=corr, row0=r, chunk_rows=chunk)
        b[r - r0:c - r0] = _sign_pm1(blk[:, supp] @ x_star[supp] + noise * _noise(c - r, seed, row0=r))
        A[r - r0:c - r0] = blk
        r = c
    return Problem("sparse_logistic_%dx%d" % (m, n), A, b, x_star, LOSS_LOGISTIC, N, M, kappa,
                   rho, gamma, iters)


def table1_sls(m=100000, n=2000, sparsity=0.9, noise=0.01, N=4, M=4, rho=1.0, gamma=10.0,
               seed=0) -> Problem:
    """The paper's timing experiment (Sec. 4, Table 1): sparse least squares over N = 4 nodes
    of m/N rows, A_i i.i.d. N(0,1) with unit-norm columns per node, x_true with
    kappa = round(n (1 - sparsity)) nonzeros (+/-U[1,2] here; the paper does not say), and
    b = A x_true + e with e ~ N(0, noise^2) (the paper leaves Sigma unstated)."""
    kappa = int(round(n * (1.0 - sparsity)))
    P = sparse_linear(m=m, n=n, nnz=kappa, noise=noise, N=N, M=M, kappa=kappa, rho=rho,
                      gamma=gamma, seed=seed, unit_columns="shard")
    P.name = "sls_table1_%dx%d_s%.1f" % (m, n, sparsity)
    return P


def sparse_sqhinge(m=4000, n=400, nnz=12, noise=0.1, N=4, M=2, kappa=12, rho=1.0,
                   gamma=10.0, iters=200, seed=0) -> Problem:
    """Sparse squared-hinge SVM: A i.i.d. N(0,1), x* +/-U[1,2] on nnz random indices,
    labels sign(A x* + N(0, noise^2))."""
    A = gaussian_rows(m, n, seed)
    x_star = planted_support(n, nnz, seed, "pm_uniform12")
    b = _sign_pm1(A @ x_star + noise * _noise(m, seed))
    return Problem("sparse_sqhinge_%dx%d" % (m, n), A, b, x_star, LOSS_SQHINGE, N, M, kappa,
                   rho, gamma, iters)


def _gumbel(m: int, K: int, seed: int, row0: int = 0, chunk_rows: int = 4096) -> np.ndarray:
    """Standard Gumbel(0, 1) draws for rows [row0, row0+m), K per row (chunked like A)."""
    out = np.empty((m, K))
    r = row0
    while r < row0 + m:
        c = r // chunk_rows
        c0, c1 = c * chunk_rows, (c + 1) * chunk_rows
        u = _rng(seed, 4, c).random((chunk_rows, K))
        lo, hi = max(r, c0), min(row0 + m, c1)
        out[lo - row0:hi - row0] = -np.log(-np.log(u[lo - c0:hi - c0] + 1e-300))
        r = hi
    return out


def planted_matrix(n: int, K: int, nnz: int, seed: int) -> np.ndarray:
    """W* (n x K, returned flattened feature-major) with nnz N(0,1) entries at uniformly
    random positions among the n*K entries."""
    g = _rng(seed, 5)
    w = np.zeros(n * K)
    idx = g.choice(n * K, size=nnz, replace=False)
    w[idx] = g.standard_normal(nnz)
    return w


def sparse_softmax(m=500000, n=2000, K=10, nnz=500, N=32, M=4, kappa=500, rho=1.0,
                   gamma=10.0, iters=200, seed=0, dtype=np.float32, rows=None,
                   scale=1.0) -> Problem:
    """Sparse softmax regression: A i.i.d. N(0,1) (times ``scale``), W* (n x K) with nnz
    N(0,1) entries at uniformly random positions, labels y_r = argmax_k (a_r W* + G_rk)
    with G standard Gumbel noise (so y is a draw from softmax(a_r W*)).  Labels are class
    indices 0..K-1 stored as floats.  Defaults are the 500000 x 2000, K = 10 workload
    (N = 32 shards, M = 4 blocks, entrywise kappa = 500).  rows=(r0, r1) generates only that
    row range of the same matrix; A is returned in ``dtype``."""
    r0, r1 = (0, m) if rows is None else rows
    W = planted_matrix(n, K, nnz, seed).reshape(n, K)
    A = np.empty((r1 - r0, n), dtype=dtype)
    b = np.empty(r1 - r0)
    chunk = 4096
    r = r0
    while r < r1:
        c = min(r1, (r // chunk + 1) * chunk)
        blk = gaussian_rows(c - r, n, seed, row0=r, chunk_rows=chunk) * scale
        b[r - r0:c - r0] = np.argmax(blk @ W + _gumbel(c - r, K, seed, row0=r, chunk_rows=chunk), axis=1)
        A[r - r0:c - r0] = blk
        r = c
    return Problem("sparse_softmax_%dx%dx%d" % (m, n, K), A, b, W.reshape(-1), LOSS_SOFTMAX,
                   N, M, kappa, rho, gamma, iters, K)


def small_problem(loss: int, m: int, n: int, nnz: int, N: int, M: int, kappa: int,
                  rho: float = 1.0, gamma: float = 10.0, seed: int = 0, noise: float = 0.1,
                  corr: float = 0.0) -> Problem:
    """Small instance of any K=1 loss, for parity and pin tests (ragged shapes welcome)."""
    A = toeplitz_rows(m, n, seed, corr=corr) if corr else gaussian_rows(m, n, seed)
    x_star = planted_support(n, nnz, seed, "pm_uniform12")
    lin = A @ x_star + noise * _noise(m, seed)
    b = lin if loss == LOSS_SQUARED else _sign_pm1(lin)
    return Problem("small_%d_%dx%d" % (loss, m, n), A, b, x_star, loss, N, M, kappa, rho,
                   gamma, 0)


def batch_instance_specs(count=256, seed=0, m_range=(1000, 50000), n_range=(100, 4000),
                         block_cols=512):
    """Shapes of a batch of uneven instances: m and n log-uniform in their ranges, kappa
    uniform in 1..5 % of n (at least 1), N uniform in 4..16 shards (at most m), M such that
    blocks have at most `block_cols` columns, loss alternating squared / squared hinge."""
    g = _rng(seed, 7)
    specs = []
    for k in range(count):
        m = int(round(math.exp(g.uniform(math.log(m_range[0]), math.log(m_range[1])))))
        n = int(round(math.exp(g.uniform(math.log(n_range[0]), math.log(n_range[1])))))
        kappa = max(1, int(round(n * g.uniform(0.01, 0.05))))
        N = min(m, int(g.integers(4, 17)))
        M = max(1, -(-n // block_cols))
        loss = LOSS_SQUARED if k % 2 == 0 else LOSS_SQHINGE
        specs.append(dict(m=m, n=n, kappa=kappa, N=N, M=M, loss=loss, seed=seed * 100003 + k))
    return specs


def batch_instance(spec, noise=0.1, dtype=np.float32) -> Problem:
    """One instance of a batch: A i.i.d. N(0,1), x* +/-U[1,2] on kappa random indices,
    b = A x* + N(0, noise^2) (squared) or its sign (squared hinge)."""
    m, n, kappa, seed = spec["m"], spec["n"], spec["kappa"], spec["seed"]
    A = gaussian_rows(m, n, seed)
    x_star = planted_support(n, kappa, seed, "pm_uniform12")
    supp = np.flatnonzero(x_star)
    lin = A[:, supp] @ x_star[supp] + noise * _noise(m, seed)
    b = lin if spec["loss"] == LOSS_SQUARED else _sign_pm1(lin)
    return Problem("batch_%d_%dx%d" % (spec["loss"], m, n), A.astype(dtype), b, x_star,
                   spec["loss"], spec["N"], spec["M"], kappa, 1.0, 10.0, 0)


def serve_request_specs(count=64, seed=0, rate=200.0, m_range=(1000, 200000),
                        n_range=(100, 10000), block_cols=512):
    """A Poisson stream of solve requests: gaps Exp(rate); m and n log-uniform in their
    ranges; kappa uniform in 1..5 % of n; N uniform in 4..16 shards; M such that blocks have
    at most `block_cols` columns; loss cycling squared / logistic / squared hinge."""
    g = _rng(seed, 8)
    t, specs = 0.0, []
    losses = (LOSS_SQUARED, LOSS_LOGISTIC, LOSS_SQHINGE)
    for k in range(count):
        t += float(g.exponential(1.0 / rate))
        m = int(round(math.exp(g.uniform(math.log(m_range[0]), math.log(m_range[1])))))
        n = int(round(math.exp(g.uniform(math.log(n_range[0]), math.log(n_range[1])))))
        kappa = max(1, int(round(n * g.uniform(0.01, 0.05))))
        N = min(m, int(g.integers(4, 17)))
        specs.append(dict(arrival=t, m=m, n=n, kappa=kappa, N=N, M=max(1, -(-n // block_cols)),
                          loss=losses[k % 3], seed=seed * 1000003 + k))
    return specs


def device_request(spec, device="cuda", noise=0.1):
    """A request's data drawn on the device (torch's seeded CUDA generator): A i.i.d. N(0,1)
    FP32, x* with kappa entries +/-U[1,2], b = A x* + N(0, noise^2) or its sign."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(spec["seed"]))
    m, n, kappa = spec["m"], spec["n"], spec["kappa"]
    A = torch.randn(m, n, generator=g, device=device, dtype=torch.float32)
    idx = torch.randperm(n, generator=g, device=device)[:kappa]
    mag = 1.0 + torch.rand(kappa, generator=g, device=device, dtype=torch.float32)
    sgn = torch.where(torch.rand(kappa, generator=g, device=device) < 0.5, -1.0, 1.0)
    lin = A[:, idx] @ (mag * sgn) + noise * torch.randn(m, generator=g, device=device)
    b = lin if spec["loss"] == LOSS_SQUARED else torch.where(lin >= 0, 1.0, -1.0)
    return A, b.double()


def round_to_f32(A: np.ndarray) -> np.ndarray:
    """FP32-rounded copy of A upcast back to FP64 (the exact values an FP32 run sees)."""
    return A.astype(np.float32).astype(np.float64)


def round_to_bf16(A: np.ndarray) -> np.ndarray:
    """BF16-rounded copy of A (round to nearest, ties to even, from the FP32 value) upcast
    back to FP64: the exact values a BF16-storage run sees when given FP32 or FP64 input."""
    f = np.ascontiguousarray(A, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def round_to_tf32(A: np.ndarray) -> np.ndarray:
    """TF32-rounded copy of A (10 mantissa bits; round to nearest, ties to even, from the
    FP32 value) upcast back to FP64: the exact values a TF32-storage run sees."""
    f = np.ascontiguousarray(A, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 13) & 1
    r = ((u + 0xFFF + lsb) >> 13) << 13
    return (r & 0xFFFFFFFF).astype(np.uint32).view(np.float32).astype(np.float64)
