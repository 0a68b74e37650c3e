"""Seeded synthetic inputs for the logistic-GLM log-posterior workloads.

This module is shared by the CPU oracle's tests and by the GPU path's tests,
smoke check and benchmark. It only draws random inputs and lays them out in
memory; it holds none of the method's arithmetic (no log-likelihood, softplus,
sigmoid, residual, gradient or prior term).

Labels are drawn from the logistic model through its latent-variable form:
y_i = 1[x_i . beta* + e_i > 0] with e_i ~ Logistic(0, 1) (inverse-CDF draw),
which has P(y_i = 1) = 1 / (1 + exp(-x_i . beta*)) — the Bernoulli-logistic
response of the paper's running example (§3.1.1) — without evaluating that
probability here.

Workload shapes (the paper's "big-data GLM" regime of §3.3.1 and the HB
extension of §4.1, at the sizes this library is measured on):

* ``small``   N=10,000,  P=50,  FP64 X, K=1 (plus 100 evaluation points, RWM)
* ``big``     N=2,000,000, P=100, FP32 X, K=1
* ``batched`` N=1,000,000, P=256, K=64 chains, X stored BF16 / FP8 E4M3
* ``hb``      G=4,000 groups, log-normal sizes (median 400, [20, 50000]), P=32
* ``serve``   16 datasets, N log-uniform [1e3, 4e6], P log-uniform [8, 512]
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 20131537


def seed_for(index: int) -> int:
    """Seed of workload number ``index`` (0 small, 1 big, 2 batched, 3 hb, 4 serve)."""
    return SEED_BASE + int(index)


def padded_ld(p: int, elem_bytes: int) -> int:
    """Smallest row stride >= p whose byte size is a multiple of 16."""
    per = 16 // elem_bytes
    return ((p + per - 1) // per) * per


def pad_columns(x: np.ndarray, ld: int) -> np.ndarray:
    """Copy an N x P matrix into an N x ld row-major array with zero padding."""
    n, p = x.shape
    if ld == p:
        return np.ascontiguousarray(x)
    out = np.zeros((n, ld), dtype=x.dtype)
    out[:, :p] = x
    return out


def design_matrix(rng: np.random.Generator, n: int, p: int, dtype=np.float64,
                  intercept: bool = True, chunk_rows: int = 1 << 18) -> np.ndarray:
    """i.i.d. N(0,1) entries, column 0 set to 1 when ``intercept``."""
    x = np.empty((n, p), dtype=dtype)
    for r0 in range(0, n, chunk_rows):
        r1 = min(n, r0 + chunk_rows)
        x[r0:r1] = rng.standard_normal((r1 - r0, p), dtype=np.float64 if dtype == np.float64 else np.float32)
    if intercept and p > 0:
        x[:, 0] = 1
    return x


def logistic_labels(rng: np.random.Generator, x: np.ndarray, beta_star: np.ndarray,
                    chunk_rows: int = 1 << 18) -> np.ndarray:
    """Bernoulli-logistic labels via the latent form y = 1[x.beta* + e > 0], e ~ Logistic(0,1)."""
    n = x.shape[0]
    y = np.empty(n, dtype=np.uint8)
    bs = np.asarray(beta_star, dtype=np.float64)
    for r0 in range(0, n, chunk_rows):
        r1 = min(n, r0 + chunk_rows)
        lin = x[r0:r1].astype(np.float64) @ bs
        u = rng.random(r1 - r0)
        u = np.clip(u, 1e-300, None)
        e = np.log(u) - np.log1p(-u)          # inverse CDF of Logistic(0, 1)
        y[r0:r1] = (lin + e > 0).astype(np.uint8)
    return y


@dataclass
class GLMData:
    """One synthetic logistic-regression dataset (row-major X, N x P)."""
    X: np.ndarray
    y: np.ndarray
    beta_star: np.ndarray
    prior_sigma: float = 10.0
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return self.X.shape[0]

    @property
    def p(self) -> int:
        return self.X.shape[1]


def make_glm(n: int, p: int, seed: int, dtype=np.float64, intercept: bool = True,
             prior_sigma: float = 10.0) -> GLMData:
    """X ~ N(0,1) (+ intercept), beta* ~ N(0, 1/P), y ~ Bernoulli-logistic(X beta*)."""
    rng = np.random.default_rng(seed)
    x = design_matrix(rng, n, p, dtype=dtype, intercept=intercept)
    beta_star = rng.standard_normal(p) / math.sqrt(max(p, 1))
    y = logistic_labels(rng, x, beta_star)
    return GLMData(X=x, y=y, beta_star=beta_star, prior_sigma=prior_sigma,
                   meta={"seed": seed, "n": n, "p": p})


def eval_points(beta_star: np.ndarray, count: int, scale: float, seed: int) -> np.ndarray:
    """``count`` vectors drawn N(beta*, scale^2 I), shape (count, P), float64."""
    rng = np.random.default_rng(seed)
    p = beta_star.shape[0]
    return beta_star[None, :] + scale * rng.standard_normal((count, p))


def rwm_streams(n_steps: int, k: int, p: int, seed: int):
    """Proposal normals z (n_steps, K, P) float32 and log-uniforms (n_steps, K) float64.

    These are the random numbers a random-walk Metropolis chain consumes; both
    the oracle chain and the device chain read the same buffers.
    """
    rng = np.random.default_rng(seed)
    z = rng.standard_normal((n_steps, k, p), dtype=np.float32)
    u = rng.random((n_steps, k))
    u = np.clip(u, 1e-300, None)
    return z, np.log(u)


def slice_streams(n_sweeps: int, p: int, s_max: int, seed: int):
    """Random numbers of Gibbs sweeps with univariate slice sampling.

    log_u0 (n_sweeps, P) float64: log of the uniform that sets each slice
    level; uni (n_sweeps, P, 2 + s_max) float32: per coordinate update the
    interval-placement uniform, the stepping-out split uniform and s_max
    shrinkage uniforms, all in (0, 1). Both the oracle and the device read
    these buffers.
    """
    rng = np.random.default_rng(seed)
    u0 = rng.random((n_sweeps, p))
    u0 = np.where(u0 > 0.0, u0, 0.5)
    uni = rng.random((n_sweeps, p, 2 + s_max)).astype(np.float32)
    uni = np.where(uni > 0.0, uni, np.float32(0.5)).astype(np.float32)
    return np.log(u0), uni


def rwm_step_size(n: int, p: int) -> float:
    """Proposal scale 2.38/sqrt(P) * 1/sqrt(N/4) (Laplace-scale guess)."""
    return 2.38 / math.sqrt(p) / math.sqrt(max(n, 1) / 4.0)


@dataclass
class GroupedData:
    """Hierarchical GLM batch: groups are contiguous row ranges of one X."""
    X: np.ndarray
    y: np.ndarray
    offsets: np.ndarray      # int64, G+1
    beta: np.ndarray         # G x P evaluation points
    mu: np.ndarray           # P
    tau: float


def group_sizes(g: int, seed: int, median: float = 400.0, sigma_ln: float = 0.945,
                lo: int = 20, hi: int = 50000) -> np.ndarray:
    rng = np.random.default_rng(seed)
    z = rng.standard_normal(g)
    n = np.rint(np.exp(math.log(median) + sigma_ln * z)).astype(np.int64)
    return np.clip(n, lo, hi)


def make_grouped(g: int, p: int, seed: int, dtype=np.float32, tau: float = 0.5,
                 sizes: np.ndarray | None = None) -> GroupedData:
    """G groups with log-normal sizes; beta_g ~ N(mu, tau^2 I), mu ~ N(0, 1/P)."""
    if sizes is None:
        sizes = group_sizes(g, seed)
    sizes = np.asarray(sizes, dtype=np.int64)
    rng = np.random.default_rng(seed + 7919)
    offsets = np.zeros(g + 1, dtype=np.int64)
    offsets[1:] = np.cumsum(sizes)
    n = int(offsets[-1])
    x = design_matrix(rng, n, p, dtype=dtype, intercept=True)
    mu = rng.standard_normal(p) / math.sqrt(p)
    beta_true = mu[None, :] + tau * rng.standard_normal((g, p))
    y = np.empty(n, dtype=np.uint8)
    for gi in range(g):
        a, b = offsets[gi], offsets[gi + 1]
        if b > a:
            y[a:b] = logistic_labels(rng, x[a:b], beta_true[gi])
    beta_eval = mu[None, :] + tau * rng.standard_normal((g, p))
    return GroupedData(X=x, y=y, offsets=offsets, beta=beta_eval, mu=mu, tau=tau)


def serving_datasets(count: int, seed: int, n_lo: float = 1e3, n_hi: float = 4e6,
                     p_lo: float = 8, p_hi: float = 512):
    """(N, P) shapes for the serving stream, log-uniform in the given ranges."""
    rng = np.random.default_rng(seed)
    ns = np.exp(rng.uniform(math.log(n_lo), math.log(n_hi), count)).astype(np.int64)
    ps = np.exp(rng.uniform(math.log(p_lo), math.log(p_hi), count)).astype(np.int64)
    return [(int(a), int(b)) for a, b in zip(ns, ps)]


def poisson_arrivals(rate: float, count: int, seed: int) -> np.ndarray:
    """Arrival times (seconds) of a Poisson process with the given rate."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate, count))


def ising_lattice(rows: int, cols: int, seed: int, flip: float = 0.1, eta: float = 1.0,
                  w: float = 2.0):
    """A noisy binary image for Ising denoising (§4.3.1): a smooth two-tone
    pattern with a fraction `flip` of its pixels flipped at random, and the
    biases of the +-1 denoising model (data strength eta, coupling J = w / 4)
    written for {0, 1} spins: with sigma = 2s - 1, J sum sigma_i sigma_j +
    eta sum sigma_i y'_i equals w sum s_i s_j + sum b_i s_i + const for
    b_i = 2 eta y'_i - (w / 2) deg_i (y' = 2y - 1, deg_i the number of
    lattice neighbours). Returns (y (rows, cols) uint8 noisy image,
    b (rows, cols) float32, the clean image)."""
    rng = np.random.default_rng(seed)
    r = np.arange(rows, dtype=np.float32)[:, None]
    c = np.arange(cols, dtype=np.float32)[None, :]
    f1, f2, p1, p2 = rng.uniform(0.01, 0.05, 2).tolist() + rng.uniform(0.0, 6.28, 2).tolist()
    clean = ((np.sin(f1 * r + p1) * np.sin(f2 * c + p2)) > 0).astype(np.uint8)
    noise = rng.random((rows, cols), dtype=np.float32) < flip
    y = np.where(noise, 1 - clean, clean).astype(np.uint8)
    deg = np.full((rows, cols), 4.0, dtype=np.float32)
    deg[0, :] -= 1
    deg[-1, :] -= 1
    deg[:, 0] -= 1
    deg[:, -1] -= 1
    b = (np.float32(2.0 * eta) * (2.0 * y.astype(np.float32) - 1.0) -
         np.float32(w / 2.0) * deg).astype(np.float32)
    return y, b, clean


def ising_uniforms(n_sweeps: int, rows: int, cols: int, seed: int):
    """Batch of uniforms for n_sweeps checkerboard sweeps: (n_sweeps, 2,
    rows, cols // 2) float32 in [0, 1), colour-plane order. Both the oracle
    and the device read this buffer."""
    rng = np.random.default_rng(seed)
    return rng.random((n_sweeps, 2, rows, cols // 2), dtype=np.float32)
