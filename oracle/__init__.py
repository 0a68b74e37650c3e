"""FP64 CPU oracle for the logistic-GLM log-posterior and gradient.

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
benchmark's ``cpu_baseline`` / ``--impl reference`` legs may import this
package; the library under ``paper_1310_1537_gb300`` never does. The oracle
shares no code with the CUDA path. The GLM arithmetic lives in
``glm_oracle.c`` (plain single-threaded C, FP64), which this module compiles
with gcc and calls through ctypes; the slice sampler, the Ising sampler and
the Hessian are plain NumPy FP64 below.

Functions and the passages they follow:

* ``logpost_grad``         — §3.1.1 log-likelihood (eq-loglike-binlogit),
  §4.2 gradient (eq-grad-expanded / eq-grad-compact), Gaussian prior N(0, s^2 I).
* ``loglik_partial``       — the same likelihood sums over a row range (the
  per-worker partials that the §4.2.2 reduction combines).
* ``logpost_grad_grouped`` — §4.1 hierarchical GLM, per-group L_m with prior
  N(mu, tau^2 I).
* ``rwm``                  — random-walk Metropolis consumer of the
  log-posterior (§2.2, §3.4.4); FP32 state, FP64 acceptance.
* ``bf16_from_f32``, ``quantize_e4m3``, ``e4m3_value`` — reduced-precision
  storage of X (bfloat16 RNE; OCP E4M3 with power-of-two column scales).
* ``slice_step``, ``slice_gibbs`` — Gibbs sweeps of univariate slice sampling
  over the coefficients (§3.4.4), evaluated with the plain log-posterior.
* ``logpost_grad_hess``    — f, g and the Hessian of the log-posterior
  (§4.2's derivatives taken one order further, as §5.2 proposes):
  H = -X^T diag(s(1 - s)) X - I / sigma^2 (NumPy, FP64).
* ``ising_half_sweep``, ``ising_gibbs``, ``ising_energy``,
  ``ising_to_plane``, ``ising_from_planes`` — checkerboard Gibbs sampling of
  the square-lattice Ising model (§4.3.1) in the natural row-major layout
  (NumPy, FP64); the colour planes only index the uniforms.

``hls_logpost_grad`` is not part of the oracle: it is the multi-core FP64 CPU
baseline the benchmark times (``cpu_hls.c``, the paper's own CPU design
restated with OpenMP), checked against ``logpost_grad`` by the tests.

Every function is pinned by ``tests/test_oracle_pins.py`` against closed
forms, extended-precision brute force, finite differences, symmetries,
library routines and quadrature.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "glm_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile glm_oracle.c into liboracle.so with gcc (-O2, no fast-math)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_HLS_SRC = os.path.join(_HERE, "cpu_hls.c")
_HLS_PATH = os.path.join(_HERE, "libcpu_hls.so")
_hls = None


def build_hls(force: bool = False) -> str:
    """Compile cpu_hls.c (the multi-core FP64 CPU baseline) with gcc -fopenmp."""
    if (not force and os.path.exists(_HLS_PATH)
            and os.path.getmtime(_HLS_PATH) >= os.path.getmtime(_HLS_SRC)):
        return _HLS_PATH
    tmp = _HLS_PATH + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O3", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-o", tmp, _HLS_SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _HLS_PATH)
    return _HLS_PATH


def _load_hls():
    global _hls
    with _lock:
        if _hls is not None:
            return _hls
        lib = C.CDLL(build_hls())
        dp = C.POINTER(C.c_double)
        lib.hls_logpost_grad.argtypes = [dp, C.c_int64, C.c_int32, C.c_int64,
                                         C.POINTER(C.c_uint8), dp, C.c_int32, C.c_double,
                                         C.c_int32, dp, dp]
        lib.hls_logpost_grad.restype = C.c_int
        lib.hls_max_threads.argtypes = []
        lib.hls_max_threads.restype = C.c_int
        _hls = lib
        return lib


def hls_max_threads() -> int:
    """Processors OpenMP sees on this host."""
    return int(_load_hls().hls_max_threads())


def hls_logpost_grad(X, y, beta, prior_sigma=10.0, p=None, threads=None):
    """The multi-core CPU baseline (``cpu_hls.c``: the paper's partial loop
    fusion, cache fusion and one combine per thread, FP64, OpenMP). Same
    arguments and results as ``logpost_grad``; not the oracle."""
    Xd = _f64_matrix(X)
    n, ld = Xd.shape
    b = np.ascontiguousarray(np.atleast_2d(beta), dtype=np.float64)
    k, pp = b.shape
    P = pp if p is None else int(p)
    if P != pp or P > ld:
        raise ValueError("beta width must equal P <= ld")
    yy = np.ascontiguousarray(y, dtype=np.uint8)
    if yy.shape[0] != n:
        raise ValueError("y length must equal N")
    nt = hls_max_threads() if threads is None else int(threads)
    f = np.empty(k, dtype=np.float64)
    g = np.empty((k, P), dtype=np.float64)
    rc = _load_hls().hls_logpost_grad(_p(Xd, C.c_double), n, P, ld, _p(yy, C.c_uint8),
                                      _p(b, C.c_double), k, float(prior_sigma), nt,
                                      _p(f, C.c_double), _p(g, C.c_double))
    if rc != 0:
        raise ValueError("hls_logpost_grad failed")
    return f, g


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = C.CDLL(build())
        dp = C.POINTER(C.c_double)
        fp = C.POINTER(C.c_float)
        u8 = C.POINTER(C.c_uint8)
        u16 = C.POINTER(C.c_uint16)
        i64p = C.POINTER(C.c_int64)
        lib.oracle_logpost_grad.argtypes = [dp, C.c_int64, C.c_int32, C.c_int64, u8, dp,
                                            C.c_int32, C.c_double, dp, dp]
        lib.oracle_loglik_partial.argtypes = [dp, C.c_int64, C.c_int64, C.c_int32, C.c_int64,
                                              u8, dp, C.c_int32, dp, dp]
        lib.oracle_logpost_grad_grouped.argtypes = [dp, C.c_int32, C.c_int64, u8, i64p,
                                                    C.c_int32, dp, dp, C.c_double, dp, dp]
        lib.oracle_rwm.argtypes = [dp, C.c_int64, C.c_int32, C.c_int64, u8, C.c_double,
                                   C.c_int32, C.c_int32, C.c_float, fp, dp, fp, dp,
                                   C.c_int32, fp, u8, dp, dp]
        lib.oracle_bf16_from_f32.argtypes = [fp, C.c_int64, u16]
        lib.oracle_bf16_from_f32.restype = None
        lib.oracle_bf16_to_f64.argtypes = [u16, C.c_int64, dp]
        lib.oracle_bf16_to_f64.restype = None
        lib.oracle_e4m3_value.argtypes = [C.c_uint8]
        lib.oracle_e4m3_value.restype = C.c_double
        lib.oracle_e4m3_from_f64.argtypes = [C.c_double]
        lib.oracle_e4m3_from_f64.restype = C.c_uint8
        lib.oracle_e4m3_column_scale.argtypes = [C.c_double]
        lib.oracle_e4m3_column_scale.restype = C.c_double
        lib.oracle_quantize_e4m3.argtypes = [fp, C.c_int64, C.c_int32, C.c_int64, u8,
                                             C.c_int64, fp]
        for name in ("oracle_logpost_grad", "oracle_loglik_partial",
                     "oracle_logpost_grad_grouped", "oracle_rwm", "oracle_quantize_e4m3"):
            getattr(lib, name).restype = C.c_int
        _lib = lib
        return lib


def _p(a, ctype):
    return a.ctypes.data_as(C.POINTER(ctype))


def _f64_matrix(X):
    X = np.asarray(X)
    if X.ndim != 2:
        raise ValueError("X must be 2-D (N x ld)")
    return np.ascontiguousarray(X, dtype=np.float64)


def logpost_grad(X, y, beta, prior_sigma=10.0, p=None):
    """f (K,) and g (K, P) of the Bayesian logistic log-posterior, FP64.

    X: N x ld (first ``p`` columns used, default all); y: N uint8 in {0,1};
    beta: (P,) or (K, P).
    """
    Xd = _f64_matrix(X)
    n, ld = Xd.shape
    b = np.ascontiguousarray(np.atleast_2d(beta), dtype=np.float64)
    k, pp = b.shape
    P = pp if p is None else int(p)
    if P != pp or P > ld:
        raise ValueError("beta width must equal P <= ld")
    yy = np.ascontiguousarray(y, dtype=np.uint8)
    if yy.shape[0] != n:
        raise ValueError("y length must equal N")
    f = np.empty(k, dtype=np.float64)
    g = np.empty((k, P), dtype=np.float64)
    rc = _load().oracle_logpost_grad(_p(Xd, C.c_double), n, P, ld, _p(yy, C.c_uint8),
                                     _p(b, C.c_double), k, float(prior_sigma),
                                     _p(f, C.c_double), _p(g, C.c_double))
    if rc != 0:
        raise ValueError("oracle_logpost_grad rejected its arguments")
    return f, g


def loglik_partial(X, y, beta, r0, r1, p=None):
    """Likelihood-only sums (no prior) over rows [r0, r1)."""
    Xd = _f64_matrix(X)
    n, ld = Xd.shape
    b = np.ascontiguousarray(np.atleast_2d(beta), dtype=np.float64)
    k, P = b.shape
    yy = np.ascontiguousarray(y, dtype=np.uint8)
    if not (0 <= r0 <= r1 <= n):
        raise ValueError("bad row range")
    f = np.empty(k, dtype=np.float64)
    g = np.empty((k, P), dtype=np.float64)
    rc = _load().oracle_loglik_partial(_p(Xd, C.c_double), int(r0), int(r1), P, ld,
                                       _p(yy, C.c_uint8), _p(b, C.c_double), k,
                                       _p(f, C.c_double), _p(g, C.c_double))
    if rc != 0:
        raise ValueError("oracle_loglik_partial rejected its arguments")
    return f, g


def logpost_grad_grouped(X, y, offsets, beta, mu, tau):
    """Per-group f (G,) and g (G, P) of the hierarchical logistic GLM."""
    Xd = _f64_matrix(X)
    n, ld = Xd.shape
    b = np.ascontiguousarray(beta, dtype=np.float64)
    G, P = b.shape
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    if off.shape[0] != G + 1 or off[0] < 0 or off[-1] > n:
        raise ValueError("offsets must have G+1 entries within [0, N]")
    m = np.ascontiguousarray(mu, dtype=np.float64)
    yy = np.ascontiguousarray(y, dtype=np.uint8)
    f = np.empty(G, dtype=np.float64)
    g = np.empty((G, P), dtype=np.float64)
    rc = _load().oracle_logpost_grad_grouped(_p(Xd, C.c_double), P, ld, _p(yy, C.c_uint8),
                                             _p(off, C.c_int64), G, _p(b, C.c_double),
                                             _p(m, C.c_double), float(tau),
                                             _p(f, C.c_double), _p(g, C.c_double))
    if rc != 0:
        raise ValueError("oracle_logpost_grad_grouped rejected its arguments")
    return f, g


def rwm(X, y, beta0, z, log_u, step, prior_sigma=10.0, p=None):
    """Run K random-walk Metropolis chains for z.shape[0] steps.

    beta0: (K, P) float32 start; z: (T, K, P) float32; log_u: (T, K) float64.
    Returns dict(samples (T,K,P) f32, accept (T,K) u8, logpost (T,K),
    log_alpha (T,K), beta (K,P) final, f (K,) final, f0 (K,) initial).
    """
    Xd = _f64_matrix(X)
    n, ld = Xd.shape
    state = np.array(np.atleast_2d(beta0), dtype=np.float32, order="C")
    k, P = state.shape
    zz = np.ascontiguousarray(z, dtype=np.float32)
    lu = np.ascontiguousarray(log_u, dtype=np.float64)
    T = zz.shape[0]
    if zz.shape != (T, k, P) or lu.shape != (T, k):
        raise ValueError("z must be (T,K,P) and log_u (T,K)")
    yy = np.ascontiguousarray(y, dtype=np.uint8)
    fs = np.zeros(k, dtype=np.float64)
    samples = np.empty((T, k, P), dtype=np.float32)
    acc = np.empty((T, k), dtype=np.uint8)
    lp = np.empty((T, k), dtype=np.float64)
    la = np.empty((T, k), dtype=np.float64)
    lib = _load()
    # initial log-posterior
    rc = lib.oracle_rwm(_p(Xd, C.c_double), n, P, ld, _p(yy, C.c_uint8), float(prior_sigma),
                        k, 0, C.c_float(step), _p(zz, C.c_float), _p(lu, C.c_double),
                        _p(state, C.c_float), _p(fs, C.c_double), 1, None, None, None, None)
    if rc != 0:
        raise ValueError("oracle_rwm rejected its arguments")
    f0 = fs.copy()
    rc = lib.oracle_rwm(_p(Xd, C.c_double), n, P, ld, _p(yy, C.c_uint8), float(prior_sigma),
                        k, T, C.c_float(step), _p(zz, C.c_float), _p(lu, C.c_double),
                        _p(state, C.c_float), _p(fs, C.c_double), 0, _p(samples, C.c_float),
                        _p(acc, C.c_uint8), _p(lp, C.c_double), _p(la, C.c_double))
    if rc != 0:
        raise ValueError("oracle_rwm rejected its arguments")
    return {"samples": samples, "accept": acc, "logpost": lp, "log_alpha": la,
            "beta": state, "f": fs, "f0": f0}


def bf16_from_f32(x):
    """uint16 bit patterns of the nearest-even bfloat16 values of float32 ``x``."""
    a = np.ascontiguousarray(x, dtype=np.float32)
    out = np.empty(a.shape, dtype=np.uint16)
    _load().oracle_bf16_from_f32(_p(a, C.c_float), a.size, _p(out, C.c_uint16))
    return out


def bf16_to_f64(bits):
    b = np.ascontiguousarray(bits, dtype=np.uint16)
    out = np.empty(b.shape, dtype=np.float64)
    _load().oracle_bf16_to_f64(_p(b, C.c_uint16), b.size, _p(out, C.c_double))
    return out


def e4m3_value(code: int) -> float:
    return _load().oracle_e4m3_value(int(code) & 0xFF)


def e4m3_from_f64(v: float) -> int:
    return int(_load().oracle_e4m3_from_f64(float(v)))


def e4m3_column_scale(amax: float) -> float:
    return _load().oracle_e4m3_column_scale(float(amax))


def e4m3_decode(codes):
    """float64 values of an array of E4M3 codes (by the format definition)."""
    table = np.array([e4m3_value(c) for c in range(256)], dtype=np.float64)
    return table[np.asarray(codes, dtype=np.uint8)]


def quantize_e4m3(X32, p=None, ld_q=None):
    """(Q uint8 N x ld_q, scale float32 P) from float32 X (N x ld)."""
    a = np.ascontiguousarray(X32, dtype=np.float32)
    n, ld = a.shape
    P = ld if p is None else int(p)
    lq = P if ld_q is None else int(ld_q)
    Q = np.empty((n, lq), dtype=np.uint8)
    s = np.empty(P, dtype=np.float32)
    rc = _load().oracle_quantize_e4m3(_p(a, C.c_float), n, P, ld, _p(Q, C.c_uint8), lq,
                                      _p(s, C.c_float))
    if rc != 0:
        raise ValueError("oracle_quantize_e4m3 rejected its arguments")
    return Q, s


def dequantize_e4m3(Q, scale, p=None):
    """FP64 values q * s_j of an E4M3 matrix (first P columns), exactly."""
    P = len(scale) if p is None else int(p)
    v = e4m3_decode(Q[:, :P])
    return v * np.asarray(scale, dtype=np.float64)[None, :P]


# ---------------------------------------------------------------------------
# Univariate slice sampling (Neal 2003: stepping out, then shrinkage) inside
# Gibbs sweeps over the coefficients, §3.4.4. The oracle evaluates every
# point with the plain definition of the log-posterior (logpost_grad); it
# does not use the differential update.
#
# Interval arithmetic is FP32 with each operation rounded separately (the
# coefficients are FP32 state): L0 = x0 - w*U, R0 = L0 + w,
# L_j = L0 - j*w, R_j = R0 + j*w, x1 = L + U*(R - L); J = floor(m*V) and
# K = m - 1 - J. The slice level is log y = g(x0) + log_u0 (FP64). After
# s_max rejected shrinkage proposals the coordinate keeps x0.

def slice_step(logdens, x0, g0, log_u0, uni, w, m, s_max):
    """One univariate slice-sampling update of a scalar.

    logdens(x: float32) -> float64 log density; x0 float32 with
    g0 = logdens(x0); uni = [U, V, shrink_0, ..., shrink_{s_max-1}] float32.
    Returns (x1, g1, n_shrink, n_evals, moved).
    """
    f32 = np.float32
    x0 = f32(x0)
    w = f32(w)
    log_y = float(g0) + float(log_u0)
    U, V = f32(uni[0]), f32(uni[1])
    L0 = f32(x0 - f32(w * U))
    R0 = f32(L0 + w)
    J = int(np.floor(f32(f32(m) * V)))
    K = (m - 1) - J
    evals = 0
    L = L0
    j = 0
    while J > 0:
        Lj = f32(L0 - f32(f32(j) * w))
        evals += 1
        if not log_y < logdens(Lj):
            L = Lj
            break
        j += 1
        J -= 1
        L = f32(L0 - f32(f32(j) * w))
    R = R0
    j = 0
    while K > 0:
        Rj = f32(R0 + f32(f32(j) * w))
        evals += 1
        if not log_y < logdens(Rj):
            R = Rj
            break
        j += 1
        K -= 1
        R = f32(R0 + f32(f32(j) * w))
    for t in range(s_max):
        x1 = f32(L + f32(f32(uni[2 + t]) * f32(R - L)))
        g1 = logdens(x1)
        evals += 1
        if log_y < g1:
            return x1, g1, t, evals, True
        if x1 < x0:
            L = x1
        else:
            R = x1
    return x0, float(g0), s_max, evals, False


def slice_gibbs(X, y, beta0, log_u0, uni, w, m, prior_sigma=10.0, p=None):
    """Gibbs sweeps of univariate slice sampling over beta (float32 state).

    log_u0 (S, P), uni (S, P, 2 + s_max) from synth.slice_streams.
    Returns dict(xk (S,P) f32: coordinate value after each update,
    gk (S,P) f64: log-posterior after each update, nshrink (S,P),
    evals (S,P), beta (P,) f32 final, f final, f0 initial).
    """
    Xd = _f64_matrix(X)
    P = Xd.shape[1] if p is None else int(p)
    beta = np.array(beta0, dtype=np.float32).reshape(P)
    S = log_u0.shape[0]
    s_max = uni.shape[2] - 2

    def f_of(b):
        f, _ = logpost_grad(Xd, y, b.astype(np.float64), prior_sigma=prior_sigma, p=P)
        return float(f[0])

    g = f_of(beta)
    f0 = g
    xk = np.empty((S, P), dtype=np.float32)
    gk = np.empty((S, P), dtype=np.float64)
    nsh = np.empty((S, P), dtype=np.int32)
    nev = np.empty((S, P), dtype=np.int32)
    for s in range(S):
        for k in range(P):
            def dens(x, k=k):
                b = beta.copy()
                b[k] = x
                return f_of(b)
            x1, g1, ns, ne, _ = slice_step(dens, beta[k], g, log_u0[s, k], uni[s, k], w, m,
                                           s_max)
            beta[k] = x1
            g = g1
            xk[s, k] = x1
            gk[s, k] = g1
            nsh[s, k] = ns
            nev[s, k] = ne
    return {"xk": xk, "gk": gk, "nshrink": nsh, "evals": nev, "beta": beta, "f": g, "f0": f0}


# ---------------------------------------------------------------------------
# Square-lattice Ising model, checkerboard Gibbs sampling (§4.3.1).
#
# Spins s_i in {0, 1} on an R x C lattice (C even), each interacting with its
# 4 lattice neighbours; free boundary (a missing neighbour contributes
# nothing). The Gibbs conditional is P(s_i = 1 | rest) = 1 / (1 + exp(-z_i)),
# z_i = b_i + w * sum_j s_j over the neighbours j of i (the paper's
# eq-ising-p); the energy consistent with it is
# E(s) = -sum_i b_i s_i - w * sum_<ij> s_i s_j, P(s) proportional to exp(-E).
# Colour c holds the sites with (row + col) % 2 == c; the two colours are
# updated in turn, each site i of the colour set to 1 iff u_i < P(s_i = 1).
# Colour plane c lists colour c's sites row by row: plane entry (r, j) is the
# site (r, 2j + ((r + c) % 2)).


def ising_to_plane(a, color):
    """Colour plane `color` of a natural-layout R x C array: (R, C // 2)."""
    a = np.asarray(a)
    R, C = a.shape
    out = np.empty((R, C // 2), dtype=a.dtype)
    for r in range(R):
        start = (r + color) % 2
        out[r] = a[r, start::2]
    return out


def ising_from_planes(p0, p1):
    """Natural R x C array from its two colour planes."""
    p0 = np.asarray(p0)
    p1 = np.asarray(p1)
    R, H = p0.shape
    out = np.empty((R, 2 * H), dtype=p0.dtype)
    for r in range(R):
        out[r, (r + 0) % 2::2] = p0[r]
        out[r, (r + 1) % 2::2] = p1[r]
    return out


def ising_energy(s, b, w):
    """E(s) = -sum_i b_i s_i - w sum over lattice edges of s_i s_j (FP64)."""
    sf = np.asarray(s, dtype=np.float64)
    bf = np.asarray(b, dtype=np.float64)
    pairs = (sf[1:, :] * sf[:-1, :]).sum() + (sf[:, 1:] * sf[:, :-1]).sum()
    return float(-(bf * sf).sum() - float(w) * pairs)


def ising_half_sweep(s, b, w, color, u_plane):
    """Update every site of colour `color` from its conditional.

    s (R, C) uint8 spins, b (R, C) biases, w the coupling, u_plane (R, C // 2)
    the colour's uniforms in plane order. Returns (new spins, P(s_i = 1) of
    every site as computed here, in the natural layout)."""
    s = np.asarray(s, dtype=np.uint8)
    R, C = s.shape
    sf = s.astype(np.float64)
    n = np.zeros((R, C))
    n[1:, :] += sf[:-1, :]          # neighbour above
    n[:-1, :] += sf[1:, :]          # below
    n[:, 1:] += sf[:, :-1]          # left
    n[:, :-1] += sf[:, 1:]          # right
    z = np.asarray(b, dtype=np.float64) + float(w) * n
    with np.errstate(over="ignore"):
        p = 1.0 / (1.0 + np.exp(-z))
    u = np.zeros((R, C))
    for r in range(R):
        u[r, (r + color) % 2::2] = np.asarray(u_plane[r], dtype=np.float64)
    rr, cc = np.indices((R, C))
    mask = ((rr + cc) % 2) == color
    out = s.copy()
    out[mask] = (u < p)[mask].astype(np.uint8)
    return out, p


def ising_gibbs(s0, b, w, u):
    """n sweeps (colour 0 then colour 1 each) from s0 with uniforms u of
    shape (n, 2, R, C // 2). Returns the final spins and the number of
    spins equal to 1 after every half-sweep, shape (n, 2)."""
    s = np.asarray(s0, dtype=np.uint8).copy()
    n = u.shape[0]
    ones = np.zeros((n, 2), dtype=np.int64)
    for t in range(n):
        for c in range(2):
            s, _ = ising_half_sweep(s, b, w, c, u[t, c])
            ones[t, c] = int(s.sum(dtype=np.int64))
    return s, ones


# ---------------------------------------------------------------------------
# Hessian of the Bayesian logistic log-posterior (§4.2 differentiated once
# more; §5.2 names the Hessian as the next derivative to parallelise).
# With mu_n = 1 / (1 + exp(-x_n . beta)): d^2 f / d beta d beta^T =
# -sum_n mu_n (1 - mu_n) x_n x_n^T - I / sigma^2.


def logpost_grad_hess(X, y, beta, prior_sigma=10.0, p=None):
    """f (float), g (P,), H (P, P) of the log-posterior at one beta, FP64.
    f and g are the plain-definition values of ``logpost_grad``."""
    X = np.asarray(X, dtype=np.float64)
    if p is not None:
        X = X[:, :p]
    P = X.shape[1]
    b = np.asarray(beta, dtype=np.float64).reshape(P)
    f, g = logpost_grad(X, y, b[None, :], prior_sigma=prior_sigma)
    eta = X @ b
    with np.errstate(over="ignore"):
        mu = 1.0 / (1.0 + np.exp(-eta))
    w = mu * (1.0 - mu)
    H = -(X.T @ (w[:, None] * X)) - np.eye(P) / (prior_sigma * prior_sigma)
    return float(f[0]), g[0], H
