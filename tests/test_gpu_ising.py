"""GPU parity of checkerboard Gibbs sampling of the square-lattice Ising
model (§4.3.1) against the FP64 oracle.

A spin is an integer decided by floating point (u < P(s_i = 1)): every device
spin must equal the oracle's decision from the device's own previous state,
except at a near tie |u - P| < 5e-6 (the device computes P in FP32 with the
hardware exponential). Plane splits and merges are bit-exact; counts of ones
are exact integers.
"""
import numpy as np
import pytest

import oracle
import synth
import paper_1310_1537_gb300 as glm
from tests.glmgpu import to_dev, torch

pytestmark = pytest.mark.gpu

TIE = 5e-6


def _planes(t, a):
    rows, cols = a.shape
    p0 = t.empty((rows, cols // 2), dtype=a.dtype, device="cuda")
    p1 = t.empty((rows, cols // 2), dtype=a.dtype, device="cuda")
    glm.glm_ising_split(a, a.element_size(), rows, cols, p0, p1)
    return p0, p1


def _natural(t, p0, p1, rows, cols):
    out = t.empty((rows, cols), dtype=p0.dtype, device="cuda")
    glm.glm_ising_merge(p0, p1, p0.element_size(), rows, cols, out)
    torch().cuda.synchronize()
    return out.cpu().numpy()


def _check_sweep(prev, nxt, b, w, u):
    """Device sweep prev -> nxt against the oracle, half by half from the
    device's own states. Returns the number of near-tie differences."""
    ties = 0
    mid = prev.copy()
    rows, cols = prev.shape
    rr, cc = np.indices((rows, cols))
    for c in (0, 1):
        want, p = oracle.ising_half_sweep(mid, b, w, c, u[c])
        mask = ((rr + cc) % 2) == c
        diff = mask & (want != nxt)
        if diff.any():
            for r, col in zip(*np.nonzero(diff)):
                uu = float(u[c][r, col // 2])
                assert abs(uu - p[r, col]) < TIE, (c, r, col, uu, p[r, col])
                ties += 1
        # continue from the device's own half-sweep result
        mid = np.where(mask, nxt, mid)
    assert np.array_equal(mid, nxt)
    return ties


def test_split_and_merge_are_exact():
    t = torch()
    rng = np.random.default_rng(1)
    for rows, cols in [(1, 2), (3, 4), (7, 34), (64, 64), (129, 998)]:
        a = (rng.random((rows, cols)) * 255).astype(np.uint8)
        f = rng.normal(size=(rows, cols)).astype(np.float32)
        for arr in (a, f):
            d = to_dev(arr)
            p0, p1 = _planes(t, d)
            t.cuda.synchronize()
            assert np.array_equal(p0.cpu().numpy(), oracle.ising_to_plane(arr, 0))
            assert np.array_equal(p1.cpu().numpy(), oracle.ising_to_plane(arr, 1))
            assert np.array_equal(_natural(t, p0, p1, rows, cols), arr)


@pytest.mark.parametrize("rows,cols,w", [
    (1, 2, 1.0), (3, 4, 2.0), (7, 34, 2.0), (64, 64, 2.0), (129, 96, 2.0), (100, 998, 1.0),
    (33, 256, -1.5), (256, 512, 2.0),
])
def test_sweeps_match_oracle(rows, cols, w):
    t = torch()
    y, b, _ = synth.ising_lattice(rows, cols, 10 + rows + cols, w=w)
    n = 4
    u = synth.ising_uniforms(n, rows, cols, 11 + rows)
    s0, s1 = _planes(t, to_dev(y))
    b0, b1 = _planes(t, to_dev(b))
    ud = to_dev(u)
    plane = rows * (cols // 2)
    ones = t.zeros(2 * n, dtype=t.int64, device="cuda")
    prev = y.copy()
    ties = 0
    for k in range(n):
        glm.glm_ising_sweeps(s0, s1, b0, b1, rows, cols, w, 1, ud[k:k + 1], ones[2 * k:2 * k + 2])
        nxt = _natural(t, s0, s1, rows, cols)
        ties += _check_sweep(prev, nxt, b, w, u[k])
        oc = ones[2 * k:2 * k + 2].cpu().numpy()
        assert oc[0] == int(oracle.ising_to_plane(nxt, 0).sum()) and \
            oc[1] == int(oracle.ising_to_plane(nxt, 1).sum())
        prev = nxt
    assert ties <= max(2, plane // 100000)
    # the same sweeps in one call: bitwise the same chain
    s0b, s1b = _planes(t, to_dev(y))
    glm.glm_ising_sweeps(s0b, s1b, b0, b1, rows, cols, w, n, ud, None)
    assert np.array_equal(_natural(t, s0b, s1b, rows, cols), prev)


def test_chain_without_ties_equals_the_oracle_chain():
    """Away from near ties the device chain is the oracle chain: compare a
    multi-sweep run with the oracle run end to end (checking that no tie
    occurred on the way)."""
    t = torch()
    rows, cols, w, n = 48, 64, 2.0, 6
    y, b, _ = synth.ising_lattice(rows, cols, 21, w=w)
    u = synth.ising_uniforms(n, rows, cols, 22)
    s = y.copy()
    for k in range(n):
        for c in (0, 1):
            s_new, p = oracle.ising_half_sweep(s, b, w, c, u[k, c])
            un = np.zeros((rows, cols))
            for r in range(rows):
                un[r, (r + c) % 2::2] = u[k, c, r]
            rr, cc = np.indices((rows, cols))
            mask = ((rr + cc) % 2) == c
            assert np.min(np.abs(un - p)[mask]) >= TIE
            s = s_new
    ref, ones_ref = oracle.ising_gibbs(y, b, w, u)
    assert np.array_equal(ref, s)
    s0, s1 = _planes(t, to_dev(y))
    b0, b1 = _planes(t, to_dev(b))
    ones = t.zeros(2 * n, dtype=t.int64, device="cuda")
    glm.glm_ising_sweeps(s0, s1, b0, b1, rows, cols, w, n, to_dev(u), ones)
    assert np.array_equal(_natural(t, s0, s1, rows, cols), ref)
    oc = ones.cpu().numpy().reshape(n, 2)
    init1 = int(oracle.ising_to_plane(y, 1).sum())
    tot = [oc[k, 0] + (oc[k - 1, 1] if k else init1) for k in range(n)]
    assert tot == [int(v) for v in ones_ref[:, 0]]
    assert [int(oc[k, 0] + oc[k, 1]) for k in range(n)] == [int(v) for v in ones_ref[:, 1]]


def test_full_size_lattice_sampled_rows():
    """8192 x 8192 denoising lattice (the benchmark workload), two sweeps;
    sampled rows (edges included) replayed in the oracle on 3-row bands of
    the device's own states."""
    t = torch()
    rows = cols = 8192
    w = 2.0
    y, b, _ = synth.ising_lattice(rows, cols, synth.seed_for(5), w=w)
    u = synth.ising_uniforms(2, rows, cols, synth.seed_for(5) + 1)
    s0, s1 = _planes(t, to_dev(y))
    b0, b1 = _planes(t, to_dev(b))
    ud = to_dev(u)
    prev = y
    for k in range(2):
        glm.glm_ising_sweeps(s0, s1, b0, b1, rows, cols, w, 1, ud[k:k + 1], None)
        nxt = _natural(t, s0, s1, rows, cols)
        for r in (0, 1, 4095, 4096, rows - 2, rows - 1):
            lo, hi = max(r - 1, 0), min(r + 2, rows)
            band_prev = prev[lo:hi]
            band_next = nxt[lo:hi]
            mid = band_prev.copy()
            for c in (0, 1):
                cb = (c + lo) % 2                       # colour in band coordinates
                want, p = oracle.ising_half_sweep(mid, b[lo:hi], w, cb, u[k, c, lo:hi])
                i = r - lo
                sel = (np.arange(cols) + i) % 2 == cb
                bad = sel & (want[i] != band_next[i])
                for col in np.nonzero(bad)[0]:
                    assert abs(float(u[k, c, r, col // 2]) - p[i, col]) < TIE
                rr, cc = np.indices(mid.shape)
                mid = np.where(((rr + cc) % 2) == cb, band_next, mid)
        prev = nxt


def test_argument_errors_launch_nothing():
    t = torch()
    s = t.zeros((4, 4), dtype=t.uint8, device="cuda")
    b = t.zeros((4, 4), dtype=t.float32, device="cuda")
    with pytest.raises(glm.GLMError):
        glm.glm_ising_sweeps(s, s, b, b, 4, 7, 1.0, 1, b, None)
    with pytest.raises(glm.GLMError):
        glm.glm_ising_split(s, 3, 4, 8, s, s)
