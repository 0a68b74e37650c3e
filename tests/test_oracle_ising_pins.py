"""Pins of the oracle's checkerboard Gibbs sampler for the square-lattice
Ising model (§4.3.1), against brute-force enumeration, closed forms and
invariants rather than against itself."""
import itertools
import math

import numpy as np

import oracle
import synth


def test_conditional_is_the_boltzmann_ratio():
    """For every site of random states, the oracle's P(s_i = 1) equals the
    ratio exp(-E(s_i=1)) / (exp(-E(s_i=1)) + exp(-E(s_i=0))) computed from
    the energy by brute force (fixes the sign convention)."""
    rng = np.random.default_rng(1)
    for _ in range(20):
        R, C = 3, 4
        s = (rng.random((R, C)) < 0.5).astype(np.uint8)
        b = rng.normal(size=(R, C)).astype(np.float32)
        w = float(rng.normal())
        for color in (0, 1):
            u = np.full((R, C // 2), 0.5, dtype=np.float32)
            _, p = oracle.ising_half_sweep(s, b, w, color, u)
            for r in range(R):
                for c in range(C):
                    s1 = s.copy()
                    s1[r, c] = 1
                    s0 = s.copy()
                    s0[r, c] = 0
                    e1, e0 = oracle.ising_energy(s1, b, w), oracle.ising_energy(s0, b, w)
                    ref = 1.0 / (1.0 + math.exp(e1 - e0))
                    assert abs(p[r, c] - ref) < 1e-12, (r, c, p[r, c], ref)


def test_no_coupling_gives_independent_sites():
    """w = 0: each updated spin is 1 iff u < 1 / (1 + exp(-b)); the other
    colour is untouched."""
    rng = np.random.default_rng(2)
    R, C = 7, 10
    s = (rng.random((R, C)) < 0.5).astype(np.uint8)
    b = rng.normal(size=(R, C)).astype(np.float32)
    for color in (0, 1):
        u = rng.random((R, C // 2)).astype(np.float32)
        out, _ = oracle.ising_half_sweep(s, b, 0.0, color, u)
        for r in range(R):
            for c in range(C):
                if (r + c) % 2 == color:
                    want = 1 if float(u[r, c // 2]) < 1.0 / (1.0 + math.exp(-float(b[r, c]))) else 0
                    assert out[r, c] == want
                else:
                    assert out[r, c] == s[r, c]


def test_update_ignores_its_own_colour():
    """A colour's new spins depend only on the other colour: changing the
    updated colour's old spins changes nothing."""
    rng = np.random.default_rng(3)
    R, C = 9, 12
    b = rng.normal(size=(R, C)).astype(np.float32)
    u = rng.random((R, C // 2)).astype(np.float32)
    s = (rng.random((R, C)) < 0.5).astype(np.uint8)
    rr, cc = np.indices((R, C))
    for color in (0, 1):
        t = s.copy()
        mask = ((rr + cc) % 2) == color
        t[mask] = 1 - t[mask]
        a, _ = oracle.ising_half_sweep(s, b, 0.7, color, u)
        c2, _ = oracle.ising_half_sweep(t, b, 0.7, color, u)
        assert np.array_equal(a, c2)


def test_planes_index_the_checkerboard():
    """Plane entry (r, j) of colour c is the site (r, 2j + (r + c) % 2), which
    has colour c; the two planes together hold every site once."""
    R, C = 5, 8
    a = np.arange(R * C).reshape(R, C)
    for c in (0, 1):
        p = oracle.ising_to_plane(a, c)
        for r in range(R):
            for j in range(C // 2):
                col = 2 * j + (r + c) % 2
                assert p[r, j] == a[r, col] and (r + col) % 2 == c
    both = np.concatenate([oracle.ising_to_plane(a, 0).ravel(), oracle.ising_to_plane(a, 1).ravel()])
    assert sorted(both.tolist()) == list(range(R * C))
    assert np.array_equal(oracle.ising_from_planes(oracle.ising_to_plane(a, 0),
                                                   oracle.ising_to_plane(a, 1)), a)


def test_chain_marginals_match_exact_enumeration():
    """3 x 4 lattice (4,096 states): the Gibbs chain's site marginals and mean
    energy agree with the exact Boltzmann distribution."""
    R, C = 3, 4
    rng = np.random.default_rng(4)
    b = (0.6 * rng.normal(size=(R, C))).astype(np.float32)
    w = 0.8
    states = np.array(list(itertools.product([0, 1], repeat=R * C)), dtype=np.uint8).reshape(-1, R, C)
    E = np.array([oracle.ising_energy(st, b, w) for st in states])
    pw = np.exp(-(E - E.min()))
    pw /= pw.sum()
    marg = (pw[:, None, None] * states).sum(axis=0)
    mean_e = float((pw * E).sum())
    n = 20000
    u = synth.ising_uniforms(n, R, C, 5)
    s = np.zeros((R, C), dtype=np.uint8)
    acc = np.zeros((R, C))
    es = np.empty(n)
    for t in range(n):
        for c in (0, 1):
            s, _ = oracle.ising_half_sweep(s, b, w, c, u[t, c])
        acc += s
        es[t] = oracle.ising_energy(s, b, w)
    burn = 200
    assert np.max(np.abs(acc / n - marg)) < 0.02, (acc / n, marg)
    nb = 40
    bm = es[burn:burn + (n - burn) // nb * nb].reshape(nb, -1).mean(axis=1)
    se = bm.std(ddof=1) / math.sqrt(nb)
    assert abs(es[burn:].mean() - mean_e) < 5 * se + 1e-3


def test_denoising_biases_match_the_pm1_model():
    """The workload's biases turn the +-1 denoising energy into the {0, 1}
    energy up to a constant: energy differences agree for random states."""
    R, C = 6, 8
    y, b, _ = synth.ising_lattice(R, C, 6, eta=1.3, w=2.0)
    J, eta = 0.5, 1.3
    yp = 2.0 * y.astype(np.float64) - 1.0
    rng = np.random.default_rng(7)

    def e_pm1(s):
        g = 2.0 * s.astype(np.float64) - 1.0
        pairs = (g[1:, :] * g[:-1, :]).sum() + (g[:, 1:] * g[:, :-1]).sum()
        return -J * pairs - eta * (g * yp).sum()
    s_ref = (rng.random((R, C)) < 0.5).astype(np.uint8)
    for _ in range(20):
        s = (rng.random((R, C)) < 0.5).astype(np.uint8)
        d01 = oracle.ising_energy(s, b, 2.0) - oracle.ising_energy(s_ref, b, 2.0)
        dpm = e_pm1(s) - e_pm1(s_ref)
        assert abs(d01 - dpm) < 1e-4 * (1 + abs(dpm))
