"""GPU parity of the device-resident random-walk Metropolis driver.

Both chains consume the same proposal normals and log-uniforms. Accept/reject
is an integer decided by floating point (FP64 on both sides, on f values that
agree to the f tolerance), so the two chains must be bitwise identical until
their first differing decision, which must be a near tie; after it, every
device transition is still checked for validity by replaying it in the oracle
from the device's own state. The FP32 proposal fmaf is exact on both sides.
"""
import numpy as np
import pytest

import oracle
import synth
import paper_1310_1537_gb300 as glm
from tests.glmgpu import Handle, to_dev, torch

pytestmark = pytest.mark.gpu


def _run_device_chain(h, K, z, lu, b0, step):
    t = torch()
    T = z.shape[0]
    P = h.p
    state = to_dev(b0.astype(np.float32))
    fst = t.zeros(K, dtype=t.float64, device="cuda")
    samples = t.empty((T, K, P), dtype=t.float32, device="cuda")
    acc = t.empty((T, K), dtype=t.uint8, device="cuda")
    lp = t.empty((T, K), dtype=t.float64, device="cuda")
    zd = to_dev(z)
    lud = to_dev(lu)
    glm.glm_rwm_run(h.h, h.X, h.x_scale, h.y, K, T, step, zd, lud, state, fst, 1, samples, acc, lp)
    assert glm.glm_sync(h.h) == glm.GLM_OK
    return samples.cpu().numpy(), acc.cpu().numpy(), lp.cpu().numpy(), state.cpu().numpy()


@pytest.mark.parametrize("K", [1, 4])
def test_rwm_chain_matches_oracle(K):
    """N=10,000, P=50: 1,000 Metropolis steps from a fixed seed.

    (1) The device chain and the oracle chain are bitwise identical up to the
        first step where their decisions differ, and that step must be a near
        tie: |log u - log alpha_oracle| within twice the f tolerance.
    (2) Every one of the 1,000 device transitions is valid: replaying it in
        the oracle from the device's own previous state gives the same
        proposal and the same decision, except at near ties.
    """
    d = synth.make_glm(10_000, 50, synth.seed_for(0), dtype=np.float64)
    X32 = d.X.astype(np.float32)
    Xs = synth.pad_columns(X32, 52)
    X64 = Xs.astype(np.float64)
    T = 1000
    z, lu = synth.rwm_streams(T, K, 50, synth.seed_for(0) + 2)
    step = synth.rwm_step_size(10_000, 50)
    b0 = np.tile(d.beta_star.astype(np.float32), (K, 1))
    h = Handle(Xs, d.y, 50, k_max=K)
    s_dev, a_dev, lp_dev, _ = _run_device_chain(h, K, z, lu, b0, step)
    ref = oracle.rwm(X64, d.y, b0, z, lu, step, p=50)
    for k in range(K):
        tie = 2e-5 * np.abs(ref["logpost"][:, k]) + 1e-6
        diff = np.nonzero(a_dev[:, k] != ref["accept"][:, k])[0]
        stop = int(diff[0]) if len(diff) else T
        if stop < T:
            assert abs(lu[stop, k] - ref["log_alpha"][stop, k]) < tie[stop], f"chain {k} step {stop}"
        np.testing.assert_array_equal(s_dev[:stop, k], ref["samples"][:stop, k])
        rel = np.abs(lp_dev[:stop, k] - ref["logpost"][:stop, k]) / np.abs(ref["logpost"][:stop, k])
        assert rel.max(initial=0.0) <= 1e-5
        # (2) replay every device transition in the oracle
        prev = b0[k:k + 1].copy()
        n_tie = 0
        for t in range(T):
            one = oracle.rwm(X64, d.y, prev, z[t:t + 1, k:k + 1], lu[t:t + 1, k:k + 1], step, p=50)
            la = one["log_alpha"][0, 0]
            if abs(lu[t, k] - la) < 2e-5 * abs(one["f"][0]) + 1e-6:
                n_tie += 1
            else:
                assert a_dev[t, k] == one["accept"][0, 0], f"chain {k} step {t}"
                np.testing.assert_array_equal(s_dev[t, k], one["samples"][0, 0])
                assert abs(lp_dev[t, k] - one["f"][0]) <= 1e-5 * abs(one["f"][0])
            prev = s_dev[t, k][None, :].copy()
        print(f"chain {k}: identical to the oracle chain for {stop} steps; all {T} transitions "
              f"valid ({n_tie} near ties); acceptance {a_dev[:, k].mean():.3f}")


def test_rwm_replay_is_deterministic():
    d = synth.make_glm(5000, 12, 123, dtype=np.float32)
    Xs = synth.pad_columns(d.X, 12)
    z, lu = synth.rwm_streams(200, 2, 12, 5)
    b0 = np.tile(d.beta_star.astype(np.float32), (2, 1))
    h = Handle(Xs, d.y, 12, k_max=2)
    r1 = _run_device_chain(h, 2, z, lu, b0, 0.02)
    r2 = _run_device_chain(h, 2, z, lu, b0, 0.02)
    for a, b in zip(r1, r2):
        np.testing.assert_array_equal(a, b)


def test_rwm_resume_equals_uninterrupted():
    """Checkpoint/resume: 150 steps then 150 more from the saved state equals 300 at once."""
    t = torch()
    d = synth.make_glm(8000, 20, 321, dtype=np.float32)
    Xs = synth.pad_columns(d.X, 20)
    z, lu = synth.rwm_streams(300, 1, 20, 6)
    b0 = d.beta_star[None, :].astype(np.float32)
    h = Handle(Xs, d.y, 20, k_max=1)
    s_all, a_all, lp_all, st_all = _run_device_chain(h, 1, z, lu, b0, 0.03)
    state = to_dev(b0)
    fst = t.zeros(1, dtype=t.float64, device="cuda")
    zd, lud = to_dev(z), to_dev(lu)
    glm.glm_rwm_run(h.h, h.X, None, h.y, 1, 150, 0.03, zd, lud, state, fst, 1)
    saved_b, saved_f = state.cpu().numpy(), fst.cpu().numpy()       # checkpoint
    state2, fst2 = to_dev(saved_b), to_dev(saved_f)                 # restore
    zd2, lud2 = to_dev(z[150:]), to_dev(lu[150:])
    glm.glm_rwm_run(h.h, h.X, None, h.y, 1, 150, 0.03, zd2, lud2, state2, fst2, 0)
    assert glm.glm_sync(h.h) == glm.GLM_OK
    np.testing.assert_array_equal(state2.cpu().numpy(), st_all)
