"""Helpers for the GPU parity tests: run the library through its C ABI on
numpy inputs and compare with the FP64 oracle at the stated tolerances."""
from __future__ import annotations

import numpy as np

import paper_1310_1537_gb300 as glm

# Tolerances of the FP32 / reduced-precision paths against the FP64 oracle run
# on the same stored (rounded) X and the same FP32 beta.
F_RTOL = 1e-5          # |f - f_o| / |f_o|
G_RTOL = 1e-4          # ||g - g_o||_2 / ||g_o||_2


def torch():
    import torch as _t
    return _t


def to_dev(a):
    t = torch()
    return t.from_numpy(np.ascontiguousarray(a)).cuda()


class Handle:
    """A glm handle plus device copies of one dataset."""

    def __init__(self, Xstore: np.ndarray, y: np.ndarray, p: int, xtype=glm.GLM_X_F32,
                 k_max: int = 8, prior_sigma: float = 10.0, x_scale=None, flags: int = 0):
        n, ld = Xstore.shape
        self.n, self.p, self.ld = n, p, ld
        self.h = glm.glm_create(n, p, ld, k_max, xtype, prior_sigma, 0, flags)
        self.X = to_dev(Xstore) if n > 0 else torch().empty(16, dtype=torch().uint8, device="cuda")
        self.y = to_dev(y) if n > 0 else torch().empty(16, dtype=torch().uint8, device="cuda")
        self.x_scale = None if x_scale is None else to_dev(np.asarray(x_scale, dtype=np.float32))

    def eval(self, beta: np.ndarray):
        t = torch()
        b = np.ascontiguousarray(np.atleast_2d(beta), dtype=np.float32)
        k = b.shape[0]
        bd = to_dev(b)
        f = t.empty(k, dtype=t.float64, device="cuda")
        g = t.empty((k, self.p), dtype=t.float32, device="cuda")
        glm.glm_logpost_grad(self.h, self.X, self.x_scale, self.y, bd, k, f, g)
        st = glm.glm_sync(self.h)
        assert st == glm.GLM_OK, glm.glm_status_str(st)
        return f.cpu().numpy(), g.cpu().numpy()

    def info(self):
        return glm.glm_get_info(self.h)

    def close(self):
        if self.h:
            glm.glm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def rel_errors(f, g, f_o, g_o):
    f = np.asarray(f, dtype=np.float64)
    g = np.asarray(g, dtype=np.float64)
    ef = np.abs(f - f_o) / np.maximum(np.abs(f_o), 1e-300)
    eg = np.linalg.norm(g - g_o, axis=-1) / np.maximum(np.linalg.norm(g_o, axis=-1), 1e-300)
    return ef, eg


def assert_close(f, g, f_o, g_o, f_rtol=F_RTOL, g_rtol=G_RTOL, what=""):
    ef, eg = rel_errors(f, g, f_o, g_o)
    assert np.all(np.isfinite(f)) and np.all(np.isfinite(g)), what
    assert ef.max() <= f_rtol, f"{what}: max rel err f {ef.max():.3e} > {f_rtol}"
    assert eg.max() <= g_rtol, f"{what}: max rel L2 err g {eg.max():.3e} > {g_rtol}"
    return ef.max(), eg.max()
