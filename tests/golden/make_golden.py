"""Writes tests/golden/tiny_glm.json: a small stored case whose expected values
come from the FP64 oracle only (the paper prints no numeric example).

Run from the repository root:  python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synth   # noqa: E402


def main():
    d = synth.make_glm(77, 5, synth.seed_for(0) + 900, dtype=np.float32)
    X = d.X.astype(np.float32)
    beta = np.stack([d.beta_star, d.beta_star + 0.25, -d.beta_star]).astype(np.float32)
    f, g = oracle.logpost_grad(X.astype(np.float64), d.y, beta.astype(np.float64), prior_sigma=10.0)
    out = {
        "what": "logistic-GLM log-posterior f and gradient g, prior N(0, 10^2 I); "
                "X and beta are float32 values, f/g from the FP64 oracle",
        "n": 77, "p": 5, "k": 3, "prior_sigma": 10.0,
        "X": X.ravel().tolist(), "y": d.y.tolist(), "beta": beta.ravel().tolist(),
        "f": f.tolist(), "g": g.ravel().tolist(),
    }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tiny_glm.json")
    with open(path, "w") as fh:
        json.dump(out, fh, indent=0)
    print("wrote", path)


if __name__ == "__main__":
    main()
