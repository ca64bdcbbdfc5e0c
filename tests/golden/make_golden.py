"""Writes tests/golden/tiny_oracle.json from the oracle alone (no CUDA code is imported).

The file freezes sampled values of the tiny workload (32^3 Gaussian-blob volume, 128^2 server
image, client rotated 5 degrees) so that an accidental change of the oracle's arithmetic shows up
as a test failure.  Re-run it only together with a commit that names the passage of the paper (or
the reading of it) that justifies the change.

    python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synth  # noqa: E402

SAMPLE = [0, 129, 2080, 4100, 6000, 7700, 8256, 8300, 9001, 10000, 11111, 12000, 13500, 15000, 16383]


def compute():
    W = synth.TINY
    cam = W.server_cam()
    rgba, depth = oracle.raycast(W.volume(), synth.tf_ramp(), cam)
    srv = rgba.astype(np.float32)
    sp = oracle.unproject(srv, depth, cam)
    out = oracle.trace(oracle.Scene(sp), synth.tiny_client_camera())
    first = oracle.trace(oracle.Scene(sp, max_hits=1), synth.tiny_client_camera())
    return {
        "n_splats": sp.n,
        "server_rgba": rgba.reshape(-1, 4)[SAMPLE].tolist(),
        "server_depth": [float(x) for x in depth.reshape(-1)[SAMPLE]],
        "client_rgba_all_hits": out["rgba"][SAMPLE].tolist(),
        "client_rgba_first_hit": first["rgba"][SAMPLE].tolist(),
        "client_alpha_sum": float(out["rgba"][:, 3].sum()),
    }


if __name__ == "__main__":
    d = compute()
    d["_about"] = ("tiny workload, oracle only; sample = flat pixel indices " + str(SAMPLE))
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "tiny_oracle.json"), "w") as f:
        json.dump(d, f, indent=1)
