"""Writes odeim_front_basis.json: the oracle's ODEIM points (Eq. odeim,
oracle.rom.odeim: DEIM greedy, then greedy oversampling by the smallest
eigenvalue of the augmented sampled Gram matrix, ties within tie_tol to the
lowest row) for bases the size of the 2048^2 benchmark's point selection
(m = 64 modes, n_p = 128 points) on 102 400 rows, in FP64 and for the same
basis rounded to FP32.

The bases come from workloads.front_basis, which uses splitmix64 draws and
IEEE-exact operations only, so the GPU test rebuilds the same bits on any
machine; the file records a SHA-256 of each basis so that the test can check
this before comparing points.  The oracle takes about 5 s per oversampling
step at this size, too long to run inside the GPU test, hence this file.

Run from the repository root:  python tests/golden/make_odeim_golden.py
"""
import hashlib
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402
from oracle import rom  # noqa: E402

CASES = [dict(nrow=102400, m=64, n_p=128, seed=2048, tie_tol=1e-12)]


def basis(case, prec):
    Phi = W.front_basis(case["nrow"], case["m"], case["seed"])
    if prec == "f32":
        Phi = Phi.astype(np.float32).astype(np.float64)
    return Phi


def digest(Phi):
    return hashlib.sha256(np.ascontiguousarray(Phi, dtype=np.float64).tobytes()).hexdigest()


def main():
    out = []
    for case in CASES:
        for prec in ("f64", "f32"):
            Phi = basis(case, prec)
            t = time.time()
            pts = rom.odeim(Phi, case["n_p"], case["tie_tol"])
            print(f"{prec}: {time.time() - t:.0f} s", file=sys.stderr)
            out.append(dict(case, prec=prec, sha256=digest(Phi), points=[int(p) for p in pts]))
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "odeim_front_basis.json")
    with open(path, "w") as f:
        json.dump({"source": "oracle.rom.odeim via tests/golden/make_odeim_golden.py",
                   "cases": out}, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
