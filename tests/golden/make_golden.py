"""Write the stored oracle values under tests/golden/.

The paper (arXiv 2409.08090) prints no worked example, so the stored values
are regression fixtures only: they are produced here by calling nothing but
``oracle/`` on the seeded ``single_small`` workload (N_d = 1000, N_f = 12000,
f0 = 0.01, df = 0.002).  Run from the repository root:

    python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2409_08090_gb300 import workloads  # noqa: E402


def main():
    s = workloads.single_small()
    rng = np.random.default_rng(2024)
    k = np.sort(np.concatenate([[0, 180, s.nf - 1], rng.choice(s.nf, 61, replace=False)]))
    k = np.unique(k).astype(np.int64)
    P = oracle.periodogram(s.t, s.y, s.dy, s.f0, s.df, k)
    out = {"workload": "single_small (seed 20240912)", "k": k.tolist(),
           "P": [float(v) for v in P], "writer": "tests/golden/make_golden.py (oracle only)"}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "single_small_oracle.json")
    with open(path, "w") as fh:
        json.dump(out, fh, indent=1)
        fh.write("\n")


if __name__ == "__main__":
    main()
