"""Writes tests/golden/oracle_steady_257_counts.json: the oracle's own work counts for the
257 x 257 steady continuation (table transport, -300 V), from oracle/ only.

Run from the repository root:  python tests/golden/make_oracle_counts.py   (a few minutes)
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402
from oracle import profile_counts  # noqa: E402


def main():
    d = W.steady_257()
    counts, wall, _ = profile_counts.steady_counts(d, tol=1e-8)
    counts["workload"] = "257x257 nodes, -300 V, table transport seed 2, sources seed 0, rho <= 1e-8"
    counts["dev_box_wall_s"] = wall
    with open(os.path.join(ROOT, "tests", "golden", "oracle_steady_257_counts.json"), "w") as fh:
        json.dump(counts, fh, indent=1)
    print(counts)


if __name__ == "__main__":
    main()
