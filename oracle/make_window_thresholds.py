"""Write paper_2202_10647_gb300/data/window_thresholds.json.

For every state k of the workload species (nitrogen and the two synthetic
ladders) it stores the lowest field in [1, 1e5] GV/m at which the oracle's ADK
rate (Eq. 1) gives W_k * 0.05 fs >= 1, or 1e30 if there is none.  The
workloads only use these numbers to place synthetic windows at the states
that the local field is burning through.  Run: python -m oracle.make_window_thresholds
"""
import json
import math
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2202_10647_gb300 import workloads  # noqa: E402  (input recipes only)

DT = 0.05


def threshold(U, l, m, Q):
    def f(E):
        return oracle.adk_rate(E, U, l, m, Q) * DT - 1.0
    grid = [10 ** (5 * i / 4000) for i in range(4001)]
    prev = grid[0]
    if f(prev) >= 0:
        return prev
    for E in grid[1:]:
        if f(E) >= 0:
            a, b = math.log(prev), math.log(E)
            for _ in range(80):
                c = 0.5 * (a + b)
                if f(math.exp(c)) >= 0:
                    b = c
                else:
                    a = c
            return math.exp(b)
        prev = E
    return 1e30


def main():
    out = {}
    for sp in (workloads.nitrogen(), workloads.argon_like(), workloads.krypton_like()):
        out[sp.name] = [threshold(sp.U[k], sp.l[k], sp.m[k], k + 1) for k in range(sp.Z)]
    path = os.path.join(ROOT, "paper_2202_10647_gb300", "data", "window_thresholds.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(path)
    for k, v in out.items():
        print(k, ["%.4g" % x for x in v])


if __name__ == "__main__":
    main()
