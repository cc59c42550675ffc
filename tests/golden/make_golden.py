"""Write the golden fixtures of this folder. It calls only oracle.exact (exact rational solve of
(I - P) X = B); rerun with `python tests/golden/make_golden.py` from the repository root.

Each fixture is a tiny graph whose exact solution of X = P.X + B (Section 1, with P oriented as
in Section 2.4) is stored as fractions. The graphs exercise every branch of the D-iteration
visit (Section 2.5 DI-CYC): dangling nodes, loop nodes (transit = F*out/(out-d)), duplicate
links, and a zero-in-degree chain (Section 2.4 E).
"""
from __future__ import annotations

import json
import os
import sys
from fractions import Fraction

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__)))))
from oracle.exact import exact_solve  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))

CASES = [
    dict(name="cycle5_uniform",
         cite="Section 1 (X = P.X + B) on a directed 5-cycle; Section 2.5 DI-CYC init B = (1-d)/N",
         n=5, edges=[(0, 1), (1, 2), (2, 3), (3, 4), (4, 0)], d="17/20", B="uniform"),
    dict(name="mixed8",
         cite="Section 2.4 (dangling, loop nodes, duplicates dropped) and Section 2.5 DI-CYC loop "
              "transit out/(out-d)",
         n=8,
         edges=[(0, 1), (0, 2), (0, 0), (1, 2), (1, 3), (2, 0), (2, 4), (2, 4), (3, 3), (3, 5),
                (4, 6), (4, 7), (4, 1), (5, 6), (6, 7), (7, 7)],
         d="17/20", B="uniform"),
    dict(name="chain_into_cycle",
         cite="Section 2.4 E: chain 0->1->2 feeds a 3-cycle 3->4->5->3; 0..2 are zero in-degree",
         n=6, edges=[(0, 1), (1, 2), (2, 3), (3, 4), (4, 5), (5, 3), (5, 5)], d="19/20",
         B=["1/10", "0", "1/5", "0", "1/20", "0"]),
    dict(name="loop_only",
         cite="Section 2.5 DI-CYC loop node: a node whose only link is itself keeps "
              "F*out/(out-d) = F/(1-d)",
         n=3, edges=[(0, 0), (1, 1), (1, 2)], d="17/20", B=["1/20", "1/20", "1/20"]),
]


def main():
    for case in CASES:
        d = Fraction(case["d"])
        n = case["n"]
        if case["B"] == "uniform":
            B = [(1 - d) / n] * n
        else:
            B = [Fraction(b) for b in case["B"]]
        X = exact_solve(n, case["edges"], d, B)
        out = dict(name=case["name"], cite=case["cite"], n=n, edges=case["edges"], d=str(d),
                   B=[str(b) for b in B], X=[str(x) for x in X],
                   note="X is exact: Gauss-Jordan over fractions on (I - P) X = B")
        with open(os.path.join(HERE, case["name"] + ".json"), "w") as f:
            json.dump(out, f, indent=1)
            f.write("\n")
        print(case["name"], [float(x) for x in X])


if __name__ == "__main__":
    main()
