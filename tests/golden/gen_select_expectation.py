"""Writes select_expectation.json: the exact expected norm of the
sample-selected column (Sec. 3.2, sample bias; Fig. selectExpect setting:
orthogonal columns with norms phi^j, j = 0..n-1, sample of l GIID rows),
computed by the oracle's quadrature.  Run from the repository root:
    python tests/golden/gen_select_expectation.py
"""
import json
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__)))))

from oracle import selection  # noqa: E402

CASES = [(phi, ell, 32) for ell in (4, 8, 16, 32) for phi in (0.5, 0.8, 0.9, 0.95, 0.98)]


def main():
    rows = [{"phi": phi, "ell": ell, "n": n, "exact": selection.select_expectation(phi, ell, n)}
            for phi, ell, n in CASES]
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "select_expectation.json")
    with open(path, "w") as f:
        json.dump({"source": "oracle.selection.select_expectation (quadrature)", "cases": rows},
                  f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
