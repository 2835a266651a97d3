"""Write tests/golden/table_restbl_reference.json: for each (n, m) row of
Table RESTBL (tests/golden/table_restbl.json, the values the paper prints),
the exact E_G = sum of the m lowest eigenvalues of the 2-D Dirichlet
Laplacian of Eq. LAPLACE, lambda_m, lambda_{m+1} and the gap, from the
closed form printed after Eq. LAPLACE (oracle.operator.laplace2d_spectrum).

Run from the repository root:
    python tests/golden/make_table_reference.py
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from oracle import operator as op  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
TABLE = os.path.join(HERE, "table_restbl.json")
OUT = os.path.join(HERE, "table_restbl_reference.json")


def rows():
    out = []
    for row in json.load(open(TABLE))["rows"]:
        n, m = row["n"], row["m"]
        lam = op.laplace2d_spectrum(n)
        out.append({"n": n, "m": m, "E_G": float(np.sum(lam[:m])),
                    "lambda_m": float(lam[m - 1]), "lambda_m1": float(lam[m]),
                    "gap": float(lam[m] - lam[m - 1])})
    return out


def main():
    data = {"source": "oracle.operator.laplace2d_spectrum (the closed form "
                      "after Eq. LAPLACE) for the rows of Table RESTBL",
            "rows": rows()}
    with open(OUT, "w") as fh:
        json.dump(data, fh, indent=1)


if __name__ == "__main__":
    main()
