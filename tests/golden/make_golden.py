"""Write the stored expected values used by the GPU parity tests.

Every value here comes from the CPU oracle (``oracle/``) on seeded synthetic
inputs; nothing is taken from the CUDA path.  Run from the repository root:

    python tests/golden/make_golden.py
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_2306_03651_gb300 import inputs as I  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "ba2000_run.json")


def main():
    w = I.ba_2000()
    g = O.Graph.of(w.graph)
    r = g.run(w.k, w.eps, w.delta, w.t, w.seed, m0=w.m0)
    doc = {
        "what": "Algorithm 1 on BA n=2000 d=4 graph seed 1; k=10 eps=0.05 delta=0.1 t=10 seed=1 m0=1000 (oracle)",
        "status": int(r["status"]),
        "S": [int(x) for x in r["S"]],
        "covered": int(r["covered"]),
        "m_final": int(r["m_final"]),
        "rounds": int(r["rounds"]),
        "log_cols": list(O.LOG_COLS),
        "log_hex": [[float(x).hex() for x in row] for row in r["log"]],
    }
    with open(OUT, "w") as f:
        json.dump(doc, f, indent=1)
    print("wrote", OUT)


if __name__ == "__main__":
    main()
