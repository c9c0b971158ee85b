"""Writes tests/golden/oracle_single_codes.json from the CPU oracle alone.

Run from the repository root:  python tests/golden/make_oracle_golden.py
Calls only ``oracle`` and the seeded generators; nothing from the CUDA path.
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2603_29942_gb300 import inputs  # noqa: E402


def main():
    out = {}
    for name in inputs.SINGLE:
        code = inputs.single(name)
        res = {}
        for mode, kw in (("default", {}), ("paper_literal", {"per_round_check": True, "defer": False})):
            r = oracle.bz(code, threads=os.cpu_count() or 1, **kw)
            res[mode] = {
                "status": r.status, "d": r.d, "L": r.L, "U": r.U, "m": r.m, "kj": r.kj,
                "evaluated": r.evaluated, "counts": r.counts,
                "passes": [list(x) for x in r.passes],
            }
        out[name] = {"p": code.p, "n": code.n, "k": code.k, "sha256": code.digest(), **res}
        print(name, res["default"]["d"], res["default"]["evaluated"])
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_single_codes.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
