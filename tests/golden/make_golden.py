"""Writes oracle_small.json: oracle values on two tiny seeded cases.

Calls only ``oracle`` and the seeded input generators in ``workloads``; the
stored values guard the oracle's arithmetic against unnoticed changes.
Run from the repository root:  python tests/golden/make_golden.py
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import workloads as W  # noqa: E402

CASES = {
    "free2d": dict(d=2, p=4, delta=3e-3, periodic=False, seed=41, max_level=3),
    "per3d": dict(d=3, p=3, delta=2e-2, periodic=True, seed=42, max_level=2),
}


def main():
    out = {}
    for name, c in CASES.items():
        tr = W.random_balanced_tree(c["d"], c["seed"], max_level=c["max_level"], periodic=c["periodic"],
                                    min_level=1)
        sig = W.random_sigma(tr, c["p"], c["seed"])
        u = oracle.box_fgt(c["d"], c["p"], c["delta"], c["periodic"], tr.level, tr.coord, sig)
        out[name] = dict(d=c["d"], p=c["p"], delta=c["delta"], periodic=c["periodic"],
                         level=tr.level.tolist(), coord=tr.coord.tolist(), sigma=sig.tolist(), u=u.tolist())
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_small.json"), "w") as f:
        json.dump(out, f, indent=0)


if __name__ == "__main__":
    main()
