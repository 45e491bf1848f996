"""Writes the stored expected values under tests/golden/ by calling only the
FP64 oracle and the seeded workload generators.

    python tests/golden/make_golden.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import workloads  # noqa: E402
from oracle import twa  # noqa: E402


def circle4():
    inst = workloads.circle4()
    prob = twa.Problem.from_instance(inst)
    st, it, res = twa.solve(prob, inst.tol, inst.max_iter)
    coll, _ = twa.min_clearance(prob, st.z)
    return {
        "workload": inst.name,
        "source": "oracle.twa.solve (FP64), stop at residual < tol",
        "tol": inst.tol,
        "iterations": it,
        "residual": res,
        "total_cost": twa.total_cost(prob, st.z),
        "min_clearance_ratio": coll,
        "z": st.z.tolist(),
    }


if __name__ == "__main__":
    out = circle4()
    with open(os.path.join(HERE, "circle4_eta4.json"), "w") as f:
        json.dump(out, f, indent=1)
    print("wrote circle4_eta4.json:", out["iterations"], out["total_cost"])
