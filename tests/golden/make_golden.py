"""Writes the oracle's reference trajectory for the 40x40x30 / 5 mm / 5-beam phantom.

Calls only the FP64 oracle (and the input generator). The stored numbers are a
regression fixture for the oracle itself: the paper prints no worked example,
so they are pinned by the tests in tests/pins.py, not by the paper.
Run:  python tests/golden/make_golden.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_0908_4421_gb300 import phantom  # noqa: E402


def main():
    case = phantom.make_case(phantom.TINY_5MM_5BEAM)
    orc = oracle.get()
    lam0 = orc.lambda0_rule(case)
    res = orc.solve(case, lambda0=lam0, eps=1e-4, alpha=2.0, delta=1e-6, max_iter=200, threads=1)
    out = {
        "what": "FP64 oracle, Sec. 2.2 projected gradient with Armijo (Eq. (5)), tiny 40x40x30 5 mm 5-beam phantom",
        "cite": "Sec. 2.1 Eq. (1)-(2), Sec. 2.2 Eq. (3)-(5) and steps 1-5",
        "m": case.m, "n": case.n, "nnz": case.nnz,
        "lambda0_rule": lam0, "eps": 1e-4, "alpha": 2.0, "delta": 1e-6, "max_iter": 200,
        "status": res.status, "iterations": res.iterations, "backtracks": res.backtracks,
        "stop_reason": res.stop_reason, "objective": res.objective, "kkt": res.kkt,
        "G": [float(g) for g in res.G],
    }
    with open(os.path.join(HERE, "tiny_5mm_5beam_oracle.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
