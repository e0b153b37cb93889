"""Writes oracle_regression.json: the oracle's Γ, WP and kept counts on a few modes of the seed-0
Morse diamond (2x2x2 and 3x3x3 meshes, T = 300 K, fixed σ = 0.1 THz and adaptive s = 1).

A regression record, not a pin: it makes any later change of the oracle's arithmetic show up in
tests/test_oracle_regression.py, where the commit that changes it must name the passage of the
paper (or the reading) that justifies the change.  Run from the repository root:

    python tests/golden/make_oracle_regression.py
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

CASES = [
    {"mesh": [2, 2, 2], "sigma": 0.1, "adaptive": False, "modes": [3, 10, 25, 47]},
    {"mesh": [3, 3, 3], "sigma": 0.1, "adaptive": False, "modes": [4, 33, 77, 161]},
    {"mesh": [3, 3, 3], "sigma": 1.0, "adaptive": True, "modes": [9, 40, 100]},
]


def compute(case):
    import oracle
    from synth import morse_system
    P = oracle.Problem(*morse_system(seed=0), tuple(case["mesh"]), T=300.0, sigma=case["sigma"],
                       sigma_adaptive=case["adaptive"])
    g, wp, cnt = P.rates(case["modes"])
    return {"gamma": g.tolist(), "wp": wp.tolist(), "counts": cnt.tolist()}


def main():
    out = {"source": "oracle (fc4_oracle.c + oracle/__init__.py), seed-0 Morse diamond, T = 300 K",
           "cases": [dict(case, **compute(case)) for case in CASES]}
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_regression.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
