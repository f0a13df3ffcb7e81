"""Writes tests/golden/small_cases.json: log-likelihood and gradient of Eq. 1 (Section 2.1) for
small seeded event sets, as computed by the FP64 CPU oracle (oracle/, the only code this
script calls besides the seeded input generator).

Each case stores its inputs (x, y, t as float64), Theta, the flags, and the oracle's
ell and gradient both for the inputs as given ("f64") and for the same inputs rounded to
float32 ("f32in", the values the mixed-precision path stores). Re-run with
    python tests/golden/make_golden.py
only when a change to the oracle's arithmetic is justified by the paper; the tests compare the
oracle and the CUDA path against these stored values.
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_2005_10123_gb300 import synth  # noqa: E402

CASES = [  # (name, n, T, seed, Theta, flags)
    ("n1", 1, 100.0, 101, synth.THETA0, 0),
    ("n2", 2, 100.0, 102, synth.THETA0, 0),
    ("n5", 5, 50.0, 103, (0.02, 0.8, 10.0, 0.6, 2.0, 0.2), 0),
    ("n50", 50, 200.0, 104, synth.THETA0, 0),
    ("n50_exclude_self", 50, 200.0, 104, synth.THETA0, oracle.EXCLUDE_SELF),
    ("n300", 300, 300.0, 105, (0.05, 1.5, 20.0, 0.4, 0.5, 0.15), 0),
    ("n777_ragged", 777, 500.0, 106, synth.THETA0, 0),
]


def main():
    out = {"source": "oracle/ (FP64, Section 2.1 Eq. 1), written by tests/golden/make_golden.py",
           "param_order": list(oracle.PARAM_NAMES), "cases": []}
    for name, n, T, seed, th, flags in CASES:
        ev = synth.simulate(n, T, seed=seed)
        case = {"name": name, "n": n, "T": T, "seed": seed, "theta": list(th), "flags": flags,
                "x": ev.x.tolist(), "y": ev.y.tolist(), "t": ev.t.tolist()}
        for key, e in (("f64", ev), ("f32in", ev.rounded32())):
            ll, g = oracle.loglik(e.x, e.y, e.t, th, flags=flags, grad=True)
            case[key] = {"loglik": float(ll), "grad": [float(v) for v in g]}
        out["cases"].append(case)
    path = os.path.join(HERE, "small_cases.json")
    with open(path, "w") as fh:  # one case per line
        head = {k: v for k, v in out.items() if k != "cases"}
        fh.write("{\n" + ",\n".join(f" {json.dumps(k)}: {json.dumps(v)}" for k, v in head.items()))
        fh.write(',\n "cases": [\n' + ",\n".join("  " + json.dumps(c) for c in out["cases"]) + "\n ]\n}\n")
    print("wrote", path, len(out["cases"]), "cases")


if __name__ == "__main__":
    main()
