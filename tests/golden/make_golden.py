"""Writes the stored oracle values the tests compare with (Section 2.1, Eq. 1 and its gradient),
as computed by the FP64 CPU oracle (oracle/, the only code this script calls besides the seeded
input generator):

  tests/golden/small_cases.json   ell and gradient for small seeded event sets;
  tests/golden/full_85k.json      ell and gradient for the N = 85,000 workload (--full);
  tests/golden/mix_cases.json     the mixture of triggering functions: small sets and the
                                  N = 85,000 workload at one mixture vector (--mix).

Each small case stores its inputs (x, y, t as float64), Theta, the flags, and the oracle's
ell and gradient both for the inputs as given ("f64") and for the same inputs rounded to
float32 ("f32in", the values the mixed-precision path stores).

The full-size file stores the generator's arguments and a SHA-256 digest of the float32-rounded
event arrays instead of the events (1 MB of floats), and the parameter vectors themselves, so that
a test can check that it regenerated the same inputs before it compares. Beside ell and the gradient
it stores sum_n |ell_n| and, per component, sum_n |d ell_n / d Theta_k|: the scales against which
the error of a sum that nearly cancels is stated. The N = 85,000 events
are float32-representable, so one oracle evaluation serves the float64 and the mixed paths.
It takes a few minutes on 8 to 16 cores (about 70 s per parameter vector on 8 x86 cores).

Re-run with
    python tests/golden/make_golden.py [--full]
only when a change to the oracle's arithmetic is justified by the paper.
"""
import hashlib
import json
import os
import sys
import time

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

# The N = 85,000 workload: Theta0, a second vector at which no gradient component is near zero,
# and four of the 64 vectors of the batched-chains workload (log-uniform within +-50% of Theta0,
# seed 20053), which the grouped kernel evaluates.
THETA_B = (0.012, 1.3, 20.0, 0.4, 1.5, 0.12)
BATCH_SEED, BATCH_K, BATCH_PICK = 20053, 64, (0, 21, 42, 63)


def events_digest(ev) -> str:
    """SHA-256 of the float32-rounded x, y, t arrays (held as float64, little-endian)."""
    h = hashlib.sha256()
    for a in (ev.x, ev.y, ev.t):
        h.update(np.ascontiguousarray(a, dtype="<f8").tobytes())
    return h.hexdigest()


def write_small():
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


# Mixture of triggering functions (the Discussion's extension): a short, narrow component (hours,
# tens of metres: multi-shot events) and a long, wide one (days to weeks: retaliation).
MIX_CASES = [  # (name, n, T, seed, mixture Theta)
    ("mix_n2", 2, 10.0, 201, (0.02, 0.8, 10.0, 0.3, 24.0, 0.05, 0.2, 0.1, 0.3)),
    ("mix_n50", 50, 100.0, 202, (0.02, 0.8, 10.0, 0.3, 24.0, 0.05, 0.2, 0.1, 0.3)),
    ("mix_n300", 300, 300.0, 203, (0.05, 1.5, 20.0, 0.25, 6.0, 0.08, 0.3, 0.3, 0.4)),
    ("mix_n777_ragged", 777, 500.0, 204, (0.01, 1.0, 30.0, 0.3, 24.0, 0.05, 0.2, 0.1, 0.3)),
]
MIX_FULL = (0.01, 1.0, 30.0, 0.3, 24.0, 0.05, 0.2, 0.1, 0.3)  # the 85k workload's mixture vector


def write_mix():
    out = {"source": "oracle/ (FP64, mixture of triggering functions), written by tests/golden/make_golden.py --mix",
           "param_order": ["mu0", "tau_x", "tau_t", "theta_1", "omega_1", "h_1", "theta_2", "omega_2", "h_2"],
           "cases": []}
    for name, n, T, seed, th in MIX_CASES:
        ev = synth.simulate(n, T, seed=seed)
        case = {"name": name, "n": n, "T": T, "seed": seed, "theta": list(th),
                "x": ev.x.tolist(), "y": ev.y.tolist(), "t": ev.t.tolist()}
        for key, e in (("f64", ev), ("f32in", ev.rounded32())):
            ll, g = oracle.loglik_mix(e.x, e.y, e.t, th, grad=True)
            case[key] = {"loglik": float(ll), "grad": [float(v) for v in g]}
        out["cases"].append(case)
    ev = synth.large_workload()
    t0 = time.time()
    ll, g = oracle.loglik_mix(ev.x, ev.y, ev.t, MIX_FULL, grad=True)
    out["full_85k"] = {"workload": {"generator": "synth.large_workload", "n": int(ev.n), "seed": 20051,
                                    "sha256_xyt_f64le": events_digest(ev)},
                       "theta": list(MIX_FULL), "loglik": float(ll), "grad": [float(v) for v in g]}
    print("mix 85k", ll, f"{time.time() - t0:.1f} s", flush=True)
    path = os.path.join(HERE, "mix_cases.json")
    with open(path, "w") as fh:
        head = {k: v for k, v in out.items() if k != "cases"}
        fh.write("{\n" + ",\n".join(f" {json.dumps(k)}: {json.dumps(v)}" for k, v in head.items()))
        fh.write(',\n "cases": [\n' + ",\n".join("  " + json.dumps(c) for c in out["cases"]) + "\n ]\n}\n")
    print("wrote", path, len(out["cases"]), "cases")


def write_full():
    ev = synth.large_workload()
    batch = synth.theta_batch(BATCH_K, seed=BATCH_SEED)
    thetas = [("theta0", tuple(synth.THETA0)), ("theta_b", THETA_B)]
    thetas += [(f"batch{BATCH_SEED}_{k}", tuple(float(v) for v in batch[k])) for k in BATCH_PICK]
    out = {"source": "oracle/ (FP64, Section 2.1 Eq. 1 and its gradient), written by "
                     "tests/golden/make_golden.py --full",
           "param_order": list(oracle.PARAM_NAMES),
           "workload": {"generator": "synth.large_workload", "n": int(ev.n), "T": 5000.0, "seed": 20051,
                        "rounded32": True, "sha256_xyt_f64le": events_digest(ev)},
           "threads": oracle.default_threads(), "cases": []}
    rows = np.arange(ev.n, dtype=np.int64)
    for name, th in thetas:
        t0 = time.time()
        r = oracle.rows(ev.x, ev.y, ev.t, th, rows, grad=True)
        # per-event gradient terms d ell_n / d Theta = (d lambda_n / d Theta) / lambda_n - d Lambda_n / d Theta;
        # their absolute sums are the scale against which a nearly cancelling component's error is stated
        terms = r["dlam"] / r["lam"][:, None] - r["dLambda"]
        case = {"name": name, "theta": [float(v) for v in th], "loglik": float(r["ell_sum"]),
                "grad": [float(v) for v in r["grad_sum"]],
                "grad_abs_sum": [float(v) for v in np.sum(np.abs(terms), axis=0)],
                "loglik_abs_sum": float(np.sum(np.abs(r["ell_n"])))}
        out["cases"].append(case)
        print(name, case["loglik"], f"{time.time() - t0:.1f} s", flush=True)
    path = os.path.join(HERE, "full_85k.json")
    with open(path, "w") as fh:
        head = {k: v for k, v in out.items() if k != "cases"}
        fh.write("{\n" + ",\n".join(f" {json.dumps(k)}: {json.dumps(v)}" for k, v in head.items()))
        fh.write(',\n "cases": [\n' + ",\n".join("  " + json.dumps(c) for c in out["cases"]) + "\n ]\n}\n")
    print("wrote", path, len(out["cases"]), "cases")


def main():
    if "--full" in sys.argv:
        write_full()
    elif "--mix" in sys.argv:
        write_mix()
    else:
        write_small()


if __name__ == "__main__":
    main()
