"""Stored oracle values of the trigger mixture (tests/golden/mix_cases.json, written by
tests/golden/make_golden.py --mix from oracle/ alone): the oracle must keep reproducing them; the
CUDA path (tests/test_gpu_mixture.py) is compared with them."""
import json
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "mix_cases.json")


def load_cases():
    with open(GOLDEN) as fh:
        return json.load(fh)["cases"]


@pytest.mark.parametrize("case", load_cases(), ids=lambda c: c["name"])
def test_oracle_reproduces_mixture_golden(case):
    x, y, t = (np.asarray(case[k], dtype=np.float64) for k in ("x", "y", "t"))
    r = lambda a: a.astype(np.float32).astype(np.float64)
    for key, (xx, yy, tt) in (("f64", (x, y, t)), ("f32in", (r(x), r(y), r(t)))):
        ll, g = oracle.loglik_mix(xx, yy, tt, case["theta"], grad=True)
        want = case[key]
        assert abs(ll - want["loglik"]) <= 1e-12 * max(1.0, abs(want["loglik"])), (key, ll, want["loglik"])
        np.testing.assert_allclose(g, want["grad"], rtol=1e-11, atol=1e-11 * max(1.0, np.max(np.abs(want["grad"]))))
