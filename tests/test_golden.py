"""Stored values (tests/golden/): the configuration values the paper prints, as this
repository's inputs, and regression values of the oracle on tiny cases (written by
tests/golden/make_oracle_regression.py, which calls only the oracle)."""
import json
import os

import numpy as np

import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _load(name):
    with open(os.path.join(GOLDEN, name)) as fh:
        return json.load(fh)


def test_paper_subdomain_shape_is_the_printed_one():
    g = _load("paper_values.json")
    nx, ny, nz = g["weak_scaling_subdomain_cells"]["value"]
    assert synth.cfg_paper_shape().shape == (nz, ny, nx)


def _close(a, b, rtol=1e-9):
    a, b = np.asarray(a, dtype=float), np.asarray(b, dtype=float)
    return np.allclose(a, b, rtol=rtol, atol=rtol * max(1e-30, float(np.max(np.abs(b)))))


def test_oracle_regression_values():
    import importlib.util
    spec = importlib.util.spec_from_file_location("make_oracle_regression",
                                                  os.path.join(GOLDEN, "make_oracle_regression.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    now, stored = mod.compute(), _load("oracle_regression.json")
    for case in stored:
        for key, val in stored[case].items():
            got = now[case][key]
            if isinstance(val, int):
                assert got == val, (case, key)
            else:
                assert _close(got, val), (case, key, got, val)
