"""Regression record of the FP64 oracle (tests/golden/oracle_dcpfphd_small.json,
written by tests/golden/make_golden.py, which calls only the oracle): a small
DCPFPHD run (Algorithm 1, Steps 1-6) recomputed and compared value by value,
so any change to the oracle's arithmetic shows here."""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "golden"))

import make_golden  # noqa: E402


def test_oracle_matches_its_regression_record():
    with open(os.path.join(HERE, "golden", "oracle_dcpfphd_small.json")) as fh:
        ref = json.load(fh)
    assert ref["seed"] == make_golden.SEED and ref["steps"] == make_golden.STEPS
    got = make_golden.run()
    assert len(got) == len(ref["record"])
    n_labels = 0
    for g, r in zip(got, ref["record"]):
        assert g["scan"] == r["scan"] and g["M"] == r["M"]
        for a, b in zip(g["C_local"], r["C_local"]):
            np.testing.assert_allclose(a, b, rtol=1e-12, atol=0)
        np.testing.assert_allclose(g["N"], r["N"], rtol=1e-12)
        assert g["local_labels"] == r["local_labels"]
        assert g["fused_labels"] == r["fused_labels"]
        np.testing.assert_allclose(np.asarray(g["fused_states"]).reshape(-1),
                                   np.asarray(r["fused_states"]).reshape(-1), rtol=1e-12, atol=1e-9)
        assert g["resample_counts"] == r["resample_counts"]
        assert g["parents_head"] == r["parents_head"]
        n_labels += len(r["fused_labels"])
    assert n_labels >= 6   # the record exercises fusion
