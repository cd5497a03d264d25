"""The oracle still reproduces its recorded configuration-0 output."""
import json
import os

import numpy as np

from tests.golden.make_golden import compute

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def test_cfg0_golden_record():
    with open(os.path.join(HERE, "cfg0_oracle.json")) as f:
        ref = json.load(f)
    got = compute()
    assert got["n_pairs"] == ref["n_pairs"]
    assert got["keys_sha256"] == ref["keys_sha256"]
    assert got["pixels"] == ref["pixels"]
    np.testing.assert_allclose(got["rgba"], ref["rgba"], atol=1e-12)
    np.testing.assert_allclose(got["mean_rgba"], ref["mean_rgba"], atol=1e-12)
