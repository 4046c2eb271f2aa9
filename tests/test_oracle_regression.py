"""The CPU oracle against its own stored outputs (written by
tests/golden/make_oracle_regression.py from the oracle alone): a change to
the oracle's arithmetic shows up here and has to be justified by the paper
passage, or the reading of it, that calls for it."""
import json
import os

import numpy as np
import pytest

from tests.golden import make_oracle_regression as gen


@pytest.fixture(scope="module")
def stored():
    with open(os.path.join(gen.HERE, "oracle_regression.json")) as f:
        return json.load(f)


@pytest.mark.parametrize("name", ["gaussian_2x12", "clustered_2x20"])
def test_oracle_outputs_are_unchanged(oracle_lib, stored, name):
    box = gen.cases()[name]
    got = gen.evaluate(box)
    want = stored[name]
    assert set(got) == set(want)
    for k, v in want.items():
        # summation orders are fixed; the tolerance only absorbs libm differences between hosts
        np.testing.assert_allclose(np.asarray(got[k]), np.asarray(v), rtol=1e-11, atol=1e-13, err_msg=k)
