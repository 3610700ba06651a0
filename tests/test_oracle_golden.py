"""The oracle still reproduces its frozen regression fixtures (tests/golden/)."""
import os

import pytest

from tests.golden.make_golden import CASES, HERE, compute, render


@pytest.mark.parametrize("name,recipe,n,params", CASES, ids=[c[0] for c in CASES])
def test_golden(name, recipe, n, params):
    with open(os.path.join(HERE, name)) as f:
        want = f.read().split("\n", 1)[1]
    assert render(compute(recipe, n, params)) == want
