"""The library's Gauss-Legendre rule (Section 2, eq. thetas), read back
through sht_plan_nodes, against the definition solved in 40-digit
arithmetic: the nodes are the zeros of P_n and the weights are
w = 2 / ((1 - x^2) P_n'(x)^2) at those zeros.  Independent of the oracle's
Newton iteration."""

import numpy as np
import pytest

from paper_0910_5435_gb300 import sht
from tests._exact import gl_root_and_weight


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


@pytest.mark.parametrize("l", [4, 64, 1024])
def test_nodes_and_weights_against_extended_precision(l):
    """Nodes to within two units in the last place.  Weights to n * 1.5e-15
    relative within 16 nodes of a pole, where the degree recurrence's
    rounding is amplified most, and to n * 1e-16 elsewhere (the recurrence's
    n roundings).  At n = 2048 the first bound is 3.1e-12: a recurrence with
    rounded square-root coefficients lands near 3e-11 there."""
    n = 2 * l
    P = sht.Plan(l, 1e-12, leaf_cols=max(2, min(64, l)), host_only=True)
    x, w = P.nodes()
    P.close()
    assert np.all(np.diff(x) > 0) and np.array_equal(x, -x[::-1]) and np.array_equal(w, w[::-1])
    sample = sorted({0, 1, 2, 3, 4, 5, 9, 15, 16, 40, n // 5, n // 3, l - 2, l - 1} & set(range(l)))
    for i in sample:
        r, wr = gl_root_and_weight(n, float(x[i]), digits=40, steps=5)
        assert abs(x[i] - float(r)) <= 2 * np.spacing(abs(x[i])), (i, x[i], float(r))
        bound = (1.5e-15 if i < 16 else 1e-16) * n
        assert abs(w[i] / float(wr) - 1) <= bound, (i, w[i], float(wr))
