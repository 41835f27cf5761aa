"""The pivot-growth rule of the library's factorisation check, on the CPU: the growth
max|U| / max|A| of an LU without pivoting, on matrices whose growth is known, and on the
oracle's local matrices of the method (Eq. 3.3; ImpRAS box matrices, Sec. 6.3), where
coercivity (Lemma 2.2) keeps the pivots away from zero and the growth stays far below the
library's default limits (1e6 for c64 factors, 1e12 for c128)."""
import numpy as np
import pytest

from oracle.problem import Problem as OracleProblem
from parity import nopivot_growth


def test_known_growth():
    e = 1e-3
    # [[e, 1], [1, 1]]: U22 = 1 - 1/e, the classic growth of elimination without pivoting
    assert abs(nopivot_growth(np.array([[e, 1.0], [1.0, 1.0]])) - (1 / e - 1)) <= 1e-9 / e
    assert nopivot_growth(3.0 * np.eye(4)) == 1.0
    # Wilkinson's matrix (1 on the diagonal and the last column, -1 below): growth 2^(n-1)
    n = 12
    W = np.tril(-np.ones((n, n)), -1) + np.eye(n)
    W[:, -1] = 1.0
    assert nopivot_growth(W) == 2.0 ** (n - 1)
    # a diagonally dominant matrix: growth at most 2 (Wilkinson)
    rng = np.random.default_rng(3)
    D = rng.standard_normal((30, 30)) + 1j * rng.standard_normal((30, 30))
    D += np.diag(np.abs(D).sum(axis=1) + 1.0)
    assert nopivot_growth(D) <= 2.0


@pytest.mark.parametrize("xi_prec,bc", [(4.0, "pec"), (16.0, "pec"), (0.0, "imp"), (4.0, "imp")])
def test_method_minors_grow_little(xi_prec, bc):
    O = OracleProblem(6, 4.0, 0.0, xi_prec, 3, 1, bc=bc)
    g = [nopivot_growth(O.dd.minor(l).toarray()) for l in range(len(O.dd.idx))]
    assert 0.1 < min(g) and max(g) < 1e3, (min(g), max(g))
