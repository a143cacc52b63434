"""Pins for the oracle's transformation matrices (Sec. II B, Eq. 12, App. A).

The oracle builds M from the basis formulas (Eqs. 7-10) and inverts it with
numpy; these tests hold both against what the paper prints.
"""

from fractions import Fraction

import numpy as np

from conftest import read_matrix, read_values
from oracle import lbm_oracle as L


def _exact_product(A, B):
    n, k, m = len(A), len(B), len(B[0])
    return [[sum((A[i][t] * B[t][j] for t in range(k)), Fraction(0)) for j in range(m)] for i in range(n)]


def test_nonorth_matrix_equals_printed_eq12():
    printed = np.array([[float(v) for v in r] for r in read_matrix("nonorth_M_eq12.txt")])
    assert printed.shape == (19, 19)
    assert np.array_equal(L.nonorth_matrix(), printed)


# As printed, rows 13 and 14 of App. A carry their m_8 coefficient (-1/4) one
# column early, under m_7.  The paper defines the matrix as the inverse of
# Eq. 12; with those two entries moved to column 8 it is that inverse exactly.
MISPLACED = [(13, 7, 8), (14, 7, 8)]


def _corrected_appendix_a():
    Minv = read_matrix("nonorth_Minv_appA.txt")
    for row, printed_col, true_col in MISPLACED:
        assert Minv[row][printed_col] == Fraction(-1, 4) and Minv[row][true_col] == 0
        Minv[row][true_col], Minv[row][printed_col] = Minv[row][printed_col], Fraction(0)
    return Minv


def test_printed_inverse_is_exact_inverse_after_two_column_fixes():
    M = read_matrix("nonorth_M_eq12.txt")
    ident = [[Fraction(int(i == j)) for j in range(19)] for i in range(19)]
    assert _exact_product(M, read_matrix("nonorth_Minv_appA.txt")) != ident
    Minv = _corrected_appendix_a()
    assert _exact_product(M, Minv) == ident
    assert _exact_product(Minv, M) == ident


def test_oracle_inverse_matches_appendix_a():
    corrected = np.array([[float(v) for v in r] for r in _corrected_appendix_a()])
    assert np.max(np.abs(L.inverse(L.nonorth_matrix()) - corrected)) < 1e-14
    printed = np.array([[float(v) for v in r] for r in read_matrix("nonorth_Minv_appA.txt")])
    bad = np.argwhere(np.abs(L.inverse(L.nonorth_matrix()) - printed) > 1e-14)
    assert sorted(map(tuple, bad)) == [(13, 7), (13, 8), (14, 7), (14, 8)]


def test_nonzero_counts():
    vals = read_values("paper_values.txt")
    M, Mo = L.nonorth_matrix(), L.orth_matrix()
    assert np.count_nonzero(M) == vals["nnz_nonorth_M"]
    assert np.count_nonzero(Mo) == vals["nnz_orth_M"]
    assert np.count_nonzero(np.abs(L.inverse(Mo)) > 1e-13) == vals["nnz_orth_Minv"]
    # The printed App. A matrix has 99 non-zeros; Sec. II B quotes 96.  The
    # printed matrix is the exact inverse (test above), so 99 is the count.
    printed = read_matrix("nonorth_Minv_appA.txt")
    nnz = sum(1 for r in printed for v in r if v != 0)
    assert nnz == 99 and vals["nnz_nonorth_Minv_quoted"] == 96


def test_orth_rows_mutually_orthogonal_with_dhumieres_norms():
    Mo = L.orth_matrix()
    gram = Mo @ Mo.T
    assert np.array_equal(gram, np.diag(np.diag(gram)))
    norms = [19, 2394, 252, 10, 40, 10, 40, 10, 40, 36, 72, 12, 24, 4, 4, 4, 8, 8, 8]
    assert np.array_equal(np.diag(gram), np.array(norms, dtype=float))
    # orthogonal rows: M^-1 = M^T diag(1/|row|^2)
    assert np.max(np.abs(L.inverse(Mo) - Mo.T / np.array(norms, float))) < 1e-15


def test_velocities_are_the_d3q19_set():
    e = L.E
    assert e.shape == (19, 3)
    assert len({tuple(r) for r in e}) == 19
    n2 = (e * e).sum(axis=1)
    assert list(n2) == [0] + [1] * 6 + [2] * 12
    # directions come in opposite pairs (1,2), (3,4), ..., (17,18)
    for a in range(1, 19, 2):
        assert np.array_equal(e[a], -e[a + 1])


def test_rest_state_is_lattice_weights_for_both_operators():
    rho = np.array([0.7, 1.3])
    for op in ("nonorth", "orth"):
        f = L.equilibrium_state(L.Params(operator=op), rho)
        want = np.multiply.outer(np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12), rho)
        assert np.max(np.abs(f - want)) < 1e-15
