"""Pins of the CPU oracle against facts the paper and the mathematics fix.

Each ``pin_*`` function raises AssertionError on a violation; the tests call
them directly, and ``test_planted_mistakes_are_caught`` re-runs them with a
deliberate mistake planted in the oracle's arithmetic to show that the pins
would notice a dropped term, a lost sign or a transposed operand.
"""
from fractions import Fraction

import numpy as np
import pytest
import scipy.linalg

import oracle
from conftest import EPS, load_golden
from paper_1612_01855_gb300 import inputs


# ---------------------------------------------------------------- helpers
def exact_solve(L, B):
    """Exact rational forward substitution (Python Fractions)."""
    n, k = B.shape
    Lf = [[Fraction(float(L[i, j])) for j in range(n)] for i in range(n)]
    X = [[Fraction(0)] * k for _ in range(n)]
    for c in range(k):
        for j in range(n):
            s = Fraction(float(B[j, c]))
            for l in range(j):
                s -= Lf[j][l] * X[l][c]
            X[j][c] = s / Lf[j][j]
    return X


def exact_inverse(L):
    n = L.shape[0]
    return exact_solve(L, np.eye(n))


def int_unit_lower(rng, n, lo=-3, hi=3):
    L = np.tril(rng.integers(lo, hi + 1, size=(n, n)).astype(np.float64), -1)
    L[np.arange(n), np.arange(n)] = 1.0
    return L


def rel_err(A, B):
    return np.max(np.abs(A - B)) / max(np.max(np.abs(B)), 1e-300)


# ---------------------------------------------------------------- pins
def pin_golden_worked_example():
    g = load_golden("worked_example_4x4.txt")
    X = oracle.forward_subst(g["L"], g["B"])
    assert np.array_equal(X, g["X"]), X
    for base in (1, 2, 4):
        Li = oracle.rec_tri_inv(g["L"], base=base)
        assert np.array_equal(Li, g["Linv"]), (base, Li)
    assert np.array_equal(oracle.tri_inv_columns(g["L"]), g["Linv"])
    Lt = oracle.diagonal_inverter(g["L"], 2, base=1)
    assert np.array_equal(Lt, g["Ltilde_n0_2"]), Lt
    for n0 in (1, 2, 3, 4):
        assert np.array_equal(oracle.it_inv_trsm(g["L"], g["B"], n0, base=1), g["X"]), n0
        assert np.array_equal(oracle.rec_trsm(g["L"], g["B"], n0), g["X"]), n0


def pin_integer_exact_solves():
    """Unit lower-triangular integer L and integer X: every intermediate is
    an integer, so each algorithm must return X bit for bit (brute force on
    n <= 8 against exact integer arithmetic)."""
    rng = np.random.default_rng(11)
    for n in range(1, 9):
        L = int_unit_lower(rng, n)
        Xt = rng.integers(-4, 5, size=(n, 3)).astype(np.float64)
        B = (L.astype(np.int64) @ Xt.astype(np.int64)).astype(np.float64)
        assert np.array_equal(oracle.forward_subst(L, B), Xt), n
        for n0 in range(1, n + 1):
            assert np.array_equal(oracle.it_inv_trsm(L, B, n0, base=1), Xt), (n, n0)
            assert np.array_equal(oracle.rec_trsm(L, B, n0), Xt), (n, n0)


def pin_integer_exact_inverse():
    """L^-1 of a unit lower-triangular integer matrix is an integer matrix;
    compare RecTriInv (every base case size) with exact rational inversion."""
    rng = np.random.default_rng(12)
    for n in (1, 2, 3, 5, 8, 12):
        L = int_unit_lower(rng, n, -2, 2)
        Linv = np.array([[float(v) for v in row] for row in exact_inverse(L)])
        assert np.array_equal(oracle.tri_inv_columns(L), Linv), n
        for base in (1, 2, 3, 16):
            assert np.array_equal(oracle.rec_tri_inv(L, base=base), Linv), (n, base)


def pin_rational_brute_force():
    """General (non-unit, dyadic) L with n <= 8 against exact Fractions:
    forward error within the classical bound for substitution."""
    rng = np.random.default_rng(13)
    for n in range(1, 9):
        L = np.tril(rng.integers(-8, 9, size=(n, n)) / 8.0, -1)
        L[np.arange(n), np.arange(n)] = rng.choice([-2.0, -1.5, 1.0, 1.25, 3.0], size=n)
        B = rng.integers(-16, 17, size=(n, 2)) / 4.0
        Xe = exact_solve(L, B)
        Xe_f = np.array([[float(v) for v in row] for row in Xe])
        for X in (oracle.forward_subst(L, B), oracle.it_inv_trsm(L, B, 2, base=1),
                  oracle.rec_trsm(L, B, 2)):
            err = np.abs(X - Xe_f)
            # |X| |L^-1| |L| style bound: loose but far below any real mistake
            assert np.all(err <= 64 * n * EPS * (np.abs(Xe_f) + 1.0)), (n, err.max())


def pin_diagonal_closed_form():
    """Diagonal L: X = D^-1 B, one correctly rounded division per entry."""
    rng = np.random.default_rng(14)
    n, k = 37, 5
    d = rng.uniform(0.5, 3.0, size=n)
    L = np.diag(d)
    B = rng.uniform(-1, 1, size=(n, k))
    assert np.array_equal(oracle.forward_subst(L, B), B / d[:, None])
    assert np.array_equal(oracle.it_inv_trsm(L, B, 8, base=4), (1.0 / d)[:, None] * B)


def pin_bidiagonal_closed_form():
    """Unit lower-bidiagonal L with sub-diagonal -a: (L^-1)_ij = a^(i-j) for
    i >= j.  With a = 1/2 or a = 3 every power is exact in FP64."""
    for a, n in ((0.5, 40), (3.0, 20)):
        L = np.eye(n) - a * np.eye(n, k=-1)
        i, j = np.indices((n, n))
        expect = np.where(i >= j, a ** (i - j).astype(np.float64), 0.0)
        assert np.array_equal(oracle.tri_inv_columns(L), expect)
        for base in (1, 2, 7, 16):
            assert np.array_equal(oracle.rec_tri_inv(L, base=base), expect), (a, base)
        for n0 in (1, 4, 13, n):
            Lt = oracle.diagonal_inverter(L, n0, base=2)
            for s in range(0, n, n0):
                m = min(n0, n - s)
                assert np.array_equal(Lt[s:s + m, s:s + m], expect[:m, :m]), (a, n0, s)


def pin_ones_closed_form():
    """All-ones lower-triangular L: L^-1 has 1 on the diagonal and -1 on the
    first sub-diagonal, zero elsewhere."""
    n = 33
    L = np.tril(np.ones((n, n)))
    expect = np.eye(n) - np.eye(n, k=-1)
    assert np.array_equal(oracle.tri_inv_columns(L), expect)
    for base in (1, 4, 16):
        assert np.array_equal(oracle.rec_tri_inv(L, base=base), expect), base


def pin_lapack_agreement():
    """Forward substitution agrees with LAPACK dtrtrs (scipy) on the
    well-conditioned workload."""
    L, B = inputs.well_conditioned(300, 7, seed=3)
    X = oracle.forward_subst(L, B)
    Xl = scipy.linalg.solve_triangular(L, B, lower=True)
    assert rel_err(X, Xl) < 1e-14


def pin_inverse_residual():
    """L_bb L_bb^-1 = I for every diagonal block (Diagonal-Inverter's
    postcondition), within a small multiple of n0 eps."""
    L = inputs.well_conditioned_L(200, seed=4)
    for n0 in (16, 64, 200):
        Lt = oracle.diagonal_inverter(L, n0, base=8)
        for s in range(0, 200, n0):
            m = min(n0, 200 - s)
            R = L[s:s + m, s:s + m] @ Lt[s:s + m, s:s + m] - np.eye(m)
            assert np.max(np.abs(R)) < 4 * m * EPS, (n0, s, np.max(np.abs(R)))


def pin_n0_family_equivalence():
    """Every block size gives the same X: n0 = 1 is substitution, n0 = n is
    full inversion (the two classical endpoints of the method)."""
    L, B = inputs.well_conditioned(97, 5, seed=5)
    X = oracle.forward_subst(L, B)
    for n0 in (1, 2, 7, 16, 32, 64, 96, 97, 200):
        assert rel_err(oracle.it_inv_trsm(L, B, n0, base=8), X) < 1e-14, n0
        assert rel_err(oracle.rec_trsm(L, B, n0), X) < 1e-14, n0


def pin_backward_error():
    """||L X - B|| / (||L|| ||X||) <= 10 n eps (triangular solves, and
    solves with inverted triangular blocks, are backward stable)."""
    n = 512
    L, B = inputs.well_conditioned(n, 16, seed=0)
    for X in (oracle.forward_subst(L, B), oracle.it_inv_trsm(L, B, 64, base=16)):
        r = np.linalg.norm(L @ X - B, np.inf) / (np.linalg.norm(L, np.inf) * np.linalg.norm(X, np.inf))
        assert r <= 10 * n * EPS, r


def pin_independent_columns():
    """A column of X depends only on the same column of B (the independent
    split): solving a subset of columns reproduces them bit for bit."""
    L, B = inputs.well_conditioned(150, 9, seed=6)
    X = oracle.forward_subst(L, B)
    cols = [0, 4, 8]
    assert np.array_equal(oracle.forward_subst_columns(L, B, cols), X[:, cols])


def pin_flop_counts():
    """Multiply-add counts of the It-Inv loop against the paper's flop
    formulas (two flops per multiply-add): update F_Upd = (n - n0) k n
    exactly when n0 divides n; solve = n (n0 + 1) k, whose leading term is
    F_Solve = n n0 k."""
    for n, n0, k in ((96, 16, 3), (64, 8, 5), (40, 40, 2)):
        L, B = inputs.well_conditioned(n, k, seed=7)
        _, (cs, cu) = oracle.it_inv_trsm(L, B, n0, base=4, return_counts=True)
        assert 2 * cu == (n - n0) * k * n, (n, n0, cu)
        assert 2 * cs == n * (n0 + 1) * k, (n, n0, cs)


def pin_double_double():
    """Double-double substitution is accurate far beyond FP64 on an
    ill-conditioned dyadic system (exact reference by Fractions)."""
    rng = np.random.default_rng(15)
    n = 14
    L = np.tril(rng.integers(-8, 9, size=(n, n)) / 8.0, -1)
    L[np.arange(n), np.arange(n)] = rng.choice([1.0 / 64, -1.0 / 32, 1.0 / 16], size=n)
    B = rng.integers(-8, 9, size=(n, 2)) / 8.0
    Xe = exact_solve(L, B)
    hi, lo = oracle.forward_subst_dd(L, B)
    for i in range(n):
        for c in range(2):
            got = Fraction(float(hi[i, c])) + Fraction(float(lo[i, c]))
            ex = Xe[i][c]
            assert abs(got - ex) <= Fraction(1, 10 ** 25) * max(abs(ex), Fraction(1)), (i, c)


PINS = [pin_golden_worked_example, pin_integer_exact_solves, pin_integer_exact_inverse,
        pin_rational_brute_force, pin_diagonal_closed_form, pin_bidiagonal_closed_form,
        pin_ones_closed_form, pin_lapack_agreement, pin_inverse_residual,
        pin_n0_family_equivalence, pin_backward_error, pin_independent_columns,
        pin_flop_counts, pin_double_double]


@pytest.mark.parametrize("pin", PINS, ids=[p.__name__ for p in PINS])
def test_pin(pin):
    pin()


@pytest.mark.parametrize("mutation", [1, 2, 3])
def test_planted_mistakes_are_caught(mutation):
    """Each planted mistake (lost sign in RecTriInv, transposed L22^-1,
    dropped substitution term) must make at least one pin fail."""
    caught = []
    oracle.set_mutation(mutation)
    try:
        for pin in PINS:
            try:
                pin()
            except (AssertionError, oracle.OracleError):
                caught.append(pin.__name__)
    finally:
        oracle.set_mutation(0)
    assert caught, f"mutation {mutation} went unnoticed"


def test_oracle_argument_errors():
    with pytest.raises(oracle.OracleError):
        oracle.forward_subst(np.diag([1.0, 0.0, 2.0]), np.ones((3, 1)))
    with pytest.raises(oracle.OracleError):
        oracle.it_inv_trsm(np.eye(4), np.ones((4, 1)), 0)


def test_oracle_threads_reported():
    assert oracle.max_threads() >= 1
