"""Pins of the update-chain oracle (Sec. 5 Eigen benchmark, stable form
X_{k+1} = X_k + c X_k A with X_0 = I and c = 1/(N T)).

Every check here compares the oracle with something other than itself:
a hand-worked example, closed forms, exact rational arithmetic, a different
algorithm (binary powering in extended precision), or an algebraic identity.
"""
from fractions import Fraction
import math

import numpy as np
import pytest

import oracle
import synth
from conftest import read_golden

EPS = np.finfo(np.float64).eps


def relF(x, ref):
    return float(np.linalg.norm(x - ref) / np.linalg.norm(ref))


def test_hand_worked_example_bit_exact():
    g = read_golden("chain_n2_t2.txt")
    n, T = int(g["n"][0]), int(g["T"][0])
    A = np.array([float(v) for v in g["A"]]).reshape(1, n, n)
    X = oracle.update_chain(A, T)
    np.testing.assert_array_equal(X.ravel(), np.array([float(v) for v in g["X"]]))


@pytest.mark.parametrize("n,T", [(1, 1), (3, 5), (8, 64), (17, 7)])
def test_zero_input_gives_identity_exactly(n, T):
    X = oracle.update_chain(np.zeros((3, n, n)), T)
    for b in range(3):
        np.testing.assert_array_equal(X[b], np.eye(n))


@pytest.mark.parametrize("n,T", [(1, 1), (2, 100), (8, 64), (5, 128)])
def test_identity_input_closed_form(n, T):
    X = oracle.update_chain(np.eye(n)[None].repeat(2, 0), T)
    c = 1.0 / (n * T)
    expect = math.pow(1.0 + c, T)
    for b in range(2):
        off = X[b] - np.diag(np.diag(X[b]))
        assert np.all(off == 0.0)
        assert np.all(np.abs(np.diag(X[b]) - expect) <= 4 * T * EPS * expect)


@pytest.mark.parametrize("n,T", [(4, 16), (12, 64)])
def test_diagonal_input_closed_form(n, T):
    a = synth.uniform_np(0x51, 0, n)
    X = oracle.update_chain(np.diag(a)[None], T)[0]
    c = 1.0 / (n * T)
    expect = np.array([math.pow(1.0 + c * ai, T) for ai in a])
    assert np.all(X - np.diag(np.diag(X)) == 0.0)
    assert np.all(np.abs(np.diag(X) - expect) <= (4 * T + 4) * EPS * np.abs(expect))


def _binary_power_longdouble(M, T):
    """(M)^T by repeated squaring in extended precision -- a different algorithm."""
    M = M.astype(np.longdouble)
    R = np.eye(M.shape[0], dtype=np.longdouble)
    while T:
        if T & 1:
            R = R @ M
        M = M @ M
        T >>= 1
    return R


@pytest.mark.parametrize("n,T", [(3, 64), (8, 100), (16, 64), (32, 64)])
def test_closed_form_binary_powering(n, T):
    A = synth.chain_inputs_np(0xC1A2, 4, n)
    X = oracle.update_chain(A, T)
    c = 1.0 / (n * T)
    for b in range(4):
        ref = _binary_power_longdouble(np.eye(n) + np.longdouble(c) * A[b].astype(np.longdouble), T)
        assert relF(X[b].astype(np.longdouble), ref) <= 1e-13


def _exact_binomial(Af, c, T):
    """X_T = sum_j C(T,j) c^j A^j in exact rationals."""
    n = len(Af)
    I = [[Fraction(int(i == j)) for j in range(n)] for i in range(n)]

    def mul(P, Q):
        return [[sum(P[i][l] * Q[l][j] for l in range(n)) for j in range(n)] for i in range(n)]

    out = [[Fraction(0)] * n for _ in range(n)]
    P = I
    for j in range(T + 1):
        coef = Fraction(math.comb(T, j)) * c ** j
        for r in range(n):
            for s in range(n):
                out[r][s] += coef * P[r][s]
        P = mul(P, Af)
    return out


@pytest.mark.parametrize("n", [1, 2, 3, 4])
def test_exact_rational_brute_force(n):
    T = 6
    A = synth.chain_inputs_np(0xB0, 1, n)
    c_fl = 1.0 / (n * T)
    Af = [[Fraction(float(A[0, i, j])) for j in range(n)] for i in range(n)]
    ref = _exact_binomial(Af, Fraction(c_fl), T)
    X = oracle.update_chain(A, T)[0]
    ref_np = np.array([[float(v) for v in row] for row in ref])
    assert relF(X, ref_np) <= 1e-14


@pytest.mark.parametrize("n,T", [(5, 64), (24, 64), (64, 128)])
def test_commutation(n, T):
    A = synth.chain_inputs_np(0xC0, 2, n)
    X = oracle.update_chain(A, T)
    for b in range(2):
        lhs = X[b] @ A[b] - A[b] @ X[b]
        assert np.linalg.norm(lhs) <= 1e-13 * np.linalg.norm(A[b]) * np.linalg.norm(X[b])


@pytest.mark.parametrize("n", [3, 7, 16])
def test_column_major_layout_bit_exact(n):
    A_row = synth.chain_inputs_np(0xC1A2, 5, n, layout=0)
    A_col = synth.chain_inputs_np(0xC1A2, 5, n, layout=1)
    np.testing.assert_array_equal(A_col, A_row.transpose(0, 2, 1))
    X_row = oracle.update_chain(A_row, 64, layout=0)
    X_col = oracle.update_chain(A_col, 64, layout=1)
    np.testing.assert_array_equal(X_col.transpose(0, 2, 1), X_row)


def test_threads_do_not_change_results():
    A = synth.chain_inputs_np(0xC1A1, 64, 8)
    np.testing.assert_array_equal(oracle.update_chain(A, 100, nthreads=1),
                                  oracle.update_chain(A, 100, nthreads=4))


def test_uneven_pool_matches_per_size_calls():
    n, t = synth.uneven_sizes(0xC1A4, 40)
    pool, off = synth.uneven_inputs_np(0xC1A4, n)
    X = oracle.update_chain_uneven(n, t, off, pool)
    for k in range(0, 40, 7):
        nk = int(n[k])
        a = pool[off[k]:off[k] + nk * nk].reshape(1, nk, nk)
        np.testing.assert_array_equal(X[off[k]:off[k] + nk * nk].reshape(nk, nk),
                                      oracle.update_chain(a, int(t[k]))[0])


def test_invalid_arguments_rejected():
    with pytest.raises(ValueError):
        oracle.update_chain(np.zeros((1, 2, 2)), 0)
    with pytest.raises(ValueError):
        oracle.update_chain(np.zeros((1, 2, 2)), 4, layout=2)


def test_paper_eigen_recurrence_exact_small():
    """Listing eigen1's literal loop M = Ones + 5e-5 (M + M M), M(i,j) = i + n j."""
    n, rep = 2, 3
    h = Fraction(5e-5)            # the double nearest 5e-5, as the C literal
    M = [[Fraction(i + n * j) for j in range(n)] for i in range(n)]
    for _ in range(rep):
        Q = [[sum(M[i][l] * M[l][j] for l in range(n)) for j in range(n)] for i in range(n)]
        M = [[1 + h * (M[i][j] + Q[i][j]) for j in range(n)] for i in range(n)]
    ref = np.array([[float(v) for v in r] for r in M])
    assert relF(oracle.eigen_bench(n, rep), ref) <= 1e-15


@pytest.mark.parametrize("n,rep", [(1, 3), (2, 2), (3, 2)])
def test_eigen_recurrence_batched_exact_small(n, rep):
    """The batched form against exact rational arithmetic on random integer
    starts (each step: Q = M M, then M = 1 + c (M + Q) with the double nearest
    the given c)."""
    rng = np.random.default_rng(n * 10 + rep)
    M0 = rng.integers(-4, 5, size=(3, n, n)).astype(np.float64)
    h = Fraction(3e-3)
    got = oracle.eigen_recurrence(M0, rep, 3e-3)
    for b in range(3):
        M = [[Fraction(int(M0[b, i, j])) for j in range(n)] for i in range(n)]
        for _ in range(rep):
            Q = [[sum(M[i][l] * M[l][j] for l in range(n)) for j in range(n)] for i in range(n)]
            M = [[1 + h * (M[i][j] + Q[i][j]) for j in range(n)] for i in range(n)]
        ref = np.array([[float(v) for v in r] for r in M])
        assert relF(got[b], ref) <= 1e-15


def test_eigen_recurrence_special_cases():
    """Zero repeats copy the start; c = 0 gives Ones after one step exactly;
    the listing's start reproduces the literal single-matrix loop bit for bit."""
    M0 = synth.uniform_np(7, 0, 2 * 5 * 5).reshape(2, 5, 5)
    np.testing.assert_array_equal(oracle.eigen_recurrence(M0, 0), M0)
    np.testing.assert_array_equal(oracle.eigen_recurrence(M0, 1, 0.0), np.ones_like(M0))
    for n, rep in ((4, 5), (16, 3)):
        start = oracle.eigen_start(n)[None]
        np.testing.assert_array_equal(oracle.eigen_recurrence(start, rep)[0], oracle.eigen_bench(n, rep))
