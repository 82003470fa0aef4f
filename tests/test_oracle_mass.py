"""Pins of the mass-operator oracle (y_e = B^T diag(op_e) B x_e, B the
Kronecker product of the 1-D basis matrix B1): closed forms of the finite-
element mass matrix, identities, exact rationals, and an independent
sum-factorized evaluation."""
import itertools
from fractions import Fraction

import numpy as np
import pytest

import oracle


def kron_dim(B1, dim):
    B = B1
    for _ in range(dim - 1):
        B = np.kron(B1, B)
    return B


@pytest.mark.parametrize("dim", [1, 2, 3])
def test_identity_basis_and_unit_data_copy_x(dim):
    D = 4
    rng = np.random.default_rng(1)
    x = rng.uniform(-1, 1, (7, D ** dim))
    y = oracle.mass(np.eye(D), np.ones((7, D ** dim)), x, dim)
    np.testing.assert_array_equal(y, x)
    y3 = oracle.mass(np.eye(D), np.full((7, D ** dim), 3.0), x, dim)
    np.testing.assert_array_equal(y3, 3.0 * x)


def gauss_legendre(q):
    return np.polynomial.legendre.leggauss(q)


def lagrange_basis(nodes, pts):
    """B1[q][d] = phi_d(pts[q]) for the Lagrange polynomials on `nodes`."""
    B = np.ones((len(pts), len(nodes)))
    for d, xd in enumerate(nodes):
        for m, xm in enumerate(nodes):
            if m != d:
                B[:, d] *= (pts - xm) / (xd - xm)
    return B


@pytest.mark.parametrize("dim", [1, 2, 3])
def test_linear_element_mass_matrix_closed_form(dim):
    """Linear elements on [-1, 1]^dim with 2-point Gauss quadrature (exact for
    the degree-2 integrands): the 1-D mass matrix is [[2, 1], [1, 2]] / 3 and
    the dim-D one its Kronecker power."""
    xq, wq = gauss_legendre(2)
    B1 = lagrange_basis(np.array([-1.0, 1.0]), xq)
    w = kron_dim(wq[None, :], dim)[0]          # tensor quadrature weights, first index fastest
    M1 = np.array([[2.0, 1.0], [1.0, 2.0]]) / 3.0
    M = kron_dim(M1, dim)
    x = np.eye(2 ** dim)                        # every unit vector: the columns of M
    y = oracle.mass(B1, np.tile(w, (2 ** dim, 1)), x, dim)
    np.testing.assert_allclose(y, M.T, rtol=0, atol=1e-15)


@pytest.mark.parametrize("dim,D,Q", [(2, 3, 4), (3, 3, 4), (2, 5, 7)])
def test_partition_of_unity_and_symmetry(dim, D, Q):
    rng = np.random.default_rng(2)
    xq, _ = gauss_legendre(Q)
    B1 = lagrange_basis(np.linspace(-1, 1, D), xq)     # rows sum to 1
    op = rng.uniform(0.5, 2.0, (3, Q ** dim))
    y1 = oracle.mass(B1, op, np.ones((3, D ** dim)), dim)
    np.testing.assert_allclose(y1.sum(axis=1), op.sum(axis=1), rtol=1e-13)
    a, b = rng.uniform(-1, 1, (2, 3, D ** dim))
    ya, yb = oracle.mass(B1, op, a, dim), oracle.mass(B1, op, b, dim)
    np.testing.assert_allclose(np.sum(ya * b, axis=1), np.sum(a * yb, axis=1), rtol=1e-12)


@pytest.mark.parametrize("dim,D,Q", [(1, 3, 5), (2, 4, 6), (3, 3, 5), (3, 4, 2)])
def test_against_sum_factorization(dim, D, Q):
    """An independent evaluation: one-dimensional contractions, one axis at a
    time (the fast algorithm), against the oracle's explicit Kronecker B."""
    rng = np.random.default_rng(3)
    B1 = rng.uniform(-1, 1, (Q, D))
    ne = 4
    x = rng.uniform(-1, 1, (ne, D ** dim))
    op = rng.uniform(-1, 1, (ne, Q ** dim))
    y = oracle.mass(B1, op, x, dim, nthreads=2)
    shp_d = (ne,) + (D,) * dim                  # axes reversed: last axis = first index (fastest)
    t = x.reshape(shp_d)
    for ax in range(dim):
        t = np.moveaxis(np.tensordot(t, B1, axes=([1 + ax], [1])), -1, 1 + ax)
    t = t * op.reshape((ne,) + (Q,) * dim)
    for ax in range(dim):
        t = np.moveaxis(np.tensordot(t, B1, axes=([1 + ax], [0])), -1, 1 + ax)
    np.testing.assert_allclose(y, t.reshape(ne, -1), rtol=1e-12, atol=1e-14)


def test_exact_rationals_small_case():
    """dim 2, D 2, Q 3 with small integers: every product and sum is exact in
    double, so the oracle equals the rational evaluation bit for bit."""
    rng = np.random.default_rng(4)
    B1 = rng.integers(-3, 4, (3, 2)).astype(float)
    op = rng.integers(-3, 4, (2, 9)).astype(float)
    x = rng.integers(-3, 4, (2, 4)).astype(float)
    y = oracle.mass(B1, op, x, 2)
    for e in range(2):
        for j in itertools.product(range(2), repeat=2):       # (j_y, j_x)
            s = Fraction(0)
            for k in itertools.product(range(3), repeat=2):   # (k_y, k_x)
                bk_j = Fraction(B1[k[0], j[0]]) * Fraction(B1[k[1], j[1]])
                u = Fraction(0)
                for jj in itertools.product(range(2), repeat=2):
                    u += Fraction(B1[k[0], jj[0]]) * Fraction(B1[k[1], jj[1]]) * Fraction(x[e, jj[0] * 2 + jj[1]])
                s += bk_j * Fraction(op[e, k[0] * 3 + k[1]]) * u
            assert y[e, j[0] * 2 + j[1]] == float(s)


def test_invalid_arguments_are_refused():
    with pytest.raises(ValueError):
        oracle.mass(np.ones((2, 2)), np.ones((1, 16)), np.ones((1, 16)), 4)
