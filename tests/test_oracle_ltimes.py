"""Pins of the LTimes oracle (Kripke LTimes, Sec. 5.2; six storage orders of
Listing kripold): out[m][g][z] = sum_d L[m][d] in[d][g][z] on logical indices.
"""
from fractions import Fraction
import itertools
import math

import numpy as np
import pytest

import oracle
import synth
from conftest import read_golden


def run(L, canon_in, lin, lout):
    M, D = L.shape
    _, G, Z = canon_in.shape
    phys = synth.to_layout(canon_in, lin)
    out = oracle.ltimes(L, phys.ravel(), G, Z, lin, lout)
    return synth.from_layout(out, lout, (M, G, Z))


def test_hand_worked_integers():
    g = read_golden("ltimes_tiny.txt")
    M, D, G, Z = (int(g[k][0]) for k in "MDGZ")
    L = np.array([float(v) for v in g["L"]]).reshape(M, D)
    x = np.array([float(v) for v in g["IN"]]).reshape(D, G, Z)
    expect = np.array([float(v) for v in g["OUT"]]).reshape(M, G, Z)
    for lin, lout in itertools.product(range(6), range(6)):
        np.testing.assert_array_equal(run(L, x, lin, lout), expect)


def test_six_orders_bit_identical():
    M, D, G, Z = 5, 7, 3, 11
    L, x = synth.ltimes_inputs_np(0xC1A3, M, D, G, Z)
    ref = run(L, x, 0, 0)
    for lin, lout in itertools.product(range(6), range(6)):
        np.testing.assert_array_equal(run(L, x, lin, lout), ref)


def test_selector_L_copies_input():
    M, D, G, Z = 4, 6, 3, 5
    _, x = synth.ltimes_inputs_np(0xC1A3, M, D, G, Z)
    L = np.zeros((M, D))
    L[np.arange(M), np.arange(M)] = 1.0
    for lin, lout in [(0, 0), (3, 5), (5, 1)]:
        np.testing.assert_array_equal(run(L, x, lin, lout), x[:M])


def test_zero_L_gives_zero():
    _, x = synth.ltimes_inputs_np(0xC1A3, 3, 4, 2, 6)
    out = run(np.zeros((3, 4)), x, 2, 4)
    assert np.all(out == 0.0)


def test_unit_input_gives_row_sums():
    M, D, G, Z = 6, 96, 2, 3
    L, _ = synth.ltimes_inputs_np(0xC1A3, M, D, G, Z)
    out = run(L, np.ones((D, G, Z)), 4, 3)
    for m in range(M):
        exact = math.fsum(L[m])
        assert np.all(np.abs(out[m] - exact) <= D * np.finfo(float).eps * np.sum(np.abs(L[m])))


@pytest.mark.parametrize("lin,lout", [(0, 0), (1, 4), (3, 2), (5, 5)])
def test_matches_library_gemm(lin, lout):
    M, D, G, Z = 4, 6, 3, 8
    L, x = synth.ltimes_inputs_np(0xC1A3, M, D, G, Z)
    ref = (L @ x.reshape(D, G * Z)).reshape(M, G, Z)
    out = run(L, x, lin, lout)
    assert np.max(np.abs(out - ref)) <= 1e-14 * np.max(np.abs(ref))


def test_exact_rational_brute_force():
    M, D, G, Z = 2, 3, 2, 2
    L, x = synth.ltimes_inputs_np(0xBB, M, D, G, Z)
    out = run(L, x, 3, 1)
    for m, gg, z in itertools.product(range(M), range(G), range(Z)):
        exact = sum(Fraction(float(L[m, d])) * Fraction(float(x[d, gg, z])) for d in range(D))
        assert abs(out[m, gg, z] - float(exact)) <= 4 * np.finfo(float).eps * float(
            sum(abs(L[m, d] * x[d, gg, z]) for d in range(D)))


def test_sampled_outputs_match_full():
    M, D, G, Z = 6, 10, 4, 9
    L, x = synth.ltimes_inputs_np(0xC1A3, M, D, G, Z)
    lin = 3
    phys = synth.to_layout(x, lin).ravel()
    full = run(L, x, lin, 0)
    idx = np.array([[1, 2, 3], [5, 3, 8], [0, 0, 0]])
    vals = oracle.ltimes_sample(L, phys, G, Z, lin, idx)
    np.testing.assert_array_equal(vals, full[idx[:, 0], idx[:, 1], idx[:, 2]])


def test_threads_do_not_change_results():
    M, D, G, Z = 6, 10, 8, 9
    L, x = synth.ltimes_inputs_np(0xC1A3, M, D, G, Z)
    phys = synth.to_layout(x, 2).ravel()
    np.testing.assert_array_equal(oracle.ltimes(L, phys, G, Z, 2, 4, nthreads=1),
                                  oracle.ltimes(L, phys, G, Z, 2, 4, nthreads=3))


# ---------------------------------------------------------------------------
# LPlusTimes (the adjoint contraction): in += Lp . out
# ---------------------------------------------------------------------------

def test_lplustimes_is_the_adjoint_of_ltimes():
    """<LTimes(L, x), y> = <x, LPlusTimes(L^T, y)> for every pair of orders."""
    M, D, G, Z = 5, 7, 3, 4
    L, x = synth.ltimes_inputs_np(0xAD, M, D, G, Z)
    y = synth.uniform_np(0xAE, 0, M * G * Z).reshape(M, G, Z)
    for lin, lout in [(0, 0), (3, 1), (5, 4), (2, 5)]:
        Lx = run(L, x, lin, lout)
        back = oracle.lplustimes(L.T.copy(), synth.to_layout(y, lout).ravel(), np.zeros(D * G * Z), G, Z, lin, lout)
        lhs = math.fsum((Lx * y).ravel())
        rhs = math.fsum((x * synth.from_layout(back, lin, (D, G, Z))).ravel())
        assert abs(lhs - rhs) <= 1e-13 * max(1.0, abs(lhs))


def test_lplustimes_accumulates_and_matches_gemm():
    M, D, G, Z = 4, 6, 2, 5
    Lp = synth.uniform_np(0xB1, 0, D * M).reshape(D, M)
    y = synth.uniform_np(0xB2, 0, M * G * Z).reshape(M, G, Z)
    base = synth.uniform_np(0xB3, 0, D * G * Z).reshape(D, G, Z)
    res = oracle.lplustimes(Lp, synth.to_layout(y, 4).ravel(), synth.to_layout(base, 1).ravel(), G, Z, 1, 4)
    got = synth.from_layout(res, 1, (D, G, Z))
    ref = base + (Lp @ y.reshape(M, G * Z)).reshape(D, G, Z)
    assert np.max(np.abs(got - ref)) <= 1e-14 * np.max(np.abs(ref))
