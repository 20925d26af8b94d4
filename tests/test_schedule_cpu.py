"""CPU checks of the lane schedule of the spectral map's Jacobi rebuild.

The GPU rebuild inserts the nodes of a discrete measure one leading row at a
time and chases each insertion's bulge down the tridiagonal; the kernel runs
32 insertions at once, lane l two rows behind lane l-1, rows stored
bottom-up.  These tests replay that schedule in plain Python (IEEE double
arithmetic, one rotation at a time in super-step order) and check:
  * within one super-step the active lanes touch disjoint rows;
  * the result is bit-identical to inserting the nodes one after another;
  * the result is a Jacobi matrix of the measure: its first eigenvector
    components squared, times the total weight, reproduce the weights, and
    its eigenvalues the nodes.
"""
import math

import numpy as np
import pytest


def _rot_sym(c, s, a, b, i):
    x, bb, cc = a[i], b[i], a[i + 1]
    cs, c2, s2 = c * s, c * c, s * s
    a[i] = c2 * x + 2.0 * cs * bb + s2 * cc
    a[i + 1] = s2 * x - 2.0 * cs * bb + c2 * cc
    b[i] = cs * (cc - x) + (c2 - s2) * bb


def _givens(x, z):
    r2 = x * x + z * z
    if r2 > 0.0:
        inv = 1.0 / math.sqrt(r2)
        return x * inv, z * inv, r2 * inv
    return 1.0, 0.0, 0.0


def _insert(x, wt, W, jn, L, m, a, b):
    a[L] = x[jn]
    b[L] = 0.0
    wj = wt[jn]
    c, s = 1.0, 0.0
    if W + wj > 0.0:
        inv = 1.0 / math.sqrt(W + wj)
        c, s = math.sqrt(wj) * inv, math.sqrt(W) * inv
    _rot_sym(c, s, a, b, L)
    bulge = 0.0
    if m > 2:
        bulge = s * b[L + 1]
        b[L + 1] *= c
    return bulge


def _chase(kk, L, m, bulge, a, b):
    c, s, rr = _givens(b[L + kk - 1], bulge)
    b[L + kk - 1] = rr
    _rot_sym(c, s, a, b, L + kk)
    if kk + 1 < m - 1:
        nb = s * b[L + kk + 1]
        b[L + kk + 1] *= c
        return nb
    return 0.0


def serial(x, wt):
    n = len(x)
    a, b = [0.0] * n, [0.0] * n
    a[n - 1] = x[0]
    W = wt[0]
    for jn in range(1, n):
        L, m = n - 1 - jn, jn + 1
        bulge = _insert(x, wt, W, jn, L, m, a, b)
        kk = 1
        while kk < m - 1 and bulge != 0.0:
            bulge = _chase(kk, L, m, bulge, a, b)
            kk += 1
        W += wt[jn]
    return a, b, W


def pipelined(x, wt, lanes=32):
    """The kernel's schedule: super-step tau, lane l at chase step tau - 2 l."""
    n = len(x)
    a, b = [0.0] * n, [0.0] * n
    Wp, W = [], 0.0
    for j in range(n):
        Wp.append(W)
        W += wt[j]
    a[n - 1] = x[0]
    for g0 in range(1, n, lanes):
        nl = min(lanes, n - g0)
        bulge = [0.0] * nl
        live = [False] * nl
        for tau in range(3 * (nl - 1) + g0):
            touched = set()
            for lane in range(nl):
                jn, kk = g0 + lane, tau - 2 * lane
                L, m = n - 1 - jn, jn + 1
                if kk == 0:
                    rows = {L, L + 1}
                    bulge[lane] = _insert(x, wt, Wp[jn], jn, L, m, a, b)
                    live[lane] = bulge[lane] != 0.0
                elif live[lane] and 1 <= kk < m - 1:
                    rows = {L + kk - 1, L + kk, L + kk + 1}
                    bulge[lane] = _chase(kk, L, m, bulge[lane], a, b)
                    live[lane] = bulge[lane] != 0.0
                else:
                    continue
                assert not (rows & touched), (g0, tau, lane)
                touched |= rows
    return a, b, W


def _measure(n, seed):
    rng = np.random.default_rng(seed)
    x = np.sort(2.0 + 30.0 * rng.random(n))
    w = rng.random(n) ** 2 * 1e-3
    w[rng.random(n) < 0.03] = 0.0
    return [float(v) for v in x], [float(v) for v in w]


@pytest.mark.parametrize("n", [1, 2, 3, 5, 31, 32, 33, 34, 64, 65, 100, 200])
def test_pipelined_rebuild_is_the_serial_rebuild_bit_for_bit(n):
    x, w = _measure(n, 1000 + n)
    a1, b1, W1 = serial(x, w)
    a2, b2, W2 = pipelined(x, w)
    assert a1 == a2 and b1[: n - 1] == b2[: n - 1] and W1 == W2


def test_rebuild_is_a_jacobi_matrix_of_the_measure():
    n = 40
    x, w = _measure(n, 7)
    w = [v + 1e-4 for v in w]   # every node carries weight
    a, b, W = pipelined(x, w)
    J = np.diag(a) + np.diag(b[: n - 1], 1) + np.diag(b[: n - 1], -1)
    th, U = np.linalg.eigh(J)
    np.testing.assert_allclose(th, x, rtol=0, atol=1e-12 * max(x))
    np.testing.assert_allclose(W * U[0] ** 2, w, rtol=1e-9, atol=1e-15)
