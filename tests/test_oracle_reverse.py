"""Pins for the oracle's exact k-step gradient (reverse mode of the three-term
recurrence) and for its Tamm-Dancoff closed-form gradient.

  * Gauss-rule identity: k Lanczos steps integrate polynomials of degree
    <= 2k - 1 exactly, so b^T C^p b = beta0^2 (T_k^p)_11 holds identically in
    (C, b) for p <= 2k - 1; its derivative through the reverse recurrence must
    then equal the textbook derivative of b^T C^p b (2 C^p b, and the sum of
    C^a b b^T C^(p-1-a)).  This checks the recurrence's adjoint on its own,
    without the spectral map or the QP equation.
  * Central differences of the oracle's own k-step QP energies (no
    reorthogonalisation) along seeded random directions in L and eps, at
    truncated k where the Krylov form of the gradient is visibly off.
  * The Tamm-Dancoff closed-form gradient against central differences of the
    Tamm-Dancoff closed-form QP energies.
  * Polynomial form (Lanczos on D = p_g(C)): the reverse Clenshaw recurrence
    gives p(C)^T u and the directional derivative of u . p(C) x (central
    differences on a dense matrix), and the whole k-step gradient matches
    central differences of the oracle's polynomial-form QP energies.
"""
import numpy as np
import pytest

import gw_inputs as gi
import oracle as O


def _spd(n, seed):
    rng = np.random.default_rng(seed)
    X = rng.normal(size=(n, n))
    lam = np.linspace(1.0, 4.0, n)
    Qm, _ = np.linalg.qr(X)
    return (Qm * lam) @ Qm.T


@pytest.mark.parametrize("p,k", [(1, 1), (2, 2), (3, 2), (5, 3), (6, 4), (7, 4)])
def test_reverse_recurrence_reproduces_polynomial_moment_gradient(p, k):
    n = 12
    C = _spd(n, 100 + p)
    b = np.random.default_rng(200 + p).normal(size=n)

    def apply_op(X):
        return X @ C.T

    alpha, beta, beta0, k_eff = O.lanczos(apply_op, b[None, :], k, reorth=False)
    ke = int(k_eff[0])
    assert ke == k
    T = np.diag(alpha[0, :ke]) + np.diag(beta[0, : ke - 1], 1) + np.diag(beta[0, : ke - 1], -1)
    e1 = np.zeros(ke)
    e1[0] = 1.0
    b0 = beta0[0]
    # F = beta0^2 (T^p)_11; dF/dT = beta0^2 sum_a T^a e1 e1^T T^(p-1-a)
    Tp = [np.linalg.matrix_power(T, a) for a in range(p)]
    Gam = b0 ** 2 * sum(np.outer(Tp[a] @ e1, Tp[p - 1 - a] @ e1) for a in range(p))
    abar = np.diag(Gam).copy()
    bbar = np.zeros(ke)
    bbar[: ke - 1] = np.diag(Gam, 1) + np.diag(Gam, -1)
    qbar0, ubar, Q, _ = O.lanczos_reverse(apply_op, b, k, abar, bbar)
    F = b0 ** 2 * (np.linalg.matrix_power(T, p) @ e1)[0]
    assert F == pytest.approx(b @ np.linalg.matrix_power(C, p) @ b, rel=1e-11)
    q0 = Q[0]
    y = (2.0 * F / b0) * q0 + (qbar0 - (qbar0 @ q0) * q0) / b0
    Cp = [np.linalg.matrix_power(C, a) for a in range(p + 1)]
    np.testing.assert_allclose(y, 2.0 * Cp[p] @ b, rtol=0, atol=1e-10 * np.abs(Cp[p] @ b).max())
    G = ubar.T @ Q
    G = 0.5 * (G + G.T)
    Gref = sum(np.outer(Cp[a] @ b, Cp[p - 1 - a] @ b) for a in range(p))
    Gref = 0.5 * (Gref + Gref.T)
    np.testing.assert_allclose(G, Gref, rtol=0, atol=1e-10 * np.abs(Gref).max())


def _wl(kf=4.0):
    return gi.make_workload("g", 3, 7, 9, [1, 2, 4], list(range(10)), 81, 5, k=21,
                            sigma_L=0.25, sigma_M=0.4, kernel_factor=kf)


def _Ek(w, k, tda):
    if tda:
        _, poles, _ = O.sigma_tda_lanczos(w, k=k, reorth=False)
    else:
        _, poles, _ = O.sigma_lanczos(w, k=k, reorth=False)
    return O.solve_all_qp(w, poles)[0]


@pytest.mark.parametrize("tda", [False, True])
@pytest.mark.parametrize("k", [4, 8, 14])
def test_recurrence_gradient_matches_central_differences(k, tda):
    wl = _wl()
    rng = np.random.default_rng(30 + k)
    dE = rng.normal(size=wl.n_t)
    dL, deps = O.qp_gradient_recurrence(wl, dE, k=k, tda=tda)
    h = 1e-6
    for trial in range(2):
        PL = rng.normal(size=wl.L.shape)
        Pe = rng.normal(size=wl.eps.shape) * 0.1
        for which in ("L", "eps"):
            wp = gi.Workload(**wl.__dict__)
            wm = gi.Workload(**wl.__dict__)
            if which == "L":
                wp.L = wl.L + h * PL
                wm.L = wl.L - h * PL
                ana = np.sum(dL * PL)
            else:
                wp.eps = wl.eps + h * Pe
                wm.eps = wl.eps - h * Pe
                ana = np.sum(deps * Pe)
            fd = (dE @ _Ek(wp, k, tda) - dE @ _Ek(wm, k, tda)) / (2 * h)
            assert ana == pytest.approx(fd, rel=1e-6, abs=1e-9), (which, trial)


def test_krylov_form_differs_from_the_k_step_derivative_at_short_k():
    """At k = 8 of 21 the Krylov form is not the derivative of E_8; the
    reverse recurrence is (the previous test).  Guards against the two
    functions collapsing into one."""
    wl = _wl()
    dE = np.random.default_rng(41).normal(size=wl.n_t)
    dLr, _ = O.qp_gradient_recurrence(wl, dE, k=8)
    dLk, _ = O.qp_gradient_lanczos(wl, dE, k=8, reorth=False)
    assert np.abs(dLr - dLk).max() > 1e-4 * np.abs(dLr).max()


@pytest.mark.parametrize("kf", [4.0, 2.0])
def test_tda_closed_form_gradient_matches_central_differences(kf):
    wl = _wl(kf)
    rng = np.random.default_rng(50)
    dE = rng.normal(size=wl.n_t)
    dL, deps = O.qp_gradient_tda_closed_form(wl, dE)
    h = 1e-6

    def E(w):
        return O.qp_energies_tda_closed_form(w)[0]

    for trial in range(2):
        PL = rng.normal(size=wl.L.shape)
        Pe = rng.normal(size=wl.eps.shape) * 0.1
        for which in ("L", "eps"):
            wp = gi.Workload(**wl.__dict__)
            wm = gi.Workload(**wl.__dict__)
            if which == "L":
                wp.L = wl.L + h * PL
                wm.L = wl.L - h * PL
                ana = np.sum(dL * PL)
            else:
                wp.eps = wl.eps + h * Pe
                wm.eps = wl.eps - h * Pe
                ana = np.sum(deps * Pe)
            fd = (dE @ E(wp) - dE @ E(wm)) / (2 * h)
            assert ana == pytest.approx(fd, rel=1e-6, abs=1e-9), (which, trial)


def test_tda_recurrence_gradient_approaches_closed_form():
    """With k = N_vc the k-step Tamm-Dancoff energies are the closed form's
    (to the loss of orthogonality of 21 plain steps), and so is the
    gradient."""
    wl = _wl()
    dE = np.random.default_rng(51).normal(size=wl.n_t)
    dLr, depsr = O.qp_gradient_recurrence(wl, dE, k=wl.n_vc, tda=True)
    dL, deps = O.qp_gradient_tda_closed_form(wl, dE)
    np.testing.assert_allclose(dLr, dL, rtol=0, atol=1e-6 * np.abs(dL).max())
    np.testing.assert_allclose(depsr, deps, rtol=0, atol=1e-6 * np.abs(deps).max())


# --------------------------------------------------------------------------
# Polynomial form: Lanczos on D = p_g(C) without reorthogonalisation
# --------------------------------------------------------------------------
def _interval(wl):
    th = np.linalg.eigvalsh(O.casida_matrix(wl.eps, wl.n_v, wl.L, wl.kernel_factor))
    return 0.9 * th.min(), 1.1 * th.max()


@pytest.mark.parametrize("g", [1, 2, 5, 8])
def test_poly_reverse_gives_transpose_product_and_directional_derivative(g):
    """xbar = p(C) u (C symmetric); the pairs' contraction with a symmetric
    direction E equals central differences of u . p(C + hE) x."""
    n = 10
    C = _spd(n, 300 + g) * 3.0
    rng = np.random.default_rng(400 + g)
    u, x = rng.normal(size=n), rng.normal(size=n)
    lo, hi = 2.5, 13.0
    c = O.chebyshev_sqrt(lo, hi, g)

    def op(M):
        return lambda X: X @ M.T

    xbar, pairs = O.apply_poly_reverse(op(C), u, x, c, lo, hi)
    np.testing.assert_allclose(xbar, O.apply_poly(op(C), u[None, :], c, lo, hi)[0],
                               rtol=0, atol=1e-12 * np.abs(xbar).max())
    E = rng.normal(size=(n, n))
    E = E + E.T
    ana = sum(coef * (pa @ E @ pb) for coef, pa, pb in pairs)
    h = 1e-5
    fp = u @ O.apply_poly(op(C + h * E), x[None, :], c, lo, hi)[0]
    fm = u @ O.apply_poly(op(C - h * E), x[None, :], c, lo, hi)[0]
    assert ana == pytest.approx((fp - fm) / (2 * h), rel=1e-7, abs=1e-10)


def _Ek_poly(w, g, lo, hi, k):
    _, poles, _ = O.sigma_poly_lanczos(w, g, lo, hi, k=k, reorth=False)
    return O.solve_all_qp(w, poles)[0]


@pytest.mark.parametrize("g,k", [(4, 4), (8, 8), (8, 14)])
def test_poly_recurrence_gradient_matches_central_differences(g, k):
    wl = _wl()
    lo, hi = _interval(wl)
    rng = np.random.default_rng(80 + g + k)
    dE = rng.normal(size=wl.n_t)
    dL, deps = O.qp_gradient_poly_recurrence(wl, dE, g, lo, hi, k=k)
    h = 1e-6
    for trial in range(2):
        PL = rng.normal(size=wl.L.shape)
        Pe = rng.normal(size=wl.eps.shape) * 0.1
        for which in ("L", "eps"):
            wp = gi.Workload(**wl.__dict__)
            wm = gi.Workload(**wl.__dict__)
            if which == "L":
                wp.L = wl.L + h * PL
                wm.L = wl.L - h * PL
                ana = np.sum(dL * PL)
            else:
                wp.eps = wl.eps + h * Pe
                wm.eps = wl.eps - h * Pe
                ana = np.sum(deps * Pe)
            # the interval [lo, hi] is a fixed input of the polynomial form
            fd = (dE @ _Ek_poly(wp, g, lo, hi, k) - dE @ _Ek_poly(wm, g, lo, hi, k)) / (2 * h)
            assert ana == pytest.approx(fd, rel=1e-6, abs=1e-9), (which, trial)


def _breakdown_wl(kf=4.0):
    """L nonzero on three pair rows only: C is block-diagonal and every start
    vector b = D L M lies in that 3-dimensional invariant subspace, so the
    recurrence stops (k_eff = 3) long before k."""
    wl = gi.make_workload("bd", 2, 6, 4, [1, 2], list(range(8)), 61, 9, k=8,
                          sigma_L=0.3, sigma_M=0.5, kernel_factor=kf)
    keep = np.zeros(wl.n_vc, dtype=bool)
    keep[[0, 3, 7]] = True
    wl.L = np.where(keep[:, None], wl.L, 0.0)
    return wl


def test_recurrence_gradient_at_breakdown_matches_central_differences():
    """At breakdown T_k stops at k_eff; a perturbation of L leaves the
    invariant subspace and adds poles of weight O(h^2), which central
    differences cancel.  The k_eff-step gradient must match."""
    wl = _breakdown_wl()
    _, _, (_, _, _, k_eff) = O.sigma_lanczos(wl, k=8, reorth=False)
    assert set(int(x) for x in k_eff) == {3}
    rng = np.random.default_rng(97)
    dE = rng.normal(size=wl.n_t)
    dL, deps = O.qp_gradient_recurrence(wl, dE, k=8)
    h = 1e-6
    for trial in range(2):
        PL = rng.normal(size=wl.L.shape)
        Pe = rng.normal(size=wl.eps.shape) * 0.1
        for which in ("L", "eps"):
            wp = gi.Workload(**wl.__dict__)
            wm = gi.Workload(**wl.__dict__)
            if which == "L":
                wp.L = wl.L + h * PL
                wm.L = wl.L - h * PL
                ana = np.sum(dL * PL)
            else:
                wp.eps = wl.eps + h * Pe
                wm.eps = wl.eps - h * Pe
                ana = np.sum(deps * Pe)
            fd = (dE @ _Ek(wp, 8, False) - dE @ _Ek(wm, 8, False)) / (2 * h)
            assert ana == pytest.approx(fd, rel=1e-6, abs=1e-9), (which, trial)
