"""Pins for the oracle's polynomial variant (Lanczos on D = p_g(C), Haydock
continued fractions at 0 and -eta z)."""
import numpy as np
import pytest

import gw_inputs as gi
import oracle as O


def test_chebyshev_interpolates_sqrt_at_its_nodes():
    lo, hi, g = 3.0, 700.0, 9
    c = O.chebyshev_sqrt(lo, hi, g)
    j = np.arange(g + 1)
    x = 0.5 * (hi + lo) + 0.5 * (hi - lo) * np.cos(np.pi * (j + 0.5) / (g + 1))
    np.testing.assert_allclose(O.chebyshev_eval(c, lo, hi, x), np.sqrt(x), rtol=1e-13)


def test_chebyshev_error_decays_at_the_bernstein_rate():
    """sqrt is analytic except at x = 0, i.e. t0 = -(hi+lo)/(hi-lo); the
    interpolation error decays like rho^-g with rho = |t0| + sqrt(t0^2 - 1)."""
    lo, hi = 4.0, 1000.0
    t0 = (hi + lo) / (hi - lo)
    rho = t0 + np.sqrt(t0 * t0 - 1.0)
    x = np.linspace(lo, hi, 20001)
    err = {g: np.abs(O.chebyshev_eval(O.chebyshev_sqrt(lo, hi, g), lo, hi, x) - np.sqrt(x)).max()
           for g in (8, 16, 24)}
    for g1, g2 in ((8, 16), (16, 24)):
        ratio = err[g2] / err[g1]
        assert 0.05 * rho ** -(g2 - g1) < ratio < 20.0 * rho ** -(g2 - g1), (g1, g2, ratio)


def test_clenshaw_on_a_diagonal_matrix():
    """p(C) v for diagonal C: at the Chebyshev nodes it is sqrt(x) v exactly,
    elsewhere the scalar series value."""
    lo, hi, g = 2.0, 50.0, 7
    c = O.chebyshev_sqrt(lo, hi, g)
    j = np.arange(g + 1)
    nodes = 0.5 * (hi + lo) + 0.5 * (hi - lo) * np.cos(np.pi * (j + 0.5) / (g + 1))
    x = np.concatenate([nodes, np.linspace(lo, hi, 13)])
    v = np.random.default_rng(1).standard_normal((3, x.size))
    got = O.apply_poly(lambda X: X * x, v, c, lo, hi)
    np.testing.assert_allclose(got[:, : g + 1], np.sqrt(nodes) * v[:, : g + 1], rtol=1e-12)
    np.testing.assert_allclose(got[:, g + 1:], O.chebyshev_eval(c, lo, hi, x[g + 1:]) *
                               v[:, g + 1:], rtol=1e-12)


def test_haydock_equals_the_gauss_pole_sum():
    rng = np.random.default_rng(2)
    n = 9
    a, b = rng.uniform(1, 5, n), rng.uniform(0.1, 1.0, n)
    T = np.diag(a) + np.diag(b[: n - 1], 1) + np.diag(b[: n - 1], -1)
    lam, U = np.linalg.eigh(T)
    z = np.array([0.3 + 0.05j, -2.0 + 0.1j, 7.0 - 0.2j, 0.0])
    ref = np.array([np.sum(1.7 ** 2 * U[0] ** 2 / (zz - lam)) for zz in z])
    np.testing.assert_allclose(O.haydock(a, b, 1.7, n, z), ref, rtol=1e-12)


def _wl():
    return gi.make_workload("p", 3, 7, 9, [1, 2, 4], list(range(10)), 61, 5, k=21,
                            sigma_L=0.25, sigma_M=0.4)


def _closed_form_with(wl, node_map):
    """Closed-form Sigma with the Casida frequencies Omega_s replaced by
    node_map(theta_s) (identity: sqrt)."""
    H = O.casida_matrix(wl.eps, wl.n_v, wl.L, wl.kernel_factor)
    theta, Y = np.linalg.eigh(H)
    P = node_map(theta)
    b = O.start_vectors(wl.eps, wl.n_v, O.coupling_vectors(wl.L, wl.M))
    eta = O.occupation_sign(wl.m_idx, wl.n_v)
    sig = np.zeros((wl.n_t, wl.omega.size), dtype=complex)
    for ti in range(wl.n_t):
        for mi, m in enumerate(wl.m_idx):
            p = Y.T @ b[ti, mi]
            z = wl.omega[:, None] - wl.eps[m] - 1j * eta[mi] * wl.delta
            sig[ti] += np.sum(p ** 2 / (P * (z + eta[mi] * P)), axis=1)
    return sig, theta


def test_full_space_reproduces_the_polynomial_closed_form():
    """k = N_vc: the Lanczos Gauss rule of D = p_g(C) is exact, so Sigma is the
    closed form with Omega_s -> p_g(theta_s) (to rounding, 1e-10)."""
    wl = _wl()
    _, theta = _closed_form_with(wl, np.sqrt)
    lo, hi, g = theta.min(), theta.max(), 6
    c = O.chebyshev_sqrt(lo, hi, g)
    ref, _ = _closed_form_with(wl, lambda th: O.chebyshev_eval(c, lo, hi, th))
    got, poles, _ = O.sigma_poly_lanczos(wl, g, lo, hi, k=wl.n_vc)
    for ti in range(wl.n_t):
        assert np.abs(got[ti] - ref[ti]).max() <= 1e-10 * np.abs(ref[ti]).max()
    # the pole form of the same rule gives the same Sigma
    pf = np.stack([O.sigma_from_poles(wl.omega, *poles[ti], wl.delta) for ti in range(wl.n_t)])
    np.testing.assert_allclose(pf, got, rtol=1e-9, atol=1e-12)


def test_error_shrinks_with_the_degree():
    """Fig. 1b analogue: QP energies of the polynomial variant approach the
    exact closed form as g grows (k = N_vc, so only the fit error is left)."""
    wl = _wl()
    sigx, polesx = O.sigma_closed_form(wl)
    Ex, _ = O.solve_all_qp(wl, polesx)
    _, theta = _closed_form_with(wl, np.sqrt)
    errs = []
    for g in (2, 4, 8, 16):
        _, poles, _ = O.sigma_poly_lanczos(wl, g, theta.min(), theta.max(), k=wl.n_vc)
        E, _ = O.solve_all_qp(wl, poles)
        errs.append(np.abs(E - Ex).max())
    print("max |dE| by degree 2/4/8/16 (eV):", errs)
    assert errs[3] < errs[2] < errs[1] < errs[0]
    assert errs[3] < 1e-4            # 0.1 meV at g = 16 (measured 0.012 meV)
