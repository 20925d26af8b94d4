"""Pins for the CPU oracle: each test fixes the oracle against something
other than itself (a closed form, an independent evaluation route, an
invariant of the mathematics, or a textbook special case)."""
import numpy as np
import pytest

import gw_inputs as gi
import oracle as O


def _denman_beavers(A, iters=60):
    """Matrix square root and inverse square root of an SPD matrix by the
    Denman-Beavers iteration (no eigensolver)."""
    Y = A.copy()
    Z = np.eye(A.shape[0])
    for _ in range(iters):
        Yi = np.linalg.inv(Y)
        Zi = np.linalg.inv(Z)
        Y, Z = 0.5 * (Y + Zi), 0.5 * (Z + Yi)
    return Y, Z


def _small(n_v=2, n_c=3, n_aux=4, seed=7, kf=4.0, scale=1.0):
    wl = gi.make_workload("t", n_v, n_c, n_aux, list(range(n_v + n_c)),
                          list(range(n_v + n_c)), 41, seed, k=n_v * n_c,
                          sigma_L=0.3 * scale, sigma_M=0.5, kernel_factor=kf)
    return wl


def test_scalar_pair_closed_form():
    """N_v = N_c = N_aux = 1: one pair, one eigenpair, everything scalar.
    Omega^2 = Delta^2 + c_K Delta L^2, b = Delta^1/2 L M, weight b^2/Omega,
    Sigma_t(w) = sum_m b_tm^2/Omega / (w - eps_m + eta_m Omega - i eta_m delta)
    (Eq. 4, text after Eq. 8, Eq. 7, Eq. 9)."""
    wl = gi.make_workload("s", 1, 1, 1, [0, 1], [0, 1], 17, 3, k=1)
    ev, ec = wl.eps
    Dl = ec - ev
    l = wl.L[0, 0]
    Om = np.sqrt(Dl * Dl + 4.0 * Dl * l * l)
    sig, poles = O.sigma_closed_form(wl)
    for ti in range(2):
        ref = np.zeros(wl.omega.shape, complex)
        for mi, (em, eta) in enumerate([(ev, 1.0), (ec, -1.0)]):
            b = np.sqrt(Dl) * l * wl.M[ti, mi, 0]
            ref += (b * b / Om) / (wl.omega - em + eta * Om - 1j * eta * wl.delta)
        np.testing.assert_allclose(sig[ti], ref, rtol=1e-13, atol=0)
    sigL, _, _ = O.sigma_lanczos(wl, k=1)
    np.testing.assert_allclose(sigL, sig, rtol=1e-13, atol=0)


@pytest.mark.parametrize("kf", [4.0, 2.0])
def test_brute_force_resolvent_route(kf):
    """Eq. 12 route: build C = (A-B)^1/2 (A+B) (A-B)^1/2 from the RPA blocks
    A = Delta + (c_K/2) K, B = (c_K/2) K (Eq. 2-4), take D = C^1/2 by
    Denman-Beavers and solve <P| [D (z + eta D)]^-1 |P> directly; no
    eigendecomposition.  Must equal the Eq. 7-9 closed form."""
    wl = _small(kf=kf)
    n_vc = wl.n_vc
    Delta = np.array([wl.eps[wl.n_v + c] - wl.eps[v]
                      for v in range(wl.n_v) for c in range(wl.n_c)])
    K = wl.L @ wl.L.T
    A = np.diag(Delta) + 0.5 * kf * K
    B = 0.5 * kf * K
    AmB_half, _ = _denman_beavers(A - B)
    C = AmB_half @ (A + B) @ AmB_half
    D, _ = _denman_beavers(C)
    sig, _ = O.sigma_closed_form(wl)
    for ti in range(wl.n_t):
        ref = np.zeros(wl.omega.shape, complex)
        for mi, m in enumerate(wl.m_idx):
            V = wl.L @ wl.M[ti, mi]
            P = V * np.sqrt(Delta)
            eta = 1.0 if m < wl.n_v else -1.0
            for fi, w in enumerate(wl.omega):
                z = w - wl.eps[m] - 1j * eta * wl.delta
                # (1/z)<P|D^-1 - (D + eta z)^-1|P>  (Eq. 12)
                x1 = np.linalg.solve(D.astype(complex), P.astype(complex))
                x2 = np.linalg.solve(D + eta * z * np.eye(n_vc), P.astype(complex))
                ref[fi] += (P @ x1 - P @ x2) / z
        np.testing.assert_allclose(sig[ti], ref, rtol=1e-10, atol=1e-13)


def test_kernel_free_limit():
    """c_K = 0: C = Delta^2, Omega_s = Delta_s, Z = I, so
    Sigma_tm = sum_vc V_vc^2 / (z_m + eta_m Delta_vc) with no eigensolver."""
    wl = _small(kf=0.0)
    sig, _ = O.sigma_closed_form(wl)
    Delta = np.array([wl.eps[wl.n_v + c] - wl.eps[v]
                      for v in range(wl.n_v) for c in range(wl.n_c)])
    for ti in range(wl.n_t):
        ref = np.zeros(wl.omega.shape, complex)
        for mi, m in enumerate(wl.m_idx):
            V = wl.L @ wl.M[ti, mi]
            eta = 1.0 if m < wl.n_v else -1.0
            z = wl.omega - wl.eps[m] - 1j * eta * wl.delta
            ref += np.sum(V[None, :] ** 2 / (z[:, None] + eta * Delta[None, :]), axis=1)
        np.testing.assert_allclose(sig[ti], ref, rtol=1e-12, atol=1e-15)


def test_rank_one_secular_equation():
    """N_aux = 1: C = Delta^2 + c_K d l l^T d is a rank-1 update of a
    diagonal.  Its eigenvalues are the roots of
    1 + c_K sum_i Delta_i l_i^2 / (Delta_i^2 - theta) = 0, one in each gap
    of the sorted Delta_i^2 and one above the largest (Golub 1973); found
    here by bisection and compared with the oracle's Omega_s^2."""
    wl = gi.make_workload("r1", 3, 5, 1, [2], [0, 1], 5, 11, sigma_L=0.4)
    Delta = O.pair_energies(wl.eps, wl.n_v)
    l = wl.L[:, 0]
    H = O.casida_matrix(wl.eps, wl.n_v, wl.L, 4.0)
    Om, _ = O.casida_eigenpairs(H)
    d2 = np.sort(Delta ** 2)
    f = lambda th: 1.0 + 4.0 * np.sum(Delta * l * l / (Delta ** 2 - th))
    hi_end = d2[-1] + 4.0 * np.sum(Delta * l * l) + 1.0
    brackets = list(zip(d2[:-1], d2[1:])) + [(d2[-1], hi_end)]
    roots = []
    for lo, hi in brackets:
        lo, hi = lo + 1e-12 * (1 + lo), hi - 1e-12 * (1 + hi) if hi != hi_end else hi
        for _ in range(200):
            mid = 0.5 * (lo + hi)
            if f(mid) > 0:       # f increases from -inf to +inf inside a gap
                hi = mid
            else:
                lo = mid
        roots.append(0.5 * (lo + hi))
    np.testing.assert_allclose(np.sort(Om ** 2), np.array(roots), rtol=1e-11)
    assert np.all(Om ** 2 >= d2 - 1e-9)


def test_spectral_invariants():
    """With weights W = p^2/Omega: sum W Omega = ||b||^2, sum W Omega^3 =
    b^T C b, and sum W / Omega = b^T C^-1 b (static limit, Cholesky solve)."""
    wl = _small(n_v=3, n_c=4, n_aux=5)
    H = O.casida_matrix(wl.eps, wl.n_v, wl.L, wl.kernel_factor)
    Om, Z = O.casida_eigenpairs(H)
    b = O.start_vectors(wl.eps, wl.n_v, O.coupling_vectors(wl.L, wl.M))
    Lc = np.linalg.cholesky(H)
    for ti in range(wl.n_t):
        for mi in range(wl.n_m):
            bb = b[ti, mi]
            W = (Z.T @ bb) ** 2 / Om
            assert np.sum(W * Om) == pytest.approx(bb @ bb, rel=1e-12)
            assert np.sum(W * Om ** 3) == pytest.approx(bb @ H @ bb, rel=1e-12)
            y = np.linalg.solve(Lc, bb)
            assert np.sum(W / Om) == pytest.approx(y @ y, rel=1e-11)


@pytest.mark.parametrize("reorth", [True, False])
def test_gauss_quadrature_moments(reorth):
    """k-step Lanczos is a k-node Gauss rule: beta0^2 e1^T T_k^p e1 =
    b^T C^p b exactly for p <= 2k-1 (Golub & Meurant), at truncated k.
    Without reorthogonalisation this pins the three-term recurrence alone."""
    wl = gi.tiny(k=6)
    H = O.casida_matrix(wl.eps, wl.n_v, wl.L, wl.kernel_factor)
    b = O.start_vectors(wl.eps, wl.n_v, O.coupling_vectors(wl.L, wl.M)).reshape(-1, wl.n_vc)
    b = b[:5]
    a, be, b0, ke = O.lanczos(lambda X: X @ H.T, b, 6, reorth=reorth)
    s = np.max(np.abs(np.linalg.eigvalsh(H)))
    for v in range(b.shape[0]):
        Om, W = O.lanczos_poles(a[v], be[v], b0[v], ke[v])
        u = W * Om                       # beta0^2 u_1j^2
        th = Om ** 2
        x = b[v].copy()
        for p in range(0, 12):
            ref = b[v] @ x               # b^T C^p b
            got = np.sum(u * th ** p)
            assert got == pytest.approx(ref, rel=1e-9 * (1 + p)), p
            x = H @ x
        assert np.isclose(np.sum(u), b[v] @ b[v], rtol=1e-13)
    del s


def test_full_lanczos_reproduces_closed_form():
    """k = N_vc Lanczos spans the whole space, so its Gauss rule is the exact
    spectral measure: Sigma equals Eq. 7 to 1e-10."""
    wl = gi.tiny(k=256)
    sig, _ = O.sigma_closed_form(wl)
    sigL, _, (a, be, b0, ke) = O.sigma_lanczos(wl, k=256)
    assert np.all(ke == 256)
    err = np.abs(sigL - sig).max() / np.abs(sig).max()
    assert err < 1e-10, err


def test_imaginary_part_sign_rule():
    """Occupied m contributes Im Sigma >= 0 and empty m Im Sigma <= 0 at every
    omega (time-ordered sign convention of Eq. 7)."""
    wl = _small(n_v=3, n_c=4, n_aux=5)
    pos, W, eta = O.closed_form_poles(wl)
    for ti in range(wl.n_t):
        occ = eta[ti] > 0
        s_occ = O.sigma_from_poles(wl.omega, pos[ti][occ], W[ti][occ], eta[ti][occ], wl.delta)
        s_emp = O.sigma_from_poles(wl.omega, pos[ti][~occ], W[ti][~occ], eta[ti][~occ], wl.delta)
        assert np.all(s_occ.imag >= 0) and np.all(s_emp.imag <= 0)
        assert np.all(W[ti] >= 0)


def test_high_frequency_tail():
    """omega Sigma_tm(omega) -> sum_s p_s^2/Omega_s = b^T C^-1/2 b as
    |omega| -> infinity; C^-1/2 from Denman-Beavers."""
    wl = _small(n_v=2, n_c=4, n_aux=3)
    H = O.casida_matrix(wl.eps, wl.n_v, wl.L, wl.kernel_factor)
    _, Hmh = _denman_beavers(H)
    b = O.start_vectors(wl.eps, wl.n_v, O.coupling_vectors(wl.L, wl.M))
    pos, W, eta = O.closed_form_poles(wl)
    big = 1e7
    for ti in range(wl.n_t):
        ref = sum(b[ti, mi] @ Hmh @ b[ti, mi] for mi in range(wl.n_m))
        got = big * O.sigma_from_poles([big], pos[ti], W[ti], eta[ti], wl.delta)[0]
        assert got.real == pytest.approx(ref, rel=1e-5)


def test_qp_single_pole_quadratic():
    """One pole, vanishing broadening: E - e0 = w / (E - E_p) is the
    quadratic (E - e0)(E - E_p) = w; Newton from e0 must land on the root
    nearer e0."""
    e0, Ep, w, delta = -5.0, -12.0, 0.8, 1e-9
    pos, W, eta = np.array([Ep]), np.array([w]), np.array([1.0])
    sfn = lambda x: O.sigma_from_poles([x], pos, W, eta, delta)[0]
    dfn = lambda x: O.dsigma_from_poles([x], pos, W, eta, delta)[0]
    E, Z = O.qp_solve(e0, sfn, dfn)
    disc = np.sqrt((e0 - Ep) ** 2 + 4 * w)
    r = [0.5 * (e0 + Ep + disc), 0.5 * (e0 + Ep - disc)]
    ref = min(r, key=lambda x: abs(x - e0))
    assert E == pytest.approx(ref, abs=1e-9)
    assert Z == pytest.approx(1.0 / (1.0 + w / (ref - Ep) ** 2), rel=1e-7)


def test_qp_bisection_fallback_agrees():
    """The grid-bracket fallback finds the same root as Newton."""
    wl = gi.tiny()
    sig, poles = O.sigma_closed_form(wl)
    pos, W, eta = poles[1]
    e0 = wl.eps[wl.targets[1]]
    sfn = lambda x: O.sigma_from_poles([x], pos, W, eta, wl.delta)[0]
    dfn = lambda x: O.dsigma_from_poles([x], pos, W, eta, wl.delta)[0]
    E1, Z1 = O.qp_solve(e0, sfn, dfn)
    E2, Z2 = O.qp_solve(e0, sfn, dfn, grid=np.linspace(e0 - 3, e0 + 3, 601), max_iter=0)
    assert E2 == pytest.approx(E1, abs=1e-8)


def test_generator_is_seeded_and_symmetric():
    a, b = gi.tiny(), gi.tiny()
    assert np.array_equal(a.L, b.L) and np.array_equal(a.M, b.M)
    # (t, m) and (m, t) share their coupling factor
    t0, t1 = 0, 1
    m_of = {int(m): j for j, m in enumerate(a.m_idx)}
    assert np.array_equal(a.M[t0, m_of[int(a.targets[t1])]], a.M[t1, m_of[int(a.targets[t0])]])
    assert np.all(np.diff(a.eps[: a.n_v]) >= 0) and np.all(np.diff(a.eps[a.n_v:]) >= 0)
