"""Pins for the Tamm-Dancoff variant and the off-diagonal element."""
import numpy as np

import gw_inputs as gi
import oracle as O


def _wl(kf=4.0):
    return gi.make_workload("tda", 3, 7, 9, [1, 2, 4], list(range(10)), 61, 5, k=21,
                            sigma_L=0.25, sigma_M=0.4, kernel_factor=kf)


def test_tda_is_the_resolvent_of_A():
    """Sigma_tm = V^T (z + eta A)^-1 V by complex linear solves (no eigenpairs)."""
    wl = _wl()
    sig, _ = O.sigma_tda_closed_form(wl)
    A = O.tda_matrix(wl.eps, wl.n_v, wl.L, wl.kernel_factor)
    V = O.coupling_vectors(wl.L, wl.M)
    eta = O.occupation_sign(wl.m_idx, wl.n_v)
    ref = np.zeros_like(sig)
    for ti in range(wl.n_t):
        for mi, m in enumerate(wl.m_idx):
            for f, w in enumerate(wl.omega):
                z = w - wl.eps[m] - 1j * eta[mi] * wl.delta
                ref[ti, f] += V[ti, mi] @ np.linalg.solve(z * np.eye(wl.n_vc) + eta[mi] * A,
                                                          V[ti, mi])
    np.testing.assert_allclose(sig, ref, rtol=1e-11, atol=1e-14)


def test_tda_and_rpa_agree_without_the_kernel():
    """K = 0: both reduce to sum_vc V^2 / (z + eta Delta)."""
    wl = _wl(kf=0.0)
    s_tda, _ = O.sigma_tda_closed_form(wl)
    s_rpa, _ = O.sigma_closed_form(wl)
    np.testing.assert_allclose(s_tda, s_rpa, rtol=1e-11, atol=1e-14)


def test_tda_lanczos_full_space_and_moments():
    wl = _wl()
    sig, poles = O.sigma_tda_closed_form(wl)
    sl, pl, co = O.sigma_tda_lanczos(wl, k=wl.n_vc)
    np.testing.assert_allclose(sl, sig, rtol=1e-10, atol=1e-13)
    # truncated k: Gauss moments sum_j w_j Om_j^p = V^T A^p V, p < 2k
    k = 4
    _, _, (al, be, b0, ke) = O.sigma_tda_lanczos(wl, k=k)
    A = O.tda_matrix(wl.eps, wl.n_v, wl.L, wl.kernel_factor)
    V = O.coupling_vectors(wl.L, wl.M).reshape(-1, wl.n_vc)
    for v in (0, 7, 29):
        T = np.diag(al[v]) + np.diag(be[v, :k - 1], 1) + np.diag(be[v, :k - 1], -1)
        Om, U = np.linalg.eigh(T)
        for p in range(2 * k):
            got = np.sum(b0[v] ** 2 * U[0] ** 2 * Om ** p)
            ref = V[v] @ np.linalg.matrix_power(A, p) @ V[v]
            assert abs(got - ref) <= 1e-9 * abs(ref)


def test_offdiagonal_by_polarisation():
    """Sigma_tt' from the closed form equals (Sigma[b_t + b_t'] - Sigma[b_t -
    b_t']) / 4 over diagonal elements of sums and differences of the start
    vectors (the identity the library's off-diagonal path uses); and it is
    symmetric in t, t'."""
    wl = _wl()
    s01 = O.sigma_offdiag_closed_form(wl, (0, 1))
    s10 = O.sigma_offdiag_closed_form(wl, (1, 0))
    np.testing.assert_allclose(s01, s10, rtol=1e-12)
    Mp = wl.M[0] + wl.M[1]
    Mm = wl.M[0] - wl.M[1]
    w2 = gi.Workload(**wl.__dict__)
    w2.targets = np.array([wl.targets[0], wl.targets[0]], dtype=np.int32)
    w2.M = np.stack([Mp, Mm])
    sd, _ = O.sigma_closed_form(w2)
    np.testing.assert_allclose((sd[0] - sd[1]) / 4.0, s01, rtol=1e-10, atol=1e-14)
