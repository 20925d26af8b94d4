"""Pins of the oracle's band Lanczos (off-diagonal Sigma_tt', the band
method for resolvent matrix elements cited after Eq. 14).

  * once the block Krylov space is exhausted (k = N_vc) every element equals
    the closed form from the Casida eigenpairs (Eq. 7-9), off-diagonal
    elements included;
  * with one target (p = 1) the band recurrence is the ordinary Lanczos
    recurrence, so Sigma_tt equals the oracle's single-vector result at the
    same k;
  * the matrix Gauss rule reproduces the block moments B C^n B^T, computed
    by repeated products with C, for n <= 2 (k / p) - 1 (block Gauss
    quadrature exactness);
  * an invariant subspace (c_K = 0, sparse coupling vectors) stops the
    recurrence early and gives the exact result.
"""
import numpy as np

import gw_inputs as gi
import oracle as O


def _apply(wl):
    return lambda X: O.apply_casida(wl.eps, wl.n_v, wl.L, X, wl.kernel_factor)


def test_full_space_equals_closed_form():
    wl = gi.make_workload("bd", 3, 6, 10, [1, 2, 3], [0, 1, 2, 5, 7], 60, 11, k=18)
    sig, recs = O.sigma_band_lanczos(wl, k=wl.n_vc)
    assert all(ke == wl.n_vc for _, _, ke in recs)
    diag, _ = O.sigma_closed_form(wl)
    for a in range(wl.n_t):
        ref = diag[a]
        assert np.abs(sig[a, a] - ref).max() <= 1e-10 * np.abs(ref).max()
        for b in range(a + 1, wl.n_t):
            ref = O.sigma_offdiag_closed_form(wl, (a, b))
            assert np.abs(sig[a, b] - ref).max() <= 1e-10 * np.abs(ref).max()
            assert np.abs(sig[b, a] - ref).max() <= 1e-10 * np.abs(ref).max()


def test_one_target_is_ordinary_lanczos():
    wl = gi.make_workload("b1", 4, 9, 20, [3], list(range(13)), 40, 5, k=12, aux_scaled=True)
    sig, _ = O.sigma_band_lanczos(wl, k=12)
    ref, _, _ = O.sigma_lanczos(wl, k=12)
    assert np.abs(sig[0, 0] - ref[0]).max() <= 1e-11 * np.abs(ref[0]).max()


def test_block_moments():
    wl = gi.make_workload("bm", 4, 12, 24, [2, 3, 4], [0, 5], 10, 7, k=12)
    apply_op = _apply(wl)
    b = O.start_vectors(wl.eps, wl.n_v, O.coupling_vectors(wl.L, wl.M))
    B = b[:, 1, :]                       # block of the three targets for one m
    p, k = B.shape[0], 12
    T, R0, ke = O.band_lanczos(apply_op, B, k)
    assert ke == k
    theta, r = O.band_gauss_rule(T, R0)
    X = B.copy()
    scale = theta.max()
    for n in range(2 * (k // p)):
        mom = (r * theta ** n) @ r.T
        ref = B @ X.T                     # B C^n B^T with X = C^n B
        assert np.abs(mom - ref).max() <= 1e-9 * np.abs(ref).max(), n
        X = apply_op(X)
    # past the exactness degree the rule no longer reproduces the moment
    X = B.copy()
    for _ in range(2 * (k // p) + 2):
        X = apply_op(X)
    n = 2 * (k // p) + 2
    assert np.abs((r * theta ** n) @ r.T - B @ X.T).max() > 1e-6 * scale ** n


def test_invariant_subspace_stops_early():
    wl = gi.make_workload("bi", 3, 5, 6, [1, 2], [0, 4], 31, 9, k=8, kernel_factor=0.0)
    V = np.zeros((2, 2, wl.n_vc))
    V[0, 0, [0, 4, 9]] = [0.3, -0.2, 0.5]
    V[1, 0, [0, 9, 11]] = [0.1, 0.4, -0.3]
    V[0, 1, [1, 7]] = [0.2, 0.6]
    V[1, 1, [7, 14]] = [-0.5, 0.1]
    Delta = O.pair_energies(wl.eps, wl.n_v)
    b = np.sqrt(Delta)[None, None, :] * V
    apply_op = _apply(wl)
    for mi, m in enumerate(wl.m_idx):
        T, R0, ke = O.band_lanczos(apply_op, b[:, mi, :], 8)
        support = np.count_nonzero(np.any(V[:, mi, :] != 0.0, axis=0))
        assert ke == support                       # the Krylov space spans the support
        theta, r = O.band_gauss_rule(T, R0)
        eta = 1.0 if m < wl.n_v else -1.0
        z = wl.omega[:, None] - wl.eps[m] - 1j * eta * wl.delta
        got = np.einsum("s,fs->f", r[0] * r[1], 1.0 / (np.sqrt(theta) * (z + eta * np.sqrt(theta))))
        # C = Delta^2: Sigma_01 = sum_vc b0 b1 / (Delta (z + eta Delta)) exactly
        ref = np.sum(b[0, mi] * b[1, mi] / (Delta * (z + eta * Delta)), axis=1)
        assert np.abs(got - ref).max() <= 1e-12 * max(1.0, np.abs(ref).max())
