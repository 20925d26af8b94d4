"""Pins for the static part and the factor convention: orbitals and a
positive definite Coulomb-like kernel on a grid give the electron-repulsion
integrals by definition; the factors built from them must reproduce those
integrals, the Casida matrix, the exchange self-energy and the couplings."""
import numpy as np

import gw_inputs as gi
import oracle as O


def _grid_system(n_v=3, n_c=5, n_grid=40, seed=3):
    rng = np.random.default_rng(seed)
    r = np.sort(rng.uniform(0, 6, n_grid))
    Vk = np.exp(-0.5 * (r[:, None] - r[None, :]) ** 2) + 0.05 * np.eye(n_grid)   # PSD kernel
    phi = rng.standard_normal((n_v + n_c, n_grid)) / np.sqrt(n_grid)
    rho = phi[:, None, :] * phi[None, :, :]                        # pair densities [p][q][r]
    eri = np.einsum("pqr,rs,tus->pqtu", rho, Vk, rho)              # (pq|tu)
    # density fitting on the grid itself: C = rho, metric = Vk
    B = O.fit_factors(rho.reshape(-1, n_grid), Vk).reshape(n_v + n_c, n_v + n_c, n_grid)
    return n_v, n_c, eri, B


def test_factors_reproduce_the_integrals():
    n_v, n_c, eri, B = _grid_system()
    np.testing.assert_allclose(np.einsum("pqk,tuk->pqtu", B, B), eri, rtol=1e-11, atol=1e-14)


def test_casida_matrix_from_factors_is_the_rpa_one():
    """C = (A-B)^1/2 (A+B) (A-B)^1/2 with A, B from the integrals (Eq. 2-4,
    real orbitals) equals the oracle's Delta^2 + 2 Delta^1/2 L L^T Delta^1/2."""
    n_v, n_c, eri, B = _grid_system()
    eps = np.concatenate([np.sort(np.random.default_rng(1).uniform(-9, -4, n_v)),
                          np.sort(np.random.default_rng(2).uniform(-2, 6, n_c))])
    vc = [(v, n_v + c) for v in range(n_v) for c in range(n_c)]
    Delta = np.array([eps[c] - eps[v] for v, c in vc])
    Am = np.diag(Delta) + np.array([[eri[v, c, v2, c2] for v2, c2 in vc] for v, c in vc])
    Bm = np.array([[eri[v, c, c2, v2] for v2, c2 in vc] for v, c in vc])
    d = np.sqrt(Delta)
    Cref = d[:, None] * (Am + Bm) * d[None, :]
    L = np.array([B[v, c] for v, c in vc])
    np.testing.assert_allclose(O.casida_matrix(eps, n_v, L, 2.0), Cref, rtol=1e-11, atol=1e-13)


def test_exchange_from_factors():
    """Sigma^ex_t = -sum_v (vt|vt) by the integrals vs the oracle's sum of
    squared pair factors over the occupied part of the summed set."""
    n_v, n_c, eri, B = _grid_system()
    targets = np.array([1, 2, 4], dtype=np.int32)
    m_idx = np.arange(n_v + n_c, dtype=np.int32)
    wl = gi.make_workload("s", n_v, n_c, B.shape[2], targets, m_idx, 3, 1)
    wl.M = np.stack([B[t][m_idx] for t in targets])
    ref = np.array([-sum(eri[v, t, v, t] for v in range(n_v)) for t in targets])
    np.testing.assert_allclose(O.sigma_x(wl), ref, rtol=1e-12)


def test_linearised_qp_is_first_order():
    """The linearised solution is one Newton step from e0, so it misses the
    graphical one by about Sigma'' (E - e0)^2 / 2: scaling Sigma by s moves
    the difference like s^3 (ratio ~8 per halving)."""
    wl = gi.tiny()
    _, poles = O.sigma_closed_form(wl)
    diffs = []
    for sc in (1.0, 0.5):
        P = [(p, w * sc, e) for p, w, e in poles]
        Eg, _ = O.solve_all_qp(wl, P)
        El, _ = O.qp_linearised(wl, P)
        diffs.append(np.abs(Eg - El).max())
    assert 5.0 < diffs[0] / diffs[1] < 12.0, diffs
