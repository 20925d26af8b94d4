"""Static part and density-fitting front end on the GPU: exchange
self-energy, the linearised QP solution, and the factors B = C chol(metric)
feeding the whole path."""
import numpy as np
import pytest

import gw_inputs as gi
import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _t(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to(DEV)


@pytest.fixture(scope="module")
def L():
    from paper_2310_20103_gb300.build import build
    build()
    from paper_2310_20103_gb300 import lgw
    return lgw


@pytest.fixture(scope="module")
def handle(L):
    h = L.lgw_create(0)
    yield h
    L.lgw_destroy(h)


def _prob(L, wl, shift=None, use_v=False):
    kw = dict(targets=_t(wl.targets), m_idx=_t(wl.m_idx), omega=_t(wl.omega), delta=wl.delta)
    if use_v:
        kw["V"] = _t(O.coupling_vectors(wl.L, wl.M))
    else:
        kw["M"] = _t(wl.M)
    if shift is not None:
        kw["static_shift"] = _t(shift)
    return L.Problem(**kw)


def test_exchange_matches_oracle(L, handle):
    wl = gi.tiny()
    s = L.lgw_prepare_system(handle, wl.n_v, wl.n_c, wl.n_aux, _t(wl.eps), _t(wl.L))
    try:
        out = torch.empty(wl.n_t, dtype=torch.float64, device=DEV)
        L.lgw_sigma_x(handle, s, _prob(L, wl), out)
        torch.cuda.synchronize()
        np.testing.assert_allclose(out.cpu().numpy(), O.sigma_x(wl), rtol=1e-12)
        with pytest.raises(L.LgwError) as ei:
            L.lgw_sigma_x(handle, s, _prob(L, wl, use_v=True), out)
        assert ei.value.status == 8
    finally:
        L.lgw_release_system(s)


@pytest.mark.parametrize("mode", ["graphical", "linearised"])
def test_qp_modes_with_static_shift(L, handle, mode):
    """E_qp with s_t = Sigma^ex_t - V_xc_t (a seeded V_xc) in both QP modes
    against the oracle on the k = 64 Lanczos poles (FP64, 1e-9)."""
    wl = gi.tiny(k=64)
    vxc = np.random.default_rng(5).uniform(-1.0, 1.0, wl.n_t)
    shift = O.sigma_x(wl) - vxc
    _, poles, _ = O.sigma_lanczos(wl, k=64)
    if mode == "graphical":
        Er, Zr = O.solve_all_qp(wl, poles, static_shift=shift)
    else:
        Er, Zr = O.qp_linearised(wl, poles, static_shift=shift)
    s = L.lgw_prepare_system(handle, wl.n_v, wl.n_c, wl.n_aux, _t(wl.eps), _t(wl.L))
    try:
        sig = torch.empty(wl.n_t, wl.omega.size, 2, dtype=torch.float64, device=DEV)
        e = torch.empty(wl.n_t, dtype=torch.float64, device=DEV)
        z = torch.empty(wl.n_t, dtype=torch.float64, device=DEV)
        L.lgw_sigma_c(handle, s, _prob(L, wl, shift=shift),
                      L.Options(k=64, precision="fp64", reorth="cgs2", qp_mode=mode), sig, e, z)
        torch.cuda.synchronize()
    finally:
        L.lgw_release_system(s)
    np.testing.assert_allclose(e.cpu().numpy(), Er, rtol=1e-9, atol=1e-9)
    np.testing.assert_allclose(z.cpu().numpy(), Zr, rtol=1e-8)


@pytest.mark.parametrize("n_pairs,n_aux", [(1000, 200), (300, 64), (50, 130)])
def test_fit_factors_match_oracle(L, handle, n_pairs, n_aux):
    rng = np.random.default_rng(n_aux)
    G = rng.standard_normal((n_aux, n_aux))
    metric = G @ G.T / n_aux + 0.1 * np.eye(n_aux)
    C = rng.standard_normal((n_pairs, n_aux))
    ref = O.fit_factors(C, metric)
    B = torch.empty(n_pairs, n_aux, dtype=torch.float64, device=DEV)
    L.lgw_fit_factors(handle, _t(C), _t(metric), B)
    torch.cuda.synchronize()
    np.testing.assert_allclose(B.cpu().numpy(), ref, rtol=1e-10, atol=1e-12)


def test_fit_factors_reject_indefinite_metric(L, handle):
    metric = np.diag([1.0, 2.0, -1.0, 3.0])
    C = np.ones((5, 4))
    B = torch.empty(5, 4, dtype=torch.float64, device=DEV)
    with pytest.raises(L.LgwError) as ei:
        L.lgw_fit_factors(handle, _t(C), _t(metric), B)
    assert ei.value.status == 5


def test_density_fitted_inputs_end_to_end(L, handle):
    """Orbitals and a positive definite kernel on a grid: the GPU builds L and M
    from the fitting coefficients (the pair densities) and the metric, and the
    whole path then matches the oracle's closed form on the same factors."""
    rng = np.random.default_rng(7)
    n_v, n_c, n_grid = 4, 12, 96
    r = np.sort(rng.uniform(0, 8, n_grid))
    metric = np.exp(-0.5 * (r[:, None] - r[None, :]) ** 2) + 0.05 * np.eye(n_grid)
    phi = rng.standard_normal((n_v + n_c, n_grid)) / np.sqrt(n_grid)
    eps = np.concatenate([np.sort(rng.uniform(-12, -5, n_v)), np.sort(rng.uniform(-3, 20, n_c))])
    vc = [(v, n_v + c) for v in range(n_v) for c in range(n_c)]
    targets = np.array([2, 3, 4, 5], dtype=np.int32)
    m_idx = np.arange(n_v + n_c, dtype=np.int32)
    C_vc = np.array([phi[v] * phi[c] for v, c in vc])
    C_tm = np.array([phi[t] * phi[m] for t in targets for m in m_idx])
    Lf = torch.empty(len(vc), n_grid, dtype=torch.float64, device=DEV)
    Mf = torch.empty(len(C_tm), n_grid, dtype=torch.float64, device=DEV)
    L.lgw_fit_factors(handle, _t(C_vc), _t(metric), Lf)
    L.lgw_fit_factors(handle, _t(C_tm), _t(metric), Mf)
    torch.cuda.synchronize()
    wl = gi.make_workload("df", n_v, n_c, n_grid, targets, m_idx, 150, 1, k=len(vc))
    wl.eps = eps
    wl.L = O.fit_factors(C_vc, metric)
    wl.M = O.fit_factors(C_tm, metric).reshape(len(targets), len(m_idx), n_grid)
    np.testing.assert_allclose(Lf.cpu().numpy(), wl.L, rtol=1e-10, atol=1e-13)
    _, polesx = O.sigma_closed_form(wl)
    Ex, _ = O.solve_all_qp(wl, polesx)
    s = L.lgw_prepare_system(handle, n_v, n_c, n_grid, _t(eps), Lf)
    try:
        prob = L.Problem(targets=_t(targets), m_idx=_t(m_idx), omega=_t(wl.omega),
                         delta=wl.delta, M=Mf.reshape(len(targets), len(m_idx), n_grid))
        sig = torch.empty(wl.n_t, wl.omega.size, 2, dtype=torch.float64, device=DEV)
        e = torch.empty(wl.n_t, dtype=torch.float64, device=DEV)
        L.lgw_sigma_c(handle, s, prob, L.Options(k=len(vc), precision="fp64", reorth="cgs2"),
                      sig, e)
        torch.cuda.synchronize()
    finally:
        L.lgw_release_system(s)
    np.testing.assert_allclose(e.cpu().numpy(), Ex, rtol=1e-9, atol=1e-9)
