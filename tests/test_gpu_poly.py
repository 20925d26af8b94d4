"""Polynomial variant on the GPU (lgw_sigma_c_poly: Lanczos on D = p_g(C),
Haydock fractions at 0 and -eta z) against the oracle."""
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


def _bounds(wl):
    th = np.linalg.eigvalsh(O.casida_matrix(wl.eps, wl.n_v, wl.L, wl.kernel_factor))
    return th.min(), th.max()


def _run(L, h, wl, g, lo, hi, opts):
    s = L.lgw_prepare_system(h, wl.n_v, wl.n_c, wl.n_aux, _t(wl.eps), _t(wl.L),
                             wl.kernel_factor)
    prob = L.Problem(targets=_t(wl.targets), m_idx=_t(wl.m_idx), omega=_t(wl.omega),
                     delta=wl.delta, M=_t(wl.M))
    try:
        sig = torch.empty(wl.n_t, wl.omega.size, 2, dtype=torch.float64, device=DEV)
        e = torch.empty(wl.n_t, dtype=torch.float64, device=DEV)
        L.lgw_sigma_c_poly(h, s, prob, opts, g, lo, hi, sig, e)
        B = wl.n_t * wl.n_m
        al = torch.empty(B, opts.k, dtype=torch.float64, device=DEV)
        be = torch.empty_like(al)
        b0 = torch.empty(B, dtype=torch.float64, device=DEV)
        ke = torch.empty(B, dtype=torch.int32, device=DEV)
        L.lgw_lanczos_coeffs_poly(h, s, prob, opts, g, lo, hi, al, be, b0, ke)
        torch.cuda.synchronize()
    finally:
        L.lgw_release_system(s)
    sg = sig.cpu().numpy()
    return (sg[..., 0] + 1j * sg[..., 1], e.cpu().numpy(),
            (al.cpu().numpy(), be.cpu().numpy(), b0.cpu().numpy(), ke.cpu().numpy()))


@pytest.mark.parametrize("g,k,reorth", [(8, 24, "cgs2"), (3, 16, "none"), (12, 40, "cgs1k")])
def test_fp64_matches_oracle(L, handle, g, k, reorth):
    wl = gi.tiny(k=k)
    lo, hi = _bounds(wl)
    ref, poles, co = O.sigma_poly_lanczos(wl, g, lo, hi, k=k, reorth=(reorth != "none"))
    Er, _ = O.solve_all_qp(wl, poles)
    sig, e, gco = _run(L, handle, wl, g, lo, hi, L.Options(k=k, precision="fp64", reorth=reorth))
    for ti in range(wl.n_t):
        assert np.abs(sig[ti] - ref[ti]).max() <= 1e-9 * np.abs(ref[ti]).max()
    assert np.abs(e - Er).max() <= 1e-9 * max(1.0, np.abs(Er).max())
    np.testing.assert_array_equal(gco[3], co[3])
    np.testing.assert_allclose(gco[0], co[0], rtol=1e-10, atol=1e-10)
    np.testing.assert_allclose(gco[1], co[1], rtol=1e-9, atol=1e-10)


def test_full_space_and_bf16(L, handle):
    """k = N_vc: the GPU reproduces the closed form with Omega_s -> p_g(theta_s)
    (FP64, 1e-9), and the BF16 contractions stay within 1 meV of it."""
    wl = gi.tiny(k=256)
    lo, hi = _bounds(wl)
    g = 10
    _, poles, _ = O.sigma_poly_lanczos(wl, g, lo, hi, k=wl.n_vc)
    Er, _ = O.solve_all_qp(wl, poles)
    _, e64, _ = _run(L, handle, wl, g, lo, hi, L.Options(k=wl.n_vc, precision="fp64",
                                                           reorth="cgs2"))
    assert np.abs(e64 - Er).max() <= 1e-9 * max(1.0, np.abs(Er).max())
    _, e16, _ = _run(L, handle, wl, g, lo, hi, L.Options(k=wl.n_vc, precision="bf16",
                                                           reorth="cgs2"))
    d = np.abs(e16 - Er).max() * 1e3
    print(f"bf16 polynomial variant vs oracle: {d:.3e} meV")
    assert d <= 1.0


def test_fig1_analogue(L, handle):
    """Synthetic analogue of Fig. 1b/1c: max |E_qp - E_exact| (meV) of the
    polynomial variant on the GPU against the closed form, vs the degree g at
    k = 64 and vs the Lanczos steps k at g = 16.  The error falls with g and
    with k until the other limit takes over."""
    wl = gi.tiny(k=64)
    lo, hi = _bounds(wl)
    _, polesx = O.sigma_closed_form(wl)
    Ex, _ = O.solve_all_qp(wl, polesx)
    by_g = {}
    for g in (2, 4, 8, 16, 32):
        _, e, _ = _run(L, handle, wl, g, lo, hi, L.Options(k=64, precision="fp64", reorth="cgs2"))
        by_g[g] = np.abs(e - Ex).max() * 1e3
    by_k = {}
    for k in (2, 4, 8, 16, 32, 64):
        _, e, _ = _run(L, handle, wl, 16, lo, hi, L.Options(k=k, precision="fp64",
                                                             reorth="cgs2"))
        by_k[k] = np.abs(e - Ex).max() * 1e3
    print("meV by g (k=64):", {g: f"{v:.3e}" for g, v in by_g.items()})
    print("meV by k (g=16):", {k: f"{v:.3e}" for k, v in by_k.items()})
    assert by_g[32] < by_g[8] < by_g[2]
    assert by_k[64] < by_k[8] < by_k[2]


def test_spectral_interval_encloses_the_spectrum(L, handle):
    """lgw_spectral_interval: x_lo = min Delta^2 lies below lambda_min (C =
    Delta^2 + a positive semidefinite term) and x_hi, the largest Ritz value
    plus its residual norm, lies above lambda_max and within 25% of it
    (tiny system, dense eigenvalues by numpy)."""
    wl = gi.tiny()
    lam_lo, lam_hi = _bounds(wl)
    s = L.lgw_prepare_system(handle, wl.n_v, wl.n_c, wl.n_aux, _t(wl.eps), _t(wl.L),
                             wl.kernel_factor)
    try:
        lo, hi = L.lgw_spectral_interval(handle, s, 32)
    finally:
        L.lgw_release_system(s)
    D = O.pair_energies(wl.eps, wl.n_v)
    assert lo == pytest.approx(float((D ** 2).min()), rel=1e-15)
    assert lo <= lam_lo
    assert lam_hi <= hi <= 1.25 * lam_hi


def test_poly_with_library_interval(L, handle):
    """x_lo = x_hi = 0 makes lgw_sigma_c_poly take lgw_spectral_interval's
    interval: the results are bit-identical to passing that interval, and
    the QP energies stay within 1 meV of the closed form at g = 16."""
    wl = gi.tiny()
    s = L.lgw_prepare_system(handle, wl.n_v, wl.n_c, wl.n_aux, _t(wl.eps), _t(wl.L),
                             wl.kernel_factor)
    try:
        lo, hi = L.lgw_spectral_interval(handle, s, 32)
    finally:
        L.lgw_release_system(s)
    opts = L.Options(k=64, precision="fp64", reorth="cgs2")
    sig_a, e_a, co_a = _run(L, handle, wl, 16, 0.0, 0.0, opts)
    sig_b, e_b, co_b = _run(L, handle, wl, 16, lo, hi, opts)
    assert np.array_equal(e_a, e_b)
    assert np.array_equal(sig_a, sig_b)
    _, polesx = O.sigma_closed_form(wl)
    Ex, _ = O.solve_all_qp(wl, polesx)
    assert np.abs(e_a - Ex).max() < 1e-3
