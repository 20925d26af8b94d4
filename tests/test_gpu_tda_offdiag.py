"""Tamm-Dancoff variant and off-diagonal elements on the GPU."""
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


def _sys(L, h, wl):
    return L.lgw_prepare_system(h, wl.n_v, wl.n_c, wl.n_aux, _t(wl.eps), _t(wl.L),
                                wl.kernel_factor)


def _prob(L, wl):
    return L.Problem(targets=_t(wl.targets), m_idx=_t(wl.m_idx), omega=_t(wl.omega),
                     delta=wl.delta, M=_t(wl.M))


def _tda(L, h, wl, opts):
    s = _sys(L, h, wl)
    try:
        sig = torch.empty(wl.n_t, wl.omega.size, 2, dtype=torch.float64, device=DEV)
        e = torch.empty(wl.n_t, dtype=torch.float64, device=DEV)
        L.lgw_sigma_c_tda(h, s, _prob(L, wl), opts, sig, e)
        torch.cuda.synchronize()
    finally:
        L.lgw_release_system(s)
    sg = sig.cpu().numpy()
    return sg[..., 0] + 1j * sg[..., 1], e.cpu().numpy()


@pytest.mark.parametrize("reorth", ["cgs2", "none"])
def test_tda_fp64_vs_oracle_lanczos(L, handle, reorth):
    wl = gi.tiny(k=48)
    ref, poles, _ = O.sigma_tda_lanczos(wl, k=48, reorth=(reorth != "none"))
    Er, _ = O.solve_all_qp(wl, poles)
    sig, e = _tda(L, handle, wl, L.Options(k=48, precision="fp64", reorth=reorth))
    for ti in range(wl.n_t):
        assert np.abs(sig[ti] - ref[ti]).max() <= 1e-9 * np.abs(ref[ti]).max()
    assert np.abs(e - Er).max() <= 1e-9 * max(1.0, np.abs(Er).max())


def test_tda_full_space_and_bf16(L, handle):
    wl = gi.tiny(k=256)
    ref, poles = O.sigma_tda_closed_form(wl)
    Er, _ = O.solve_all_qp(wl, poles)
    sig, e = _tda(L, handle, wl, L.Options(k=256, precision="fp64", reorth="cgs2"))
    for ti in range(wl.n_t):
        assert np.abs(sig[ti] - ref[ti]).max() <= 1e-9 * np.abs(ref[ti]).max()
    assert np.abs(e - Er).max() <= 1e-9 * max(1.0, np.abs(Er).max())
    _, e16 = _tda(L, handle, wl, L.Options(k=256, precision="bf16", reorth="cgs2"))
    d = np.abs(e16 - Er).max() * 1e3
    print(f"TDA bf16 vs closed form: {d:.3e} meV")
    assert d <= 1.0


def test_offdiagonal_vs_closed_form(L, handle):
    """k = N_vc: Sigma_tt' equals the closed form (FP64, 1e-9 of its scale);
    pairs (0,1), (2,3), (1,3) and the diagonal pair (2,2) (= Sigma_tt)."""
    wl = gi.tiny(k=256)
    pairs = np.array([[0, 1], [2, 3], [1, 3], [2, 2]], dtype=np.int32)
    s = _sys(L, handle, wl)
    try:
        od = torch.empty(len(pairs), wl.omega.size, 2, dtype=torch.float64, device=DEV)
        L.lgw_sigma_offdiag(handle, s, _prob(L, wl), L.Options(k=256, precision="fp64",
                                                                reorth="cgs2"),
                            _t(pairs.ravel()), od)
        torch.cuda.synchronize()
    finally:
        L.lgw_release_system(s)
    got = od.cpu().numpy()
    got = got[..., 0] + 1j * got[..., 1]
    sigx, _ = O.sigma_closed_form(wl)
    for i, (a, b) in enumerate(pairs):
        ref = O.sigma_offdiag_closed_form(wl, (a, b))
        scale = max(np.abs(ref).max(), np.abs(sigx).max() * 1e-3)
        assert np.abs(got[i] - ref).max() <= 1e-9 * scale, (a, b)
    np.testing.assert_allclose(got[3], sigx[2], rtol=1e-9, atol=1e-9 * np.abs(sigx[2]).max())
