"""GPU band Lanczos (lgw_sigma_band): the self-energy matrix Sigma_tt'(omega)
of a request's targets from one band recurrence per summed orbital.

Bars:
  * FP64 contractions vs the oracle's band recurrence at the same k: every
    element within 1e-9 of the largest |Sigma| of the matrix (per target
    pair, max over the grid);
  * k = N_vc (block Krylov space exhausted) vs the closed form (Eq. 7-9) and
    its off-diagonal elements: 1e-9;
  * one target: equal to lgw_sigma_c's Sigma_t at the same k (1e-9);
  * BF16 contractions: within 1% of the largest |Sigma| (the bar of the
    diagonal BF16 test on the grid);
  * an invariant subspace stops each recurrence early with the exact result.
"""
import numpy as np
import pytest

import gw_inputs as gi
import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


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


def _t(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to(DEV)


def _band(L, h, wl, opts, V=None, report=False):
    s = L.lgw_prepare_system(h, wl.n_v, wl.n_c, wl.n_aux, _t(wl.eps), _t(wl.L),
                             wl.kernel_factor)
    try:
        kw = dict(targets=_t(wl.targets), m_idx=_t(wl.m_idx), omega=_t(wl.omega),
                  delta=wl.delta)
        if V is None:
            kw["M"] = _t(wl.M)
        else:
            kw["V"] = _t(V)
        sig = torch.empty(wl.n_t, wl.n_t, wl.omega.size, 2, dtype=torch.float64, device=DEV)
        rep = L.lgw_sigma_band(h, s, L.Problem(**kw), opts, sig, report=report)
        torch.cuda.synchronize()
    finally:
        L.lgw_release_system(s)
    g = sig.cpu().numpy()
    return g[..., 0] + 1j * g[..., 1], rep


def _err(got, ref):
    return np.abs(got - ref).max() / np.abs(ref).max()


def test_fp64_vs_oracle_band(L, handle):
    wl = gi.tiny()
    ref, _ = O.sigma_band_lanczos(wl, k=64)
    got, rep = _band(L, handle, wl, L.Options(k=64, precision="fp64"), report=True)
    assert _err(got, ref) < 1e-9
    assert np.abs(got - np.swapaxes(got, 0, 1)).max() == 0.0
    assert rep["gpu_launches"] > 0


def test_full_space_vs_closed_form(L, handle):
    wl = gi.tiny()
    got, _ = _band(L, handle, wl, L.Options(k=wl.n_vc, precision="fp64"))
    diag, _ = O.sigma_closed_form(wl)
    ref = np.zeros_like(got)
    for a in range(wl.n_t):
        ref[a, a] = diag[a]
        for b in range(a + 1, wl.n_t):
            ref[a, b] = ref[b, a] = O.sigma_offdiag_closed_form(wl, (a, b))
    assert _err(got, ref) < 1e-9
    gotb, _ = _band(L, handle, wl, L.Options(k=wl.n_vc, precision="bf16"))
    assert _err(gotb, ref) < 1e-2


def test_one_target_equals_sigma_c(L, handle):
    wl = gi.make_workload("b1", 4, 9, 20, [3], list(range(13)), 40, 5, k=12, aux_scaled=True)
    got, _ = _band(L, handle, wl, L.Options(k=12, precision="fp64"))
    s = L.lgw_prepare_system(handle, wl.n_v, wl.n_c, wl.n_aux, _t(wl.eps), _t(wl.L))
    sig = torch.empty(1, wl.omega.size, 2, dtype=torch.float64, device=DEV)
    e = torch.empty(1, dtype=torch.float64, device=DEV)
    L.lgw_sigma_c(handle, s, L.Problem(targets=_t(wl.targets), m_idx=_t(wl.m_idx),
                                       omega=_t(wl.omega), delta=wl.delta, M=_t(wl.M)),
                  L.Options(k=12, precision="fp64", reorth="cgs2"), sig, e)
    torch.cuda.synchronize()
    L.lgw_release_system(s)
    sc = sig.cpu().numpy()[0]
    sc = sc[:, 0] + 1j * sc[:, 1]
    assert np.abs(got[0, 0] - sc).max() <= 1e-9 * np.abs(sc).max()


def test_mid_ragged_sub_batches(L, handle):
    """N_vc = 13 * 347 (several 2048-element chunks, ragged tail), three
    targets, 21 summed orbitals in sub-batches of 8 groups, k = 40."""
    wl = gi.make_workload("bm", 13, 347, 300, [11, 12, 13], list(range(21)), 120, 2, k=40,
                          aux_scaled=True)
    ref, _ = O.sigma_band_lanczos(wl, k=40)
    got, _ = _band(L, handle, wl, L.Options(k=40, precision="fp64", b_sub=8))
    assert _err(got, ref) < 1e-9
    gotb, _ = _band(L, handle, wl, L.Options(k=40, precision="bf16"))
    assert _err(gotb, ref) < 1e-2


def test_invariant_subspace(L, handle):
    wl = gi.make_workload("bi", 3, 5, 6, [1, 2], [0, 4], 31, 9, k=8, kernel_factor=0.0)
    V = np.zeros((2, 2, wl.n_vc))
    V[0, 0, [0, 4, 9]] = [0.3, -0.2, 0.5]
    V[1, 0, [0, 9, 11]] = [0.1, 0.4, -0.3]
    V[0, 1, [1, 7]] = [0.2, 0.6]
    V[1, 1, [7, 14]] = [-0.5, 0.1]
    got, _ = _band(L, handle, wl, L.Options(k=8, precision="fp64"), V=V)
    Delta = O.pair_energies(wl.eps, wl.n_v)
    b = np.sqrt(Delta)[None, None, :] * V
    ref = np.zeros_like(got)
    for mi, m in enumerate(wl.m_idx):
        eta = 1.0 if m < wl.n_v else -1.0
        z = wl.omega[:, None] - wl.eps[m] - 1j * eta * wl.delta
        for a in range(2):
            for c in range(2):
                ref[a, c] += np.sum(b[a, mi] * b[c, mi] / (Delta * (z + eta * Delta)), axis=1)
    assert _err(got, ref) < 1e-10
