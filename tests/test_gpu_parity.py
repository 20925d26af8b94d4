"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Tolerances
  * FP64 path vs oracle Lanczos at the same k: 1e-9 relative on Sigma
    (max over the grid, per target) and 1e-9 * max(1, |E|) eV on E_qp.
  * FP64 path at k = N_vc vs the closed form (Eq. 7-9): same bounds.
  * BF16 contractions vs the oracle on the FP64 factor: 1 meV on E_qp.
"""
import numpy as np
import pytest

import gw_inputs as gi
import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


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


DEV = "cuda:0"


def _t(x, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(x))
    if dtype is not None:
        t = t.to(dtype)
    return t.to(DEV)


def _system(L, h, wl):
    return L.lgw_prepare_system(h, wl.n_v, wl.n_c, wl.n_aux, _t(wl.eps), _t(wl.L),
                                wl.kernel_factor)


def _problem(L, wl, use_V=False):
    kw = dict(targets=_t(wl.targets), m_idx=_t(wl.m_idx), omega=_t(wl.omega), delta=wl.delta)
    if use_V:
        kw["V"] = _t(O.coupling_vectors(wl.L, wl.M))
    else:
        kw["M"] = _t(wl.M)
    return L.Problem(**kw)


def _run(L, h, wl, opts, use_V=False, report=False):
    s = _system(L, h, wl)
    try:
        sig = torch.empty(wl.n_t, wl.omega.size, 2, dtype=torch.float64, device=DEV)
        e = torch.empty(wl.n_t, dtype=torch.float64, device=DEV)
        z = torch.empty(wl.n_t, dtype=torch.float64, device=DEV)
        rep = L.lgw_sigma_c(h, s, _problem(L, wl, use_V), opts, sig, e, z, report=report)
        torch.cuda.synchronize()
    finally:
        L.lgw_release_system(s)
    sg = sig.cpu().numpy()
    return sg[..., 0] + 1j * sg[..., 1], e.cpu().numpy(), z.cpu().numpy(), rep


def _rel_sigma_err(a, b):
    return max(np.abs(a[i] - b[i]).max() / np.abs(b[i]).max() for i in range(a.shape[0]))


# ---------------------------------------------------------------------------
# the contractions alone
# ---------------------------------------------------------------------------
def _apply(L, h, wl, X, prec):
    s = _system(L, h, wl)
    try:
        Xd = _t(X)
        Y = torch.empty_like(Xd)
        L.lgw_apply_casida(h, s, Xd, Y, prec)
        torch.cuda.synchronize()
    finally:
        L.lgw_release_system(s)
    return Y.cpu().numpy()


@pytest.mark.parametrize("shape", [(8, 32, 128, 5), (7, 131, 200, 70), (16, 300, 384, 300)])
def test_apply_fp64_matches_oracle(L, handle, shape):
    n_v, n_c, A, nvec = shape
    wl = gi.make_workload("a", n_v, n_c, A, [0], [0], 3, 5, aux_scaled=True)
    X = np.random.default_rng(1).standard_normal((nvec, wl.n_vc))
    Y = _apply(L, handle, wl, X, "fp64")
    ref = O.apply_casida(wl.eps, wl.n_v, wl.L, X, wl.kernel_factor)
    assert np.abs(Y - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("shape", [(8, 32, 128, 5), (7, 131, 200, 70), (16, 300, 384, 300),
                                   (32, 256, 256, 512)])
def test_apply_bf16_tensor_core_exact(L, handle, shape):
    """Delta = 1 and ternary L, x: every product and partial sum is an
    integer that BF16/FP32 hold exactly, so the tcgen05 contractions must
    reproduce the FP64 product bit for bit (tiles, K splits, ragged M, N, K)."""
    n_v, n_c, A, nvec = shape
    rng = np.random.default_rng(3)
    eps = np.concatenate([np.full(n_v, -0.5), np.full(n_c, 0.5)])
    wl = gi.make_workload("x", n_v, n_c, A, [0], [0], 3, 5)
    wl.eps = eps
    p = min(0.3, 6.0 / np.sqrt(wl.n_vc))
    wl.L = (rng.choice([-1.0, 0.0, 1.0], size=(wl.n_vc, A), p=[p / 2, 1 - p, p / 2]))
    X = rng.choice([-1.0, 0.0, 1.0], size=(nvec, wl.n_vc), p=[p / 2, 1 - p, p / 2])
    Y = (X @ wl.L)
    assert np.abs(Y).max() <= 256   # bf16-exact intermediate
    ref = X + wl.kernel_factor * (Y @ wl.L.T)
    got = _apply(L, handle, wl, X, "bf16")
    np.testing.assert_array_equal(got, ref)


# ---------------------------------------------------------------------------
# full path, tiny workload
# ---------------------------------------------------------------------------
@pytest.fixture(scope="module")
def tiny_ref():
    wl = gi.tiny()
    sig64, poles64, co64 = O.sigma_lanczos(wl, k=64)
    E64, Z64 = O.solve_all_qp(wl, poles64)
    sigx, polesx = O.sigma_closed_form(wl)
    Ex, Zx = O.solve_all_qp(wl, polesx)
    return wl, (sig64, E64, Z64, co64), (sigx, Ex, Zx)


@pytest.mark.parametrize("arith", ["fp64", "split"])
@pytest.mark.parametrize("reorth", ["cgs2", "cgs1k"])
def test_tiny_fp64_k64_vs_oracle_lanczos(L, handle, tiny_ref, reorth, arith):
    """FP64 contractions with either reorthogonalisation arithmetic: the
    split (double-float) basis must be as accurate as the FP64 one."""
    wl, (sig64, E64, Z64, _), _ = tiny_ref
    sig, e, z, _ = _run(L, handle, wl, L.Options(k=64, precision="fp64", reorth=reorth,
                                                 reorth_arith=arith))
    assert _rel_sigma_err(sig, sig64) < 1e-9
    assert np.all(np.abs(e - E64) <= 1e-9 * np.maximum(1, np.abs(E64)))
    assert np.all(np.abs(z - Z64) <= 1e-8)


def test_float_basis_option(L, handle, tiny_ref):
    """Float-only basis (split32): w is orthogonalised against fl32(q_i), so
    orthogonality to the FP64 q_i is ~2^-24 / sqrt(N_vc) ~ 4e-9 here and T_k
    inherits errors of that relative size; Sigma within 1e-6 relative and
    E_qp within 1e-8 eV of the oracle (FP64 contractions)."""
    wl, (sig64, E64, _, _), _ = tiny_ref
    for reorth in ("cgs2", "cgs1k"):
        sig, e, _, _ = _run(L, handle, wl, L.Options(k=64, precision="fp64", reorth=reorth,
                                                     reorth_arith="split32"))
        assert _rel_sigma_err(sig, sig64) < 1e-6
        assert np.abs(e - E64).max() < 1e-8


@pytest.mark.parametrize("arith", ["fp64", "split"])
def test_tiny_fp64_full_k_vs_closed_form(L, handle, tiny_ref, arith):
    wl, _, (sigx, Ex, Zx) = tiny_ref
    sig, e, z, _ = _run(L, handle, wl, L.Options(k=wl.n_vc, precision="fp64", reorth="cgs2",
                                                 reorth_arith=arith))
    assert _rel_sigma_err(sig, sigx) < 1e-9
    assert np.all(np.abs(e - Ex) <= 1e-9 * np.maximum(1, np.abs(Ex)))


def test_tiny_bf16_within_1meV(L, handle, tiny_ref):
    """BF16 contractions: QP energies within 1 meV of the FP64 closed form.
    On the grid, with k = N_vc (Gauss nodes = Casida eigenvalues, so only
    the BF16 perturbation of C moves them), Sigma stays within 1% of the
    closed form; near a pole |dSigma| ~ (w/delta^2) dOmega, and BF16
    rounding (2^-9) of the coupling moves Omega by well under delta."""
    wl, _, (sigx, Ex, Zx) = tiny_ref
    sig, e, z, _ = _run(L, handle, wl, L.Options(k=64, precision="bf16", reorth="cgs2"))
    assert np.abs(e - Ex).max() < 1e-3
    sigf, ef, _, _ = _run(L, handle, wl, L.Options(k=wl.n_vc, precision="bf16", reorth="cgs2"))
    assert np.abs(ef - Ex).max() < 1e-3
    assert _rel_sigma_err(sigf, sigx) < 1e-2


def test_coefficients_vs_oracle(L, handle, tiny_ref):
    wl, (_, _, _, (a_ref, b_ref, b0_ref, k_ref)), _ = tiny_ref
    s = _system(L, handle, wl)
    B, k = wl.n_t * wl.n_m, 64
    al = torch.empty(B, k, dtype=torch.float64, device=DEV)
    be = torch.empty(B, k, dtype=torch.float64, device=DEV)
    b0 = torch.empty(B, dtype=torch.float64, device=DEV)
    ke = torch.empty(B, dtype=torch.int32, device=DEV)
    L.lgw_lanczos_coeffs(handle, s, _problem(L, wl), L.Options(k=k, precision="fp64"), al, be,
                         b0, ke)
    torch.cuda.synchronize()
    L.lgw_release_system(s)
    assert np.array_equal(ke.cpu().numpy(), k_ref)
    np.testing.assert_allclose(b0.cpu().numpy(), b0_ref, rtol=1e-13)
    np.testing.assert_allclose(al.cpu().numpy(), a_ref, rtol=1e-9)
    np.testing.assert_allclose(be.cpu().numpy(), b_ref, rtol=1e-7)


def test_sigma_from_oracle_coefficients(L, handle, tiny_ref):
    """Spectral map + continued fractions + QP alone: feed the oracle's own
    tridiagonals and compare with the oracle's pole sums."""
    wl, (sig64, E64, Z64, (a0, b0, bb0, k0)), _ = tiny_ref
    s = _system(L, handle, wl)
    sig = torch.empty(wl.n_t, wl.omega.size, 2, dtype=torch.float64, device=DEV)
    e = torch.empty(wl.n_t, dtype=torch.float64, device=DEV)
    z = torch.empty(wl.n_t, dtype=torch.float64, device=DEV)
    L.lgw_sigma_from_coeffs(handle, s, _problem(L, wl), L.Options(k=64, precision="fp64"),
                            _t(a0), _t(b0), _t(bb0), _t(k0.astype(np.int32)), sig, e, z)
    torch.cuda.synchronize()
    L.lgw_release_system(s)
    sg = sig.cpu().numpy()
    assert _rel_sigma_err(sg[..., 0] + 1j * sg[..., 1], sig64) < 1e-11
    assert np.abs(e.cpu().numpy() - E64).max() < 1e-10
    assert np.abs(z.cpu().numpy() - Z64).max() < 1e-9


def test_host_buffers_match_device_buffers(L, handle, tiny_ref):
    wl, (sig64, E64, _, _), _ = tiny_ref
    s = L.lgw_prepare_system(handle, wl.n_v, wl.n_c, wl.n_aux, wl.eps.copy(), wl.L.copy())
    prob = L.Problem(targets=wl.targets.copy(), m_idx=wl.m_idx.copy(), omega=wl.omega.copy(),
                     delta=wl.delta, M=wl.M.copy())
    sig = np.empty((wl.n_t, wl.omega.size, 2))
    e = np.empty(wl.n_t)
    L.lgw_sigma_c(handle, s, prob, L.Options(k=64, precision="fp64"), sig, e)
    L.lgw_release_system(s)
    assert _rel_sigma_err(sig[..., 0] + 1j * sig[..., 1], sig64) < 1e-9
    assert np.abs(e - E64).max() < 1e-9


def test_coupling_vectors_given_directly(L, handle, tiny_ref):
    wl, (sig64, E64, _, _), _ = tiny_ref
    sig, e, _, _ = _run(L, handle, wl, L.Options(k=64, precision="fp64"), use_V=True)
    assert _rel_sigma_err(sig, sig64) < 1e-9
    assert np.abs(e - E64).max() < 1e-9


# ---------------------------------------------------------------------------
# edge cases
# ---------------------------------------------------------------------------
def test_exact_breakdown_small_space(L, handle):
    """N_vc = 6 with k = 6: the Krylov space is exhausted, the result is the
    closed form; a zero coupling vector gives k_eff = 0 and no poles."""
    wl = gi.make_workload("e", 2, 3, 4, [0, 1, 2], [0, 1, 3, 4], 31, 9, k=6, sigma_L=0.3)
    wl.M[0, 1] = 0.0
    sigx, polesx = O.sigma_closed_form(wl)
    Ex, _ = O.solve_all_qp(wl, polesx)
    sig, e, _, _ = _run(L, handle, wl, L.Options(k=6, precision="fp64", reorth="cgs2"))
    assert _rel_sigma_err(sig, sigx) < 1e-9
    assert np.abs(e - Ex).max() < 1e-9


def test_early_breakdown_invariant_subspace(L, handle):
    """c_K = 0 makes C diagonal; a coupling vector with three nonzeros spans
    a 3-dimensional Krylov space, so the recurrence must stop at k_eff = 3
    and still give the exact closed form."""
    wl = gi.make_workload("b", 3, 5, 6, [1], [0, 4], 41, 12, k=8, kernel_factor=0.0)
    V = np.zeros((1, 2, wl.n_vc))
    V[0, 0, [0, 4, 9]] = [0.3, -0.2, 0.5]
    V[0, 1, [1, 7, 14]] = [0.1, 0.4, -0.3]
    s = _system(L, handle, wl)
    B, k = 2, 8
    al = torch.empty(B, k, dtype=torch.float64, device=DEV)
    be = torch.empty(B, k, dtype=torch.float64, device=DEV)
    b0 = torch.empty(B, dtype=torch.float64, device=DEV)
    ke = torch.empty(B, dtype=torch.int32, device=DEV)
    prob = L.Problem(targets=_t(wl.targets), m_idx=_t(wl.m_idx), omega=_t(wl.omega),
                     delta=wl.delta, V=_t(V))
    L.lgw_lanczos_coeffs(handle, s, prob, L.Options(k=k, precision="fp64"), al, be, b0, ke)
    sig = torch.empty(1, wl.omega.size, 2, dtype=torch.float64, device=DEV)
    e = torch.empty(1, dtype=torch.float64, device=DEV)
    L.lgw_sigma_c(handle, s, prob, L.Options(k=k, precision="fp64"), sig, e)
    torch.cuda.synchronize()
    L.lgw_release_system(s)
    assert list(ke.cpu().numpy()) == [3, 3]
    Delta = O.pair_energies(wl.eps, wl.n_v)
    ref = np.zeros(wl.omega.size, complex)
    for mi, m in enumerate(wl.m_idx):
        eta = 1.0 if m < wl.n_v else -1.0
        z = wl.omega - wl.eps[m] - 1j * eta * wl.delta
        ref += np.sum(V[0, mi][None, :] ** 2 / (z[:, None] + eta * Delta[None, :]), axis=1)
    sg = sig.cpu().numpy()[0]
    assert np.abs(sg[:, 0] + 1j * sg[:, 1] - ref).max() < 1e-10 * np.abs(ref).max()


def test_k_one_and_no_reorth(L, handle):
    wl = gi.make_workload("k1", 4, 9, 20, [2, 3, 4], list(range(13)), 51, 4, k=1)
    for k, reorth in [(1, "cgs2"), (1, "none"), (5, "none")]:
        ref, poles, _ = O.sigma_lanczos(wl, k=k, reorth=(reorth != "none"))
        Er, _ = O.solve_all_qp(wl, poles)
        sig, e, _, _ = _run(L, handle, wl, L.Options(k=k, precision="fp64", reorth=reorth))
        assert _rel_sigma_err(sig, ref) < 1e-9
        assert np.abs(e - Er).max() < 1e-9


def test_mid_ragged_fp64_and_bf16(L, handle):
    """Several vector chunks and GEMM tiles with ragged tails: N_vc = 13*347
    (not a multiple of 128 or 2048), N_aux = 300, 3 targets x 21 m."""
    wl = gi.make_workload("m", 13, 347, 300, [11, 12, 13], list(range(21)), 120, 2, k=40,
                          aux_scaled=True)
    ref, poles, _ = O.sigma_lanczos(wl, k=40)
    Er, _ = O.solve_all_qp(wl, poles)
    for arith in ("fp64", "split"):
        sig, e, _, rep = _run(L, handle, wl, L.Options(k=40, precision="fp64", b_sub=32,
                                                       reorth_arith=arith), report=True)
        assert rep["n_sub_batches"] == 2
        assert _rel_sigma_err(sig, ref) < 1e-9
        assert np.abs(e - Er).max() < 1e-9
    for reorth in ("cgs2", "cgs1k"):
        for arith in ("auto", "split32"):
            sigb, eb, _, _ = _run(L, handle, wl, L.Options(k=40, precision="bf16", reorth=reorth,
                                                           reorth_arith=arith))
            assert np.abs(eb - Er).max() < 1e-3


def test_errors_are_reported(L, handle):
    wl = gi.tiny()
    s = _system(L, handle, wl)
    sig = torch.empty(wl.n_t, wl.omega.size, 2, dtype=torch.float64, device=DEV)
    e = torch.empty(wl.n_t, dtype=torch.float64, device=DEV)
    with pytest.raises(L.LgwError) as ei:
        L.lgw_sigma_c(handle, s, _problem(L, wl), L.Options(k=0), sig, e)
    assert ei.value.status == 1
    bad = _problem(L, wl)
    bad.targets = _t(np.array([0, 1, 2, 999], dtype=np.int32))
    with pytest.raises(L.LgwError) as ei:
        L.lgw_sigma_c(handle, s, bad, L.Options(k=8), sig, e)
    assert ei.value.status == 2
    L.lgw_release_system(s)
    wl2 = gi.tiny()
    wl2.eps = wl2.eps.copy()
    wl2.eps[wl2.n_v] = wl2.eps[0] - 1.0    # a conduction level below a valence level
    with pytest.raises(L.LgwError) as ei:
        _system(L, handle, wl2)
    assert ei.value.status == 5
