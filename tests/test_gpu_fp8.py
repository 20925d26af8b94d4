"""E4M3 tensor-core contractions (precision "fp8").

  * bit-exact matvec on small-integer operands: Delta = 1, ternary L and x
    with every column of L holding a +-1 and |L^T x| <= 16, so the power-of-
    two scales map them onto E4M3 integers and every product, FP32 sum and
    rescaling is exact;
  * the matvec on Gaussian operands against a PyTorch emulation of the same
    quantisation (torch.float8_e4m3fn, power-of-two scales, FP64 sums);
  * the full path's QP energies against the FP64 GPU path, in meV.
"""
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


def _apply(L, h, wl, X, prec):
    s = L.lgw_prepare_system(h, wl.n_v, wl.n_c, wl.n_aux, _t(wl.eps), _t(wl.L), wl.kernel_factor)
    try:
        Xd = _t(X)
        Y = torch.empty_like(Xd)
        L.lgw_apply_casida(h, s, Xd, Y, prec)
        torch.cuda.synchronize()
    finally:
        L.lgw_release_system(s)
    return Y.cpu().numpy()


@pytest.mark.parametrize("shape", [(8, 32, 128, 5), (7, 131, 256, 70), (16, 300, 384, 300),
                                   (32, 256, 512, 512)])
def test_apply_fp8_exact_small_integers(L, handle, shape):
    n_v, n_c, A, nvec = shape
    rng = np.random.default_rng(4)
    wl = gi.make_workload("x8", n_v, n_c, A, [0], [0], 3, 5)
    wl.eps = np.concatenate([np.full(n_v, -0.5), np.full(n_c, 0.5)])
    p = min(0.2, 2.0 / np.sqrt(wl.n_vc))
    Lm = rng.choice([-1.0, 0.0, 1.0], size=(wl.n_vc, A), p=[p / 2, 1 - p, p / 2])
    Lm[rng.integers(0, wl.n_vc, size=A), np.arange(A)] = rng.choice([-1.0, 1.0], size=A)
    wl.L = Lm
    X = rng.choice([-1.0, 0.0, 1.0], size=(nvec, wl.n_vc), p=[p / 2, 1 - p, p / 2])
    Y = X @ Lm
    assert np.abs(Y).max() <= 16            # E4M3-exact intermediate
    ref = X + wl.kernel_factor * (Y @ Lm.T)
    np.testing.assert_array_equal(_apply(L, handle, wl, X, "fp8"), ref)


def _pow2(amax):
    """Smallest power of two s with amax / s <= 448 (1 for amax = 0)."""
    amax = np.asarray(amax, dtype=np.float64)
    out = np.ones_like(amax)
    nz = amax > 0
    m, e = np.frexp(amax[nz] / 448.0)
    e = e - (m == 0.5)
    out[nz] = np.ldexp(1.0, e)
    return out


def _e4m3(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).to(
        torch.float8_e4m3fn).to(torch.float64).numpy()


def test_apply_fp8_matches_emulation(L, handle):
    """Gaussian operands: the GPU result against the same quantisation done
    by PyTorch on the host (FP64 sums).  The two differ only where FP32
    accumulation order flips an E4M3 rounding of y; relative norm 1e-3."""
    wl = gi.make_workload("e8", 16, 256, 512, [0], [0], 3, 6, aux_scaled=True)
    X = np.random.default_rng(2).standard_normal((64, wl.n_vc))
    got = _apply(L, handle, wl, X, "fp8")
    Delta = O.pair_energies(wl.eps, wl.n_v)
    d = np.sqrt(Delta)
    xh = torch.from_numpy(d * X).to(torch.bfloat16).to(torch.float64).numpy()
    sx = _pow2(np.abs(xh).max(axis=1))
    x8 = _e4m3(xh / sx[:, None])
    sL = _pow2(np.abs(wl.L).max(axis=0))
    L8 = _e4m3(wl.L / sL[None, :])
    y = (x8 @ L8) * sx[:, None] * sL[None, :]
    yp = y * sL[None, :]
    ty = _pow2(np.abs(yp).max(axis=1))
    y8 = _e4m3(yp / ty[:, None])
    U = (y8 @ L8.T) * ty[:, None]
    ref = Delta ** 2 * X + wl.kernel_factor * d * U
    rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    exact = O.apply_casida(wl.eps, wl.n_v, wl.L, X, wl.kernel_factor)
    coup = np.linalg.norm(wl.kernel_factor * d * (d * X @ wl.L @ wl.L.T))
    print(f"fp8 apply vs emulation {rel:.2e}; coupling-term error vs FP64 "
          f"{np.linalg.norm(got - exact) / coup:.2e}")
    assert rel <= 1e-3


@pytest.mark.parametrize("wl_name,bound_mev", [("tiny", 1.0), ("mid2x64", 0.01)])
def test_fp8_path_qp_energies(L, handle, wl_name, bound_mev):
    """Full path with E4M3 contractions (CGS2 against the split basis) vs the
    FP64 GPU path on the same system: QP energies within 1 meV on the tiny
    system (unscaled L, strong coupling; measured 0.29 meV) and within 0.01
    meV on a mid-size slice (N_vc 131072, N_aux 2048, 2 targets x 64
    orbitals, k 200; measured 5.5e-4 meV)."""
    if wl_name == "tiny":
        wl, k = gi.tiny(k=64), 64
    else:
        wl, k = gi.custom(128, 1024, 2048, 2, 64, 1000, 1, k=200), 200
    s = L.lgw_prepare_system(handle, wl.n_v, wl.n_c, wl.n_aux, _t(wl.eps), _t(wl.L))
    prob = L.Problem(targets=_t(wl.targets), m_idx=_t(wl.m_idx), omega=_t(wl.omega),
                     delta=wl.delta, M=_t(wl.M))
    e = {}
    try:
        for prec in ("fp64", "fp8"):
            sig = torch.empty(wl.n_t, wl.omega.size, 2, dtype=torch.float64, device=DEV)
            ee = torch.empty(wl.n_t, dtype=torch.float64, device=DEV)
            L.lgw_sigma_c(handle, s, prob, L.Options(k=k, precision=prec, reorth="cgs2"), sig, ee)
            torch.cuda.synchronize()
            e[prec] = ee.cpu().numpy()
    finally:
        L.lgw_release_system(s)
    d = np.abs(e["fp8"] - e["fp64"]).max() * 1e3
    print(f"{wl_name}: |E_fp8 - E_fp64| = {d:.3e} meV")
    assert d <= bound_mev


def test_system_flags(L, handle):
    """Copies of L per LGW_SYS_* flag: a system without the FP64 copy (E4M3
    copies made at preparation, straight from the caller's L) gives the same
    BF16 and FP8 results as a full system, and refuses FP64 requests and the
    adjoint; a system without the BF16 copies gives the same FP64 results,
    refuses BF16, and runs FP8 with FP64 start vectors."""
    wl = gi.custom(16, 96, 256, 2, 32, 100, 9, k=40)
    prob = L.Problem(targets=_t(wl.targets), m_idx=_t(wl.m_idx), omega=_t(wl.omega),
                     delta=wl.delta, M=_t(wl.M))

    def run(flags, prec):
        s = L.lgw_prepare_system(handle, wl.n_v, wl.n_c, wl.n_aux, _t(wl.eps), _t(wl.L),
                                 flags=flags)
        try:
            sig = torch.empty(wl.n_t, wl.omega.size, 2, dtype=torch.float64, device=DEV)
            e = torch.empty(wl.n_t, dtype=torch.float64, device=DEV)
            L.lgw_sigma_c(handle, s, prob, L.Options(k=40, precision=prec, reorth="cgs2"), sig, e)
            torch.cuda.synchronize()
            return sig.cpu().numpy(), e.cpu().numpy()
        finally:
            L.lgw_release_system(s)

    full = {p: run(0, p) for p in ("fp64", "bf16", "fp8")}
    lean = L.SYS_NO_FP64 | L.SYS_FP8
    for p in ("bf16", "fp8"):
        got = run(lean, p)
        np.testing.assert_array_equal(got[0], full[p][0])
    with pytest.raises(L.LgwError) as ei:
        run(lean, "fp64")
    assert ei.value.status == 8
    s = L.lgw_prepare_system(handle, wl.n_v, wl.n_c, wl.n_aux, _t(wl.eps), _t(wl.L), flags=lean)
    try:
        with pytest.raises(L.LgwError) as ei:
            L.lgw_sigma_c_backward(handle, s, prob, L.Options(k=40, precision="bf16"),
                                   _t(np.ones(wl.n_t)))
        assert ei.value.status == 8
    finally:
        L.lgw_release_system(s)
    np.testing.assert_array_equal(run(L.SYS_NO_BF16, "fp64")[0], full["fp64"][0])
    with pytest.raises(L.LgwError) as ei:
        run(L.SYS_NO_BF16, "bf16")
    assert ei.value.status == 8
    e8 = run(L.SYS_NO_BF16, "fp8")[1]
    assert np.abs(e8 - full["fp8"][1]).max() < 1e-8     # start vectors by FP64 instead of split BF16
    with pytest.raises(L.LgwError) as ei:
        run(L.SYS_NO_FP64 | L.SYS_NO_BF16, "fp8")
    assert ei.value.status == 1


@pytest.mark.parametrize("prec,bound_mev", [("bf16", 0.1), ("fp8", 1.0)])
def test_tensor_core_path_without_reorth(L, handle, prec, bound_mev):
    """Tensor-core contractions without reorthogonalisation (the large-system
    mode: store-only FP32 contraction epilogue, FP64 assembly of w and alpha
    on the vector pass) against the oracle's plain FP64 recurrence, k 24 on
    the tiny system and on a ragged shape (N_vc = 13*347, N_aux = 300)."""
    for wl in (gi.tiny(k=24), gi.make_workload("rg", 13, 347, 300, [11, 12, 13],
                                               list(range(21)), 120, 3, k=24, aux_scaled=True)):
        ref, poles, _ = O.sigma_lanczos(wl, k=24, reorth=False)
        Er, _ = O.solve_all_qp(wl, poles)
        s = L.lgw_prepare_system(handle, wl.n_v, wl.n_c, wl.n_aux, _t(wl.eps), _t(wl.L))
        prob = L.Problem(targets=_t(wl.targets), m_idx=_t(wl.m_idx), omega=_t(wl.omega),
                         delta=wl.delta, M=_t(wl.M))
        try:
            sig = torch.empty(wl.n_t, wl.omega.size, 2, dtype=torch.float64, device=DEV)
            e = torch.empty(wl.n_t, dtype=torch.float64, device=DEV)
            L.lgw_sigma_c(handle, s, prob, L.Options(k=24, precision=prec, reorth="none"), sig, e)
            torch.cuda.synchronize()
        finally:
            L.lgw_release_system(s)
        d = np.abs(e.cpu().numpy() - Er).max() * 1e3
        print(f"{wl.name} {prec} no-reorth: |dE| = {d:.3e} meV")
        assert d <= bound_mev
