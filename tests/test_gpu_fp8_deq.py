"""E4M3 L widened to FP16 in shared memory (precision "fp8_deq").

L is stored in E4M3 with one power-of-two scale per column (the copies of
precision "fp8"), the TMA brings its tiles in as bytes and the epilogue warps
widen them to FP16 in the swizzled layout the tensor cores read; the moving
operands x and y are FP16 with one power-of-two scale per vector.

  * bit-exact matvec on small-integer operands (Delta = 1, ternary L and x,
    |L^T x| <= 16): every quantisation, product, FP32 sum and rescaling is
    exact, so any error in the widening (byte order, swizzle, K offsets of
    the half K blocks) shows;
  * the matvec on Gaussian operands against a PyTorch emulation of the same
    quantisation (torch.float8_e4m3fn for L, float16 for x and y,
    power-of-two scales, FP64 sums): 1e-4 relative;
  * the full path's QP energies against the FP64 GPU path, in meV, with
    CGS2, the delayed Gram-Schmidt and without reorthogonalisation;
  * a system prepared without the FP64 copy gives the same results.
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
def test_apply_deq_exact_small_integers(L, handle, shape):
    n_v, n_c, A, nvec = shape
    rng = np.random.default_rng(7)
    wl = gi.make_workload("d16", n_v, n_c, A, [0], [0], 3, 5)
    wl.eps = np.concatenate([np.full(n_v, -0.5), np.full(n_c, 0.5)])
    p = min(0.2, 2.0 / np.sqrt(wl.n_vc))
    Lm = rng.choice([-1.0, 0.0, 1.0], size=(wl.n_vc, A), p=[p / 2, 1 - p, p / 2])
    Lm[rng.integers(0, wl.n_vc, size=A), np.arange(A)] = rng.choice([-1.0, 1.0], size=A)
    wl.L = Lm
    X = rng.choice([-1.0, 0.0, 1.0], size=(nvec, wl.n_vc), p=[p / 2, 1 - p, p / 2])
    Y = X @ Lm
    assert np.abs(Y).max() <= 16
    ref = X + wl.kernel_factor * (Y @ Lm.T)
    np.testing.assert_array_equal(_apply(L, handle, wl, X, "fp8_deq"), ref)


def _pow2(amax, top):
    """Smallest power of two s with amax / s <= top (1 for amax = 0)."""
    amax = np.asarray(amax, dtype=np.float64)
    out = np.ones_like(amax)
    nz = amax > 0
    m, e = np.frexp(amax[nz] / top)
    e = e - (m == 0.5)
    out[nz] = np.ldexp(1.0, e)
    return out


def _cast(x, dt):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).to(dt).to(
        torch.float64).numpy()


def test_apply_deq_matches_emulation(L, handle):
    wl = gi.make_workload("e16", 16, 256, 512, [0], [0], 3, 6, aux_scaled=True)
    X = np.random.default_rng(3).standard_normal((64, wl.n_vc))
    got = _apply(L, handle, wl, X, "fp8_deq")
    Delta = O.pair_energies(wl.eps, wl.n_v)
    d = np.sqrt(Delta)
    xh = torch.from_numpy(d * X).to(torch.bfloat16).to(torch.float64).numpy()
    sx = _pow2(np.abs(xh).max(axis=1), 32768.0)
    x16 = _cast(xh / sx[:, None], torch.float16)
    sL = _pow2(np.abs(wl.L).max(axis=0), 448.0)
    L8 = _cast(wl.L / sL[None, :], torch.float8_e4m3fn)
    y = (x16 @ L8) * sx[:, None] * sL[None, :]
    yp = y * sL[None, :]
    ty = _pow2(np.abs(yp).max(axis=1), 32768.0)
    y16 = _cast(yp / ty[:, None], torch.float16)
    U = (y16 @ L8.T) * ty[:, None]
    ref = Delta ** 2 * X + wl.kernel_factor * d * U
    rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    exact = O.apply_casida(wl.eps, wl.n_v, wl.L, X, wl.kernel_factor)
    coup = np.linalg.norm(wl.kernel_factor * d * (d * X @ wl.L @ wl.L.T))
    e8 = np.linalg.norm(_apply(L, handle, wl, X, "fp8") - exact) / coup
    e16 = np.linalg.norm(got - exact) / coup
    print(f"deq apply vs emulation {rel:.2e}; coupling-term error vs FP64: deq {e16:.2e}, "
          f"fp8 {e8:.2e}")
    assert rel <= 1e-4
    assert e16 < e8            # only L is rounded to 8 bits


@pytest.mark.parametrize("reorth", ["cgs2", "dcgs", "none"])
def test_deq_path_qp_energies(L, handle, reorth):
    """Tiny system (unscaled L, strong coupling) within 1 meV of the FP64 GPU
    path; k 24 without reorthogonalisation, k 64 otherwise."""
    k = 24 if reorth == "none" else 64
    wl = gi.tiny(k=k)
    s = L.lgw_prepare_system(handle, wl.n_v, wl.n_c, wl.n_aux, _t(wl.eps), _t(wl.L))
    prob = L.Problem(targets=_t(wl.targets), m_idx=_t(wl.m_idx), omega=_t(wl.omega),
                     delta=wl.delta, M=_t(wl.M))
    e = {}
    try:
        for prec in ("fp64", "fp8_deq"):
            sig = torch.empty(wl.n_t, wl.omega.size, 2, dtype=torch.float64, device=DEV)
            ee = torch.empty(wl.n_t, dtype=torch.float64, device=DEV)
            L.lgw_sigma_c(handle, s, prob, L.Options(k=k, precision=prec, reorth=reorth), sig,
                          ee)
            torch.cuda.synchronize()
            e[prec] = ee.cpu().numpy()
    finally:
        L.lgw_release_system(s)
    d = np.abs(e["fp8_deq"] - e["fp64"]).max() * 1e3
    print(f"{reorth}: |E_deq - E_fp64| = {d:.3e} meV")
    assert d <= 1.0


def test_deq_mid_slice(L, handle):
    """Mid-size slice (N_vc 131072, N_aux 2048, 2 targets x 64 orbitals, k 200,
    delayed Gram-Schmidt): within 0.01 meV of the FP64 GPU path, and closer
    to it than the all-E4M3 contractions."""
    wl = gi.custom(128, 1024, 2048, 2, 64, 1000, 1, k=200)
    s = L.lgw_prepare_system(handle, wl.n_v, wl.n_c, wl.n_aux, _t(wl.eps), _t(wl.L))
    prob = L.Problem(targets=_t(wl.targets), m_idx=_t(wl.m_idx), omega=_t(wl.omega),
                     delta=wl.delta, M=_t(wl.M))
    e = {}
    try:
        for prec in ("fp64", "fp8", "fp8_deq"):
            sig = torch.empty(wl.n_t, wl.omega.size, 2, dtype=torch.float64, device=DEV)
            ee = torch.empty(wl.n_t, dtype=torch.float64, device=DEV)
            r = "cgs1k" if prec == "fp64" else "dcgs"
            L.lgw_sigma_c(handle, s, prob, L.Options(k=200, precision=prec, reorth=r), sig, ee)
            torch.cuda.synchronize()
            e[prec] = ee.cpu().numpy()
    finally:
        L.lgw_release_system(s)
    d16 = np.abs(e["fp8_deq"] - e["fp64"]).max() * 1e3
    d8 = np.abs(e["fp8"] - e["fp64"]).max() * 1e3
    print(f"mid slice: |E_deq - E_fp64| = {d16:.3e} meV, |E_fp8 - E_fp64| = {d8:.3e} meV")
    assert d16 <= 0.01
    assert d16 <= d8


def test_deq_lean_system(L, handle):
    """A system without the FP64 copy (E4M3 copies made at preparation)
    gives the same bits as a full system."""
    wl = gi.custom(16, 96, 256, 2, 32, 100, 9, k=40)
    prob = L.Problem(targets=_t(wl.targets), m_idx=_t(wl.m_idx), omega=_t(wl.omega),
                     delta=wl.delta, M=_t(wl.M))

    def run(flags):
        s = L.lgw_prepare_system(handle, wl.n_v, wl.n_c, wl.n_aux, _t(wl.eps), _t(wl.L),
                                 flags=flags)
        try:
            sig = torch.empty(wl.n_t, wl.omega.size, 2, dtype=torch.float64, device=DEV)
            e = torch.empty(wl.n_t, dtype=torch.float64, device=DEV)
            L.lgw_sigma_c(handle, s, prob, L.Options(k=40, precision="fp8_deq", reorth="cgs2"),
                          sig, e)
            torch.cuda.synchronize()
            return sig.cpu().numpy()
        finally:
            L.lgw_release_system(s)

    np.testing.assert_array_equal(run(L.SYS_NO_FP64 | L.SYS_FP8), run(0))
