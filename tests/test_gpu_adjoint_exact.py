"""GPU adjoint in its exact k-step form and the Tamm-Dancoff adjoint.

With FP64 contractions and no reorthogonalisation, lgw_sigma_c_backward
takes the three-term recurrence back step by step (reverse mode), from
Krylov checkpoints every ckpt_every steps, so the gradient is the
derivative of the k-step QP energies at any k:
  * against the oracle's reverse mode of the same recurrence, 1e-9 relative
    to the largest entry, for several checkpoint intervals (one segment,
    several, a ragged last segment);
  * sub-batched recomputation equals the single pass;
  * against central differences of the GPU's own FP64 forward at k = 8 and
    k = 40 on the differentiation workload's shapes (N_vc 32768,
    N_aux 1024), where the Krylov form of the gradient is far off;
  * Tamm-Dancoff: the exact form against the oracle's reverse mode, and the
    Krylov form at k = N_vc against the closed-form Tamm-Dancoff gradient;
  * the polynomial form (Lanczos on D = p_g(C), reverse Clenshaw recurrence)
    against the oracle's reverse mode and against central differences of
    the GPU's polynomial-form energies at the differentiation shapes;
  * through torch.autograd with tda=True.
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


def _problem(L, wl):
    return L.Problem(targets=_t(wl.targets), m_idx=_t(wl.m_idx), omega=_t(wl.omega),
                     delta=wl.delta, M=_t(wl.M))


def _system(L, h, wl):
    return L.lgw_prepare_system(h, wl.n_v, wl.n_c, wl.n_aux, _t(wl.eps), _t(wl.L),
                                wl.kernel_factor)


def _grad(L, h, wl, dE, opts, tda=False):
    s = _system(L, h, wl)
    try:
        dL = torch.empty(wl.n_vc, wl.n_aux, dtype=torch.float64, device=DEV)
        de = torch.empty(wl.n_v + wl.n_c, dtype=torch.float64, device=DEV)
        fn = L.lgw_sigma_c_tda_backward if tda else L.lgw_sigma_c_backward
        fn(h, s, _problem(L, wl), opts, _t(dE), dL, de)
        torch.cuda.synchronize()
    finally:
        L.lgw_release_system(s)
    return dL.cpu().numpy(), de.cpu().numpy()


def _energies(L, h, wl, opts, tda=False):
    s = _system(L, h, wl)
    try:
        sig = torch.empty(wl.n_t, wl.omega.size, 2, dtype=torch.float64, device=DEV)
        e = torch.empty(wl.n_t, dtype=torch.float64, device=DEV)
        fn = L.lgw_sigma_c_tda if tda else L.lgw_sigma_c
        fn(h, s, _problem(L, wl), opts, sig, e)
        torch.cuda.synchronize()
    finally:
        L.lgw_release_system(s)
    return e.cpu().numpy()


def _close(got, ref, rel):
    scale = np.abs(ref).max()
    err = np.abs(got - ref).max()
    assert err <= rel * scale, f"max err {err:.3e} vs {rel:.0e} * {scale:.3e}"


def _exact(k, ckpt=0, b_sub=0):
    from paper_2310_20103_gb300 import lgw
    return lgw.Options(k=k, precision="fp64", reorth="none", ckpt_every=ckpt, b_sub=b_sub)


@pytest.mark.parametrize("k,ckpt", [(1, 0), (8, 0), (24, 0), (24, 5), (24, 64), (40, 16)])
def test_exact_reverse_vs_oracle(L, handle, k, ckpt):
    wl = gi.tiny(k=k)
    dE = np.random.default_rng(20 + k).normal(size=wl.n_t)
    dLr, der = O.qp_gradient_recurrence(wl, dE, k=k)
    dL, de = _grad(L, handle, wl, dE, _exact(k, ckpt))
    _close(dL, dLr, 1e-9)
    _close(de, der, 1e-9)


def test_exact_checkpoint_intervals_agree(L, handle):
    """The checkpoint interval changes only where the recurrence restarts;
    the recomputed steps are the forward's, so the gradients agree to
    rounding."""
    wl = gi.tiny(k=24)
    dE = np.random.default_rng(22).normal(size=wl.n_t)
    a = _grad(L, handle, wl, dE, _exact(24, 3))
    b = _grad(L, handle, wl, dE, _exact(24, 24))
    for x, y in zip(a, b):
        _close(x, y, 1e-12)


def test_exact_sub_batches_equal_single_pass(L, handle):
    wl = gi.tiny(k=24)
    dE = np.random.default_rng(23).normal(size=wl.n_t)
    a = _grad(L, handle, wl, dE, _exact(24, 8))
    b = _grad(L, handle, wl, dE, _exact(24, 8, b_sub=48))
    for x, y in zip(a, b):
        _close(x, y, 1e-12)


@pytest.mark.parametrize("k,ckpt", [(8, 0), (40, 16)])
def test_exact_central_differences_differentiation_shapes(L, handle, k, ckpt):
    """N_v 64, N_c 512 (N_vc 32768), N_aux 1024, sigma/sqrt(A) distributions,
    2 targets x 4 summed orbitals, k 8 (the polynomial form's depth) and 40
    (three checkpoint segments, the last ragged).  Directional derivatives
    along seeded unit-normal directions vs central differences (h = 1e-6)
    of the GPU FP64 forward without reorthogonalisation, 1e-5 relative plus
    2e-9 absolute: the rounding of E (about 1e-15 eV at E ~ 10 eV) over the
    step 2h = 2e-6 (measured differences 2e-11 to 1.3e-10)."""
    wl = gi.make_workload("diff", 64, 512, 1024, [62, 64], [0, 30, 63, 64], 200, 4,
                          k=k, aux_scaled=True)
    rng = np.random.default_rng(27 + k)
    dE = rng.normal(size=wl.n_t)
    opts = _exact(k, ckpt)
    opts.qp_tol = 1e-13
    dL, de = _grad(L, handle, wl, dE, opts)
    h = 1e-6
    for trial in range(2):
        PL = rng.normal(size=wl.L.shape)
        Pe = rng.normal(size=wl.eps.shape)
        for which in ("L", "eps"):
            wp = gi.Workload(**wl.__dict__)
            wm = gi.Workload(**wl.__dict__)
            if which == "L":
                wp.L, wm.L = wl.L + h * PL, wl.L - h * PL
                ana = np.sum(dL * PL)
            else:
                wp.eps, wm.eps = wl.eps + h * Pe, wl.eps - h * Pe
                ana = np.sum(de * Pe)
            fd = (dE @ _energies(L, handle, wp, opts) - dE @ _energies(L, handle, wm, opts)) / (2 * h)
            print(f"k {k} {which} trial {trial}: analytic {ana:.10e} fd {fd:.10e}")
            assert ana == pytest.approx(fd, rel=1e-5, abs=2e-9), (which, trial)


@pytest.mark.parametrize("ckpt", [0, 2])
def test_exact_reverse_at_breakdown_vs_oracle(L, handle, ckpt):
    """L nonzero on three pair rows: every start vector lies in a
    3-dimensional invariant subspace of C, so the recurrence stops at
    k_eff = 3 of k = 8 (with interval 2 the checkpoints straddle the stop).
    The k_eff-step gradient (pinned by central differences in the oracle
    tests) against the oracle, 1e-9."""
    wl = gi.make_workload("bd", 2, 6, 4, [1, 2], list(range(8)), 61, 9, k=8,
                          sigma_L=0.3, sigma_M=0.5)
    keep = np.zeros(wl.n_vc, dtype=bool)
    keep[[0, 3, 7]] = True
    wl.L = np.where(keep[:, None], wl.L, 0.0)
    dE = np.random.default_rng(98).normal(size=wl.n_t)
    dLr, der = O.qp_gradient_recurrence(wl, dE, k=8)
    dL, de = _grad(L, handle, wl, dE, _exact(8, ckpt))
    _close(dL, dLr, 1e-9)
    _close(de, der, 1e-9)


@pytest.mark.parametrize("k,ckpt", [(8, 0), (24, 5)])
def test_tda_exact_reverse_vs_oracle(L, handle, k, ckpt):
    wl = gi.tiny(k=k)
    dE = np.random.default_rng(60 + k).normal(size=wl.n_t)
    dLr, der = O.qp_gradient_recurrence(wl, dE, k=k, tda=True)
    dL, de = _grad(L, handle, wl, dE, _exact(k, ckpt), tda=True)
    _close(dL, dLr, 1e-9)
    _close(de, der, 1e-9)


@pytest.mark.parametrize("kf", [4.0, 2.0])
def test_tda_krylov_form_full_k_equals_closed_form(L, handle, kf):
    """Tamm-Dancoff, k = N_vc with CGS2: the Krylov form is exact and equals
    the closed-form Tamm-Dancoff gradient."""
    wl = gi.tiny(k=256)
    wl.kernel_factor = kf
    dE = np.random.default_rng(70).normal(size=wl.n_t)
    dLr, der = O.qp_gradient_tda_closed_form(wl, dE)
    dL, de = _grad(L, handle, wl, dE, L.Options(k=wl.n_vc, precision="fp64", reorth="cgs2"),
                   tda=True)
    _close(dL, dLr, 1e-8)
    _close(de, der, 1e-8)


def test_backward_rejects_linearised_qp_and_negative_interval(L, handle):
    wl = gi.tiny(k=8)
    dE = np.ones(wl.n_t)
    o = _exact(8)
    o.qp_mode = "linearised"
    with pytest.raises(L.LgwError) as e:
        _grad(L, handle, wl, dE, o)
    assert e.value.status == 8
    o = _exact(8, -1)
    with pytest.raises(L.LgwError) as e:
        _grad(L, handle, wl, dE, o)
    assert e.value.status == 1
    # the handle stays usable
    dLr, der = O.qp_gradient_recurrence(wl, dE, k=8)
    dL, de = _grad(L, handle, wl, dE, _exact(8))
    _close(dL, dLr, 1e-9)


def test_autograd_tda_exact(L, handle):
    from paper_2310_20103_gb300.autograd import qp_energies
    wl = gi.tiny(k=16)
    opts = _exact(16, 6)
    Lt = _t(wl.L).requires_grad_(True)
    et = _t(wl.eps).requires_grad_(True)
    E = qp_energies(Lt, et, wl.n_v, wl.n_c, _problem(L, wl), opts, handle, wl.kernel_factor,
                    tda=True)
    np.testing.assert_array_equal(E.detach().cpu().numpy(), _energies(L, handle, wl, opts, True))
    w = torch.linspace(-1.0, 2.0, wl.n_t, dtype=torch.float64, device=DEV)
    (w * E).sum().backward()
    dL, de = _grad(L, handle, wl, w.cpu().numpy(), opts, tda=True)
    np.testing.assert_array_equal(Lt.grad.cpu().numpy(), dL)
    np.testing.assert_array_equal(et.grad.cpu().numpy(), de)


# --------------------------------------------------------------------------
# Polynomial form
# --------------------------------------------------------------------------
def _interval(wl):
    th = np.linalg.eigvalsh(O.casida_matrix(wl.eps, wl.n_v, wl.L, wl.kernel_factor))
    return 0.9 * th.min(), 1.1 * th.max()


def _poly_grad(L, h, wl, dE, opts, g, lo, hi):
    s = _system(L, h, wl)
    try:
        dL = torch.empty(wl.n_vc, wl.n_aux, dtype=torch.float64, device=DEV)
        de = torch.empty(wl.n_v + wl.n_c, dtype=torch.float64, device=DEV)
        L.lgw_sigma_c_poly_backward(h, s, _problem(L, wl), opts, g, lo, hi, _t(dE), dL, de)
        torch.cuda.synchronize()
    finally:
        L.lgw_release_system(s)
    return dL.cpu().numpy(), de.cpu().numpy()


def _poly_energies(L, h, wl, opts, g, lo, hi):
    s = _system(L, h, wl)
    try:
        sig = torch.empty(wl.n_t, wl.omega.size, 2, dtype=torch.float64, device=DEV)
        e = torch.empty(wl.n_t, dtype=torch.float64, device=DEV)
        L.lgw_sigma_c_poly(h, s, _problem(L, wl), opts, g, lo, hi, sig, e)
        torch.cuda.synchronize()
    finally:
        L.lgw_release_system(s)
    return e.cpu().numpy()


@pytest.mark.parametrize("g,k,ckpt", [(1, 4, 0), (4, 8, 0), (8, 16, 5)])
def test_poly_exact_reverse_vs_oracle(L, handle, g, k, ckpt):
    wl = gi.tiny(k=k)
    lo, hi = _interval(wl)
    dE = np.random.default_rng(90 + g + k).normal(size=wl.n_t)
    dLr, der = O.qp_gradient_poly_recurrence(wl, dE, g, lo, hi, k=k)
    dL, de = _poly_grad(L, handle, wl, dE, _exact(k, ckpt), g, lo, hi)
    _close(dL, dLr, 1e-9)
    _close(de, der, 1e-9)


def test_poly_central_differences_differentiation_shapes(L, handle):
    """The paper's depths (g 8, k 8) at N_vc 32768, N_aux 1024: directional
    derivatives vs central differences (h = 1e-6) of the GPU's FP64
    polynomial-form energies on a fixed interval, 1e-6 relative."""
    wl = gi.make_workload("diff", 64, 512, 1024, [62, 64], [0, 30, 63, 64], 200, 4,
                          k=8, aux_scaled=True)
    s = _system(L, handle, wl)
    try:
        lo, hi = L.lgw_spectral_interval(handle, s, 32)
    finally:
        L.lgw_release_system(s)
    rng = np.random.default_rng(95)
    dE = rng.normal(size=wl.n_t)
    opts = _exact(8)
    opts.qp_tol = 1e-13
    dL, de = _poly_grad(L, handle, wl, dE, opts, 8, lo, hi)
    h = 1e-6
    for trial in range(2):
        PL = rng.normal(size=wl.L.shape)
        Pe = rng.normal(size=wl.eps.shape)
        for which in ("L", "eps"):
            wp = gi.Workload(**wl.__dict__)
            wm = gi.Workload(**wl.__dict__)
            if which == "L":
                wp.L, wm.L = wl.L + h * PL, wl.L - h * PL
                ana = np.sum(dL * PL)
            else:
                wp.eps, wm.eps = wl.eps + h * Pe, wl.eps - h * Pe
                ana = np.sum(de * Pe)
            fd = (dE @ _poly_energies(L, handle, wp, opts, 8, lo, hi)
                  - dE @ _poly_energies(L, handle, wm, opts, 8, lo, hi)) / (2 * h)
            print(f"poly {which} trial {trial}: analytic {ana:.10e} fd {fd:.10e}")
            assert ana == pytest.approx(fd, rel=1e-5, abs=2e-9), (which, trial)


def test_poly_backward_needs_the_exact_form(L, handle):
    wl = gi.tiny(k=8)
    lo, hi = _interval(wl)
    o = L.Options(k=8, precision="fp64", reorth="cgs2")
    with pytest.raises(L.LgwError) as e:
        _poly_grad(L, handle, wl, np.ones(wl.n_t), o, 4, lo, hi)
    assert e.value.status == 8
