"""Pins for the oracle's QP-energy gradient: central finite differences of
the closed-form QP energies along seeded random directions in L and eps."""
import numpy as np
import pytest

import gw_inputs as gi
import oracle as O


def _wl(kf=4.0):
    return gi.make_workload("g", 3, 7, 9, [1, 2, 4], list(range(10)), 81, 5, k=21,
                            sigma_L=0.25, sigma_M=0.4, kernel_factor=kf)


def _E(wl):
    E, _ = O.qp_energies_closed_form(wl)
    return E


@pytest.mark.parametrize("kf", [4.0, 2.0])
def test_gradient_matches_central_differences(kf):
    wl = _wl(kf)
    rng = np.random.default_rng(3)
    dE = rng.normal(size=wl.n_t)
    dL, deps = O.qp_gradient_closed_form(wl, dE)
    h = 1e-6
    for trial in range(3):
        PL = rng.normal(size=wl.L.shape)
        Pe = rng.normal(size=wl.eps.shape) * 0.1
        for which in ("L", "eps"):
            wp = gi.Workload(**wl.__dict__)
            wm = gi.Workload(**wl.__dict__)
            if which == "L":
                wp.L = wl.L + h * PL
                wm.L = wl.L - h * PL
                ana = np.sum(dL * PL)
            else:
                wp.eps = wl.eps + h * Pe
                wm.eps = wl.eps - h * Pe
                ana = np.sum(deps * Pe)
            fd = (dE @ _E(wp) - dE @ _E(wm)) / (2 * h)
            assert ana == pytest.approx(fd, rel=1e-6, abs=1e-9), (which, trial)


def test_krylov_gradient_at_full_k_equals_closed_form():
    """With k = N_vc the Lanczos basis spans the space and the Krylov form
    of the gradient is the closed form."""
    wl = _wl()
    rng = np.random.default_rng(4)
    dE = rng.normal(size=wl.n_t)
    E, Z = O.qp_energies_closed_form(wl)
    b = O.start_vectors(wl.eps, wl.n_v, O.coupling_vectors(wl.L, wl.M)).reshape(-1, wl.n_vc)
    H = O.casida_matrix(wl.eps, wl.n_v, wl.L, wl.kernel_factor)
    Qs = []
    for v in range(b.shape[0]):
        # explicit Lanczos basis with CGS2 (test-side, to build the Krylov form)
        q = b[v] / np.linalg.norm(b[v])
        Q = [q]
        for j in range(wl.n_vc - 1):
            w = H @ Q[-1]
            for _ in range(2):
                w = w - np.array(Q).T @ (np.array(Q) @ w)
            Q.append(w / np.linalg.norm(w))
        Qm = np.array(Q).T
        T = Qm.T @ H @ Qm
        th, U = np.linalg.eigh((T + T.T) / 2)
        Qs.append((Qm @ U, th))
    dLk, depsk = O.qp_gradient(wl, dE, E, Z, lambda v: Qs[v])
    dL, deps = O.qp_gradient_closed_form(wl, dE)
    np.testing.assert_allclose(dLk, dL, rtol=1e-7, atol=1e-10)
    np.testing.assert_allclose(depsk, deps, rtol=1e-7, atol=1e-10)


def test_lanczos_gradient_at_full_k_equals_closed_form():
    """The oracle's Krylov-form gradient (its own Lanczos basis) reproduces
    the closed form when k = N_vc."""
    wl = _wl()
    rng = np.random.default_rng(6)
    dE = rng.normal(size=wl.n_t)
    dLk, depsk = O.qp_gradient_lanczos(wl, dE, k=wl.n_vc)
    dL, deps = O.qp_gradient_closed_form(wl, dE)
    np.testing.assert_allclose(dLk, dL, rtol=1e-7, atol=1e-10)
    np.testing.assert_allclose(depsk, deps, rtol=1e-7, atol=1e-10)


def test_lanczos_gradient_truncated_k_tracks_finite_differences():
    """At truncated k the Krylov-form gradient approximates the derivative
    of the k-step QP energies; the gap shrinks as k grows and closes at
    k = N_vc."""
    wl = _wl()
    rng = np.random.default_rng(7)
    dE = rng.normal(size=wl.n_t)
    PL = rng.normal(size=wl.L.shape)
    h = 1e-6

    def Ek(w, k):
        _, poles, _ = O.sigma_lanczos(w, k=k)
        return O.solve_all_qp(w, poles)[0]

    errs = []
    for k in (8, 14, wl.n_vc):
        dLk, _ = O.qp_gradient_lanczos(wl, dE, k=k)
        wp = gi.Workload(**wl.__dict__)
        wm = gi.Workload(**wl.__dict__)
        wp.L = wl.L + h * PL
        wm.L = wl.L - h * PL
        fd = (dE @ Ek(wp, k) - dE @ Ek(wm, k)) / (2 * h)
        errs.append(abs(np.sum(dLk * PL) - fd) / abs(fd))
    print("relative gap by k:", errs)
    assert errs[-1] < 1e-6
    assert errs[1] < errs[0]
