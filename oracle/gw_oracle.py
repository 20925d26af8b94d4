"""FP64 CPU oracle for the Lanczos full-frequency GW hot path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module.  It shares no code
with the CUDA library and never calls it.

Everything here is plain numpy float64, written for a reader checking it
against the paper (Gao, Tang, Zhao, Chelikowsky, "Efficient Full-frequency GW
Calculations using a Lanczos Method", arXiv 2310.20103).  Index names follow
the code convention: ``t`` is the target orbital (the paper's m in
Sigma_mm), ``m`` is the summed orbital (the paper's n in Eq. 10), ``vc`` the
electron-hole pair, ``s`` a Casida eigenpair.

Readings of the paper used below (each is listed with its reason in the
design notes of the repository):
  * the Casida matrix is C = (A-B)^1/2 (A+B) (A-B)^1/2 with A-B = diag(Delta)
    and A+B = Delta + (c_K/2) K, i.e. C = Delta^2 + c_K Delta^1/2 K Delta^1/2,
    with c_K = 4 by default (closed-shell spin sum) and K = L L^T;
  * the sign factor eta and the energy in z belong to the summed orbital m;
  * z_m = omega - eps_m - i eta_m delta (Eq. 11), and Eq. 11 equals
    sum_s p_s^2 / (Omega_s (z_m + eta_m Omega_s)), which is Eq. 7 with
    W^s_{tm} = p_s Omega_s^-1/2 (Eq. 9);
  * a k-step Lanczos gives a k x k tridiagonal T_k (alpha_1..alpha_k on the
    diagonal, beta_2..beta_k off it); Sigma follows from the Gauss rule of
    T_k mapped through Omega = sqrt(theta) (Eq. 12 with D = C^1/2);
  * the quasiparticle equation is E = eps_t + s_t + Re Sigma_t(E) (the paper
    does not print it), solved by Newton from eps_t + s_t, falling back to
    a bracketed bisection on the frequency grid.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "pair_energies", "occupation_sign", "casida_matrix", "apply_casida",
    "coupling_vectors", "start_vectors", "casida_eigenpairs",
    "closed_form_poles", "lanczos", "lanczos_poles", "sigma_from_poles",
    "dsigma_from_poles", "sigma_closed_form", "sigma_lanczos", "qp_solve",
    "solve_all_qp", "qp_gradient", "qp_energies_closed_form", "qp_gradient_closed_form",
    "qp_gradient_lanczos", "lanczos_reverse", "qp_gradient_recurrence",
    "qp_energies_tda_closed_form", "qp_gradient_tda_closed_form", "chebyshev_sqrt", "chebyshev_eval", "apply_poly",
    "sigma_poly_lanczos", "apply_poly_reverse", "qp_gradient_poly_recurrence", "haydock", "sigma_x", "qp_linearised", "fit_factors",
    "tda_matrix", "sigma_tda_closed_form", "sigma_tda_lanczos", "sigma_offdiag_closed_form",
    "band_lanczos", "band_gauss_rule", "sigma_band_lanczos",
]


# --------------------------------------------------------------------------
# Eq. 2-4: pair energies and the reduced Casida matrix
# --------------------------------------------------------------------------
def pair_energies(eps, n_v):
    """Delta_vc = eps_c - eps_v, pair index vc = v * n_c + c.

    Diagonal of A - B in Eq. 2-3 (the Coulomb terms cancel in A - B)."""
    eps = np.asarray(eps, dtype=np.float64)
    ev, ec = eps[:n_v], eps[n_v:]
    return (ec[None, :] - ev[:, None]).reshape(-1)


def occupation_sign(m, n_v):
    """eta_m: +1 for an occupied orbital, -1 for an empty one (Eq. 7)."""
    return np.where(np.asarray(m) < n_v, 1.0, -1.0)


def casida_matrix(eps, n_v, L, kernel_factor=4.0):
    """Dense C = Delta^2 + c_K Delta^1/2 (L L^T) Delta^1/2 (Eq. 4)."""
    Delta = pair_energies(eps, n_v)
    d = np.sqrt(Delta)
    K = L @ L.T
    H = kernel_factor * (d[:, None] * K * d[None, :])
    H[np.diag_indices_from(H)] += Delta ** 2
    return H


def apply_casida(eps, n_v, L, X, kernel_factor=4.0):
    """C applied to the rows of X ([n_vec, N_vc]) through the low-rank factor."""
    Delta = pair_energies(eps, n_v)
    d = np.sqrt(Delta)
    Y = (X * d[None, :]) @ L          # L^T (Delta^1/2 x), one row per vector
    U = Y @ L.T                       # L y
    return (Delta ** 2)[None, :] * X + kernel_factor * d[None, :] * U


# --------------------------------------------------------------------------
# Start vectors |P_tm> (text after Eq. 8): (P)_vc = (tm|vc) (eps_c - eps_v)^1/2
# --------------------------------------------------------------------------
def coupling_vectors(L, M):
    """(tm|vc) = sum_mu L[vc, mu] M^{tm}[mu]  ->  V[t, m, vc] (Eq. 16 fitted form)."""
    return np.einsum("vu,tmu->tmv", L, M)


def start_vectors(eps, n_v, V):
    """b_tm = Delta^1/2 * V_tm, the vector |P_tm> of the text after Eq. 8."""
    d = np.sqrt(pair_energies(eps, n_v))
    return V * d


# --------------------------------------------------------------------------
# Closed form: Eq. 7-9 with the Casida eigenpairs
# --------------------------------------------------------------------------
def casida_eigenpairs(H):
    """C Z^s = Z^s Omega_s^2 (Eq. 4).  Returns (Omega, Z).

    Raises if C is not positive definite (Omega_s must be real, > 0)."""
    theta, Z = np.linalg.eigh(H)
    if theta.min() <= 0.0:
        raise ValueError("Casida matrix is not positive definite")
    return np.sqrt(theta), Z


def closed_form_poles(wl, Omega=None, Z=None):
    """Pole list of Sigma_t(omega) from the Casida eigenpairs.

    For every target t, summed m and eigenpair s the pole is
        W_tms / (omega - eps_m + eta_m Omega_s - i eta_m delta)      (Eq. 7)
    with W_tms = (W^s_tm)^2 = p_s^2 / Omega_s, p_s = <P_tm|Z^s> (Eq. 9).
    Returns arrays (pos, weight, eta) of shape [n_t, n_m * N_vc] where
    pos = eps_m - eta_m Omega_s (the real part of the pole).
    """
    if Omega is None:
        Omega, Z = casida_eigenpairs(casida_matrix(wl.eps, wl.n_v, wl.L, wl.kernel_factor))
    b = start_vectors(wl.eps, wl.n_v, coupling_vectors(wl.L, wl.M))   # [n_t, n_m, N_vc]
    p = b @ Z                                                          # [n_t, n_m, N_vc]
    W = p ** 2 / Omega[None, None, :]
    eps_m = wl.eps[wl.m_idx]
    eta = occupation_sign(wl.m_idx, wl.n_v)
    pos = eps_m[:, None] - eta[:, None] * Omega[None, :]               # [n_m, N_vc]
    n_t = wl.n_t
    pos = np.broadcast_to(pos, (n_t,) + pos.shape).reshape(n_t, -1)
    etas = np.broadcast_to(eta[:, None], (wl.n_m, Omega.shape[0]))
    etas = np.broadcast_to(etas, (n_t,) + etas.shape).reshape(n_t, -1)
    return pos.copy(), W.reshape(n_t, -1), etas.copy()


def sigma_from_poles(omega, pos, weight, eta, delta):
    """Sigma(omega) = sum_p weight_p / (omega - pos_p - i eta_p delta)  (Eq. 7).

    ``omega`` is a 1-D grid; pos/weight/eta are 1-D pole lists for one target.
    Each term is evaluated as written; the sum runs over all poles."""
    omega = np.asarray(omega, dtype=np.float64)
    out = np.empty(omega.shape[0], dtype=np.complex128)
    for i, w in enumerate(omega):
        out[i] = np.sum(weight / ((w - pos) - 1j * eta * delta))
    return out


def dsigma_from_poles(omega, pos, weight, eta, delta):
    """d Sigma / d omega of ``sigma_from_poles``."""
    omega = np.atleast_1d(np.asarray(omega, dtype=np.float64))
    out = np.empty(omega.shape[0], dtype=np.complex128)
    for i, w in enumerate(omega):
        den = (w - pos) - 1j * eta * delta
        out[i] = -np.sum(weight / den ** 2)
    return out


def sigma_closed_form(wl):
    """Sigma_t(omega_f) for every target on the workload grid, Eq. 7-9.

    Returns complex [n_t, n_freq] and the per-target pole lists used."""
    pos, W, eta = closed_form_poles(wl)
    poles = [(pos[i], W[i], eta[i]) for i in range(wl.n_t)]
    sig = np.stack([sigma_from_poles(wl.omega, *poles[i], wl.delta)
                    for i in range(wl.n_t)])
    return sig, poles


# --------------------------------------------------------------------------
# Lanczos tridiagonalisation (Eq. 13), run on C itself from |P_tm>
# --------------------------------------------------------------------------
def lanczos(apply_op, b, k, reorth=True, breakdown_tol=1e-13, return_basis=False):
    """k-step Lanczos from each row of ``b`` ([n_vec, N]).

    Every row is an independent recurrence (own basis, own coefficients); the
    rows are only processed side by side.  Step j:
        w = C q_j - beta_j q_{j-1}
        alpha_j = q_j . w ;  w = w - alpha_j q_j
        (reorth) twice: w = w - Q_j (Q_j^T w)     (classical Gram-Schmidt)
        beta_{j+1} = ||w|| ;  q_{j+1} = w / beta_{j+1}
    A row stops (k_eff = j) when beta_{j+1} <= breakdown_tol * max_i |alpha_i|.

    Returns alpha [n_vec, k], beta [n_vec, k] (beta[:, j] couples steps j and
    j+1, i.e. the paper's b_{j+1}; beta[:, k-1] is the residual norm),
    beta0 = ||b|| [n_vec] and k_eff [n_vec]; with return_basis also the
    basis Q [k, n_vec, N] (rows past k_eff are zero).
    """
    b = np.atleast_2d(np.asarray(b, dtype=np.float64))
    n_vec, N = b.shape
    k = int(min(k, N))
    alpha = np.zeros((n_vec, k))
    beta = np.zeros((n_vec, k))
    beta0 = np.sqrt(np.einsum("vi,vi->v", b, b))
    k_eff = np.full(n_vec, k, dtype=np.int64)
    active = beta0 > 0.0
    k_eff[~active] = 0
    Q = np.zeros((k + 1, n_vec, N)) if (reorth or return_basis) else None
    q = np.where(active[:, None], b / np.where(active, beta0, 1.0)[:, None], 0.0)
    q_prev = np.zeros_like(q)
    beta_j = np.zeros(n_vec)
    amax = np.zeros(n_vec)
    for j in range(k):
        if Q is not None:
            Q[j] = q
        w = apply_op(q) - beta_j[:, None] * q_prev
        a = np.einsum("vi,vi->v", q, w)
        w = w - a[:, None] * q
        if reorth:
            for _ in range(2):
                h = np.einsum("jvi,vi->jv", Q[: j + 1], w)
                w = w - np.einsum("jvi,jv->vi", Q[: j + 1], h)
        bn = np.sqrt(np.einsum("vi,vi->v", w, w))
        alpha[:, j] = np.where(active, a, 0.0)
        amax = np.maximum(amax, np.abs(alpha[:, j]))
        beta[:, j] = np.where(active, bn, 0.0)
        stop = active & (bn <= breakdown_tol * amax)
        k_eff[stop] = j + 1
        active = active & ~stop
        q_prev = q
        q = np.where(active[:, None], w / np.where(active, bn, 1.0)[:, None], 0.0)
        beta_j = np.where(active, bn, 0.0)
    if return_basis:
        return alpha, beta, beta0, k_eff, Q[:k]
    return alpha, beta, beta0, k_eff


def lanczos_poles(alpha, beta, beta0, k_eff):
    """Gauss rule of one tridiagonal: nodes theta_j, weights beta0^2 u_1j^2.

    Mapped to the D = C^1/2 spectrum (Eq. 12): Omega_j = sqrt(theta_j) and the
    Eq. 7 weight p^2/Omega becomes beta0^2 u_1j^2 / Omega_j."""
    ke = int(k_eff)
    if ke == 0:
        return np.zeros(0), np.zeros(0)
    T = np.diag(alpha[:ke])
    if ke > 1:
        off = beta[: ke - 1]
        T += np.diag(off, 1) + np.diag(off, -1)
    theta, U = np.linalg.eigh(T)
    if theta.min() <= 0.0:
        raise ValueError("Lanczos tridiagonal is not positive definite")
    Om = np.sqrt(theta)
    return Om, beta0 ** 2 * U[0, :] ** 2 / Om


def sigma_lanczos(wl, k=None, reorth=True, apply_op=None, coeffs=None):
    """Sigma_t(omega_f) from k-step Lanczos on C for every (t, m) start vector.

    Returns (sigma [n_t, n_freq], pole lists, (alpha, beta, beta0, k_eff))."""
    k = wl.k if k is None else k
    if coeffs is None:
        b = start_vectors(wl.eps, wl.n_v, coupling_vectors(wl.L, wl.M))
        b = b.reshape(wl.n_t * wl.n_m, -1)
        if apply_op is None:
            def apply_op(X):
                return apply_casida(wl.eps, wl.n_v, wl.L, X, wl.kernel_factor)
        coeffs = lanczos(apply_op, b, k, reorth=reorth)
    alpha, beta, beta0, k_eff = coeffs
    eta_all = occupation_sign(wl.m_idx, wl.n_v)
    poles = []
    for ti in range(wl.n_t):
        P, Wt, E = [], [], []
        for mi, m in enumerate(wl.m_idx):
            v = ti * wl.n_m + mi
            Om, wt = lanczos_poles(alpha[v], beta[v], beta0[v], k_eff[v])
            P.append(wl.eps[m] - eta_all[mi] * Om)
            Wt.append(wt)
            E.append(np.full(Om.shape[0], eta_all[mi]))
        poles.append((np.concatenate(P), np.concatenate(Wt), np.concatenate(E)))
    sig = np.stack([sigma_from_poles(wl.omega, *poles[ti], wl.delta) for ti in range(wl.n_t)])
    return sig, poles, coeffs


# --------------------------------------------------------------------------
# Quasiparticle equation (not printed in the paper; reading stated above)
# --------------------------------------------------------------------------
def qp_solve(e0, sigma_fn, dsigma_fn, grid=None, tol=1e-10, max_iter=50):
    """Solve E = e0 + Re Sigma(E) with e0 = eps_t + s_t.

    Newton from E = e0 with f(E) = E - e0 - Re Sigma(E), f' = 1 - Re Sigma'(E);
    converged when |dE| <= tol * max(1, |E|).  If Newton fails, scan ``grid``
    for sign changes of f, bisect each bracket, and keep the root closest to
    e0 (ties: larger Z).  Returns (E, Z) with Z = 1 / (1 - Re Sigma'(E))."""
    E = float(e0)
    ok = False
    for _ in range(max_iter):
        f = E - e0 - sigma_fn(E).real
        fp = 1.0 - dsigma_fn(E).real
        if fp == 0.0 or not np.isfinite(f / fp):
            break
        dE = f / fp
        E -= dE
        if abs(dE) <= tol * max(1.0, abs(E)):
            ok = True
            break
    if ok:
        return E, 1.0 / (1.0 - dsigma_fn(E).real)
    if grid is None:
        raise RuntimeError("quasiparticle equation did not converge")
    g = np.asarray(grid, dtype=np.float64)
    fg = g - e0 - np.array([sigma_fn(x).real for x in g])
    best = None
    for i in range(len(g) - 1):
        if fg[i] == 0.0 or fg[i] * fg[i + 1] < 0.0:
            lo, hi, flo = g[i], g[i + 1], fg[i]
            for _ in range(200):
                mid = 0.5 * (lo + hi)
                fm = mid - e0 - sigma_fn(mid).real
                if (fm < 0.0) == (flo < 0.0):
                    lo, flo = mid, fm
                else:
                    hi = mid
                if hi - lo <= tol * max(1.0, abs(mid)):
                    break
            r = 0.5 * (lo + hi)
            Zr = 1.0 / (1.0 - dsigma_fn(r).real)
            key = (abs(r - e0), -Zr)
            if best is None or key < best[0]:
                best = (key, r, Zr)
    if best is None:
        raise RuntimeError("quasiparticle equation has no root on the grid")
    return best[1], best[2]


def solve_all_qp(wl, poles, static_shift=None):
    """QP energies and renormalisation factors for every target."""
    E = np.empty(wl.n_t)
    Z = np.empty(wl.n_t)
    for ti, t in enumerate(wl.targets):
        pos, W, eta = poles[ti]
        e0 = wl.eps[t] + (0.0 if static_shift is None else static_shift[ti])

        def sfn(x, pos=pos, W=W, eta=eta):
            return sigma_from_poles([x], pos, W, eta, wl.delta)[0]

        def dfn(x, pos=pos, W=W, eta=eta):
            return dsigma_from_poles([x], pos, W, eta, wl.delta)[0]

        E[ti], Z[ti] = qp_solve(e0, sfn, dfn, grid=wl.omega)
    return E, Z


# --------------------------------------------------------------------------
# Gradients of the QP energies (implicit function of the QP equation)
# --------------------------------------------------------------------------
def _f_and_divdiff(Om, z, eta):
    """f(theta) = 1 / (sqrt(theta) (z + eta sqrt(theta))) at theta = Om^2 and
    its divided differences f[theta_s, theta_t] (f' on the diagonal), through
    g(Om) = 1/(Om (z + eta Om)):  f[.,.] = g[Om_s, Om_t] / (Om_s + Om_t),
    g[Om_s, Om_t] = -(z + eta (Om_s + Om_t)) / (Om_s Om_t (z+eta Om_s)(z+eta Om_t))."""
    a = z + eta * Om
    f = 1.0 / (Om * a)
    num = -(z + eta * (Om[:, None] + Om[None, :]))
    den = (Om[:, None] * Om[None, :]) * (a[:, None] * a[None, :]) * (Om[:, None] + Om[None, :])
    return f, num / den


def qp_gradient(wl, dE, E, Z, basis):
    """d(sum_t dE[t] E_t)/dL and /d(eps) of the QP energies.

    E_t = eps_t + s_t + Re Sigma_t(E_t) gives dE_t = Z_t (d eps_t + Re dSigma_t)
    at fixed omega = E_t.  Each term F = b^T f(C) b of Sigma_t (Eq. 7-9 with
    f(theta) = 1/(sqrt(theta)(z_m + eta_m sqrt(theta)))) varies as
        dF = 2 (f(C) b) . db + tr(G dC) - (dF/dz) d eps_m,
        G = Y (F_div o (p p^T)) Y^T,   p = Y^T b          (Daleckii-Krein)
    where `basis(v)` returns (Y, theta) for start vector v: the Casida
    eigenvectors and eigenvalues (closed form) or a Lanczos basis Q_k with
    the eigen-decomposition of T_k (Q_k U, theta) (Krylov form; exact at
    k = N_vc).  With C = Delta^2 + c_K D L L^T D, D = diag(Delta^1/2),
    b = D L M:
        dF/dL     = 2 c_K D G D L + (D y) M^T,     y = 2 f(C) b
        dF/dDelta = 2 Delta diag(G) + c_K diag(K D G)/d + y V / (2 d).
    Returns (dL [N_vc, N_aux], deps [n_v + n_c])."""
    Delta = pair_energies(wl.eps, wl.n_v)
    d = np.sqrt(Delta)
    V_all = coupling_vectors(wl.L, wl.M)                       # [n_t, n_m, N_vc]
    eta_all = occupation_sign(wl.m_idx, wl.n_v)
    SC = np.zeros_like(wl.L)          # sum c G D L (C path)
    SB = np.zeros_like(wl.L)          # sum (D y) M^T (b path)
    dDelta = np.zeros(wl.n_vc)
    deps = np.zeros(wl.n_v + wl.n_c)
    for ti, t in enumerate(wl.targets):
        cw = dE[ti] * Z[ti]
        deps[t] += cw
        for mi, m in enumerate(wl.m_idx):
            v = ti * wl.n_m + mi
            Y, theta = basis(v)
            Om = np.sqrt(theta)
            b = d * V_all[ti, mi]
            p = Y.T @ b
            z = E[ti] - wl.eps[m] - 1j * eta_all[mi] * wl.delta
            f, F = _f_and_divdiff(Om, z, eta_all[mi])
            y = 2.0 * (Y @ (f * p)).real                       # dF/db
            Gm = (Y @ ((F * np.outer(p, p)).real) @ Y.T)       # dF/dC
            dFdz = -np.sum(p * p / (Om * (z + eta_all[mi] * Om) ** 2))
            SC += cw * (Gm @ (d[:, None] * wl.L))
            SB += cw * np.outer(d * y, wl.M[ti, mi])
            dDelta += cw * (2.0 * Delta * np.diag(Gm) + y * V_all[ti, mi] / (2.0 * d))
            deps[m] -= cw * dFdz.real
    dL = 2.0 * wl.kernel_factor * d[:, None] * SC + SB
    dDelta += wl.kernel_factor * np.sum(wl.L * SC, axis=1) / d
    # Delta_vc = eps_c - eps_v, vc = v * n_c + c
    dD = dDelta.reshape(wl.n_v, wl.n_c)
    deps[wl.n_v:] += dD.sum(axis=0)
    deps[: wl.n_v] -= dD.sum(axis=1)
    return dL, deps


def qp_energies_closed_form(wl):
    """E_t and Z_t from the closed form (Eq. 7-9)."""
    _, poles = sigma_closed_form(wl)
    return solve_all_qp(wl, poles)


def qp_gradient_lanczos(wl, dE, k=None, reorth=True):
    """Krylov form of the gradient at k Lanczos steps: E_t, Z_t from the
    k-step pole sums and, per start vector, (Y, theta) = (Q_k U, theta) with
    T_k = U diag(theta) U^T.  Equals the closed form at k = N_vc."""
    k = wl.k if k is None else k
    b = start_vectors(wl.eps, wl.n_v, coupling_vectors(wl.L, wl.M)).reshape(wl.n_t * wl.n_m, -1)
    alpha, beta, beta0, k_eff, Q = lanczos(
        lambda X: apply_casida(wl.eps, wl.n_v, wl.L, X, wl.kernel_factor), b, k, reorth=reorth,
        return_basis=True)
    _, poles, _ = sigma_lanczos(wl, coeffs=(alpha, beta, beta0, k_eff))
    E, Z = solve_all_qp(wl, poles)

    def basis(v):
        ke = int(k_eff[v])
        T = np.diag(alpha[v, :ke])
        if ke > 1:
            T += np.diag(beta[v, : ke - 1], 1) + np.diag(beta[v, : ke - 1], -1)
        theta, U = np.linalg.eigh(T)
        return Q[:ke, v, :].T @ U, theta

    return qp_gradient(wl, dE, E, Z, basis)


def qp_gradient_closed_form(wl, dE):
    """Gradient of sum_t dE[t] E_t with the Casida eigenpairs (exact)."""
    E, Z = qp_energies_closed_form(wl)
    theta, Y = np.linalg.eigh(casida_matrix(wl.eps, wl.n_v, wl.L, wl.kernel_factor))
    return qp_gradient(wl, dE, E, Z, lambda v: (Y, theta))


# --------------------------------------------------------------------------
# Exact derivative of the k-step QP energies: reverse mode of the three-term
# recurrence (Eq. 13 without reorthogonalisation), the Gauss rule of T_k
# (Eq. 12, 14) and the QP equation.  Unlike the Krylov form above, which is
# the derivative of the converged f(C) seen through the k-step basis, this
# differentiates exactly what k steps compute, so it is the derivative of
# E_k at any k.
# --------------------------------------------------------------------------
def lanczos_reverse(apply_op, b, k, abar, bbar, breakdown_tol=1e-13):
    """Reverse mode of ``lanczos(apply_op, b, k, reorth=False)`` for one
    start vector b [N] (C symmetric, given by apply_op on rows).

    Forward step j (q_{-1} = 0, beta_0 = 0 as the coupling of q_{-1}):
        u = C q_j ;  w1 = u - beta_j q_{j-1} ;  alpha_j = q_j . w1
        w2 = w1 - alpha_j q_j ;  beta_{j+1} = ||w2|| ;  q_{j+1} = w2 / beta_{j+1}
    T_k holds alpha_0..alpha_{ke-1} and beta_1..beta_{ke-1}; the last
    residual beta_{ke} and q_{ke} do not enter it.  Given the adjoints
    abar[j] = dF/dalpha_j and bbar[j] = dF/dbeta[j] (beta[j] the coupling of
    steps j and j+1, as ``lanczos`` returns it), the steps are taken back
    in reverse order, j = ke-1 .. 0:
        w2bar = (qbar_{j+1} - (qbar_{j+1} . q_{j+1}) q_{j+1}) / beta_{j+1}
                + bbar[j] q_{j+1}                       (0 for j = ke-1)
        abar_j' = abar[j] - w2bar . q_j
        qbar_j += -alpha_j w2bar + abar_j' w1
        ubar_j = w1bar = w2bar + abar_j' q_j
        bbar[j-1] -= w1bar . q_{j-1} ;  qbar_{j-1} -= beta_j w1bar
        qbar_j += C ubar_j                              (C symmetric)
    Returns (qbar_0 = dF/dq_0 at fixed C, ubar [ke, N], Q [ke, N], (alpha,
    beta, beta0, ke)); the derivative with respect to C is
    dF/dC = sum_j ubar_j q_j^T (its symmetric part for a symmetric dC)."""
    b = np.asarray(b, dtype=np.float64)
    alpha, beta, beta0, k_eff, Q = lanczos(apply_op, b[None, :], k, reorth=False,
                                           breakdown_tol=breakdown_tol, return_basis=True)
    alpha, beta, ke = alpha[0], beta[0], int(k_eff[0])
    Q = Q[:ke, 0, :]
    N = b.size
    zero = np.zeros(N)
    bb = np.array(bbar, dtype=np.float64)[: max(ke, 1)].copy()
    qbar = np.zeros((ke + 1, N))
    ubar = np.zeros((ke, N))
    for j in range(ke - 1, -1, -1):
        qj = Q[j]
        qm = Q[j - 1] if j > 0 else zero
        bj = beta[j - 1] if j > 0 else 0.0
        w1 = apply_op(qj[None, :])[0] - bj * qm
        if j < ke - 1:
            q1 = Q[j + 1]
            w2bar = (qbar[j + 1] - (qbar[j + 1] @ q1) * q1) / beta[j] + bb[j] * q1
        else:
            w2bar = zero
        at = abar[j] - w2bar @ qj
        qbar[j] += -alpha[j] * w2bar + at * w1
        w1bar = w2bar + at * qj
        if j > 0:
            bb[j - 1] -= w1bar @ qm
            qbar[j - 1] -= bj * w1bar
        qbar[j] += apply_op(w1bar[None, :])[0]
        ubar[j] = w1bar
    return qbar[0], ubar, Q, (alpha, beta, beta0[0], ke)


def _tridiag(alpha, beta, ke):
    T = np.diag(alpha[:ke])
    if ke > 1:
        T += np.diag(beta[: ke - 1], 1) + np.diag(beta[: ke - 1], -1)
    return T


def _tda_f_and_divdiff(theta, z, eta):
    """f(theta) = 1 / (z + eta theta) and f[theta_s, theta_t] = -eta / ((z +
    eta theta_s)(z + eta theta_t)) (Tamm-Dancoff form of Eq. 7, no square
    root)."""
    a = z + eta * theta
    return 1.0 / a, -eta / (a[:, None] * a[None, :])


def qp_gradient_recurrence(wl, dE, k=None, tda=False, breakdown_tol=1e-13):
    """Exact gradient of sum_t dE[t] E_t^(k) with respect to L and eps, E^(k)
    the QP energies of k-step Lanczos without reorthogonalisation
    (``sigma_lanczos(reorth=False)``, or ``sigma_tda_lanczos(reorth=False)``
    with tda) and the QP equation.

    Per start vector, F = beta0^2 Re e_1^T f(T_k) e_1 at z = E_t - eps_m -
    i eta_m delta (the Gauss rule of Eq. 12-14), weighted by c = dE_t Z_t:
        dF/dT_k = c beta0^2 Re U (F_div o u1 u1^T) U^T   (Daleckii-Krein on T_k)
    gives abar_j (diagonal) and bbar_j (twice the off-diagonal); the
    recurrence's reverse mode (``lanczos_reverse``) gives qbar_0 and the
    pairs (ubar_j, q_j); beta0 = ||b|| enters directly with
    dF/dbeta0 = 2 c beta0 Re e_1^T f(T_k) e_1, so
        y = dF/db = (dF/dbeta0) q_0 + (qbar_0 - (qbar_0 . q_0) q_0) / beta0,
        G = dF/dC = sym(sum_j ubar_j q_j^T).
    Assembly as in ``qp_gradient`` (C = Delta^2 + c_K D L L^T D, b = D L M):
        dL = 2 c_K D G D L + (D y) M^T,
        dDelta = 2 Delta diag(G) + c_K diag(K D G) / d + y V / (2 d);
    Tamm-Dancoff (A = Delta + c_K/2 L L^T, b = V = L M):
        dL = c_K G L + y M^T,  dDelta = diag(G).
    eps_m enters z: deps[m] -= c Re dF/dz.  Returns (dL, deps)."""
    k = wl.k if k is None else k
    Delta = pair_energies(wl.eps, wl.n_v)
    d = np.sqrt(Delta)
    V_all = coupling_vectors(wl.L, wl.M)                       # [n_t, n_m, N_vc]
    eta_all = occupation_sign(wl.m_idx, wl.n_v)
    if tda:
        Amat = tda_matrix(wl.eps, wl.n_v, wl.L, wl.kernel_factor)

        def apply_op(X):
            return X @ Amat.T

        b_all = V_all
        _, poles, coeffs = sigma_tda_lanczos(wl, k=k, reorth=False)
    else:
        def apply_op(X):
            return apply_casida(wl.eps, wl.n_v, wl.L, X, wl.kernel_factor)

        b_all = d * V_all
        _, poles, coeffs = sigma_lanczos(wl, k=k, reorth=False)
    E, Z = solve_all_qp(wl, poles)
    alpha, beta, beta0, k_eff = coeffs
    SC = np.zeros_like(wl.L)          # G D L (G L for Tamm-Dancoff)
    SB = np.zeros_like(wl.L)          # (D y) M^T
    dDelta = np.zeros(wl.n_vc)
    deps = np.zeros(wl.n_v + wl.n_c)
    for ti, t in enumerate(wl.targets):
        cw = dE[ti] * Z[ti]
        deps[t] += cw
        for mi, m in enumerate(wl.m_idx):
            v = ti * wl.n_m + mi
            ke = int(k_eff[v])
            if ke == 0:
                continue
            eta = eta_all[mi]
            z = E[ti] - wl.eps[m] - 1j * eta * wl.delta
            theta, U = np.linalg.eigh(_tridiag(alpha[v], beta[v], ke))
            u1 = U[0]
            if tda:
                f, Fd = _tda_f_and_divdiff(theta, z, eta)
                dfdz = -1.0 / (z + eta * theta) ** 2
            else:
                Om = np.sqrt(theta)
                f, Fd = _f_and_divdiff(Om, z, eta)
                dfdz = -1.0 / (Om * (z + eta * Om) ** 2)
            b0 = beta0[v]
            Gam = cw * b0 ** 2 * (U @ (Fd * np.outer(u1, u1)).real @ U.T)
            abar = np.diag(Gam).copy()
            bbar = np.zeros(ke)
            bbar[: ke - 1] = 2.0 * np.diag(Gam, 1)
            qbar0, ubar, Q, _ = lanczos_reverse(apply_op, b_all[ti, mi], k, abar, bbar,
                                                breakdown_tol)
            q0 = Q[0]
            b0bar = 2.0 * cw * b0 * np.sum(u1 * u1 * f).real
            y = b0bar * q0 + (qbar0 - (qbar0 @ q0) * q0) / b0
            Cbar = ubar.T @ Q
            G = 0.5 * (Cbar + Cbar.T)
            deps[m] -= cw * (b0 ** 2 * np.sum(u1 * u1 * dfdz)).real
            if tda:
                SC += G @ wl.L
                SB += np.outer(y, wl.M[ti, mi])
                dDelta += np.diag(G)
            else:
                SC += G @ (d[:, None] * wl.L)
                SB += np.outer(d * y, wl.M[ti, mi])
                dDelta += 2.0 * Delta * np.diag(G) + y * V_all[ti, mi] / (2.0 * d)
    if tda:
        dL = wl.kernel_factor * SC + SB
    else:
        dL = 2.0 * wl.kernel_factor * d[:, None] * SC + SB
        dDelta += wl.kernel_factor * np.sum(wl.L * SC, axis=1) / d
    dD = dDelta.reshape(wl.n_v, wl.n_c)
    deps[wl.n_v:] += dD.sum(axis=0)
    deps[: wl.n_v] -= dD.sum(axis=1)
    return dL, deps


def qp_energies_tda_closed_form(wl):
    """E_t and Z_t of the Tamm-Dancoff closed form."""
    _, poles = sigma_tda_closed_form(wl)
    return solve_all_qp(wl, poles)


def qp_gradient_tda_closed_form(wl, dE):
    """Gradient of sum_t dE[t] E_t for the Tamm-Dancoff closed form, from the
    eigenpairs (Omega_s, X_s) of A = Delta + c_K/2 L L^T: each term
    F = V^T (z + eta A)^-1 V varies as
        dF = 2 (f(A) V) . dV + tr(G dA) - (dF/dz) d eps_m,
        G = X (F_div o p p^T) X^T,  p = X^T V,  f(theta) = 1/(z + eta theta)
    (Daleckii-Krein), and with V = L M, dA = diag(dDelta) + c_K/2 (dL L^T +
    L dL^T):  dL = c_K G L + y M^T (y = 2 f(A) V),  dDelta = diag(G)."""
    E, Z = qp_energies_tda_closed_form(wl)
    theta, X = np.linalg.eigh(tda_matrix(wl.eps, wl.n_v, wl.L, wl.kernel_factor))
    V_all = coupling_vectors(wl.L, wl.M)
    eta_all = occupation_sign(wl.m_idx, wl.n_v)
    SC = np.zeros_like(wl.L)
    SB = np.zeros_like(wl.L)
    dDelta = np.zeros(wl.n_vc)
    deps = np.zeros(wl.n_v + wl.n_c)
    for ti, t in enumerate(wl.targets):
        cw = dE[ti] * Z[ti]
        deps[t] += cw
        for mi, m in enumerate(wl.m_idx):
            eta = eta_all[mi]
            z = E[ti] - wl.eps[m] - 1j * eta * wl.delta
            p = X.T @ V_all[ti, mi]
            f, Fd = _tda_f_and_divdiff(theta, z, eta)
            y = 2.0 * (X @ (f * p)).real
            G = X @ (Fd * np.outer(p, p)).real @ X.T
            deps[m] -= cw * np.sum(-p * p / (z + eta * theta) ** 2).real
            SC += cw * (G @ wl.L)
            SB += cw * np.outer(y, wl.M[ti, mi])
            dDelta += cw * np.diag(G)
    dL = wl.kernel_factor * SC + SB
    dD = dDelta.reshape(wl.n_v, wl.n_c)
    deps[wl.n_v:] += dD.sum(axis=0)
    deps[: wl.n_v] -= dD.sum(axis=1)
    return dL, deps


# --------------------------------------------------------------------------
# Polynomial variant: Lanczos on D = p_g(C) ~ C^1/2 (paper text after Eq. 12,
# Eq. 13-14).  p_g fits sqrt on the spectral interval [lo, hi] of C; here it
# is the degree-g Chebyshev interpolant (reading: the paper's monomial sum is
# the same polynomial, evaluated stably in the Chebyshev basis).
# --------------------------------------------------------------------------
def chebyshev_sqrt(lo, hi, g):
    """Coefficients c_0..c_g with p(x) = sum_k c_k T_k(t), t = (2x - hi - lo) /
    (hi - lo), interpolating sqrt at the g+1 Chebyshev points of the first
    kind t_j = cos(pi (j + 1/2) / (g + 1))."""
    n = g + 1
    j = np.arange(n)
    tj = np.cos(np.pi * (j + 0.5) / n)
    fj = np.sqrt(0.5 * (hi + lo) + 0.5 * (hi - lo) * tj)
    c = np.empty(n)
    for k in range(n):
        c[k] = 2.0 / n * np.sum(fj * np.cos(k * np.pi * (j + 0.5) / n))
    c[0] *= 0.5
    return c


def chebyshev_eval(c, lo, hi, x):
    """p(x) = sum_k c_k T_k(t) by the three-term recurrence of T_k."""
    t = (2.0 * np.asarray(x, dtype=np.float64) - hi - lo) / (hi - lo)
    tk_1, tk = np.ones_like(t), t
    out = c[0] * tk_1
    if len(c) > 1:
        out = out + c[1] * tk
    for k in range(2, len(c)):
        tk_1, tk = tk, 2.0 * t * tk - tk_1
        out = out + c[k] * tk
    return out


def apply_poly(apply_op, V, c, lo, hi):
    """p(C) V for the Chebyshev series c on [lo, hi], with C given by apply_op
    (rows of V are vectors): Clenshaw's recurrence in S = (2C - (hi+lo)) /
    (hi - lo),  b_k = c_k V + 2 S b_{k+1} - b_{k+2},  p(C) V = c_0 V + S b_1 - b_2."""
    V = np.atleast_2d(np.asarray(V, dtype=np.float64))
    g = len(c) - 1
    a_s, b_s = 2.0 / (hi - lo), -(hi + lo) / (hi - lo)

    def S(X):
        return a_s * apply_op(X) + b_s * X

    b1 = np.zeros_like(V)
    b2 = np.zeros_like(V)
    for k in range(g, 0, -1):
        b1, b2 = c[k] * V + 2.0 * S(b1) - b2, b1
    return c[0] * V + S(b1) - b2


def haydock(alpha, beta, beta0, k_eff, zeta):
    """<P|(zeta - T)^-1|P> = beta0^2 / (zeta - a_0 - b_1^2 / (zeta - a_1 - ...))
    for the tridiagonal (alpha, beta) of one start vector (Eq. 14), at
    complex points zeta (array)."""
    ke = int(k_eff)
    zeta = np.asarray(zeta, dtype=np.complex128)
    if ke == 0:
        return np.zeros_like(zeta)
    t = zeta - alpha[ke - 1]
    for i in range(ke - 2, -1, -1):
        t = zeta - alpha[i] - beta[i] ** 2 / t
    return beta0 ** 2 / t


def sigma_poly_lanczos(wl, g, lo, hi, k=None, reorth=True):
    """Sigma_t(omega_f) with Lanczos on D = p_g(C) from each |P_tm> and
    Sigma_tm(omega) = (1/z) <P|D^-1 - (D + eta z)^-1|P>
                    = (1/z) [G(-eta z) - G(0)],  G(zeta) = <P|(zeta - D_L)^-1|P>,
    z = omega - eps_m - i eta delta (the resolvent form after Eq. 12 and
    Eq. 14).  Returns (sigma [n_t, n_freq], pole lists of the equivalent Gauss
    rule, coefficients)."""
    k = wl.k if k is None else k
    c = chebyshev_sqrt(lo, hi, g)
    b = start_vectors(wl.eps, wl.n_v, coupling_vectors(wl.L, wl.M)).reshape(wl.n_t * wl.n_m, -1)
    coeffs = lanczos(lambda X: apply_poly(
        lambda Y: apply_casida(wl.eps, wl.n_v, wl.L, Y, wl.kernel_factor), X, c, lo, hi),
        b, k, reorth=reorth)
    alpha, beta, beta0, k_eff = coeffs
    eta_all = occupation_sign(wl.m_idx, wl.n_v)
    sig = np.zeros((wl.n_t, wl.omega.size), dtype=np.complex128)
    poles = []
    for ti in range(wl.n_t):
        P, Wt, E = [], [], []
        for mi, m in enumerate(wl.m_idx):
            v = ti * wl.n_m + mi
            eta = eta_all[mi]
            z = wl.omega - wl.eps[m] - 1j * eta * wl.delta
            G0 = haydock(alpha[v], beta[v], beta0[v], k_eff[v], np.array([0.0]))[0]
            sig[ti] += (haydock(alpha[v], beta[v], beta0[v], k_eff[v], -eta * z) - G0) / z
            # the same sum as poles: nodes Om_j of D_L, weights beta0^2 u_1j^2
            ke = int(k_eff[v])
            if ke:
                T = np.diag(alpha[v, :ke])
                if ke > 1:
                    T += np.diag(beta[v, : ke - 1], 1) + np.diag(beta[v, : ke - 1], -1)
                Om, U = np.linalg.eigh(T)
                P.append(wl.eps[m] - eta * Om)
                Wt.append(beta0[v] ** 2 * U[0] ** 2 / Om)
                E.append(np.full(ke, eta))
        poles.append((np.concatenate(P), np.concatenate(Wt), np.concatenate(E)))
    return sig, poles, coeffs


def apply_poly_reverse(apply_op, u, x, c, lo, hi):
    """Reverse mode of ``apply_poly`` for one vector: y = p(C) x by
    Clenshaw's recurrence in S = a_s C + b_s I,
        b_g = c_g x,  b_k = c_k x + 2 S b_{k+1} - b_{k+2} (k = g-1 .. 1),
        y = c_0 x + S b_1 - b_2,
    and the scalar u . y.  Taking the recurrence back with ybar = u gives
        bbar_1 = S u,  bbar_k = 2 S bbar_{k-1} - bbar_{k-2}  (bbar_0 = u),
        xbar = c_0 u + sum_{k>=1} c_k bbar_k      (= p(C)^T u),
        Sbar = u b_1^T + 2 sum_{k=1}^{g-1} bbar_k b_{k+1}^T,  Cbar = a_s Sbar.
    Returns (xbar, pairs) with d(u . p(C) x)/dC = sum (coef * a) b^T over the
    pairs (coef, a, b)."""
    g = len(c) - 1
    a_s, b_s = 2.0 / (hi - lo), -(hi + lo) / (hi - lo)

    def S(X):
        return a_s * apply_op(X[None, :])[0] + b_s * X

    bk = [None] * (g + 2)
    bk[g + 1] = np.zeros_like(x)
    if g >= 1:
        bk[g] = c[g] * x
        for k in range(g - 1, 0, -1):
            bk[k] = c[k] * x + 2.0 * S(bk[k + 1]) - (bk[k + 2] if k + 2 <= g else 0.0)
    xbar = c[0] * u
    pairs = []
    if g == 0:
        return xbar, pairs
    bbar = [u, S(u)]
    pairs.append((a_s, u, bk[1]))
    for k in range(2, g + 1):
        bbar.append(2.0 * S(bbar[k - 1]) - bbar[k - 2])
    for k in range(1, g + 1):
        xbar = xbar + c[k] * bbar[k]
        if k <= g - 1:
            pairs.append((2.0 * a_s, bbar[k], bk[k + 1]))
    return xbar, pairs


def qp_gradient_poly_recurrence(wl, dE, g, lo, hi, k=None, breakdown_tol=1e-13):
    """Exact gradient of sum_t dE[t] E_t^(k) for the polynomial form: k-step
    Lanczos on D = p_g(C) without reorthogonalisation
    (``sigma_poly_lanczos(reorth=False)``) and the QP equation.

    Per start vector the Gauss rule of D's tridiagonal gives
    F = beta0^2 Re e_1^T f(T_k) e_1 with f(Om) = 1 / (Om (z + eta Om)) on D's
    nodes Om (no square root: D already approximates C^1/2), so
        dF/dT_k = c beta0^2 Re U (F_div o u1 u1^T) U^T,
        F_div[s, t] = -(z + eta (Om_s + Om_t)) / (Om_s Om_t (z + eta Om_s)(z + eta Om_t)).
    The recurrence is taken back with operator D (``lanczos_reverse``),
    giving dF/dD = sum_j ubar_j q_j^T; each term passes to C through the
    reverse of the Clenshaw recurrence (``apply_poly_reverse``):
        dF/dC = sum_j sum_pairs coef a b^T   (a, b from ubar_j and q_j).
    Assembly as in ``qp_gradient_recurrence`` (Casida C, b = D L M)."""
    k = wl.k if k is None else k
    c = chebyshev_sqrt(lo, hi, g)
    Delta = pair_energies(wl.eps, wl.n_v)
    d = np.sqrt(Delta)
    V_all = coupling_vectors(wl.L, wl.M)
    eta_all = occupation_sign(wl.m_idx, wl.n_v)

    def apply_C(X):
        return apply_casida(wl.eps, wl.n_v, wl.L, X, wl.kernel_factor)

    def apply_D(X):
        return apply_poly(apply_C, X, c, lo, hi)

    _, poles, coeffs = sigma_poly_lanczos(wl, g, lo, hi, k=k, reorth=False)
    E, Z = solve_all_qp(wl, poles)
    alpha, beta, beta0, k_eff = coeffs
    SC = np.zeros_like(wl.L)
    SB = np.zeros_like(wl.L)
    dDelta = np.zeros(wl.n_vc)
    deps = np.zeros(wl.n_v + wl.n_c)
    for ti, t in enumerate(wl.targets):
        cw = dE[ti] * Z[ti]
        deps[t] += cw
        for mi, m in enumerate(wl.m_idx):
            v = ti * wl.n_m + mi
            ke = int(k_eff[v])
            if ke == 0:
                continue
            eta = eta_all[mi]
            z = E[ti] - wl.eps[m] - 1j * eta * wl.delta
            Om, U = np.linalg.eigh(_tridiag(alpha[v], beta[v], ke))
            u1 = U[0]
            a = z + eta * Om
            f = 1.0 / (Om * a)
            Fd = -(z + eta * (Om[:, None] + Om[None, :])) / (
                (Om[:, None] * Om[None, :]) * (a[:, None] * a[None, :]))
            b0 = beta0[v]
            Gam = cw * b0 ** 2 * (U @ (Fd * np.outer(u1, u1)).real @ U.T)
            abar = np.diag(Gam).copy()
            bbar = np.zeros(ke)
            bbar[: ke - 1] = 2.0 * np.diag(Gam, 1)
            bvec = d * V_all[ti, mi]
            qbar0, ubar, Q, _ = lanczos_reverse(apply_D, bvec, k, abar, bbar, breakdown_tol)
            q0 = Q[0]
            y = 2.0 * cw * b0 * np.sum(u1 * u1 * f).real * q0 + (qbar0 - (qbar0 @ q0) * q0) / b0
            Cbar = np.zeros((wl.n_vc, wl.n_vc))
            for j in range(ke):
                _, pairs = apply_poly_reverse(apply_C, ubar[j], Q[j], c, lo, hi)
                for coef, pa, pb in pairs:
                    Cbar += coef * np.outer(pa, pb)
            G = 0.5 * (Cbar + Cbar.T)
            deps[m] -= cw * (b0 ** 2 * np.sum(u1 * u1 * (-1.0 / (Om * a ** 2)))).real
            SC += G @ (d[:, None] * wl.L)
            SB += np.outer(d * y, wl.M[ti, mi])
            dDelta += 2.0 * Delta * np.diag(G) + y * V_all[ti, mi] / (2.0 * d)
    dL = 2.0 * wl.kernel_factor * d[:, None] * SC + SB
    dDelta += wl.kernel_factor * np.sum(wl.L * SC, axis=1) / d
    dD = dDelta.reshape(wl.n_v, wl.n_c)
    deps[wl.n_v:] += dD.sum(axis=0)
    deps[: wl.n_v] -= dD.sum(axis=1)
    return dL, deps


# --------------------------------------------------------------------------
# Static part (text around Eq. 5-6): exchange from the pair factors and the
# linearised QP solution; density-fitting factors from a metric.
# --------------------------------------------------------------------------
def sigma_x(wl):
    """Sigma^ex_t = -sum_v (vt|vt) over the occupied orbitals v of the summed
    set.  The pair factors M share L's metric-folded form, (pq|rs) =
    sum_mu B_pq,mu B_rs,mu, so (vt|vt) = sum_mu M[t, v, mu]^2."""
    occ = np.asarray(wl.m_idx) < wl.n_v
    return -np.einsum("tmu,tmu->t", wl.M[:, occ, :], wl.M[:, occ, :])


def qp_linearised(wl, poles, static_shift=None):
    """E_t = e0 + Z Re Sigma_t(e0), Z = 1 / (1 - Re Sigma_t'(e0)),
    e0 = eps_t + s_t (first-order expansion of the QP equation at e0)."""
    E = np.empty(wl.n_t)
    Z = np.empty(wl.n_t)
    for ti, t in enumerate(wl.targets):
        pos, W, eta = poles[ti]
        e0 = wl.eps[t] + (0.0 if static_shift is None else static_shift[ti])
        S = sigma_from_poles([e0], pos, W, eta, wl.delta)[0]
        dS = dsigma_from_poles([e0], pos, W, eta, wl.delta)[0]
        Z[ti] = 1.0 / (1.0 - dS.real)
        E[ti] = e0 + Z[ti] * S.real
    return E, Z


def fit_factors(C, metric):
    """Density-fitting pair factors B = C R with metric = R R^T (Cholesky, R
    lower), so that (ab|cd) = sum_{mu,nu} C_ab,mu metric_mu,nu C_cd,nu =
    sum_kappa B_ab,kappa B_cd,kappa (the L and M of this problem)."""
    R = np.linalg.cholesky(np.asarray(metric, dtype=np.float64))
    return np.asarray(C, dtype=np.float64) @ R


# --------------------------------------------------------------------------
# Tamm-Dancoff variant (B = 0): the excitations are the eigenpairs of A
# alone, A = Delta + (c_K / 2) L L^T (A holds the kernel once, A + B twice),
# and W^s_tm = sum_vc (tm|vc) X^s_vc, so
#   Sigma_tm(omega) = sum_s (V . X_s)^2 / (z + eta Omega_s) = V^T (z + eta A)^-1 V.
# --------------------------------------------------------------------------
def tda_matrix(eps, n_v, L, kernel_factor=4.0):
    Delta = pair_energies(eps, n_v)
    return np.diag(Delta) + 0.5 * kernel_factor * (L @ L.T)


def sigma_tda_closed_form(wl):
    """Sigma_t(omega) and its pole lists from the eigenpairs of A."""
    Om, X = np.linalg.eigh(tda_matrix(wl.eps, wl.n_v, wl.L, wl.kernel_factor))
    V = coupling_vectors(wl.L, wl.M)                       # [n_t, n_m, N_vc]
    p = V @ X
    eta = occupation_sign(wl.m_idx, wl.n_v)
    poles = []
    for ti in range(wl.n_t):
        pos = (wl.eps[wl.m_idx][:, None] - eta[:, None] * Om[None, :]).ravel()
        poles.append((pos, (p[ti] ** 2).ravel(), np.repeat(eta, Om.size)))
    sig = np.stack([sigma_from_poles(wl.omega, *poles[ti], wl.delta) for ti in range(wl.n_t)])
    return sig, poles


def sigma_tda_lanczos(wl, k=None, reorth=True):
    """k-step Lanczos on A from each V_tm; Sigma_tm = -eta G(-eta z) with
    G(zeta) = <V|(zeta - A_k)^-1|V> the Haydock fraction of the tridiagonal;
    also the equivalent Gauss-rule poles (nodes of A_k, weights beta0^2 u1^2)."""
    k = wl.k if k is None else k
    A = tda_matrix(wl.eps, wl.n_v, wl.L, wl.kernel_factor)
    V = coupling_vectors(wl.L, wl.M).reshape(wl.n_t * wl.n_m, -1)
    coeffs = lanczos(lambda X: X @ A.T, V, k, reorth=reorth)
    alpha, beta, beta0, k_eff = coeffs
    eta_all = occupation_sign(wl.m_idx, wl.n_v)
    sig = np.zeros((wl.n_t, wl.omega.size), dtype=np.complex128)
    poles = []
    for ti in range(wl.n_t):
        P, Wt, E = [], [], []
        for mi, m in enumerate(wl.m_idx):
            v = ti * wl.n_m + mi
            eta = eta_all[mi]
            z = wl.omega - wl.eps[m] - 1j * eta * wl.delta
            sig[ti] += -eta * haydock(alpha[v], beta[v], beta0[v], k_eff[v], -eta * z)
            ke = int(k_eff[v])
            if ke:
                T = np.diag(alpha[v, :ke])
                if ke > 1:
                    T += np.diag(beta[v, : ke - 1], 1) + np.diag(beta[v, : ke - 1], -1)
                Om, U = np.linalg.eigh(T)
                P.append(wl.eps[m] - eta * Om)
                Wt.append(beta0[v] ** 2 * U[0] ** 2)
                E.append(np.full(ke, eta))
        poles.append((np.concatenate(P), np.concatenate(Wt), np.concatenate(E)))
    return sig, poles, coeffs


def sigma_offdiag_closed_form(wl, t_pair):
    """Off-diagonal element Sigma_tt'(omega) = sum_m sum_s W^s_tm W^s_t'm /
    (Omega_s (z + eta Omega_s)) (Eq. 7 with the two targets of t_pair, given as
    indices into wl.targets; RPA, from the Casida eigenpairs)."""
    Om, Z = casida_eigenpairs(casida_matrix(wl.eps, wl.n_v, wl.L, wl.kernel_factor))
    b = start_vectors(wl.eps, wl.n_v, coupling_vectors(wl.L, wl.M))
    i, j = t_pair
    eta = occupation_sign(wl.m_idx, wl.n_v)
    out = np.zeros(wl.omega.size, dtype=np.complex128)
    for mi, m in enumerate(wl.m_idx):
        pa, pb = b[i, mi] @ Z, b[j, mi] @ Z
        z = wl.omega[:, None] - wl.eps[m] - 1j * eta[mi] * wl.delta
        out += np.sum(pa * pb / (Om * (z + eta[mi] * Om)), axis=1)
    return out


# --------------------------------------------------------------------------
# Band Lanczos for off-diagonal elements: the band-Lanczos method for
# matrix elements of a resolvent that the paper cites after Eq. 14, here in
# the one-vector-per-step form with full reorthogonalisation.
# --------------------------------------------------------------------------
def band_lanczos(apply_op, B, k, breakdown_tol=1e-13):
    """Band Lanczos from the p rows of B ([p, N]).

    The start block is orthonormalised by classical Gram-Schmidt (twice):
    b_a = sum_i R0[i, a] q_i, R0 [p, p] upper triangular, q_0..q_{p-1} the
    first basis vectors.  Step j applies C to q_j (the j-th basis vector):
        u = C q_j ;  twice: h = Q^T u, u = u - Q h     (all n vectors so far)
        T[i, j] = T[j, i] = (sum of both passes' h_i)  for j <= i < n
        beta = ||u||: unless beta <= breakdown_tol * max|T|, a new vector
        q_n = u / beta with T[n, j] = T[j, n] = beta.
    T on the first k basis vectors is Q^T C Q, banded with bandwidth p.  The
    recurrence ends after k steps, or earlier once every basis vector has
    been multiplied (the block's Krylov space is exhausted); vectors past
    the k-th are not formed.
    Returns (T [ke, ke], R0 [p, p], ke) with ke <= k the number of steps."""
    B = np.atleast_2d(np.asarray(B, dtype=np.float64))
    p, N = B.shape
    Q = np.zeros((max(k, p), N))
    R0 = np.zeros((p, p))
    n = 0
    scale = 0.0
    for a in range(p):
        u = B[a].copy()
        h = np.zeros(n)
        for _ in range(2):
            d = Q[:n] @ u
            u = u - Q[:n].T @ d
            h = h + d
        r = np.linalg.norm(u)
        R0[:n, a] = h
        scale = max(scale, np.linalg.norm(B[a]))
        if r > breakdown_tol * scale:
            R0[n, a] = r
            Q[n] = u / r
            n += 1
    T = np.zeros((k, k))
    tmax = 0.0
    j = 0
    while j < k and j < n:
        u = apply_op(Q[j][None, :])[0]
        h = np.zeros(n)
        for _ in range(2):
            d = Q[:n] @ u
            u = u - Q[:n].T @ d
            h = h + d
        for i in range(j, min(n, k)):
            T[i, j] = T[j, i] = h[i]
        tmax = max(tmax, np.abs(h[j:n]).max())
        beta = np.linalg.norm(u)
        # vectors past the first k are never multiplied and do not enter T
        if n < k and beta > breakdown_tol * tmax:
            T[n, j] = T[j, n] = beta
            Q[n] = u / beta
            n += 1
        j += 1
    return T[:j, :j], R0, j


def band_gauss_rule(T, R0):
    """Matrix-valued Gauss rule of the band recurrence: nodes theta_s and
    vectors r_s = R0^T U[:p, s] (U the eigenvectors of T), so that
    b_a . f(C) b_b ~ sum_s f(theta_s) r_s[a] r_s[b]; exact once the block's
    Krylov space is exhausted."""
    theta, U = np.linalg.eigh(T)
    p = R0.shape[0]
    return theta, R0.T @ U[:p, :]


def sigma_band_lanczos(wl, k=None, breakdown_tol=1e-13):
    """Sigma_tt'(omega) for every pair of the workload's targets: one band
    recurrence per summed orbital m from the block [b_tm over t], then
        Sigma_tt'(omega) = sum_m sum_s r_s[t] r_s[t'] / (Omega_s (z_m + eta_m Omega_s)),
    Omega_s = sqrt(theta_s), z_m = omega - eps_m - i eta_m delta (Eq. 7 with
    the square-root map of Eq. 12).  Returns sigma [n_t, n_t, n_freq] and the
    per-m recurrences [(T, R0, ke)]."""
    k = wl.k if k is None else k
    b = start_vectors(wl.eps, wl.n_v, coupling_vectors(wl.L, wl.M))   # [n_t, n_m, N]
    eta = occupation_sign(wl.m_idx, wl.n_v)

    def apply_op(X):
        return apply_casida(wl.eps, wl.n_v, wl.L, X, wl.kernel_factor)

    out = np.zeros((wl.n_t, wl.n_t, wl.omega.size), dtype=np.complex128)
    recs = []
    for mi, m in enumerate(wl.m_idx):
        T, R0, ke = band_lanczos(apply_op, b[:, mi, :], k, breakdown_tol)
        recs.append((T, R0, ke))
        if ke == 0:
            continue
        theta, r = band_gauss_rule(T, R0)
        if theta.min() <= 0.0:
            raise ValueError("band tridiagonal is not positive definite")
        Om = np.sqrt(theta)
        z = wl.omega[:, None] - wl.eps[m] - 1j * eta[mi] * wl.delta
        g = 1.0 / (Om * (z + eta[mi] * Om))           # [n_freq, ke]
        out += np.einsum("as,bs,fs->abf", r, r, g)
    return out, recs
