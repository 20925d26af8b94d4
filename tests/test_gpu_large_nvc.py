"""Parity at the large cluster's pair dimension.

N_v=400, N_c=4000 (N_vc 1.6M, as in the large cluster-sized system) with a
reduced auxiliary basis, N_aux 256, so that the oracle's FP64 L stays at
3.3 GB, and that system's entry distributions for L and M (same coupling
strength).  This is the regime where a row block of the contraction operands
spans hundreds of pages (the K-block-major layouts), GEMM1 runs many K
splits, and every vector pass has 782 chunks per vector.

  * sampled start vectors with BF16 and E4M3 contractions, plain recurrence
    and CGS1K, against the oracle's FP64 recurrence: each Sigma_tm(omega)
    contribution within 1/n_m meV, so the n_m contributions of a target stay
    within 1 meV;
  * the FP64 GPU path on one sampled vector at 1e-9 relative;
  * E_qp from BF16 and E4M3 against the FP64 GPU path within 1 meV.

Targets HOMO and LUMO, summed over 32 valence and 32 conduction orbitals
(64 start vectors per target), k = 24, 200 frequencies, seed 11.
"""
import numpy as np
import pytest

import gw_inputs as gi
import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"
K = 24
SAMPLE = [0, 40, 64 + 5, 64 + 63]      # vector index = t_index * n_m + m_index


def _t(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to(DEV)


@pytest.fixture(scope="module")
def large():
    from paper_2310_20103_gb300.build import build
    build()
    from paper_2310_20103_gb300 import lgw as L
    n_v, n_c = 400, 4000
    m_idx = list(range(32)) + list(range(n_v, n_v + 32))
    # the large system's distributions: L ~ N(0, (0.05/sqrt(8192))^2) and M ~
    # N(0, (0.1/sqrt(8192))^2), so C has the same coupling strength at the
    # smaller N_aux (sigma_L^2 N_vc is what sets it)
    r = np.sqrt(256 / 8192)
    wl = gi.make_workload("large_nvc", n_v, n_c, 256, [n_v - 1, n_v], m_idx, 200, 11, k=K,
                          aux_scaled=True, sigma_L=0.05 * r, sigma_M=0.1 * r)
    h = L.lgw_create(0)
    s = L.lgw_prepare_system(h, wl.n_v, wl.n_c, wl.n_aux, _t(wl.eps), _t(wl.L))
    prob = L.Problem(targets=_t(wl.targets), m_idx=_t(wl.m_idx), omega=_t(wl.omega),
                     delta=wl.delta, M=_t(wl.M))
    yield dict(wl=wl, L=L, h=h, s=s, prob=prob)
    L.lgw_release_system(s)
    L.lgw_destroy(h)


def _coeffs(d, opts, prob=None, B=None):
    L, wl = d["L"], d["wl"]
    B = B or wl.n_t * wl.n_m
    al = torch.empty(B, K, dtype=torch.float64, device=DEV)
    be = torch.empty_like(al)
    b0 = torch.empty(B, dtype=torch.float64, device=DEV)
    ke = torch.empty(B, dtype=torch.int32, device=DEV)
    L.lgw_lanczos_coeffs(d["h"], d["s"], prob or d["prob"], opts, al, be, b0, ke)
    torch.cuda.synchronize()
    return (al.cpu().numpy(), be.cpu().numpy(), b0.cpu().numpy(),
            ke.cpu().numpy().astype(np.int64))


def _sigma_tm(wl, v, co, row):
    m = int(wl.m_idx[v % wl.n_m])
    eta = 1.0 if m < wl.n_v else -1.0
    Om, W = O.lanczos_poles(co[0][row], co[1][row], co[2][row], co[3][row])
    return O.sigma_from_poles(wl.omega, wl.eps[m] - eta * Om, W, np.full(Om.size, eta),
                              wl.delta)


@pytest.fixture(scope="module")
def oracle_ref(large):
    """The oracle's FP64 recurrences of the sampled start vectors, with and
    without reorthogonalisation (start vectors only for the sample)."""
    wl = large["wl"]
    Ms = wl.M.reshape(-1, wl.n_aux)[SAMPLE]
    b = O.start_vectors(wl.eps, wl.n_v, (wl.L @ Ms.T).T)
    op = lambda X: O.apply_casida(wl.eps, wl.n_v, wl.L, X, wl.kernel_factor)
    return {True: O.lanczos(op, b, K, reorth=True), False: O.lanczos(op, b, K, reorth=False)}


@pytest.mark.parametrize("prec,reorth", [("bf16", "none"), ("fp8", "none"), ("bf16", "cgs1k"),
                                         ("fp8", "cgs1k")])
def test_sampled_vectors_vs_oracle(large, oracle_ref, prec, reorth):
    wl, L = large["wl"], large["L"]
    co = _coeffs(large, L.Options(k=K, precision=prec, reorth=reorth))
    ref = oracle_ref[reorth != "none"]
    assert np.all(co[3] == K)
    for i, v in enumerate(SAMPLE):
        err_mev = np.abs(_sigma_tm(wl, v, co, v) - _sigma_tm(wl, v, ref, i)).max() * 1e3
        print(f"{prec}/{reorth} vector {v}: max|dSigma_tm| = {err_mev:.3e} meV")
        assert err_mev <= 1.0 / wl.n_m


def test_fp64_path_vs_oracle(large, oracle_ref):
    """One sampled vector through the FP64 GPU path (its own one-target,
    one-orbital problem), CGS2, against the oracle at 1e-9 relative."""
    wl, L = large["wl"], large["L"]
    v = SAMPLE[2]
    ti, mi = divmod(v, wl.n_m)
    prob = L.Problem(targets=_t(wl.targets[ti:ti + 1]), m_idx=_t(wl.m_idx[mi:mi + 1]),
                     omega=_t(wl.omega), delta=wl.delta, M=_t(wl.M[ti:ti + 1, mi:mi + 1]))
    co = _coeffs(large, L.Options(k=K, precision="fp64", reorth="cgs2"), prob=prob, B=1)
    g = _sigma_tm(wl, v, co, 0)
    r = _sigma_tm(wl, v, oracle_ref[True], 2)
    assert np.abs(g - r).max() <= 1e-9 * np.abs(r).max()


def test_qp_energies_vs_fp64_path(large):
    """E_qp with BF16 and E4M3 contractions against the FP64 GPU path at
    the same k and reorthogonalisation (1 meV)."""
    wl, L = large["wl"], large["L"]
    out = {}
    for prec in ("fp64", "bf16", "fp8"):
        sig = torch.empty(wl.n_t, wl.omega.size, 2, dtype=torch.float64, device=DEV)
        e = torch.empty(wl.n_t, dtype=torch.float64, device=DEV)
        L.lgw_sigma_c(large["h"], large["s"], large["prob"],
                      L.Options(k=K, precision=prec, reorth="cgs1k"), sig, e)
        torch.cuda.synchronize()
        out[prec] = e.cpu().numpy()
    for prec in ("bf16", "fp8"):
        d = np.abs(out[prec] - out["fp64"]).max() * 1e3
        print(f"{prec}: max |dE_qp| = {d:.3e} meV")
        assert d <= 1.0
