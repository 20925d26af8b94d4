"""CUDA-graph replay of the Lanczos sub-batches, the tile autotuner, and the
batched call over systems of uneven size.

  * use_graph = 1 gives bit-identical results to eager launches, on the
    capture call and on replays, for both precisions, and reports the same
    launch count;
  * releasing a system drops the graphs that reference it;
  * lgw_sigma_c_batched over systems of the batched-uneven workload (shapes
    drawn per system, seed 100+i) equals one lgw_sigma_c per system, and
    sampled start vectors match the oracle.
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


def _prob(L, wl):
    return L.Problem(targets=_t(wl.targets), m_idx=_t(wl.m_idx), omega=_t(wl.omega),
                     delta=wl.delta, M=_t(wl.M))


def _sigma(L, h, s, wl, opts, report=False, prob=None):
    """One lgw_sigma_c call.  Graphs are keyed on the problem's device
    buffers, so replay tests pass the same Problem every time."""
    sig = torch.empty(wl.n_t, wl.omega.size, 2, dtype=torch.float64, device=DEV)
    e = torch.empty(wl.n_t, dtype=torch.float64, device=DEV)
    rep = L.lgw_sigma_c(h, s, prob if prob is not None else _prob(L, wl), opts, sig, e,
                        report=report)
    torch.cuda.synchronize()
    return sig.cpu().numpy(), e.cpu().numpy(), rep


@pytest.mark.parametrize("prec,reorth", [("fp64", "cgs2"), ("bf16", "cgs1k"), ("bf16", "none")])
def test_graph_replay_bit_identical(L, handle, prec, reorth):
    wl = gi.custom(16, 96, 256, 2, 64, 300, 3, k=48)
    s = L.lgw_prepare_system(handle, wl.n_v, wl.n_c, wl.n_aux, _t(wl.eps), _t(wl.L))
    prob = _prob(L, wl)
    try:
        eager = _sigma(L, handle, s, wl, L.Options(k=48, precision=prec, reorth=reorth, b_sub=64),
                       report=True, prob=prob)
        og = L.Options(k=48, precision=prec, reorth=reorth, b_sub=64, use_graph=1)
        for _ in range(3):          # capture (possibly twice while buffers settle), replays
            got = _sigma(L, handle, s, wl, og, report=True, prob=prob)
            np.testing.assert_array_equal(got[0], eager[0])
            np.testing.assert_array_equal(got[1], eager[1])
            assert got[2]["gpu_launches"] == eager[2]["gpu_launches"]
    finally:
        L.lgw_release_system(s)


def test_release_drops_graphs(L, handle):
    """Two systems prepared one after the other (the second may reuse the
    first one's addresses) each get their own, correct, graphs."""
    out = []
    for seed in (5, 6):
        wl = gi.custom(16, 96, 256, 1, 64, 200, seed, k=40)
        s = L.lgw_prepare_system(handle, wl.n_v, wl.n_c, wl.n_aux, _t(wl.eps), _t(wl.L))
        prob = _prob(L, wl)
        try:
            og = L.Options(k=40, precision="bf16", reorth="cgs2", b_sub=64, use_graph=1)
            a = _sigma(L, handle, s, wl, og, prob=prob)
            b = _sigma(L, handle, s, wl, og, prob=prob)
            eager = _sigma(L, handle, s, wl, L.Options(k=40, precision="bf16", reorth="cgs2",
                                                       b_sub=64), prob=prob)
            np.testing.assert_array_equal(b[0], eager[0])
            np.testing.assert_array_equal(a[0], eager[0])
            out.append(eager[1])
        finally:
            L.lgw_release_system(s)
    assert not np.array_equal(out[0], out[1])


def test_autotuned_tiles_match_default(L, handle, monkeypatch):
    """The autotuner changes only tile shapes and split counts: the BF16 QP
    energies agree with the untuned heuristic within FP32 summation noise."""
    wl = gi.custom(32, 256, 512, 2, 128, 200, 8, k=40)
    res = {}
    for tune in ("0", "1"):
        monkeypatch.setenv("LGW_AUTOTUNE", tune)
        s = L.lgw_prepare_system(handle, wl.n_v, wl.n_c, wl.n_aux, _t(wl.eps), _t(wl.L))
        try:
            res[tune] = _sigma(L, handle, s, wl, L.Options(k=40, precision="bf16",
                                                           reorth="cgs2"))[1]
        finally:
            L.lgw_release_system(s)
    assert np.abs(res["0"] - res["1"]).max() < 1e-6       # eV


@pytest.fixture(scope="module")
def batch(L, handle):
    """Three systems of the batched-uneven workload (the smallest ones:
    N_vc 6384, 6272, 4975), two targets each, k 150."""
    wls = [gi.batched_uneven(i, max_targets=2) for i in (2, 11, 13)]
    systems = [L.lgw_prepare_system(handle, w.n_v, w.n_c, w.n_aux, _t(w.eps), _t(w.L))
               for w in wls]
    yield wls, systems
    for s in systems:
        L.lgw_release_system(s)


@pytest.mark.parametrize("use_graph", [0, 1])
def test_batched_equals_single_calls(L, handle, batch, use_graph):
    wls, systems = batch
    opts = L.Options(k=150, precision="bf16", reorth="cgs1k", use_graph=use_graph)
    sig = [torch.empty(w.n_t, w.omega.size, 2, dtype=torch.float64, device=DEV) for w in wls]
    e = [torch.empty(w.n_t, dtype=torch.float64, device=DEV) for w in wls]
    probs = [_prob(L, w) for w in wls]
    for _ in range(3):
        rep = L.lgw_sigma_c_batched(handle, systems, probs, opts, sig, e, report=True)
        torch.cuda.synchronize()
    assert rep["n_vectors"] == sum(w.n_t * w.n_m for w in wls)
    for w, s, sg, ee in zip(wls, systems, sig, e):
        one = _sigma(L, handle, s, w, L.Options(k=150, precision="bf16", reorth="cgs1k"))
        np.testing.assert_array_equal(sg.cpu().numpy(), one[0])
        np.testing.assert_array_equal(ee.cpu().numpy(), one[1])


def test_batched_sampled_vectors_vs_oracle(L, handle, batch):
    """Sampled start vectors of each system: the BF16 path's Sigma_tm(omega)
    against the oracle's FP64 recurrence, in meV (each of the n_m
    contributions within 1/n_m meV)."""
    wls, systems = batch
    for w, s in zip(wls, systems):
        B = w.n_t * w.n_m
        al = torch.empty(B, 150, dtype=torch.float64, device=DEV)
        be = torch.empty_like(al)
        b0 = torch.empty(B, dtype=torch.float64, device=DEV)
        ke = torch.empty(B, dtype=torch.int32, device=DEV)
        L.lgw_lanczos_coeffs(handle, s, _prob(L, w), L.Options(k=150, precision="bf16",
                                                               reorth="cgs1k"), al, be, b0, ke)
        co = (al.cpu().numpy(), be.cpu().numpy(), b0.cpu().numpy(),
              ke.cpu().numpy().astype(np.int64))
        vs = [0, w.n_m // 2, B - 1]
        b = O.start_vectors(w.eps, w.n_v, O.coupling_vectors(w.L, w.M)).reshape(-1, w.n_vc)
        ref = O.lanczos(lambda X: O.apply_casida(w.eps, w.n_v, w.L, X, w.kernel_factor), b[vs],
                        150)
        for i, v in enumerate(vs):
            m = int(w.m_idx[v % w.n_m])
            eta = 1.0 if m < w.n_v else -1.0
            Om, W = O.lanczos_poles(co[0][v], co[1][v], co[2][v], co[3][v])
            g = O.sigma_from_poles(w.omega, w.eps[m] - eta * Om, W, np.full(Om.size, eta),
                                   w.delta)
            Om, W = O.lanczos_poles(ref[0][i], ref[1][i], ref[2][i], ref[3][i])
            r = O.sigma_from_poles(w.omega, w.eps[m] - eta * Om, W, np.full(Om.size, eta),
                                   w.delta)
            assert np.abs(g - r).max() * 1e3 <= 1.0 / w.n_m, (w.name, v)


def test_gemm2_pipeline_variants_bit_identical():
    """GEMM2 (L y with the store-only c_K Delta^1/2 epilogue) runs as one CTA
    per tile, as the half-depth pipeline (two CTAs per SM) or as the
    persistent kernel with two TMEM accumulators; all keep the same K order
    per output element, so the Lanczos tridiagonals must agree bit for bit
    (ragged N_vc, several M tiles per CTA, both tile orders through the
    tuner's choice)."""
    import os
    from paper_2310_20103_gb300.build import build
    build()
    from paper_2310_20103_gb300 import lgw as L
    wl = gi.make_workload("p2", 24, 700, 384, [22, 23, 24], list(range(48)), 50, 9, k=24,
                          aux_scaled=True)
    h = L.lgw_create(0)
    s = L.lgw_prepare_system(h, wl.n_v, wl.n_c, wl.n_aux, _t(wl.eps), _t(wl.L))
    prob = L.Problem(targets=_t(wl.targets), m_idx=_t(wl.m_idx), omega=_t(wl.omega),
                     delta=wl.delta, M=_t(wl.M))
    B = wl.n_t * wl.n_m
    res = []
    try:
        for pipe in ("0", "1", "2"):
            os.environ["LGW_GEMM2_PIPE"] = pipe
            al = torch.empty(B, 24, dtype=torch.float64, device=DEV)
            be = torch.empty_like(al)
            b0 = torch.empty(B, dtype=torch.float64, device=DEV)
            ke = torch.empty(B, dtype=torch.int32, device=DEV)
            L.lgw_lanczos_coeffs(h, s, prob, L.Options(k=24, precision="bf16", reorth="dcgs"),
                                 al, be, b0, ke)
            torch.cuda.synchronize()
            res.append((al.cpu().numpy(), be.cpu().numpy()))
    finally:
        os.environ.pop("LGW_GEMM2_PIPE", None)
        L.lgw_release_system(s)
        L.lgw_destroy(h)
    for a, b in res[1:]:
        assert np.array_equal(a, res[0][0])
        assert np.array_equal(b, res[0][1])
