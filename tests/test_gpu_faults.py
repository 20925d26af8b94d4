"""Failure paths in safe forms: nothing here faults, traps or hangs the GPU.

  * Bounded device wait: the tensor-core pipeline's mbarrier wait, run by a
    diagnostic kernel with a 50 ms limit on a barrier that nothing completes,
    must give LGW_ERR_TIMEOUT; with the barrier completed it gives LGW_OK;
    afterwards the handle computes correct results (the context survived).
  * Allocation failure injected on the host: a workspace byte limit below
    what the call needs gives LGW_ERR_OOM before the allocation; the handle
    stays usable once the limit is lifted, and releasing the workspace
    returns its memory.
"""
import time

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


def _t(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to(DEV)


def _tiny_call(L, h, wl):
    s = L.lgw_prepare_system(h, wl.n_v, wl.n_c, wl.n_aux, _t(wl.eps), _t(wl.L))
    try:
        prob = L.Problem(targets=_t(wl.targets), m_idx=_t(wl.m_idx), omega=_t(wl.omega),
                         delta=wl.delta, M=_t(wl.M))
        sig = torch.empty(wl.n_t, wl.omega.size, 2, dtype=torch.float64, device=DEV)
        e = torch.empty(wl.n_t, dtype=torch.float64, device=DEV)
        L.lgw_sigma_c(h, s, prob, L.Options(k=32, precision="bf16", reorth="dcgs"), sig, e)
        torch.cuda.synchronize()
        return e.cpu().numpy()
    finally:
        L.lgw_release_system(s)


@pytest.fixture(scope="module")
def ref():
    wl = gi.tiny(k=32)
    _, poles, _ = O.sigma_lanczos(wl, k=32)
    E, _ = O.solve_all_qp(wl, poles)
    return wl, E


def test_bounded_wait_times_out_and_context_survives(L, ref):
    wl, E = ref
    h = L.lgw_create(0)
    try:
        L.lgw_selftest_bounded_wait(h, True, 0.05)           # completed barrier: no timeout
        t0 = time.perf_counter()
        with pytest.raises(L.LgwError) as ei:
            L.lgw_selftest_bounded_wait(h, False, 0.05)      # nothing arrives
        dt = time.perf_counter() - t0
        assert ei.value.status == 7                           # LGW_ERR_TIMEOUT
        assert "bounded device wait" in str(ei.value)
        assert dt < 5.0
        # the context and the handle are intact: a full call is still exact
        e = _tiny_call(L, h, wl)
        assert np.abs(e - E).max() < 1e-3
        L.lgw_selftest_bounded_wait(h, True, 0.05)
        with pytest.raises(L.LgwError) as ei:
            L.lgw_selftest_bounded_wait(h, False, 10.0)      # outside [1e-4, 2] s
        assert ei.value.status == 1
    finally:
        L.lgw_destroy(h)


def test_workspace_limit_gives_oom_and_handle_recovers(L, ref):
    wl, E = ref
    h = L.lgw_create(0)
    try:
        e0 = _tiny_call(L, h, wl)
        need = L.lgw_workspace_bytes(h)
        assert need > 0
        L.lgw_release_workspace(h)
        assert L.lgw_workspace_bytes(h) == 0
        L.lgw_set_workspace_limit(h, need // 4)
        with pytest.raises(L.LgwError) as ei:
            _tiny_call(L, h, wl)
        assert ei.value.status == 4                           # LGW_ERR_OOM
        assert "workspace limit" in str(ei.value)
        assert L.lgw_workspace_bytes(h) <= need // 4
        L.lgw_set_workspace_limit(h, 0)
        e1 = _tiny_call(L, h, wl)
        assert np.array_equal(e0, e1)
        assert np.abs(e1 - E).max() < 1e-3
        # a limit that fits changes nothing
        L.lgw_set_workspace_limit(h, L.lgw_workspace_bytes(h))
        assert np.array_equal(_tiny_call(L, h, wl), e0)
    finally:
        L.lgw_destroy(h)
