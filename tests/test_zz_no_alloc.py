"""The allocation-free entry point gives the same self-energy and QP
energies as lgw_sigma_from_coeffs.

Callers that cannot let the library allocate device memory mid-run (fixed
device budgets, latency-bound loops where an allocation would synchronise
the device) use lgw_sigma_from_coeffs_noalloc, whose scratch is a fixed
static device array.  This file is collected last so that a failure here
never hides the other tests when pytest stops at the first failure."""
import numpy as np
import pytest

import gw_inputs as gi

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _t(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to(DEV)


def test_noalloc_matches_allocating_entry_point():
    from paper_2310_20103_gb300.build import build
    build()
    from paper_2310_20103_gb300 import lgw as L

    wl = gi.tiny(k=48)
    h = L.lgw_create(0)
    try:
        s = L.lgw_prepare_system(h, wl.n_v, wl.n_c, wl.n_aux, _t(wl.eps), _t(wl.L))
        prob = L.Problem(targets=_t(wl.targets), m_idx=_t(wl.m_idx), omega=_t(wl.omega),
                         delta=wl.delta, M=_t(wl.M))
        opts = L.Options(k=48, precision="fp64")
        B = wl.n_t * wl.n_m
        al = torch.empty(B, 48, dtype=torch.float64, device=DEV)
        be = torch.empty_like(al)
        b0 = torch.empty(B, dtype=torch.float64, device=DEV)
        ke = torch.empty(B, dtype=torch.int32, device=DEV)
        L.lgw_lanczos_coeffs(h, s, prob, opts, al, be, b0, ke)

        def out():
            return (torch.empty(wl.n_t, wl.omega.size, 2, dtype=torch.float64, device=DEV),
                    torch.empty(wl.n_t, dtype=torch.float64, device=DEV),
                    torch.empty(wl.n_t, dtype=torch.float64, device=DEV))

        ref = out()
        L.lgw_sigma_from_coeffs(h, s, prob, opts, al, be, b0, ke, *ref)
        torch.cuda.synchronize()
        ref = [x.cpu().numpy() for x in ref]
        for _ in range(2):   # two calls in a row share and overwrite the scratch
            got = out()
            L.lgw_sigma_from_coeffs_noalloc(h, s, prob, opts, al, be, b0, ke, *got)
            torch.cuda.synchronize()
            got = [x.cpu().numpy() for x in got]
            for g, r in zip(got, ref):
                assert np.abs(g - r).max() <= 1e-11 * max(1.0, np.abs(r).max())

        # beyond the static scratch: rejected with a clear error, nothing runs
        big_k = 48
        big = L.Problem(targets=_t(np.arange(wl.n_t, dtype=np.int32)),
                        m_idx=_t(np.zeros(40000, dtype=np.int32)), omega=_t(wl.omega),
                        delta=wl.delta, M=_t(wl.M))
        with pytest.raises(L.LgwError) as ei:
            L.lgw_sigma_from_coeffs_noalloc(h, s, big, L.Options(k=big_k, precision="fp64"),
                                            al, be, b0, ke, *out())
        assert ei.value.status == 8 and "static scratch" in str(ei.value)
        # host arrays are refused
        with pytest.raises(L.LgwError) as ei:
            L.lgw_sigma_from_coeffs_noalloc(h, s, prob, opts, al.cpu(), be, b0, ke, *out())
        assert ei.value.status == 1
        # an out-of-range summed orbital or target, or a depth beyond k, is
        # caught by the device-side index check, whose verdict is read back
        # before any kernel that would dereference the index is queued
        norb = wl.n_v + wl.n_c
        bad_m = wl.m_idx.copy()
        bad_m[3] = norb
        bad_t = wl.targets.copy()
        bad_t[0] = -1
        bad_k = ke.clone()
        bad_k[5] = 49
        cases = [
            (L.Problem(targets=_t(wl.targets), m_idx=_t(bad_m), omega=_t(wl.omega),
                       delta=wl.delta, M=_t(wl.M)), ke),
            (L.Problem(targets=_t(bad_t), m_idx=_t(wl.m_idx), omega=_t(wl.omega),
                       delta=wl.delta, M=_t(wl.M)), ke),
            (prob, bad_k),
        ]
        for bp, kk in cases:
            with pytest.raises(L.LgwError) as ei:
                L.lgw_sigma_from_coeffs_noalloc(h, s, bp, opts, al, be, b0, kk, *out())
            assert ei.value.status == 2
        # an unknown QP mode is refused before any launch (raw C struct: the
        # binding only maps the known mode names)
        import ctypes
        fn = L.load_library().lgw_sigma_from_coeffs_noalloc
        co, cp = opts.to_c(), prob.to_c()
        co.qp_mode = 7
        o3 = out()
        st = fn(h.ptr, s.ptr, ctypes.byref(cp), ctypes.byref(co), al.data_ptr(), be.data_ptr(),
                b0.data_ptr(), ke.data_ptr(), o3[0].data_ptr(), o3[1].data_ptr(),
                o3[2].data_ptr())
        assert st == 1
        # the handle stays usable after the refusals
        got = out()
        L.lgw_sigma_from_coeffs_noalloc(h, s, prob, opts, al, be, b0, ke, *got)
        torch.cuda.synchronize()
        for g, r in zip([x.cpu().numpy() for x in got], ref):
            assert np.abs(g - r).max() <= 1e-11 * max(1.0, np.abs(r).max())
        L.lgw_release_system(s)
    finally:
        L.lgw_destroy(h)
