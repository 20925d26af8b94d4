"""torch.autograd.Function over the QP energies of the C library.

Forward: ``lgw_sigma_c`` (E_t for the targets of a request), or
``lgw_sigma_c_tda`` with ``tda=True``.  Backward: ``lgw_sigma_c_backward``
(``lgw_sigma_c_tda_backward``), the hand-written adjoint (implicit function
for the QP equation; the exact reverse mode of the three-term recurrence
for FP64 runs without reorthogonalisation, else the Daleckii-Krein
derivative of f(C) in the Krylov basis; Eq. 7-14), giving dE/dL and
dE/deps.  Gradients flow to L and eps; the
coupling factors M are treated as constants.  Both passes run in the CUDA
library on the handle's stream; this module only allocates outputs.
"""
from __future__ import annotations

import torch

from . import lgw as _lgw


class QPEnergies(torch.autograd.Function):
    """E = QPEnergies.apply(L, eps, n_v, n_c, problem, options, handle, kernel_factor, tda).

    L [n_v*n_c, n_aux] and eps [n_v+n_c] are float64 CUDA tensors; problem is
    an :class:`lgw.Problem` with M (not V) when dL should include the
    coupling-vector path V = L M; options an :class:`lgw.Options`."""

    @staticmethod
    def forward(ctx, L, eps, n_v, n_c, problem, options, handle, kernel_factor=4.0, tda=False):
        L = L.detach().contiguous()
        eps = eps.detach().contiguous()
        s = _lgw.lgw_prepare_system(handle, n_v, n_c, L.shape[1], eps, L, kernel_factor)
        try:
            n_t = _lgw._numel(problem.targets)
            n_f = _lgw._numel(problem.omega)
            sig = torch.empty(n_t, n_f, 2, dtype=torch.float64, device=L.device)
            e = torch.empty(n_t, dtype=torch.float64, device=L.device)
            (_lgw.lgw_sigma_c_tda if tda else _lgw.lgw_sigma_c)(handle, s, problem, options,
                                                                 sig, e)
        finally:
            _lgw.lgw_release_system(s)
        ctx.save_for_backward(L, eps)
        ctx.meta = (n_v, n_c, problem, options, handle, kernel_factor, tda)
        return e

    @staticmethod
    def backward(ctx, gE):
        L, eps = ctx.saved_tensors
        n_v, n_c, problem, options, handle, kernel_factor, tda = ctx.meta
        dL = torch.empty_like(L) if ctx.needs_input_grad[0] else None
        deps = torch.empty_like(eps) if ctx.needs_input_grad[1] else None
        if dL is None and deps is None:
            return (None,) * 9
        s = _lgw.lgw_prepare_system(handle, n_v, n_c, L.shape[1], eps, L, kernel_factor)
        try:
            bw = _lgw.lgw_sigma_c_tda_backward if tda else _lgw.lgw_sigma_c_backward
            bw(handle, s, problem, options, gE.detach().to(torch.float64).contiguous(), dL, deps)
        finally:
            _lgw.lgw_release_system(s)
        return dL, deps, None, None, None, None, None, None, None


def qp_energies(L, eps, n_v, n_c, problem, options, handle, kernel_factor=4.0, tda=False):
    """Differentiable QP energies E_t (see :class:`QPEnergies`)."""
    return QPEnergies.apply(L, eps, n_v, n_c, problem, options, handle, kernel_factor, tda)
