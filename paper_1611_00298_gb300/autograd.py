"""torch.autograd wrapper of the EOFA action and its adjoint force kernel.

S_f(U) = phi^+ M_EOFA(U) phi (Eq. (5)) as a function of the gauge links.
Forward runs the two solves of Eq. (5) / (7) in libeofa and keeps chi_L and
chi_R; backward calls the adjoint kernel (eofa_grad_from_chi_dev), which
rebuilds the spin projections of chi at every link instead of storing them
and returns dS/dRe U and dS/dIm U.  No derivative is taken by torch itself.

The links enter as a real float64 CUDA tensor of shape (T, Z, Y, X, 4, 3, 3, 2)
(the real view of the canonical complex layout); they must be SU(3)
(libeofa checks unitarity on load).
"""
from __future__ import annotations

import torch

from . import eofa as _eofa


class EOFAAction(torch.autograd.Function):
    """S = EOFAAction.apply(U_real, phi, lattice, alpha, M5, m1, m2, precision, tol)."""

    @staticmethod
    def forward(ctx, U_real, phi, lattice, alpha, M5, m1, m2, precision=_eofa.PREC_F64, tol=1e-12):
        assert U_real.is_cuda and U_real.dtype == torch.float64 and U_real.shape[-1] == 2
        lattice.gauge_load_dev(U_real.contiguous())
        chiL = torch.empty(lattice.shape5, dtype=torch.complex128, device=U_real.device)
        chiR = torch.empty_like(chiL)
        S, info = lattice.pseudofermion_solutions_dev(phi, chiL, chiR, alpha, M5, m1, m2, precision, tol)
        k, _, _ = _eofa.coefficients(lattice.Ls, alpha, m1, m2)
        ctx.save_for_backward(chiL, chiR)
        ctx.lattice = lattice
        ctx.k = k
        ctx.shape = U_real.shape
        return torch.tensor(S, dtype=torch.float64, device=U_real.device)

    @staticmethod
    def backward(ctx, grad_S):
        chiL, chiR = ctx.saved_tensors
        G = torch.empty(ctx.lattice.shapeU, dtype=torch.complex128, device=chiL.device)
        ctx.lattice.grad_from_chi_dev(ctx.k, chiL, chiR, G)
        g = torch.view_as_real(G).reshape(ctx.shape) * grad_S
        return g, None, None, None, None, None, None, None, None


def eofa_action(U_real, phi, lattice, alpha, M5, m1, m2, precision=_eofa.PREC_F64, tol=1e-12):
    """Differentiable EOFA action (see EOFAAction)."""
    return EOFAAction.apply(U_real, phi, lattice, alpha, M5, m1, m2, precision, tol)
