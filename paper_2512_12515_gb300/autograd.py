"""torch.autograd wrapper: (L, eps) -> lowest two-electron addition energies.

Forward runs pprpa_solve on the device; backward contracts the incoming
gradient with the Hellmann-Feynman derivatives of the roots in one
pprpa_grad_sum call (Sec. "Analytic Gradient": d omega = z^T (dM) z for
z^T W z = 1), computed in FP64 by the library.  Both directions stay in the
CUDA library; this class only moves tensors across the C ABI.
"""
from __future__ import annotations

import numpy as np
import torch

from ._lib import DEVICE, METHOD_DAVIDSON, PREC_FP64, Context


class PPRPARoots(torch.autograd.Function):
    """omega = PPRPARoots.apply(L, eps, nocc, mult, nroots, method, precision, conv_tol).

    L: (naux, n, n) float64 CUDA tensor of active-space fitted integrals
    (occupied orbitals first), eps: (n,) float64 orbital energies (any
    device), nocc: number of occupied orbitals among the n.
    Returns omega (nroots,) on L's device.  The library context holding the
    solve's eigenvectors lives as long as the autograd graph, so backward
    may run more than once (retain_graph=True).
    """

    @staticmethod
    def forward(ctx, L, eps, nocc, mult=1, nroots=5, method=METHOD_DAVIDSON,
                precision=PREC_FP64, conv_tol=1e-7):
        if not (L.is_cuda and L.dtype == torch.float64):
            raise TypeError("L must be a float64 CUDA tensor")
        n = L.shape[1]
        e = eps.detach().to("cpu", torch.float64).numpy()
        occ = np.concatenate([np.ones(nocc), np.zeros(n - nocc)])
        c = Context(L.device.index or 0)
        c.set_orbitals(occ, e)
        c.set_mo(L.detach().contiguous())
        res = c.solve(mult=mult, nroots=nroots, method=method, precision=precision,
                      conv_tol=conv_tol)
        ctx.pprpa = c  # closed when the graph (and this ctx) is freed
        ctx.shape = L.shape
        ctx.eps_device = eps.device
        return torch.as_tensor(res["omega"], dtype=torch.float64, device=L.device)

    @staticmethod
    def backward(ctx, g):
        naux, n, _ = ctx.shape
        dL = torch.empty(ctx.shape, dtype=torch.float64, device=g.device)
        de = torch.empty(n, dtype=torch.float64, device=g.device)
        ctx.pprpa.grad_sum(g.detach().to("cpu", torch.float64).numpy(), dL, de)
        return dL, de.to(ctx.eps_device), None, None, None, None, None, None


__all__ = ["PPRPARoots", "DEVICE"]
