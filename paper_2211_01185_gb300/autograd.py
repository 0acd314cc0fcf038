"""PyTorch autograd front end of the coupling step and its adjoint.

``coupling_step(ctx, x, r, u_p, u_nodal, p_nodal)`` runs one coupling step
(steps a1-a7: void fraction, its smoothed L2 projection, the particle forces
and the fluid source) through ``cfdem_coupling_step`` and returns
``(f, f_drag, eps_h, F_elem)`` as tensors that take part in autograd.  Their
backward pass is ``cfdem_adjoint``: given the incoming gradients of f, f_D and
eps_h it returns dJ/dx and dJ/du_nodal.  ``mass_norm(ctx, eps_h)`` is
||eps_h||_M = sqrt(eps_h^T M eps_h) with M the consistent mass matrix
(``cfdem_mass_apply``), whose gradient is M eps_h / ||eps_h||_M.

Marshalling only: every derivative is computed by the CUDA library.  The
library differentiates with respect to the particle positions and the nodal
fluid velocity; asking for gradients of r, u_p or p_nodal raises.  The
fluid source F_elem is returned without a gradient (the adjoint does not
differentiate it).  Each forward call starts the projection from zero, so
the forward result does not depend on earlier calls.
"""
from __future__ import annotations

import torch

from . import cfdem as cf


def _contig(t):
    return t.detach().contiguous()


class CouplingFn(torch.autograd.Function):
    """(x, u_nodal) -> (f, f_drag, eps_h, F_elem); see module docstring."""

    @staticmethod
    def forward(ctx, x, u_nodal, handle, r, u_p, p_nodal):
        st = cf.cfdem_get_stats(handle.h)
        n = x.shape[0]
        dev = x.device
        x_, u_ = _contig(x), _contig(u_nodal)
        r_, up_, p_ = _contig(r), _contig(u_p), _contig(p_nodal)
        eps = torch.zeros(st.n_nodes, dtype=torch.float64, device=dev)
        f = torch.empty((n, 3), dtype=torch.float64, device=dev)
        fd = torch.empty((n, 3), dtype=torch.float64, device=dev)
        Fe = torch.empty((st.n_elem, 3), dtype=torch.float64, device=dev)
        cf.cfdem_coupling_step(handle.h, n, x_, r_, up_, u_, p_, eps, f, fd, Fe)
        cf.cfdem_synchronize(handle.h)
        ctx.handle = handle
        ctx.set_materialize_grads(False)   # unused outputs reach backward as None
        ctx.save_for_backward(x_, u_, r_, up_, p_, eps)
        ctx.mark_non_differentiable(Fe)
        return f, fd, eps, Fe

    @staticmethod
    def backward(ctx, g_f, g_fd, g_eps, g_Fe):
        if any(ctx.needs_input_grad[3:]):
            raise RuntimeError("the coupling-step adjoint gives dJ/dx and dJ/du_nodal only "
                               "(r, u_p and p_nodal must not require grad)")
        x, u, r, up, p, eps = ctx.saved_tensors
        h = ctx.handle.h
        n = x.shape[0]
        dJdx = torch.zeros((n, 3), dtype=torch.float64, device=x.device)
        dJdu = torch.zeros_like(u) if ctx.needs_input_grad[1] else None
        cf.cfdem_adjoint(h, n, x, r, up, u, p, eps,
                         None if g_f is None else _contig(g_f),
                         None if g_fd is None else _contig(g_fd),
                         None if g_eps is None else _contig(g_eps), dJdx, dJdu)
        cf.cfdem_synchronize(h)
        return (dJdx if ctx.needs_input_grad[0] else None, dJdu, None, None, None, None)


class MassNormFn(torch.autograd.Function):
    """eps_h -> ||eps_h||_M = sqrt(eps_h^T M eps_h)."""

    @staticmethod
    def forward(ctx, eps, handle):
        e = _contig(eps)
        Me = torch.empty_like(e)
        cf.cfdem_mass_apply(handle.h, e, Me)
        cf.cfdem_synchronize(handle.h)
        norm = torch.sqrt(torch.dot(e, Me))
        ctx.save_for_backward(Me, norm)
        return norm

    @staticmethod
    def backward(ctx, g):
        Me, norm = ctx.saved_tensors
        return g * Me / norm, None


def coupling_step(handle, x, r, u_p, u_nodal, p_nodal):
    """One coupling step on the context ``handle`` (a ``cfdem.Context``);
    returns (f, f_drag, eps_h, F_elem), differentiable in x and u_nodal."""
    return CouplingFn.apply(x, u_nodal, handle, r, u_p, p_nodal)


def mass_norm(handle, eps_h):
    """||eps_h||_M on the context's mesh, differentiable in eps_h."""
    return MassNormFn.apply(eps_h, handle)
