"""torch.autograd binding of the pseudo-fermion actions.

The action of one pseudo-fermion term (Sec. 1 eq. (3): |W1^-1 phi|^2,
|R^-1 phi|^2, |W2^-1 phi|^2, |R2^-1 phi|^2 and the mass-preconditioned
S2 / S1) becomes a differentiable function of the Lie-algebra coordinates
omega of the links, S(omega) = S[exp(i omega^a T^a) U].  The forward pass
rotates the links and evaluates S through the C-ABI; the backward pass
calls the library's force kernel, which recomputes the solver solutions
instead of keeping them from the forward pass.  The gradient is the force
dS/domega^a at the rotated links, i.e. the exact gradient at omega = 0 (the
point where the molecular dynamics uses it) and the left-trivialised
derivative elsewhere.  Both passes leave the lattice handle holding the
caller's links U again (they install the rotated links only while they
evaluate).  Argument marshalling only: every step runs in the library's
kernels.
"""
import torch

from . import lqcd

_EO_TERMS = (lqcd.TERM_S2, lqcd.TERM_S1)


def _evaluate(lat, term, phi, kappa, rho, precision, tol, max_iter, force):
    if term in _EO_TERMS:
        return lat.pf_force_eo(phi, kappa, rho, term, precision, tol, max_iter, force)
    return lat.pf_force(phi, kappa, term, precision, tol, max_iter, force)


class PseudoFermionAction(torch.autograd.Function):
    """S = PseudoFermionAction.apply(omega, lat, U, phi, kappa, term,
    precision, tol, max_iter, rho); omega: float64 (4, V, 8) on the device."""

    @staticmethod
    def forward(ctx, omega, lat, U, phi, kappa, term, precision=lqcd.PREC_F64, tol=1e-12, max_iter=20000,
                rho=0.0):
        Uw = lat.link_update(U, omega.detach().contiguous(), 1.0)
        S, _ = _evaluate(lat, term, phi, kappa, rho, precision, tol, max_iter, False)
        lat.set_gauge(U)
        ctx.lat, ctx.U, ctx.Uw, ctx.phi = lat, U, Uw, phi
        ctx.args = (kappa, term, precision, tol, max_iter, rho)
        return torch.tensor(S, dtype=torch.float64, device=omega.device)

    @staticmethod
    def backward(ctx, grad_out):
        kappa, term, precision, tol, max_iter, rho = ctx.args
        ctx.lat.set_gauge(ctx.Uw)
        _, F = _evaluate(ctx.lat, term, ctx.phi, kappa, rho, precision, tol, max_iter, True)
        ctx.lat.set_gauge(ctx.U)
        return (grad_out * F,) + (None,) * 9


def pseudofermion_action(omega, lat, U, phi, kappa, term, precision=lqcd.PREC_F64, tol=1e-12, max_iter=20000,
                         rho=0.0):
    return PseudoFermionAction.apply(omega, lat, U, phi, kappa, term, precision, tol, max_iter, rho)
