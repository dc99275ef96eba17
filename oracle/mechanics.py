"""Mechanics sub-problem: Fourier-Galerkin strain solver (Sec. 3.1.1).  Test infrastructure only.

Unknown: the zero-mean, compatible polarisation strain eps* (eps = eps_bar + eps*).
Nodal equilibrium (Eq. elasticity_nodal): G-hat : sigma-hat = 0 at every mode,
i.e. R(eps*) := P sigma(eps_bar + eps*) = 0 with P = F^-1 Gamma F.

Newton (Eq. mech_newton): eps*_{m+1} = eps*_m + theta_m with theta_m from CG on
Eq. elasticity_newton_linear, read with the sign restored:
P C_m theta = -P sigma_m.  Starting CG from theta = 0, every iterate stays in
range(P), where P C_m is symmetric in the Frobenius inner product.

Stopping (Sec. 3.1.1 text; reading of the unspecified norms): ell_2 norms over
the grid of the Frobenius norm; Newton stops when ||R|| <= mech_tol * ||C_0:eps_bar||
(C_0: undamaged stiffness of the pixel).  Linear (isotropic-stress) models take a
single Newton step whose CG is solved to that same absolute target.  Nonlinear
splits solve each Newton update with CG to max(target, mech_cg_rtol * ||R_m||).
"""
import numpy as np

from . import constitutive as cm
from .fourier import project


def inner(a, b):
    """Frobenius inner product summed over the grid."""
    return float(np.sum(a * b))


def residual(eps_star, eps_bar, phi, E, par):
    """R = P sigma(eps_bar + eps*, phi) (Eq. elasticity_nodal)."""
    lam, mu = cm.lame(E, par.nu)
    sig = cm.stress(eps_bar[None, None] + eps_star, phi, lam, mu, par.split)
    return project(sig, par.dx)


def reference_norm(eps_bar, E, par):
    """||C_0(E(x)) : eps_bar|| over the grid (scale of the stopping tests)."""
    lam, mu = cm.lame(E, par.nu)
    tr = eps_bar[0, 0] + eps_bar[1, 1]
    s = 2.0 * mu[..., None, None] * eps_bar[None, None] + (lam * tr)[..., None, None] * np.eye(2)
    return np.sqrt(np.sum(s * s))


def cg(apply_A, b, target, max_iter):
    """Plain conjugate gradients for A x = b from x = 0; stops when ||r|| <= target."""
    x = np.zeros_like(b)
    r = b.copy()
    p = r.copy()
    rr = inner(r, r)
    it = 0
    while np.sqrt(rr) > target and it < max_iter:
        Ap = apply_A(p)
        pAp = inner(p, Ap)
        if pAp <= 0.0:
            break
        alpha = rr / pAp
        x += alpha * p
        r -= alpha * Ap
        rr_new = inner(r, r)
        p = r + (rr_new / rr) * p
        rr = rr_new
        it += 1
    return x, it, np.sqrt(rr)


def solve(eps_star, eps_bar, phi, E, par):
    """Newton-CG solve of the mechanics sub-problem; returns (eps_star, info)."""
    eps_star = eps_star.copy()
    lam, mu = cm.lame(E, par.nu)
    target = par.mech_tol * reference_norm(eps_bar, E, par)
    linear = cm.is_linear(par.split)
    info = {"newton": 0, "cg": 0, "res": None}
    for m in range(par.mech_max_newton):
        eps = eps_bar[None, None] + eps_star
        sig = cm.stress(eps, phi, lam, mu, par.split)
        R = project(sig, par.dx)
        rn = np.sqrt(inner(R, R))
        info["res"] = rn
        if rn <= target:
            break
        tang = cm.Tangent(eps, phi, lam, mu, par.split)

        def apply_A(p):
            return project(tang(p), par.dx)

        cg_target = target if linear else max(target, par.mech_cg_rtol * rn)
        theta, it, _ = cg(apply_A, -R, cg_target, par.mech_max_cg)
        eps_star += theta
        info["newton"] += 1
        info["cg"] += it
        if linear:
            break
    return eps_star, info
