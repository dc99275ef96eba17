"""Phase-field sub-problem: Fourier collocation and BCCG (Sec. 3.1.2, Algorithm 1).  Test infrastructure only.

Readings of the paper used here (each a place where the printed text is
inconsistent with itself; the chosen reading is the one that reproduces the
paper's own closed forms, Eqs. AT1_analytical / AT2_analytical and the G_c
normalisation of Eq. Ff):
  * AT2 local energy f(phi) = phi^2 with c_w = 2 (Eq. fracturelocal prints
    phi^2/2, whose optimal profile would be exp(-|x|/(sqrt(2) ell)) and whose
    crack energy would not be G_c).  AT1: f = phi, c_w = 8/3.
  * F_phi is the exact variation of Eq. functional:
      F_phi = h'(phi) psi_0^+ + (G_c/(c_w ell)) (f'(phi) - 2 ell^2 nabla^2 phi)
    (Eq. F_phi prints ell^2, which would give the AT1 profile a support of
    sqrt(2) ell instead of 2 ell).
  * J = eta/dt + h'' psi_0^+ + (G_c/(c_w ell)) (f'' - 2 ell^2 nabla^2_N), with
    h'' = 2, f'' = 0 (AT1) or 2 (AT2) -- the linearisation of the above, which
    is exact because F_phi is affine in phi for these f and h.
  * Irreversibility bound on the update v = phi_new - phi_old (text after the
    Jacobian): phi_new >= phi_con(phi_old) gives v >= v_con with
    v_con = phi_con(phi_old) - phi_old (the printed difference has its operands
    swapped, which would demand phi_new >= 2 phi_old - phi_con).
  * Crack set: phi_con = phi where phi >= 0.9 (the inequality of Eq.
    constraint_field), else 0.
  * Algorithm 1: alpha = -(r.p)/(p.Jp) (the printed ratio has the wrong sign for
    r = Jv - b and p = -r); beta as printed, r^m.(r^m - r^{m-1}) / (alpha p.Jp);
    loop while ||r|| exceeds the tolerance; initial v^0 = 0 (the algorithm's
    "e.g." choice v^0 = b is dimensionally a force); points count as bound when
    v = v_con holds exactly after the clamp.
"""
import numpy as np

from .fourier import laplacian
from .params import AT1, CRACK_SET


def f_local(phi, par):
    """f(phi) of Eq. fracturelocal (AT2 read as phi^2)."""
    return phi if par.fracture == AT1 else phi ** 2


def df_local(phi, par):
    return np.ones_like(phi) if par.fracture == AT1 else 2.0 * phi


def d2f_local(par):
    return 0.0 if par.fracture == AT1 else 2.0


def phi_con(phi, par):
    """Constraining field of Eq. constraint_field."""
    if par.irreversibility == CRACK_SET:
        return np.where(phi >= par.crack_set_threshold, phi, 0.0)
    return phi.copy()


def resistance(phi, lap_phi, par):
    """R_f = -(G_c/(c_w ell)) (f'(phi) - 2 ell^2 nabla^2 phi): the fracture part of -F_phi."""
    return -par.c() * (df_local(phi, par) - 2.0 * par.ell ** 2 * lap_phi)


def driving(phi, psi):
    """Crack driving force -h'(phi) psi_0^+ = 2 (1 - phi) psi_0^+."""
    return 2.0 * (1.0 - phi) * psi


def minus_F_phi(phi, psi, par, lap_phi=None):
    """-F_phi (Eq. F_phi with the reading above)."""
    if lap_phi is None:
        lap_phi = laplacian(phi, par.dx)
    return driving(phi, psi) + resistance(phi, lap_phi, par)


def J_apply(v, psi, par):
    """Jacobian of Eq. phase_field_euler applied to v (Sec. 3.1.2)."""
    diag = par.eta_dt() + 2.0 * psi + par.c() * d2f_local(par)
    return diag * v - 2.0 * par.c() * par.ell ** 2 * laplacian(v, par.dx)


def bccg(apply_J, b, vcon, rtol, atol, max_iter):
    """Bound-constrained CG, Algorithm 1, with the readings of the module docstring.

    Returns (v, info); info has the iteration count, final ||r||, and the
    boolean active set (v = v_con and r > 0 before masking) of the last iterate.
    """
    v = np.zeros_like(b)
    v = np.where(v < vcon, vcon, v)
    r = apply_J(v) - b
    active = (v == vcon) & (r > 0)
    r[active] = 0.0
    p = -r
    tol = max(rtol * np.sqrt(np.sum(r * r)), atol)
    it = 0
    while np.sqrt(np.sum(r * r)) > tol and it < max_iter:
        Jp = apply_J(p)
        pJp = float(np.sum(p * Jp))
        if pJp <= 0.0:
            break
        alpha = -float(np.sum(r * p)) / pJp
        v = v + alpha * p
        v = np.where(v < vcon, vcon, v)
        r_old = r
        r = apply_J(v) - b
        active = (v == vcon) & (r > 0)
        r[active] = 0.0
        beta = float(np.sum(r * (r - r_old))) / (alpha * pJp)
        p = -r + beta * p
        p[active] = 0.0
        it += 1
    return v, {"iters": it, "res": float(np.sqrt(np.sum(r * r))), "active": active, "tol": tol}


def solve(phi, psi, par, lap_phi=None, constraint=None, eta_dt=None):
    """One phase-field sub-problem from phi_n with fixed psi_0^+ (Algorithm 1 on Eq. phase_field_update).

    constraint: the constraining field phi_con (default phi_con(phi_n)); eta_dt:
    eta/dt of Eq. phase_field_euler (default par.eta_dt()).  Returns (phi_new, v, info).
    """
    if lap_phi is None:
        lap_phi = laplacian(phi, par.dx)
    if eta_dt is not None:
        par = _with_eta_dt(par, eta_dt)
    b = minus_F_phi(phi, psi, par, lap_phi)
    pc = phi_con(phi, par) if constraint is None else constraint
    vcon = pc - phi
    v, info = bccg(lambda x: J_apply(x, psi, par), b, vcon, par.pf_tol, par.pf_atol, par.pf_max_iter)
    return phi + v, v, info


def _with_eta_dt(par, eta_dt):
    import dataclasses
    return dataclasses.replace(par, eta_over_dt=eta_dt)
