"""Near-equilibrium evolution (Sec. 3.2.3, Algorithm 4), energies and step reports.  Test infrastructure only.

One call of ``load_step`` is one pass of the while-loop of Algorithm 4:
mechanics solve, rescale test, phase-field solve, stiffness, strain increment.

Readings of Algorithm 4 used here:
  * The trigger of its first "if" and the denominator of gamma use the crack
    driving force D = -h'(phi) psi_0^+ = 2(1-phi) psi_0^+ (the algorithm prints
    -h psi_0^+, which is never positive, and h' psi_0^+ without the minus sign;
    the accompanying text names -h' psi_0^+).
  * gamma^2 D(x*) + R_f(x*) = (-F_phi)_max with R_f = -F_phi - D, i.e.
    gamma = sqrt(((-F_phi)_max - R_f(x*)) / D(x*)); the rescale is skipped when
    the numerator or the denominator is not positive.  Flag stays set once set.
  * x* = first maximiser in row-major (y, x) order.
  * The whole strain eps = eps_bar + eps* is scaled, i.e. both eps_bar and eps*.
  * C-bar = sigma-bar_ij / eps-bar_ij at the component (i, j) where |eps-bar| is
    largest (Sec. 3.2.1 text: ratio of the largest components).
  * ||phi_{n+1} - phi_n||_1 (Sec. 3.2.1) is measured with lengths in units of
    ell (Sec. 3.3 scales lengths by ell): (dx/ell)^2 sum |delta phi|.
  * The increment test compares with (dphi)_min and adds Delta eps_bar to the
    (possibly rescaled) eps_bar_n.
"""
from dataclasses import dataclass, field

import numpy as np

from . import constitutive as cm
from . import mechanics, phasefield
from .fourier import laplacian


@dataclass
class State:
    E: np.ndarray
    phi: np.ndarray
    eps_star: np.ndarray
    eps_bar: np.ndarray
    flag: bool = False
    n: int = 0
    history: list = field(default_factory=list)

    @staticmethod
    def initial(E, phi0=None):
        ny, nx = E.shape
        phi = np.zeros((ny, nx)) if phi0 is None else np.array(phi0, dtype=float)
        return State(E=np.array(E, dtype=float), phi=phi,
                     eps_star=np.zeros((ny, nx, 2, 2)), eps_bar=np.zeros((2, 2)))


def energies(eps, phi, E, par, lap_phi=None):
    """(F_e, F_f): Eq. Fe with the contact-model density, and Eq. Ff written with
    sum |grad phi|^2 = -sum phi nabla^2_N phi (Parseval on the trigonometric interpolant)."""
    lam, mu = cm.lame(E, par.nu)
    dA = par.dx ** 2
    Fe = float(np.sum(cm.energy_density(eps, phi, lam, mu, par.split))) * dA
    if lap_phi is None:
        lap_phi = laplacian(phi, par.dx)
    Ff = par.c() * float(np.sum(phasefield.f_local(phi, par) - par.ell ** 2 * phi * lap_phi)) * dA
    return Fe, Ff


def stiffness(eps_bar, sig_bar):
    """C-bar: ratio of sigma-bar and eps-bar at the largest |eps-bar| component."""
    i, j = np.unravel_index(np.argmax(np.abs(eps_bar)), (2, 2))
    if eps_bar[i, j] == 0.0:
        return np.inf
    return float(sig_bar[i, j] / eps_bar[i, j])


def rescale_factor(phi, psi, eps_bar, par, flag, lap_phi):
    """Lines 4-10 of Algorithm 4; returns (gamma, flag, diagnostics)."""
    D = phasefield.driving(phi, psi)
    Rf = phasefield.resistance(phi, lap_phi, par)
    mF = D + Rf
    istar = int(np.argmax(mF))
    mF_max = float(mF.flat[istar])
    if mF_max > par.fmax() and float(D.max()) > par.thr():
        flag = True
    gamma = 1.0
    if mF_max > par.fmax() and flag:
        num = par.fmax() - float(Rf.flat[istar])
        den = float(D.flat[istar])
        if num > 0.0 and den > 0.0:
            gamma = np.sqrt(num / den)
            d_eps = np.asarray(par.d_eps_bar, dtype=float)
            emax = np.abs(eps_bar).max()
            if emax > 0.0:
                gamma = min(gamma, 1.0 + np.abs(d_eps).max() / emax)
    return gamma, flag, {"mF_max": mF_max, "istar": istar, "D_max": float(D.max())}


def load_step(st, par, compute_energies=True):
    """One iteration of Algorithm 4 on state ``st`` (modified in place); returns a report dict."""
    lam, mu = cm.lame(st.E, par.nu)
    # line 3: elasticity sub-problem at eps_bar_n, phi_n
    st.eps_star, minfo = mechanics.solve(st.eps_star, st.eps_bar, st.phi, st.E, par)
    # lines 4-10: rescale
    eps = st.eps_bar[None, None] + st.eps_star
    psi = cm.psi_plus(eps, lam, mu, par.split)
    lap_phi = laplacian(st.phi, par.dx)
    gamma, st.flag, rinfo = rescale_factor(st.phi, psi, st.eps_bar, par, st.flag, lap_phi)
    if gamma != 1.0:
        st.eps_star = gamma * st.eps_star
        st.eps_bar = gamma * st.eps_bar
        eps = st.eps_bar[None, None] + st.eps_star
        psi = cm.psi_plus(eps, lam, mu, par.split)
    # line 11: phase-field sub-problem with phi_con(phi_n) and dt = (dt)_max
    phi_new, v, pinfo = phasefield.solve(st.phi, psi, par, lap_phi)
    # line 12: stiffness from eps_n and phi_{n+1}
    sig = cm.stress(eps, phi_new, lam, mu, par.split)
    sig_bar = sig.mean(axis=(0, 1))
    eps_bar_n = st.eps_bar.copy()
    C_bar = stiffness(eps_bar_n, sig_bar)
    dphi = (par.dx / par.ell) ** 2 * float(np.sum(np.abs(v)))
    incremented = dphi < par.dphi_min
    st.phi = phi_new
    if incremented:
        st.eps_bar = st.eps_bar + np.asarray(par.d_eps_bar, dtype=float)
    C_broken = par.C_broken if par.C_broken is not None else 0.01 * float(st.E.mean())
    rep = {"n": st.n, "eps_bar": eps_bar_n, "sig_bar": sig_bar, "C_bar": C_bar, "gamma": gamma,
           "rescaled": gamma != 1.0, "incremented": incremented, "dphi_L1": dphi,
           "newton": minfo["newton"], "mech_cg": minfo["cg"], "bccg": pinfo["iters"],
           "n_active": int(np.sum(pinfo["active"])), "active": pinfo["active"],
           "broken": C_bar < C_broken, **rinfo}
    if compute_energies:
        rep["F_e"], rep["F_f"] = energies(eps, phi_new, st.E, par)
    st.n += 1
    st.history.append({k: v for k, v in rep.items() if k != "active"})
    return rep


def run(E, par, max_steps=5000, phi0=None, max_increments=None, stop_when_broken=True):
    """Algorithm 4 until C-bar < C_broken (or a step / increment cap); returns (state, reports)."""
    st = State.initial(E, phi0)
    reps = []
    n_inc = 0
    for _ in range(max_steps):
        rep = load_step(st, par)
        reps.append(rep)
        n_inc += int(rep["incremented"])
        if stop_when_broken and rep["broken"]:
            break
        if max_increments is not None and n_inc >= max_increments:
            break
    return st, reps


# ---------------------------------------------------------------------------
# Alternating minimisation (Sec. 3.2.1, Algorithm 2) and time-dependent evolution
# (Sec. 3.2.2, Algorithm 3).  Readings: eta/dt = 0 in the alternating
# minimisation's phase-field solves (as the algorithm states); the increment's
# constraint field phi_con(phi_{s,0}) stays fixed over its inner loop; the inner
# loop ends when ||phi_{s,n+1} - phi_{s,n}||_1 < Tol_AM (the printed "> Tol" is the
# continuation test); time steps are in units of t~ = eta/(G_c/ell), so
# eta/dt = (G_c/ell) / dt; the doubling of dt is capped at (dt)_max.


def am_increment(st, par, tol_am=1e-3, max_inner=1000):
    """One strain increment s of Algorithm 2 on state ``st``; returns a report."""
    lam, mu = cm.lame(st.E, par.nu)
    st.eps_bar = st.eps_bar + np.asarray(par.d_eps_bar, dtype=float)
    con = phasefield.phi_con(st.phi, par)            # phi_con(phi_{s,0})
    inner = 0
    mech_cg = bccg = 0
    while True:
        st.eps_star, minfo = mechanics.solve(st.eps_star, st.eps_bar, st.phi, st.E, par)
        eps = st.eps_bar[None, None] + st.eps_star
        psi = cm.psi_plus(eps, lam, mu, par.split)
        phi_new, v, pinfo = phasefield.solve(st.phi, psi, par, constraint=con, eta_dt=0.0)
        dphi = (par.dx / par.ell) ** 2 * float(np.sum(np.abs(v)))
        st.phi = phi_new
        inner += 1
        mech_cg += minfo["cg"]
        bccg += pinfo["iters"]
        if dphi < tol_am or inner >= max_inner:
            break
    sig = cm.stress(eps, st.phi, lam, mu, par.split)
    sig_bar = sig.mean(axis=(0, 1))
    C_bar = stiffness(st.eps_bar, sig_bar)
    C_broken = par.C_broken if par.C_broken is not None else 0.01 * float(st.E.mean())
    st.n += 1
    return {"eps_bar": st.eps_bar.copy(), "sig_bar": sig_bar, "C_bar": C_bar, "inner": inner, "dphi_L1": dphi,
            "mech_cg": mech_cg, "bccg": bccg, "broken": C_bar < C_broken}


def td_step(st, par, dt, dt_min=2.0 ** -16, dt_max=2.0 ** 16, dphi_max=1.5):
    """One time step n of Algorithm 3 on ``st`` with current step ``dt`` (units of
    t~); returns (report, dt for the next step)."""
    lam, mu = cm.lame(st.E, par.nu)
    st.eps_star, minfo = mechanics.solve(st.eps_star, st.eps_bar, st.phi, st.E, par)
    eps = st.eps_bar[None, None] + st.eps_star
    psi = cm.psi_plus(eps, lam, mu, par.split)
    lap_phi = laplacian(st.phi, par.dx)
    tries = 0
    while True:
        eta_dt = (par.Gc / par.ell) / dt
        phi_new, v, pinfo = phasefield.solve(st.phi, psi, par, lap_phi, eta_dt=eta_dt)
        dphi = (par.dx / par.ell) ** 2 * float(np.sum(np.abs(v)))
        tries += 1
        if dphi < dphi_max or dt <= dt_min:
            if dphi < dphi_max / 2:
                dt = min(2.0 * dt, dt_max)
            break
        dt = dt / 2.0
    st.phi = phi_new
    eps_bar_n = st.eps_bar.copy()
    incremented = dphi < par.dphi_min and dt >= dt_max
    if incremented:
        st.eps_bar = st.eps_bar + np.asarray(par.d_eps_bar, dtype=float)
    sig_bar = cm.stress(eps, st.phi, lam, mu, par.split).mean(axis=(0, 1))
    C_bar = stiffness(eps_bar_n, sig_bar)
    C_broken = par.C_broken if par.C_broken is not None else 0.01 * float(st.E.mean())
    st.n += 1
    return ({"eps_bar": eps_bar_n, "sig_bar": sig_bar, "C_bar": C_bar, "dt": dt, "tries": tries, "dphi_L1": dphi,
             "incremented": incremented, "mech_cg": minfo["cg"], "bccg": pinfo["iters"], "broken": C_bar < C_broken},
            dt)
