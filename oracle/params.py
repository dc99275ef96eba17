"""Model parameters of the oracle (Sec. 3.3 "Non-Dimensionalization and Simulation
Parameters").  Test infrastructure only.

Defaults follow the paper's Sec. 3.3 values where it gives them: sub-solver
tolerances 1e-6, (dphi)_min = 1e-3, (-F_phi)_max = 0.7 G_c/ell,
(-h psi_0^+)_thresh = 1 G_c/ell, near-equilibrium time step (Delta t)_max =
2^16 eta/(G_c/ell) so that eta/Delta t = 2^-16 G_c/ell.
"""
from dataclasses import dataclass, field

AT1, AT2 = 1, 2                      # Eq. fracturelocal
ISOTROPIC, SPECTRAL, SPECTRAL_STRESSFREE, VOLDEV, SPECTRAL_VOLDEV = 0, 1, 2, 3, 4
# Eqs. isotropic_en, strain_spectral_en, vol_dev_en; the non-variational pairings of
# Sec. 4.2 (strain-spectral driving force with the stress-free / vol.-dev. contact model)
CRACK_SET, DAMAGE = 0, 1             # Eq. constraint_field


@dataclass
class Params:
    nu: float = 0.2
    Gc: float = 1.0
    ell: float = 2.0
    dx: float = 1.0
    fracture: int = AT1
    split: int = SPECTRAL
    irreversibility: int = CRACK_SET
    crack_set_threshold: float = 0.9          # Eq. constraint_field (phi >= 0.9)
    # mechanics sub-problem (Sec. 3.1.1)
    mech_tol: float = 1e-6                    # Newton stop: ||P sigma|| <= mech_tol * ||C0:eps_bar||
    mech_cg_rtol: float = 1e-4                # inner CG relative tolerance for nonlinear splits
    mech_max_newton: int = 50
    mech_max_cg: int = 5000
    # phase-field sub-problem (Sec. 3.1.2)
    pf_tol: float = 1e-6                      # BCCG stop: ||r|| <= max(pf_tol*||r0||, pf_atol)
    pf_atol: float = 1e-12
    pf_max_iter: int = 20000
    eta_over_dt: float | None = None          # default 2^-16 G_c/ell (Algorithm 4 uses (Delta t)_max)
    # near-equilibrium evolution (Algorithm 4)
    F_max: float | None = None                # default 0.7 G_c/ell
    thresh: float | None = None               # default 1.0 G_c/ell
    dphi_min: float = 1e-3
    d_eps_bar: tuple = field(default_factory=lambda: ((0.0, 0.0), (0.0, 1e-4)))
    C_broken: float | None = None             # default 0.01 * mean(E)

    def eta_dt(self):
        return self.eta_over_dt if self.eta_over_dt is not None else 2.0 ** -16 * self.Gc / self.ell

    def fmax(self):
        return self.F_max if self.F_max is not None else 0.7 * self.Gc / self.ell

    def thr(self):
        return self.thresh if self.thresh is not None else 1.0 * self.Gc / self.ell

    def cw(self):
        """c_w of Eq. fracturelocal."""
        return 8.0 / 3.0 if self.fracture == AT1 else 2.0

    def c(self):
        """Prefactor G_c/(c_w ell) of Eq. Ff."""
        return self.Gc / (self.cw() * self.ell)
