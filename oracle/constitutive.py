"""Pointwise constitutive model (Sec. 2.1).  Test infrastructure only.

Strains and stresses are full symmetric 2x2 tensors on the last two axes.

Readings of the paper used here:
  * Lame parameters (text after Eq. isotropic_en): mu = E/(2+2nu),
    lambda = E nu/(1-nu-2nu^2), applied to the in-plane 2x2 strain (plane strain:
    these are the 3-D Lame constants, and Sec. 3.3 quotes (lambda+2mu) = 10/9 E_0
    at nu = 0.2, which only plane strain gives).
  * Degradation h(phi) = (1-phi)^2 with no residual stiffness (Eq. isotropic_en).
  * Ramp functions <x>_+ / <x>_- of Eq. strain_spectral_en; their derivatives use
    H(x) = 1 for x > 0 and 0 otherwise for the + branch, 1 - H for the - branch.
  * Volumetric-deviatoric split: Eq. vol_dev_en taken literally with the sums over
    the d = 2 in-plane components and the 1/3 of the 3-D deviator (this is the form
    whose value 2 mu (a^2 + ab + 5b^2/18) the paper quotes in Sec. 4.2.1); its stress
    is the exact gradient of that energy.
  * Non-variational pairings (Sec. 2.1, Sec. 4.2): "strain-spectral/stress-free"
    (driving force psi_0^+ from the spectral split, stress from the isotropic model)
    and "strain-spectral/vol.-dev." (stress from the volumetric-deviatoric model).
"""
import numpy as np

from .params import ISOTROPIC, SPECTRAL, SPECTRAL_STRESSFREE, SPECTRAL_VOLDEV, VOLDEV


def lame(E, nu):
    """(lambda, mu) from Young's modulus and Poisson ratio (text after Eq. isotropic_en)."""
    lam = E * nu / (1.0 - nu - 2.0 * nu * nu)
    mu = E / (2.0 + 2.0 * nu)
    return lam, mu


def h(phi):
    """Degradation h(phi) = (1-phi)^2 (Eq. isotropic_en)."""
    return (1.0 - phi) ** 2


def dh(phi):
    """h'(phi) = -2(1-phi)."""
    return -2.0 * (1.0 - phi)


def trace(t):
    return t[..., 0, 0] + t[..., 1, 1]


def _v(x):
    """Material constant with one trailing axis (principal-value arrays)."""
    return np.asarray(x)[..., None]


def _t(x):
    """Material constant with two trailing axes (tensor arrays)."""
    return np.asarray(x)[..., None, None]


def _eye_like(t):
    e = np.zeros_like(t)
    e[..., 0, 0] = 1.0
    e[..., 1, 1] = 1.0
    return e


def ramp_p(x):
    return np.where(x > 0, x, 0.0)


def ramp_m(x):
    return np.where(x < 0, x, 0.0)


def heav(x):
    return (x > 0).astype(float)


def _eig(eps):
    """Principal strains and directions (numpy.linalg.eigh on each 2x2)."""
    w, V = np.linalg.eigh(eps)
    return w, V


def _from_principal(vals, V):
    """sum_a vals_a n^a (x) n^a."""
    return np.einsum("...ia,...a,...ja->...ij", V, vals, V)


def energy_parts(eps, lam, mu, split):
    """(psi_0^+, psi_0^-) of Eqs. isotropic_en / strain_spectral_en / vol_dev_en."""
    tr = trace(eps)
    if split == ISOTROPIC:
        pp = 0.5 * lam * tr ** 2 + mu * np.einsum("...ij,...ij->...", eps, eps)
        return pp, np.zeros_like(pp)
    if split == SPECTRAL:
        w, _ = _eig(eps)
        pp = 0.5 * lam * ramp_p(tr) ** 2 + mu * np.sum(ramp_p(w) ** 2, axis=-1)
        pm = 0.5 * lam * ramp_m(tr) ** 2 + mu * np.sum(ramp_m(w) ** 2, axis=-1)
        return pp, pm
    if split == VOLDEV:
        K = lam + 2.0 * mu / 3.0
        dev = eps - (tr / 3.0)[..., None, None] * _eye_like(eps)
        pp = 0.5 * K * ramp_p(tr) ** 2 + mu * np.einsum("...ij,...ij->...", dev, dev)
        pm = 0.5 * K * ramp_m(tr) ** 2
        return pp, pm
    raise ValueError(split)


def stress_parts(eps, lam, mu, split):
    """(sigma_0^+, sigma_0^-) = d psi_0^pm / d eps (Eqs. stress_iso, stress_spectral, stress_voldev)."""
    tr = trace(eps)
    I = _eye_like(eps)
    if split == ISOTROPIC:
        sp = _t(lam) * tr[..., None, None] * I + 2.0 * _t(mu) * eps
        return sp, np.zeros_like(sp)
    if split == SPECTRAL:
        w, V = _eig(eps)
        sp = _from_principal(_v(lam) * ramp_p(tr)[..., None] + 2.0 * _v(mu) * ramp_p(w), V)
        sm = _from_principal(_v(lam) * ramp_m(tr)[..., None] + 2.0 * _v(mu) * ramp_m(w), V)
        return sp, sm
    if split == VOLDEV:
        K = _t(lam + 2.0 * mu / 3.0)
        sp = K * ramp_p(tr)[..., None, None] * I + 2.0 * _t(mu) * (eps - (4.0 / 9.0) * tr[..., None, None] * I)
        sm = K * ramp_m(tr)[..., None, None] * I
        return sp, sm
    raise ValueError(split)


def contact_split(split):
    """Split that supplies the stress (the contact model of Sec. 2.1)."""
    return {SPECTRAL_STRESSFREE: ISOTROPIC, SPECTRAL_VOLDEV: VOLDEV}.get(split, split)


def driving_split(split):
    """Split that supplies psi_0^+ in the crack driving force (Sec. 2.1)."""
    return SPECTRAL if split in (SPECTRAL_STRESSFREE, SPECTRAL_VOLDEV) else split


def stress(eps, phi, lam, mu, split):
    """sigma = sigma_0^+ h(phi) + sigma_0^- of the contact model (Sec. 2.1)."""
    sp, sm = stress_parts(eps, lam, mu, contact_split(split))
    return h(phi)[..., None, None] * sp + sm


def psi_plus(eps, lam, mu, split):
    """psi_0^+ of the crack-driving-force model."""
    return energy_parts(eps, lam, mu, driving_split(split))[0]


def energy_density(eps, phi, lam, mu, split):
    """psi = psi_0^+ h + psi_0^- of the contact model (Eq. psi_schema)."""
    pp, pm = energy_parts(eps, lam, mu, contact_split(split))
    return h(phi) * pp + pm


class Tangent:
    """Consistent tangent C = d sigma / d eps at a fixed strain (Sec. 3.1.1, Eq. elasticity_newton_linear).

    The paper cites the literature for C.  For the spectral split the derivative
    of eps -> sum_a <eps_a>_+ n^a (x) n^a is written in the eigenbasis with
    divided differences (Daleckii-Krein): diagonal entries H(eps_a), off-diagonal
    (<eps_1>_+ - <eps_2>_+)/(eps_1 - eps_2), replaced by H(eps_1) when the two
    principal strains coincide to 1e-12 relative.
    """

    def __init__(self, eps, phi, lam, mu, split):
        self.split = contact_split(split)
        self.hphi = h(phi)
        self.lam, self.mu = lam, mu
        self.tr = trace(eps)
        if self.split == SPECTRAL:
            w, V = _eig(eps)
            self.V = V
            g = np.empty(w.shape[:-1] + (2, 2))
            Hw = heav(w)
            g[..., 0, 0] = Hw[..., 0]
            g[..., 1, 1] = Hw[..., 1]
            dw = w[..., 0] - w[..., 1]
            scale = np.maximum(np.abs(w).max(axis=-1), 1e-300)
            degenerate = np.abs(dw) <= 1e-12 * scale
            off = np.where(degenerate, Hw[..., 0],
                           (ramp_p(w[..., 0]) - ramp_p(w[..., 1])) / np.where(degenerate, 1.0, dw))
            g[..., 0, 1] = off
            g[..., 1, 0] = off
            self.g = g

    def __call__(self, p):
        lam, mu = _t(self.lam), _t(self.mu)
        trp = trace(p)
        I = _eye_like(p)
        hh = self.hphi[..., None, None]
        if self.split == ISOTROPIC:
            return hh * (lam * trp[..., None, None] * I + 2.0 * mu * p)
        if self.split == SPECTRAL:
            V = self.V
            pt = np.einsum("...ia,...ij,...jb->...ab", V, p, V)     # p in the eigenbasis
            dplus = np.einsum("...ia,...ab,...jb->...ij", V, self.g * pt, V)
            Ht = heav(self.tr)[..., None, None]
            plus = lam * Ht * trp[..., None, None] * I + 2.0 * mu * dplus
            minus = lam * (1.0 - Ht) * trp[..., None, None] * I + 2.0 * mu * (p - dplus)
            return hh * plus + minus
        if self.split == VOLDEV:
            K = lam + 2.0 * mu / 3.0
            Ht = heav(self.tr)[..., None, None]
            plus = K * Ht * trp[..., None, None] * I + 2.0 * mu * (p - (4.0 / 9.0) * trp[..., None, None] * I)
            minus = K * (1.0 - Ht) * trp[..., None, None] * I
            return hh * plus + minus
        raise ValueError(self.split)


def is_linear(split):
    """Whether the stress is linear in eps (one Newton step suffices, Sec. 3.1.1)."""
    return contact_split(split) == ISOTROPIC
