"""Pins of the oracle's pointwise constitutive model (Sec. 2.1, Sec. 3.3, Sec. 4.2.1)."""
import numpy as np
import pytest

from oracle import constitutive as cm
from oracle.params import ISOTROPIC, SPECTRAL, SPECTRAL_STRESSFREE, VOLDEV


def rot(theta):
    c, s = np.cos(theta), np.sin(theta)
    return np.array([[c, -s], [s, c]])


def test_plane_strain_numbers_of_sec_3_3():
    # Sec. 3.3: nu = 0.2 gives (lambda + 2 mu) = 10/9 E0, eps_M ~= 0.005809, sigma_M ~= 64.55 Gc/ell
    E0, nu, Gc, ell = 1e4, 0.2, 1.0, 1.0
    lam, mu = cm.lame(E0, nu)
    assert lam + 2 * mu == pytest.approx(10.0 / 9.0 * E0, rel=1e-14)
    epsM = np.sqrt(3 * Gc / (8 * ell * (lam + 2 * mu)))
    sigM = np.sqrt(3 * Gc * (lam + 2 * mu) / (8 * ell))
    assert round(epsM, 6) == 0.005809
    assert round(sigM, 2) == 64.55
    # and the oracle's driving force at eps_M balances the AT1 threshold: -h'(0) psi = 3 Gc/(8 ell) f'(0)
    eps = np.array([[0.0, 0.0], [0.0, epsM]])
    for split in (ISOTROPIC, SPECTRAL, VOLDEV):
        psi = cm.psi_plus(eps, lam, mu, split)
        if split == VOLDEV:
            continue   # Sec. 3.3 states equality for uniaxial strain only among models identical there
        assert 2 * psi == pytest.approx(3 * Gc / (8 * ell), rel=1e-12)


def test_pure_shear_numbers_of_sec_4_2_2():
    # eps_12,M = (1/4) sqrt(3 Gc/(ell mu)) = 0.007246, sigma_12,M = 51.75 for nu = 0.4, E = 1e4
    E0, nu, Gc, ell = 1e4, 0.4, 1.0, 1.0
    lam, mu = cm.lame(E0, nu)
    e12 = 0.25 * np.sqrt(3 * Gc / (ell * mu))
    assert round(e12, 6) == 0.007246
    assert round(2 * mu * e12, 2) == 51.75
    eps = np.array([[0.0, e12], [e12, 0.0]])
    psi = cm.psi_plus(eps, lam, mu, SPECTRAL)
    assert 2 * psi == pytest.approx(3 * Gc / (8 * ell), rel=1e-12)
    sig = cm.stress(eps, np.array(0.0), lam, mu, SPECTRAL)
    assert sig[0, 1] == pytest.approx(51.75, abs=5e-3)


@pytest.mark.parametrize("theta", [0.0, 0.3, 1.1])
@pytest.mark.parametrize("a,b", [(1.0, 0.0), (0.7, 0.4), (0.2, 1.5)])
def test_psi_plus_shear_plus_compression_sec_4_2_1(theta, a, b):
    lam, mu = cm.lame(2.5, 0.3)
    R = rot(theta)
    eps = R @ np.diag([a, -a - b]) @ R.T
    assert cm.psi_plus(eps, lam, mu, ISOTROPIC) == pytest.approx(0.5 * lam * b * b + 2 * mu * (a * a + a * b + b * b / 2), rel=1e-12)
    assert cm.psi_plus(eps, lam, mu, SPECTRAL) == pytest.approx(mu * a * a, rel=1e-12)
    assert cm.psi_plus(eps, lam, mu, VOLDEV) == pytest.approx(2 * mu * (a * a + a * b + 5 * b * b / 18), rel=1e-12)
    assert cm.psi_plus(eps, lam, mu, SPECTRAL_STRESSFREE) == pytest.approx(mu * a * a, rel=1e-12)


def test_contact_stresses_at_phi_one_sec_4_2_1():
    lam, mu = cm.lame(3.0, 0.25)
    b = 0.37
    one = np.array(1.0)
    eps = np.array([[0.0, 0.0], [0.0, -b]])
    np.testing.assert_allclose(cm.stress(eps, one, lam, mu, ISOTROPIC), 0.0, atol=1e-15)
    np.testing.assert_allclose(cm.stress(eps, one, lam, mu, SPECTRAL), np.diag([-lam * b, -(lam + 2 * mu) * b]), rtol=1e-13)
    np.testing.assert_allclose(cm.stress(eps, one, lam, mu, VOLDEV), -(lam + 2 * mu / 3) * b * np.eye(2), rtol=1e-13)
    np.testing.assert_allclose(cm.stress(eps, one, lam, mu, SPECTRAL_STRESSFREE), 0.0, atol=1e-15)
    eps = np.array([[0.0, b], [b, 2 * b]])
    s2 = np.sqrt(2.0)
    expect = mu / s2 * np.array([[-b, (s2 - 1) * b], [(s2 - 1) * b, (2 * s2 - 3) * b]])
    np.testing.assert_allclose(cm.stress(eps, one, lam, mu, SPECTRAL), expect, rtol=1e-12)
    np.testing.assert_allclose(cm.stress(eps, one, lam, mu, ISOTROPIC), 0.0, atol=1e-15)
    np.testing.assert_allclose(cm.stress(eps, one, lam, mu, VOLDEV), 0.0, atol=1e-15)


def _rand_strains(n, seed):
    rng = np.random.default_rng(seed)
    e = rng.standard_normal((n, 2, 2))
    return 0.5 * (e + np.swapaxes(e, -1, -2))


@pytest.mark.parametrize("split", [ISOTROPIC, SPECTRAL, VOLDEV])
def test_stress_is_gradient_of_energy(split):
    # sigma = d psi / d eps (Eq. F_strain) by central differences along symmetric directions
    lam, mu = cm.lame(1.7, 0.2)
    eps = _rand_strains(50, 1)
    phi = np.random.default_rng(2).uniform(0, 1, 50)
    sig = cm.stress(eps, phi, lam, mu, split)
    hstep = 1e-6
    for (i, j) in [(0, 0), (1, 1), (0, 1)]:
        d = np.zeros((2, 2)); d[i, j] = 1.0; d[j, i] = 1.0
        ep = cm.energy_density(eps + hstep * d, phi, lam, mu, split)
        em = cm.energy_density(eps - hstep * d, phi, lam, mu, split)
        fd = (ep - em) / (2 * hstep)
        np.testing.assert_allclose(np.einsum("nij,ij->n", sig, d), fd, rtol=1e-6, atol=1e-8)


@pytest.mark.parametrize("split", [ISOTROPIC, SPECTRAL, VOLDEV, SPECTRAL_STRESSFREE])
def test_tangent_matches_finite_differences(split):
    lam, mu = cm.lame(1.3, 0.2)
    eps = _rand_strains(60, 4)
    phi = np.random.default_rng(5).uniform(0, 1, 60)
    p = _rand_strains(60, 6)
    tang = cm.Tangent(eps, phi, lam, mu, split)
    hstep = 1e-7
    fd = (cm.stress(eps + hstep * p, phi, lam, mu, split) - cm.stress(eps - hstep * p, phi, lam, mu, split)) / (2 * hstep)
    np.testing.assert_allclose(tang(p), fd, rtol=1e-5, atol=1e-7)


@pytest.mark.parametrize("split", [ISOTROPIC, SPECTRAL, VOLDEV])
def test_homogeneity(split):
    # Sec. 3.2.3: psi_0^+ is degree-2 and sigma degree-1 homogeneous
    lam, mu = cm.lame(1.0, 0.2)
    eps = _rand_strains(30, 8)
    phi = np.random.default_rng(9).uniform(0, 1, 30)
    g = 0.731
    np.testing.assert_allclose(cm.psi_plus(g * eps, lam, mu, split), g * g * cm.psi_plus(eps, lam, mu, split), rtol=1e-12)
    np.testing.assert_allclose(cm.stress(g * eps, phi, lam, mu, split), g * cm.stress(eps, phi, lam, mu, split), rtol=1e-12, atol=1e-15)


def test_spectral_split_sums_to_isotropic():
    lam, mu = cm.lame(1.0, 0.3)
    eps = _rand_strains(40, 11)
    pp, pm = cm.energy_parts(eps, lam, mu, SPECTRAL)
    iso, _ = cm.energy_parts(eps, lam, mu, ISOTROPIC)
    np.testing.assert_allclose(pp + pm, iso, rtol=1e-12)
    sp, sm = cm.stress_parts(eps, lam, mu, SPECTRAL)
    si, _ = cm.stress_parts(eps, lam, mu, ISOTROPIC)
    np.testing.assert_allclose(sp + sm, si, rtol=1e-12, atol=1e-14)
