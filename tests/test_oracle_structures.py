"""Pins of the oracle's initial conditions and microstructure generators
(Sec. 3.3, Sec. 4.1.1, Eqs. init_crack, AT1_analytical, sigmoid, ACsmooth)
against closed forms, the 1-D analytical crack profile, exact single-step
responses and the properties the paper asks of each construction."""
import numpy as np
import pytest

from oracle import structures as st
from paper_2203_16467_gb300.inputs import white_noise


def test_crack_cross_section_is_the_AT1_profile():
    # across the middle of the crack the profile is Eq. AT1_analytical
    ny, nx, ell = 96, 128, 3.0
    phi = st.phi_init(ny, nx, 1.0, ell, 64.0, 40.0, 30.0)
    col = phi[:, 64]
    y = np.arange(ny) - 40.0
    ref = np.where(np.abs(y) <= 2 * ell, (1 - np.abs(y) / (2 * ell)) ** 2, 0.0)
    np.testing.assert_allclose(col, ref, atol=1e-15)
    assert phi.max() == 1.0 and np.all(phi >= 0.0)


@pytest.mark.parametrize("length", [0.0, 60.0])
def test_crack_integral_closed_form(length):
    # int phi dA = 4 L ell / 3 (strip) + 2 pi ell^2 / 3 (two half-disc tips)
    ny, nx, ell = 256, 256, 12.0
    phi = st.phi_init(ny, nx, 1.0, ell, 128.0, 128.0, length)
    exact = 4.0 * length * ell / 3.0 + 2.0 * np.pi * ell ** 2 / 3.0
    assert abs(phi.sum() - exact) / exact < 3e-3


def test_crack_is_periodic_and_void_is_round():
    ny, nx, ell = 64, 64, 2.5
    a = st.phi_init(ny, nx, 1.0, ell, 32.0, 32.0, 20.0)
    b = st.phi_init(ny, nx, 1.0, ell, 2.0, 61.0, 20.0)      # centre near a corner: wraps
    np.testing.assert_allclose(np.roll(np.roll(a, -30, axis=1), 29, axis=0), b, atol=1e-15)
    v = st.phi_init(ny, nx, 1.0, ell, 32.0, 32.0, 0.0)
    np.testing.assert_allclose(v, v.T, atol=1e-15)
    np.testing.assert_allclose(v, v[::-1, :][np.r_[ny - 1, 0:ny - 1], :], atol=1e-15)


def test_edge_crack_is_the_printed_equation():
    # the notch runs from the periodic cut x = -Lx/2 (relative to the centre) to the tip
    ny, nx, ell, L = 64, 128, 2.0, 40.0
    phi = st.phi_init(ny, nx, 1.0, ell, 64.0, 32.0, L, mode="edge")
    assert np.all(phi[32, 0:85] == 1.0) and phi[32, 85] < 1.0        # tip at x = 64 + 20
    np.testing.assert_allclose(phi[32, 84:90], [1.0, 0.5625, 0.25, 0.0625, 0.0, 0.0], atol=1e-15)
    assert phi[32, 127] == 0.0                                        # sharp cut at the periodic edge
    np.testing.assert_allclose(phi[:, 10], st.phi_init(ny, nx, 1.0, ell, 64.0, 32.0, 100.0)[:, 64], atol=1e-15)


def test_modulus_crack_is_degraded_modulus():
    E = st.modulus_with_crack(64, 64, 1.0, 2.0, 32.0, 32.0, 16.0, 3.0)
    assert E[32, 32] == 0.0 and E[0, 0] == 3.0
    assert np.all((E >= 0.0) & (E <= 3.0))


def test_lowpass_keeps_exactly_the_band():
    ny, nx, dx, Lc = 64, 96, 0.5, 3.7
    xi = white_noise(ny, nx, 5)
    f = st.lowpass(xi, dx, Lc)
    F, X = np.fft.fft2(f), np.fft.fft2(xi)
    qx = 2 * np.pi * np.fft.fftfreq(nx, d=dx)
    qy = 2 * np.pi * np.fft.fftfreq(ny, d=dx)
    q = np.hypot(qy[:, None], qx[None, :])
    band = (q > 0) & (q <= 2 * np.pi / Lc)
    assert band.sum() > 10 and (~band).sum() > 10
    np.testing.assert_allclose(F[band], X[band], atol=1e-10)
    assert np.abs(F[~band]).max() < 1e-10
    assert abs(f.mean()) < 1e-15


def test_sigmoid_floor_properties():
    xm = 0.01
    x = np.linspace(-50.0, 3.0, 20001)
    s = st.sigmoid_floor(x, xm)
    assert np.all(s > xm - 1e-15) and np.all(np.diff(s) > -1e-15)  # bounded below, monotone
    core = (x > -1.0)
    assert np.all(np.diff(s[core]) > 0)
    np.testing.assert_array_equal(s[x >= 1.0], x[x >= 1.0])        # untouched at and above 1
    assert abs(st.sigmoid_floor(np.array([-1e6]), xm)[0] - xm) < 1e-12   # tends to xi_min
    h = 1e-6                                                       # slope 1 at xi_r = 1
    assert abs((1.0 - st.sigmoid_floor(np.array([1.0 - h]), xm)[0]) / h - 1.0) < 1e-9


def test_random_field_hits_target_std_and_mean():
    xi = white_noise(128, 128, 3)
    # a floor far below the values leaves the scaled field untouched: STD_t exactly, mean 1
    f = st.random_field(xi, 1.0, 10.0, std_target=0.3, xi_min=-1e9)
    assert abs(f.std() - 0.3) < 1e-12 and abs(f.mean() - 1.0) < 1e-12
    g = st.random_field(xi, 1.0, 10.0)
    assert g.min() > 0.01 and abs(g.mean() - 1.0) < 0.02


def test_allen_cahn_step_exact_responses():
    n = 8
    d = np.zeros((n, n))
    d[0, 0] = 1.0                              # delta at a corner: 5-point stencil with wrap
    s = st.allen_cahn_step(d)
    assert s[0, 0] == pytest.approx(0.6, abs=1e-15)
    for (j, i) in ((0, 1), (1, 0), (0, n - 1), (n - 1, 0)):
        assert s[j, i] == pytest.approx(0.1, abs=1e-15)
    assert np.count_nonzero(s) == 5
    for c, want in ((1.0, 1.0), (-1.0, -1.0), (0.0, 0.0), (0.5, 0.5 - 0.1 * (0.125 - 0.5))):
        np.testing.assert_allclose(st.allen_cahn_step(np.full((n, n), c)), want, atol=1e-15)
    x = white_noise(n, n, 1)                   # the Laplacian part conserves the sum
    assert st.allen_cahn_step(x).sum() == pytest.approx(x.sum() - 0.1 * (x ** 3 - x).sum(), abs=1e-12)


def test_two_phase_has_the_phase_ratio():
    # a = 0.875 gives the ratio (1 + a) / (1 - a) = 15 between the bulk phases
    # (the smoothing moves points up to 21 pixels from an interface, so the deep
    # bulk of a coarse structure keeps the bulk values to high accuracy)
    xi = white_noise(256, 256, 7)
    E = st.two_phase_field(xi, 1.0, 64.0, a=0.875)
    assert E.min() >= 0.125 - 1e-12 and E.max() <= 1.875 + 1e-12
    assert E.max() / E.min() == pytest.approx(15.0, rel=1e-6)
    bulk = np.isclose(E, 0.125, atol=1e-3) | np.isclose(E, 1.875, atol=1e-3)
    assert bulk.mean() > 0.4


def _cbar_2222(phi, ell):
    from oracle import constitutive as cm
    from oracle import mechanics
    from oracle.params import ISOTROPIC, Params
    ny, nx = phi.shape
    E = np.ones((ny, nx))
    eb = np.array([[0.0, 0.0], [0.0, 1e-3]])
    es, _ = mechanics.solve(np.zeros((ny, nx, 2, 2)), eb, phi, E, Params(split=ISOTROPIC, ell=ell, mech_tol=1e-8))
    lam, mu = cm.lame(E, 0.2)
    sig = cm.stress(eb[None, None] + es, phi, lam, mu, ISOTROPIC).mean(axis=(0, 1))
    return sig[1, 1] / eb[1, 1] / (1.0 * (lam[0, 0] + 2 * mu[0, 0]))


def test_homogenised_stiffness_of_the_crack_and_void_ICs():
    # Sec. 4.1.1: a 100 ell periodic domain with E = E0, nu = 0.2, stress-free contact,
    # crack IC (L_crack = 50 ell): C-bar_2222 = 0.65 sigma_M/eps_M; void IC: nearly 1
    # (printed for 511^2; here 128^2, ell = 1.28 px)
    n = 128
    ell = n / 100.0
    crack = st.phi_init(n, n, 1.0, ell, n / 2, n / 2, 50 * ell, mode="edge")
    void = st.phi_init(n, n, 1.0, ell, n / 2, n / 2, 0.0)
    assert abs(_cbar_2222(crack, ell) - 0.65) < 0.03
    assert _cbar_2222(void, ell) > 0.99


def _cbar_2222_modulus(E):
    from oracle import constitutive as cm
    from oracle import mechanics
    from oracle.params import ISOTROPIC, Params
    ny, nx = E.shape
    eb = np.array([[0.0, 0.0], [0.0, 1e-3]])
    zero = np.zeros((ny, nx))
    es, _ = mechanics.solve(np.zeros((ny, nx, 2, 2)), eb, zero, E, Params(split=ISOTROPIC, mech_tol=1e-6))
    lam, mu = cm.lame(E, 0.2)
    sig = cm.stress(eb[None, None] + es, zero, lam, mu, ISOTROPIC).mean(axis=(0, 1))
    return sig[1, 1] / eb[1, 1] / (10.0 / 9.0)      # (lambda + 2 mu)(E0 = 1) = 10/9 at nu = 0.2


def test_homogenised_stiffness_of_generated_structures():
    # Sec. 4.1.2 prints C-bar_2222 = 0.94 sigma_M/eps_M for a smooth random structure
    # (STD_t 0.3) and 0.42-0.44 for two-phase ones (a = 0.875), L_cut = 6 ell, 100 ell
    # domains at N = 511; single realisations, so a loose band.  The random field's
    # stiffness barely depends on resolution (128^2 here); the two-phase one depends on
    # the 2-pixel interface width and is checked at the paper's resolution (512^2).
    xi = white_noise(128, 128, 0)
    assert abs(_cbar_2222_modulus(st.modulus_field("random", xi, 1.0, 6 * 1.28)) - 0.94) < 0.03
    xi = white_noise(512, 512, 0)
    assert abs(_cbar_2222_modulus(st.modulus_field("two_phase", xi, 1.0, 6 * 5.12)) - 0.43) < 0.03
