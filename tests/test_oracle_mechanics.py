"""Pins of the oracle's mechanics solver (Sec. 3.1.1): closed forms and dense direct solves."""
import numpy as np
import pytest

from oracle import constitutive as cm
from oracle import fourier, mechanics
from oracle.params import ISOTROPIC, SPECTRAL, SPECTRAL_STRESSFREE, VOLDEV, Params


def test_homogeneous_modulus_gives_zero_polarisation():
    par = Params(split=SPECTRAL, mech_tol=1e-12)
    E = np.full((16, 16), 1.3)
    phi = np.zeros((16, 16))
    eps_bar = np.array([[0.01, 0.003], [0.003, -0.02]])
    es, info = mechanics.solve(np.zeros((16, 16, 2, 2)), eps_bar, phi, E, par)
    assert np.abs(es).max() < 1e-14
    assert info["newton"] == 0


@pytest.mark.parametrize("split", [ISOTROPIC, SPECTRAL, SPECTRAL_STRESSFREE])
def test_laminate_closed_form(split):
    # Properties varying with y only, uniaxial eps_bar_yy = e > 0: equilibrium forces sigma_yy const,
    # compatibility forces eps_xx = 0, so eps_yy(y) = e M(y)^-1 / <M^-1> with M = h(phi)(lambda + 2 mu).
    # Odd grid (as in the paper): the closed form has content at every frequency, and an even
    # grid drops the Nyquist mode from the projection.
    ny, nx = 33, 9
    y = np.arange(ny)
    Ey = 1.0 + 0.5 * np.sin(2 * np.pi * y / ny) + 0.2 * np.cos(6 * np.pi * y / ny)
    phiy = 0.3 + 0.25 * np.cos(2 * np.pi * y / ny)
    E = np.repeat(Ey[:, None], nx, axis=1)
    phi = np.repeat(phiy[:, None], nx, axis=1)
    e = 0.01
    par = Params(split=split, nu=0.2, mech_tol=1e-12, mech_cg_rtol=1e-6)
    eps_bar = np.array([[0.0, 0.0], [0.0, e]])
    es, info = mechanics.solve(np.zeros((ny, nx, 2, 2)), eps_bar, phi, E, par)
    lam, mu = cm.lame(E, par.nu)
    M = cm.h(phi) * (lam + 2 * mu)
    expect_yy = e * (1.0 / M) / np.mean(1.0 / M[:, 0])
    eps = eps_bar[None, None] + es
    np.testing.assert_allclose(eps[..., 1, 1], expect_yy, rtol=1e-9)
    np.testing.assert_allclose(eps[..., 0, 0], 0.0, atol=1e-11)
    np.testing.assert_allclose(eps[..., 0, 1], 0.0, atol=1e-11)


def _range_basis(ny, nx):
    """Orthonormal basis of range(P) in the space of symmetric tensor fields (3 comps per pixel)."""
    cols = []
    for j in range(ny):
        for i in range(nx):
            for (a, b) in [(0, 0), (1, 1), (0, 1)]:
                z = np.zeros((ny, nx, 2, 2))
                z[j, i, a, b] = 1.0
                z[j, i, b, a] = 1.0
                cols.append(fourier.project(z).ravel())
    A = np.array(cols).T
    U, s, _ = np.linalg.svd(A, full_matrices=False)
    return U[:, s > 1e-10 * s[0]]


@pytest.mark.parametrize("split", [ISOTROPIC, SPECTRAL, VOLDEV])
def test_newton_cg_matches_dense_direct_solve_8x8(split):
    ny = nx = 8
    rng = np.random.default_rng(21)
    E = np.exp(0.5 * rng.standard_normal((ny, nx)))
    phi = rng.uniform(0.0, 0.6, (ny, nx))
    eps_bar = np.array([[0.002, 0.004], [0.004, 0.01]])
    par = Params(split=split, mech_tol=1e-13, mech_cg_rtol=1e-8)
    es, info = mechanics.solve(np.zeros((ny, nx, 2, 2)), eps_bar, phi, E, par)
    lam, mu = cm.lame(E, par.nu)
    Q = _range_basis(ny, nx)
    shape = (ny, nx, 2, 2)
    # Newton on the reduced coordinates y (eps* = Q y) with a dense Jacobian from the tangent
    yv = np.zeros(Q.shape[1])
    for _ in range(30):
        eps = eps_bar[None, None] + (Q @ yv).reshape(shape)
        Rv = Q.T @ cm.stress(eps, phi, lam, mu, split).ravel()
        if np.linalg.norm(Rv) < 1e-15:
            break
        tang = cm.Tangent(eps, phi, lam, mu, split)
        Jm = np.array([Q.T @ tang(Q[:, k].reshape(shape)).ravel() for k in range(Q.shape[1])]).T
        yv = yv - np.linalg.solve(Jm, Rv)
    direct = (Q @ yv).reshape(shape)
    np.testing.assert_allclose(es, direct, atol=1e-10 * np.abs(direct).max(), rtol=0)
    # and the converged field satisfies the nodal equilibrium equations
    R = mechanics.residual(es, eps_bar, phi, E, par)
    assert np.linalg.norm(R) <= 1e-12 * mechanics.reference_norm(eps_bar, E, par)


def test_solution_minimises_elastic_energy_isotropic():
    # Variational model: the converged eps* minimises F_e over compatible perturbations.
    ny = nx = 16
    rng = np.random.default_rng(5)
    E = np.exp(0.4 * rng.standard_normal((ny, nx)))
    phi = rng.uniform(0, 0.5, (ny, nx))
    par = Params(split=ISOTROPIC, mech_tol=1e-13)
    eps_bar = np.array([[0.0, 0.0], [0.0, 0.01]])
    es, _ = mechanics.solve(np.zeros((ny, nx, 2, 2)), eps_bar, phi, E, par)
    lam, mu = cm.lame(E, par.nu)

    def Fe(x):
        return np.sum(cm.energy_density(eps_bar[None, None] + x, phi, lam, mu, ISOTROPIC))
    base = Fe(es)
    for k in range(5):
        d = rng.standard_normal((ny, nx, 2, 2)); d = fourier.project(d + np.swapaxes(d, -1, -2))
        d *= 1e-3 / np.abs(d).max()
        assert Fe(es + d) > base
        assert Fe(es - d) > base
