"""Pins of the oracle's Fourier operators (Sec. 3.1) against closed forms and brute force."""
import numpy as np
import pytest

from oracle import fourier


@pytest.mark.parametrize("ny,nx", [(16, 16), (15, 21), (8, 32)])
def test_laplacian_of_cosine_closed_form(ny, nx):
    # nabla^2 cos(2 pi (kx x / Lx + ky y / Ly)) = -|2 pi q|^2 cos(...)
    dx = 0.7
    y, x = np.meshgrid(np.arange(ny) * dx, np.arange(nx) * dx, indexing="ij")
    Lx, Ly = nx * dx, ny * dx
    kx, ky = 3, 2
    arg = 2 * np.pi * (kx * x / Lx + ky * y / Ly)
    g = np.cos(arg) + 0.5 * np.sin(2 * np.pi * (x / Lx - 2 * y / Ly))
    lap = fourier.laplacian(g, dx)
    expect = (-(2 * np.pi) ** 2 * ((kx / Lx) ** 2 + (ky / Ly) ** 2) * np.cos(arg)
              - 0.5 * (2 * np.pi) ** 2 * ((1 / Lx) ** 2 + (2 / Ly) ** 2) * np.sin(2 * np.pi * (x / Lx - 2 * y / Ly)))
    np.testing.assert_allclose(lap, expect, atol=1e-10)


def test_laplacian_matches_trig_polynomial_from_paper_dft():
    # Odd grid: build the trigonometric interpolant with the paper's DFT pair
    # (forward carries 1/|N|, indices k in Z_N centred on 0, Sec. 3.1) by explicit sums
    # and differentiate it analytically at the grid points.
    rng = np.random.default_rng(3)
    ny, nx, dx = 5, 7, 1.3
    Lx, Ly = nx * dx, ny * dx
    v = rng.standard_normal((ny, nx))
    ks_x = np.arange(-(nx // 2), nx // 2 + 1)
    ks_y = np.arange(-(ny // 2), ny // 2 + 1)
    xs = np.arange(nx) * dx
    ys = np.arange(ny) * dx
    vhat = {}
    for ky in ks_y:
        for kx in ks_x:
            s = 0j
            for j in range(ny):
                for i in range(nx):
                    s += v[j, i] * np.exp(-2j * np.pi * (kx * xs[i] / Lx + ky * ys[j] / Ly))
            vhat[(ky, kx)] = s / (nx * ny)
    lap = np.zeros((ny, nx))
    for j in range(ny):
        for i in range(nx):
            s = 0j
            for (ky, kx), c in vhat.items():
                q2 = (kx / Lx) ** 2 + (ky / Ly) ** 2
                s += -(2 * np.pi) ** 2 * q2 * c * np.exp(2j * np.pi * (kx * xs[i] / Lx + ky * ys[j] / Ly))
            lap[j, i] = s.real
    np.testing.assert_allclose(fourier.laplacian(v, dx), lap, atol=1e-10)


def _sym_grad_field(ny, nx, dx, modes):
    """Analytic sym(grad u) of u = sum A_m cos(2 pi q_m . x + c_m) e_m (band-limited, no Nyquist)."""
    y, x = np.meshgrid(np.arange(ny) * dx, np.arange(nx) * dx, indexing="ij")
    Lx, Ly = nx * dx, ny * dx
    eps = np.zeros((ny, nx, 2, 2))
    for (kx, ky, ax, ay, c) in modes:
        q = np.array([kx / Lx, ky / Ly])
        arg = 2 * np.pi * (q[0] * x + q[1] * y) + c
        d = -2 * np.pi * np.sin(arg)               # derivative factor of cos(arg) w.r.t. (q . x)
        a = np.array([ax, ay])
        for i in range(2):
            for j in range(2):
                eps[..., i, j] += 0.5 * (a[i] * q[j] + a[j] * q[i]) * d
    return eps


def _airy_stress(ny, nx, dx, modes):
    """sigma from an Airy stress function chi = sum A cos(2 pi q . x + c): divergence free."""
    y, x = np.meshgrid(np.arange(ny) * dx, np.arange(nx) * dx, indexing="ij")
    Lx, Ly = nx * dx, ny * dx
    sig = np.zeros((ny, nx, 2, 2))
    for (kx, ky, A, c) in modes:
        qx, qy = 2 * np.pi * kx / Lx, 2 * np.pi * ky / Ly
        arg = qx * x + qy * y + c
        cc = -A * np.cos(arg)                      # second derivative factor
        sig[..., 0, 0] += qy * qy * cc             # chi_yy
        sig[..., 1, 1] += qx * qx * cc             # chi_xx
        sig[..., 0, 1] += -qx * qy * cc            # -chi_xy
        sig[..., 1, 0] += -qx * qy * cc
    return sig


@pytest.mark.parametrize("ny,nx", [(16, 16), (9, 15), (16, 8)])
def test_projection_keeps_compatible_and_kills_equilibrated(ny, nx):
    dx = 1.0
    modes_u = [(1, 2, 0.3, -0.7, 0.4), (3, -1, 1.1, 0.2, -1.0), (0, 2, 0.5, 0.9, 0.3), (2, 0, -0.4, 0.6, 2.0)]
    eps = _sym_grad_field(ny, nx, dx, modes_u)
    np.testing.assert_allclose(fourier.project(eps, dx), eps, atol=1e-12)
    modes_s = [(1, 1, 0.7, 0.1), (2, -3, -0.4, 1.3), (0, 1, 1.0, 0.0), (3, 0, 0.5, -0.2)]
    sig = _airy_stress(ny, nx, dx, modes_s)
    np.testing.assert_allclose(fourier.project(sig, dx), 0.0, atol=1e-12)
    const = np.zeros((ny, nx, 2, 2)) + np.array([[0.3, -0.1], [-0.1, 0.7]])
    np.testing.assert_allclose(fourier.project(const, dx), 0.0, atol=1e-12)


@pytest.mark.parametrize("ny,nx", [(16, 16), (9, 15)])
def test_projection_is_orthogonal_projector(ny, nx):
    rng = np.random.default_rng(7)
    a = rng.standard_normal((ny, nx, 2, 2)); a = a + np.swapaxes(a, -1, -2)
    b = rng.standard_normal((ny, nx, 2, 2)); b = b + np.swapaxes(b, -1, -2)
    Pa = fourier.project(a)
    np.testing.assert_allclose(fourier.project(Pa), Pa, atol=1e-12)
    np.testing.assert_allclose(np.sum(Pa * b), np.sum(a * fourier.project(b)), rtol=1e-12)
    np.testing.assert_allclose(Pa, np.swapaxes(Pa, -1, -2), atol=1e-13)
    # projection of the trace-free-free part: P is not the identity on generic fields
    assert np.linalg.norm(Pa - a) > 0.1 * np.linalg.norm(a)
