"""Discretisation and Fourier-space operators (Sec. 3.1).  Test infrastructure only.

Grid (Sec. 3.1): N = (nx, ny) points with spacing dx, L = N dx, wavevector
q^k = k / L.  The forward DFT of Sec. 3.1 carries 1/|N|; every operator here
is F^-1 M F, in which the normalisation cancels, so ``numpy.fft.fft2`` /
``ifft2`` are used directly as the DFT pair.

Even grids.  The paper works with odd N only (Eq. trapezoidal).  For even N the
Nyquist index k = -N/2 has no conjugate partner with the opposite wavevector,
and the cross term n_x n_y of the projection differs between the modes
(-N/2, k_y) and (-N/2, -k_y).  Reading used here: the projection Gamma is set to
zero on every mode whose k_x or k_y is the Nyquist index (an orthogonal
projection that keeps fields real), while the Laplacian multiplier |2 pi q|^2,
which is even in each component, is kept on those modes.  Odd grids have no
Nyquist index, so nothing is dropped there.
"""
import numpy as np


def wavevectors(ny, nx, dx=1.0):
    """Return (qy, qx) arrays of shape (ny, nx): q^k = k/L in numpy FFT order (Sec. 3.1)."""
    qx = np.fft.fftfreq(nx, d=dx)
    qy = np.fft.fftfreq(ny, d=dx)
    QY, QX = np.meshgrid(qy, qx, indexing="ij")
    return QY, QX


def nyquist_mask(ny, nx):
    """True on modes whose kx or ky index is the Nyquist index of an even grid."""
    m = np.zeros((ny, nx), dtype=bool)
    if nx % 2 == 0:
        m[:, nx // 2] = True
    if ny % 2 == 0:
        m[ny // 2, :] = True
    return m


def fft2(f):
    """DFT over the two grid axes (axes 0, 1) of a field with optional trailing tensor axes."""
    return np.fft.fft2(f, axes=(0, 1))


def ifft2_real(fh):
    """Inverse DFT over the grid axes, real part (the fields of Sec. 3.1 are real)."""
    return np.fft.ifft2(fh, axes=(0, 1)).real


def gamma_hat_apply(zeta_hat, ny, nx, dx=1.0):
    """Apply the compatibility projection Gamma(q) mode by mode.

    The paper defers the form of G-hat to its references (Sec. 3.1.1, text
    after Eq. elasticity_weak_discrete).  Used here: the orthogonal projection of
    a symmetric 2x2 tensor onto the compatible strains sym(a (x) n) at wave
    direction n = q/|q|:  Gamma(n):zeta = n (x) (zeta n) + (zeta n) (x) n - (n.zeta n) n (x) n,
    and Gamma(0) = 0 (the mean strain is the applied eps_bar).
    zeta_hat has shape (ny, nx, 2, 2).
    """
    QY, QX = wavevectors(ny, nx, dx)
    qn = np.sqrt(QX ** 2 + QY ** 2)
    zero = (qn == 0) | nyquist_mask(ny, nx)
    safe = np.where(zero, 1.0, qn)
    n = np.stack([QX / safe, QY / safe], axis=-1)          # (ny, nx, 2), components (x, y)
    s = np.einsum("...ij,...j->...i", zeta_hat, n)          # zeta n
    t = np.einsum("...i,...i->...", n, s)                   # n . zeta n
    out = (np.einsum("...i,...j->...ij", n, s) + np.einsum("...i,...j->...ij", s, n)
           - t[..., None, None] * np.einsum("...i,...j->...ij", n, n))
    out[zero] = 0.0
    return out


def project(zeta, dx=1.0):
    """Real-space projection P zeta = F^-1 Gamma F zeta of a tensor field (ny, nx, 2, 2)."""
    ny, nx = zeta.shape[:2]
    return ifft2_real(gamma_hat_apply(fft2(zeta), ny, nx, dx))


def laplacian(g, dx=1.0):
    """Collocation Laplacian nabla^2_N g = -F^-1 |2 pi q|^2 F g (Sec. 3.1.2)."""
    ny, nx = g.shape
    QY, QX = wavevectors(ny, nx, dx)
    mult = (2.0 * np.pi) ** 2 * (QX ** 2 + QY ** 2)
    return ifft2_real(-mult * fft2(g))
