"""Initial conditions and microstructure generators (Sec. 3.3 and Sec. 4.1.1).
Test infrastructure only.

Initial crack / void (Eq. init_crack): a generalisation of the AT1 profile
(Eq. AT1_analytical),
    phi_init(x) = (1 - |r| / (2 ell))^2  where |r| <= 2 ell,  0 elsewhere.
Readings:
  * the printed support condition "|r| <= 2" is read in units of ell (the
    profile reaches zero at |r| = 2 ell, where it must stop);
  * "edge" crack, the equation as printed: r = (max(x - L_crack/2, 0), y) with
    x, y measured from the domain centre (xc, yc) and x in [-Lx/2, Lx/2), i.e.
    a notch from the periodic cut at x = -Lx/2 to a rounded tip at x = L_crack/2
    (the periodic single-edge-notched specimen of Sec. 3.3; this reading gives
    the printed homogenised stiffness C-bar_2222 = 0.65 sigma_M/eps_M of
    Sec. 4.1.1 for L_crack = 50 ell in a 100 ell domain);
  * "segment" crack: r = (max(|x| - L_crack/2, 0), y), a crack of length
    L_crack with two rounded tips; L_crack = 0 gives the small void of
    Sec. 4.1.1 (r = (x, y));
  * y (and x for the segment) is the nearest periodic image; the grid point
    (i, j) sits at (i dx, j dx).
Crack in E (Sec. 4.2.2): E = h(phi_init) E0 = (1 - phi_init)^2 E0.

Random structures (Sec. 3.3): xi ~ N(0, 1) per grid point (drawn by the caller
and passed in), low-pass filtered in Fourier space, then
  * random field: xi_r = xi STD_t / STD(xi) + 1 followed by the algebraic
    sigmoid of Eq. sigmoid on the points with xi_r < 1;
  * two-phase: xi_p = sgn(xi), smoothed by iterations of Eq. ACsmooth (an
    explicit Allen-Cahn step with the 5-point periodic Laplacian in pixel
    units), then scaled xi_p := a xi_p + 1.
E = E0 xi.  Readings:
  * the filter keeps the modes with 0 < |q| <= 2 pi / L_cut (the printed
    condition zeroes |q| < 2 pi / L_cut, which would be a high-pass, while the
    text asks to remove wavelengths shorter than L_cut and a zero-mean result);
    with |q| = 2 pi |k / L| the test is kx^2/Lx^2 + ky^2/Ly^2 <= 1/L_cut^2,
    evaluated as kx^2 (Ly L_cut)^2 + ky^2 (Lx L_cut)^2 <= (Lx Ly)^2 (exact for
    integer lengths, so that both implementations take the same decision);
  * STD is the population standard deviation over the grid points;
  * Eq. sigmoid is read as xi_r := 1 - d D / (d^10 + D^10)^(1/10) with
    d = 1 - xi_r and D = 1 - xi_min, applied where xi_r < 1 (the printed
    "+ 1" and the missing tenth root would map values below 1 above 1 and
    would not bound xi_r below by xi_min);
  * Eq. ACsmooth runs for n = 0, 1, ..., n_iter - 1 with n_iter = 21 (the
    printed n = 0..20), with the cubic term at the same point as the update.
"""
import numpy as np


# ---------------------------------------------------------------- initial conditions
def crack_distance(ny, nx, dx, xc, yc, length, mode="segment"):
    """|r| of Eq. init_crack for a horizontal crack centred at (xc, yc) (readings above)."""
    Lx, Ly = nx * dx, ny * dx
    x = np.arange(nx) * dx
    y = np.arange(ny) * dx
    ddx = x[None, :] - xc
    ddy = y[:, None] - yc
    ddx = ddx - Lx * np.floor(ddx / Lx + 0.5)   # into [-Lx/2, Lx/2)
    ddy = ddy - Ly * np.floor(ddy / Ly + 0.5)
    if mode == "segment":
        rx = np.maximum(np.abs(ddx) - 0.5 * length, 0.0)
    elif mode == "edge":
        rx = np.maximum(ddx - 0.5 * length, 0.0)
    else:
        raise ValueError(mode)
    return np.sqrt(rx * rx + ddy * ddy)


def phi_init(ny, nx, dx, ell, xc, yc, length, mode="segment"):
    """Eq. init_crack."""
    r = crack_distance(ny, nx, dx, xc, yc, length, mode)
    return np.where(r <= 2.0 * ell, (1.0 - r / (2.0 * ell)) ** 2, 0.0)


def modulus_with_crack(ny, nx, dx, ell, xc, yc, length, E0, mode="segment"):
    """Crack in E (Sec. 4.2.2): E = h(phi_init) E0 with h = (1 - phi)^2."""
    return (1.0 - phi_init(ny, nx, dx, ell, xc, yc, length, mode)) ** 2 * E0


# ---------------------------------------------------------------- random structures
def lowpass_keep(ny, nx, dx, L_cut):
    """Boolean mask of the kept Fourier modes (numpy FFT order): 0 < |q| <= 2 pi / L_cut."""
    kx = np.fft.fftfreq(nx, d=1.0 / nx)          # integer mode indices
    ky = np.fft.fftfreq(ny, d=1.0 / ny)
    Lx, Ly = nx * dx, ny * dx
    lhs = (kx[None, :] ** 2) * (Ly * L_cut) ** 2 + (ky[:, None] ** 2) * (Lx * L_cut) ** 2
    keep = lhs <= (Lx * Ly) ** 2
    keep[0, 0] = False
    return keep


def lowpass(xi, dx, L_cut):
    """Sec. 3.3: zero the Fourier components outside the kept band, transform back."""
    ny, nx = xi.shape
    return np.fft.ifft2(np.fft.fft2(xi) * lowpass_keep(ny, nx, dx, L_cut)).real


def sigmoid_floor(xi_r, xi_min):
    """Eq. sigmoid (reading above): values below 1 are pulled smoothly above xi_min."""
    D = 1.0 - xi_min
    d = 1.0 - xi_r
    low = xi_r < 1.0
    out = np.array(xi_r, dtype=float, copy=True)
    dl = d[low]
    out[low] = 1.0 - dl * D / (dl ** 10 + D ** 10) ** 0.1
    return out


def random_field(xi, dx, L_cut, std_target=0.3, xi_min=0.01):
    """Smooth random structure xi_r of Sec. 3.3."""
    f = lowpass(xi, dx, L_cut)
    xr = f * (std_target / f.std()) + 1.0
    return sigmoid_floor(xr, xi_min)


def allen_cahn_step(xi):
    """One iteration of Eq. ACsmooth (periodic, pixel units)."""
    lap5 = 4.0 * xi - np.roll(xi, 1, axis=1) - np.roll(xi, 1, axis=0) - np.roll(xi, -1, axis=1) - np.roll(xi, -1, axis=0)
    return xi - 0.1 * ((xi ** 3 - xi) + lap5)


def two_phase_field(xi, dx, L_cut, a=0.875, n_iter=21):
    """Two-phase structure xi_p of Sec. 3.3."""
    f = lowpass(xi, dx, L_cut)
    xp = np.sign(f)
    for _ in range(n_iter):
        xp = allen_cahn_step(xp)
    return a * xp + 1.0


def modulus_field(kind, xi, dx, L_cut, E0=1.0, std_target=0.3, xi_min=0.01, a=0.875, n_iter=21):
    """E = E0 xi for kind 'random' or 'two_phase'."""
    if kind == "random":
        return E0 * random_field(xi, dx, L_cut, std_target, xi_min)
    if kind == "two_phase":
        return E0 * two_phase_field(xi, dx, L_cut, a, n_iter)
    raise ValueError(kind)
