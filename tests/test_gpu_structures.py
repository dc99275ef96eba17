"""GPU initial conditions and microstructure generators (Sec. 3.3, Sec. 4.1.1,
Sec. 4.2.2) against the oracle on the same inputs, element by element, on small
non-square grids and at the 512^2 size of the paper's structures; then the
homogenised stiffnesses the paper prints, computed end to end on the GPU."""
import numpy as np
import pytest

from oracle import structures as st
from paper_2203_16467_gb300.inputs import white_noise

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pff():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2203_16467_gb300 import pff as m
    return m


def _problem(pff, nx, ny, prec, dx=1.0, ell=2.0):
    p = pff.Problem(nx, ny, prec, E=np.ones((ny, nx)))
    p.set_params(dx=dx, ell=ell, nu=0.2)
    return p


def _tol(prec, scale=1.0):
    return dict(rtol=0, atol=(1e-13 if prec == 0 else 2e-7) * scale)


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "mixed"])
@pytest.mark.parametrize("shape", ["segment", "edge"])
@pytest.mark.parametrize("ny,nx,dx,ell,xc,yc,length", [(64, 128, 0.5, 1.5, 20.3, 31.9, 30.0),
                                                       (512, 512, 1.0, 5.12, 256.0, 256.0, 256.0),
                                                       (64, 64, 1.0, 3.0, 1.0, 62.5, 0.0)])
def test_crack_initial_condition_parity(pff, prec, shape, ny, nx, dx, ell, xc, yc, length):
    p = _problem(pff, nx, ny, prec, dx, ell)
    code = pff.CRACK_SEGMENT if shape == "segment" else pff.CRACK_EDGE
    p.init_crack(pff.IC_PHASE_FIELD, code, xc, yc, length)
    ref = st.phi_init(ny, nx, dx, ell, xc, yc, length, mode=shape)
    np.testing.assert_allclose(p.get_fields(pff.FIELD_PHI), ref, **_tol(prec))
    p.init_crack(pff.IC_MODULUS, code, xc, yc, length, 2.5)
    ref = st.modulus_with_crack(ny, nx, dx, ell, xc, yc, length, 2.5, mode=shape)
    np.testing.assert_allclose(p.get_fields(pff.FIELD_MODULUS), ref, **_tol(prec, 2.5))
    p.close()


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "mixed"])
@pytest.mark.parametrize("kind", ["random", "two_phase"])
@pytest.mark.parametrize("ny,nx,dx,L_cut", [(64, 128, 0.5, 5.3), (512, 512, 1.0, 30.72), (32, 32, 1.0, 4.0)])
def test_microstructure_generator_parity(pff, prec, kind, ny, nx, dx, L_cut):
    xi = white_noise(ny, nx, nx + 7 * ny)
    p = _problem(pff, nx, ny, prec, dx)
    code = pff.MICRO_RANDOM if kind == "random" else pff.MICRO_TWO_PHASE
    p.generate_modulus(xi, code, L_cut=L_cut, E0=1.7)
    got = p.get_fields(pff.FIELD_MODULUS)
    ref = st.modulus_field(kind, xi, dx, L_cut, E0=1.7)
    # the two-phase sign decision: no filtered value sits within rounding of zero here
    f = st.lowpass(xi, dx, L_cut)
    assert np.abs(f).min() > 1e-10 * np.abs(f).max()
    np.testing.assert_allclose(got, ref, **_tol(prec, 1.7 * (1e3 if kind == "two_phase" and prec == 0 else 10.0)))
    p.close()


def test_generator_rejects_bad_parameters(pff):
    p = _problem(pff, 32, 32, pff.MIXED)
    xi = white_noise(32, 32, 0)
    for kw in (dict(L_cut=0.0), dict(E0=-1.0), dict(a=1.5, kind=pff.MICRO_TWO_PHASE), dict(xi_min=2.0)):
        kind = kw.pop("kind", pff.MICRO_RANDOM)
        with pytest.raises(pff.PffError):
            p.generate_modulus(xi, kind, **kw)
    with pytest.raises(pff.PffError):
        p.init_crack(7, pff.CRACK_EDGE, 1.0, 1.0, 3.0)
    p.close()


def _cbar(pff, p, E0=1.0):
    em = 1e-3
    p.set_strain(np.zeros(3 * 512 * 512), (0.0, em, 0.0))
    p.solve_mechanics()
    sig = p.get_fields(pff.FIELD_STRESS)
    return sig[1].mean() / em / (10.0 / 9.0 * E0)     # (lambda + 2 mu) = 10/9 E0 at nu = 0.2


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "mixed"])
def test_paper_stiffnesses_on_gpu(pff, prec):
    # Sec. 4.1.1 / 4.1.2 print C-bar_2222 in sigma_M/eps_M for 100 ell domains at N = 511:
    # edge crack of 50 ell 0.65, small void ~1, smooth random 0.94, two-phase 0.42-0.44
    n, ell = 512, 5.12
    p = pff.Problem(n, n, prec, E=np.ones((n, n)), model=("AT1", "ISOTROPIC", "DAMAGE"))
    p.set_params(ell=ell, nu=0.2, mech_tol=1e-7)
    p.init_crack(pff.IC_PHASE_FIELD, pff.CRACK_EDGE, n / 2, n / 2, 50 * ell)
    assert abs(_cbar(pff, p) - 0.65) < 0.03
    p.init_crack(pff.IC_PHASE_FIELD, pff.CRACK_SEGMENT, n / 2, n / 2, 0.0)
    assert _cbar(pff, p) > 0.99
    p.set_phase_field(np.zeros((n, n)))
    xi = white_noise(n, n, 0)
    p.generate_modulus(xi, pff.MICRO_RANDOM, L_cut=6 * ell)
    assert abs(_cbar(pff, p) - 0.94) < 0.03
    p.generate_modulus(xi, pff.MICRO_TWO_PHASE, L_cut=6 * ell)
    assert abs(_cbar(pff, p) - 0.43) < 0.03
    p.close()
