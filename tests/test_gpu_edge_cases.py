"""Degenerate and edge cases of the load step on the GPU: zero macroscopic strain,
a homogeneous modulus (the exact solution eps* = 0 of Sec. 3.1.1), a line of
fully broken pixels (phi = 1, where h(phi) = 0), and extreme aspect ratios
against the oracle (16 x 512 and 512 x 16 grids, several load steps)."""
import numpy as np
import pytest

from oracle import evolution as ev
from oracle.params import AT1, AT2, CRACK_SET, DAMAGE, ISOTROPIC, SPECTRAL, Params
from paper_2203_16467_gb300.inputs import eps_M, modulus_field
from tests.helpers import bar3, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pff():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2203_16467_gb300 import pff as m
    return m


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "mixed"])
def test_zero_load_is_a_fixed_point(pff, prec):
    n = 64
    p = pff.Problem(n, n, prec, E=modulus_field(n, n, 8.0, 1), model=("AT1", "SPECTRAL", "CRACK_SET"))
    p.set_params(ell=2.0, d_eps_bar=(0.0, 0.0, 0.0))
    reps = p.step_load(2)
    assert len(reps) == 2
    for r in reps:
        assert np.all(np.isfinite(r["eps_bar"])) and r["eps_bar"] == [0.0, 0.0, 0.0]
        assert r["bccg_iters"] == 0 and not r["rescaled"]
    assert np.all(p.get_fields(pff.FIELD_EPS_STAR) == 0.0)
    assert np.all(p.get_fields(pff.FIELD_PHI) == 0.0)
    p.close()


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "mixed"])
@pytest.mark.parametrize("split", ["ISOTROPIC", "SPECTRAL"])
def test_homogeneous_modulus_has_no_fluctuation(pff, prec, split):
    n = 128
    em = eps_M(1.0, 0.2, 1.0, 2.0)
    p = pff.Problem(n, n, prec, E=np.full((n, n), 1.7), model=("AT2", split, "DAMAGE"))
    p.set_params(ell=2.0)
    p.set_strain(None, (0.3 * em, 0.7 * em, 0.2 * em))
    p.solve_mechanics()
    es = p.get_fields(pff.FIELD_EPS_STAR)
    assert np.abs(es).max() < (1e-12 if prec == 0 else 1e-7) * em
    p.close()


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "mixed"])
def test_broken_line_stays_finite_and_irreversible(pff, prec):
    # a segment crack puts phi = 1 (h = 0, zero stiffness) on a line of pixels
    n = 64
    em = eps_M(1.0, 0.2, 1.0, 2.0)
    p = pff.Problem(n, n, prec, E=modulus_field(n, n, 8.0, 2), model=("AT1", "SPECTRAL", "CRACK_SET"))
    p.set_params(ell=2.0, d_eps_bar=(0.0, em / 10, 0.0))
    p.init_crack(pff.IC_PHASE_FIELD, pff.CRACK_SEGMENT, 32.0, 32.0, 24.0)
    phi0 = p.get_fields(pff.FIELD_PHI)
    assert phi0.max() == 1.0
    p.set_strain(None, (0.0, 0.5 * em, 0.0))
    reps = p.step_load(5)
    phi = p.get_fields(pff.FIELD_PHI)
    assert all(np.all(np.isfinite(r["sig_bar"])) for r in reps)
    assert np.all(np.isfinite(p.get_fields(pff.FIELD_STRESS)))
    crack_set = phi0 >= 0.9
    assert np.all(phi[crack_set] >= phi0[crack_set] - 1e-7)     # irreversibility within the crack set
    assert phi.min() >= -1e-7 and phi.max() <= 1.0 + 1e-6
    p.close()


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "mixed"])
@pytest.mark.parametrize("ny,nx", [(16, 512), (512, 16)])
def test_extreme_aspect_ratio_load_steps(pff, prec, ny, nx):
    ell = 2.0
    em = eps_M(1.0, 0.2, 1.0, ell)
    E = modulus_field(ny, nx, 4.0, 7)
    par = Params(fracture=AT2, split=SPECTRAL, irreversibility=DAMAGE, ell=ell, mech_tol=1e-10, pf_tol=1e-10,
                 pf_atol=1e-14, d_eps_bar=((0.0, 0.0), (0.0, em / 5)))
    st = ev.State.initial(E)
    p = pff.Problem(nx, ny, prec, E=E, model=("AT2", "SPECTRAL", "DAMAGE"))
    p.set_params(nu=par.nu, ell=ell, mech_tol=par.mech_tol, pf_tol=par.pf_tol, pf_atol=par.pf_atol,
                 d_eps_bar=(0.0, em / 5, 0.0))
    nsteps = 12
    reps = p.step_load(nsteps)
    for k in range(nsteps):
        r = ev.load_step(st, par)
        np.testing.assert_allclose(reps[k]["eps_bar"], bar3(r["eps_bar"]), rtol=1e-5 if prec else 1e-9, atol=1e-12)
        assert reps[k]["incremented"] == r["incremented"]
    assert rel_l2(p.get_fields(pff.FIELD_PHI), st.phi) < (1e-7 if prec == 0 else 1e-4)
    p.close()
