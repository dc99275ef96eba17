"""Alternating minimisation (Algorithm 2) and time-dependent evolution (Algorithm 3)
through the C ABI against the FP64 oracle."""
import numpy as np
import pytest

from oracle import evolution as ev
from oracle.params import AT1, AT2, CRACK_SET, DAMAGE, SPECTRAL, Params
from paper_2203_16467_gb300.inputs import eps_M, modulus_field
from tests.helpers import bar3, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pff():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2203_16467_gb300 import pff as m
    return m


def _setup(pff, prec, par, E, evolution, eb0):
    ny, nx = E.shape
    p = pff.Problem(nx, ny, prec, E=E)
    p.set_model(par.fracture, par.split, par.irreversibility)
    p.set_params(nu=par.nu, ell=par.ell, mech_tol=par.mech_tol, pf_tol=par.pf_tol, pf_atol=par.pf_atol,
                 dphi_min=par.dphi_min, d_eps_bar=(0.0, par.d_eps_bar[1][1], 0.0), evolution=evolution)
    p.set_strain(None, (0.0, eb0, 0.0))
    return p


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "mixed"])
@pytest.mark.parametrize("fracture,irr", [(AT1, DAMAGE), (AT2, CRACK_SET)])
def test_alternating_minimisation_parity(pff, prec, fracture, irr):
    ell = 2.0
    em = eps_M(1.0, 0.2, 1.0, ell)
    par = Params(fracture=fracture, split=SPECTRAL, irreversibility=irr, ell=ell,
                 d_eps_bar=((0.0, 0.0), (0.0, em / 8)), mech_tol=1e-10, pf_tol=1e-10, pf_atol=1e-14)
    E = modulus_field(32, 32, 4.0, 3)
    st = ev.State.initial(E)
    st.eps_bar = np.array([[0.0, 0.0], [0.0, 0.9 * em]])
    p = _setup(pff, prec, par, E, pff.ALTERNATING_MIN, 0.9 * em)
    for s in range(4):
        r = ev.am_increment(st, par)
        g = p.step_load(1)[0]
        np.testing.assert_allclose(g["eps_bar"], bar3(st.eps_bar), rtol=1e-12)
        if prec == 0:
            assert g["inner_iters"] == r["inner"]
        assert abs(g["C_bar"] - r["C_bar"]) <= (1e-8 if prec == 0 else 1e-4) * abs(r["C_bar"])
    phi = p.get_fields(pff.FIELD_PHI)
    assert rel_l2(phi, st.phi) < (1e-7 if prec == 0 else 1e-4)
    p.close()


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "mixed"])
def test_time_dependent_parity(pff, prec):
    ell = 2.0
    em = eps_M(1.0, 0.2, 1.0, ell)
    par = Params(fracture=AT1, split=SPECTRAL, irreversibility=DAMAGE, ell=ell,
                 d_eps_bar=((0.0, 0.0), (0.0, em / 8)), mech_tol=1e-10, pf_tol=1e-10, pf_atol=1e-14)
    E = modulus_field(32, 32, 4.0, 3)
    st = ev.State.initial(E)
    st.eps_bar = np.array([[0.0, 0.0], [0.0, 1.2 * em]])
    p = _setup(pff, prec, par, E, pff.TIME_DEPENDENT, 1.2 * em)
    dt = 2.0 ** 16
    for n in range(12):
        r, dt = ev.td_step(st, par, dt)
        g = p.step_load(1)[0]
        assert g["dt"] == dt
        assert g["inner_iters"] == r["tries"]
        assert g["incremented"] == r["incremented"]
        np.testing.assert_allclose(g["dphi_L1"], r["dphi_L1"], rtol=1e-8 if prec == 0 else 1e-4, atol=1e-12)
    phi = p.get_fields(pff.FIELD_PHI)
    assert rel_l2(phi, st.phi) < (1e-7 if prec == 0 else 1e-4)
    p.close()
