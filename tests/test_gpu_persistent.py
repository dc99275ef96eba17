"""The persistent BCCG solve (one cooperative launch per phase-field sub-problem
of a single FP32 512 x 512 problem) against the oracle on the same input
state, and against the per-phase kernels over several load steps.  Its dot
products are summed in a different (fixed) order than the per-phase kernels',
so the comparison between the two GPU paths is within the mixed-precision
tolerance, not bitwise."""
import ctypes

import numpy as np
import pytest

from oracle import constitutive as cm
from oracle import mechanics, phasefield
from oracle.params import AT1, AT2, CRACK_SET, DAMAGE, SPECTRAL, Params
from paper_2203_16467_gb300.inputs import eps_M, gaussian_field, modulus_field
from tests.helpers import bar3, rel_l2, to3

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pff():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2203_16467_gb300 import pff as m
    return m


@pytest.mark.parametrize("fracture,irr", [(AT1, CRACK_SET), (AT2, DAMAGE)])
def test_persistent_phase_field_solve_parity_512(pff, fracture, irr):
    n, ell = 512, 4.0
    E = modulus_field(n, n, 32.0, 5)
    z = gaussian_field(n, n, 16.0, 6)
    phi0 = 0.95 * (z - z.min()) / (z.max() - z.min())
    em = eps_M(1.0, 0.2, 1.0, ell)
    par = Params(fracture=fracture, split=SPECTRAL, irreversibility=irr, ell=ell, mech_tol=1e-10, pf_tol=1e-10,
                 pf_atol=1e-14)
    eb = np.array([[0.0, 0.0], [0.0, 1.3 * em]])
    # a strain state that is not the mechanical equilibrium is a valid input of the sub-problem
    es = 0.05 * em * np.stack([np.stack([z, 0.3 * z], -1), np.stack([0.3 * z, -z], -1)], -2)
    lam, mu = cm.lame(E, 0.2)
    psi = cm.psi_plus(eb[None, None] + es, lam, mu, SPECTRAL)
    phi_ref, v_ref, info = phasefield.solve(phi0, psi, par)
    for persistent in (True, False):
        pff.set_persistent(persistent)
        p = pff.Problem(n, n, pff.MIXED, E=E)
        p.set_model(par.fracture, par.split, par.irreversibility)
        p.set_params(nu=0.2, ell=ell, pf_tol=1e-10, pf_atol=1e-14)
        p.set_phase_field(phi0)
        p.set_strain(to3(es), bar3(eb))
        rep = p.solve_phase_field()
        phi = p.get_fields(pff.FIELD_PHI)
        err = rel_l2(phi, phi_ref)
        assert err < 1e-5, (persistent, err, rep["bccg_iters"], info["iters"])
        act = p.get_fields(pff.FIELD_ACTIVE) > 0.5
        assert int(np.sum(act != info["active"])) <= act.size // 2000
        assert phi.min() >= -1e-12
        p.close()
    pff.set_persistent(False)


@pytest.mark.parametrize("model", [("AT1", "SPECTRAL", "CRACK_SET"), ("AT2", "ISOTROPIC", "DAMAGE")])
def test_persistent_load_steps_match_per_phase_kernels(pff, model):
    import torch
    n, ell = 512, 4.0
    em = eps_M(1.0, 0.2, 1.0, ell)
    E = modulus_field(n, n, 32.0, 0)
    out = {}
    try:
        for persistent in (True, False):
            pff.set_persistent(persistent)
            stream = torch.cuda.Stream()
            p = pff.Problem(n, n, pff.MIXED, stream=stream.cuda_stream, E=E, model=model,
                            params=dict(nu=0.2, ell=ell, mech_tol=1e-8, pf_tol=1e-8, d_eps_bar=(0.0, em / 20, 0.0)))
            p.set_strain(None, (0.0, 1.0 * em, 0.0))
            reps = p.step_load(3)
            out[persistent] = (reps, p.get_fields(pff.FIELD_PHI))
            p.close()
    finally:
        pff.set_persistent(False)
    (ra, pa), (rb, pb) = out[True], out[False]
    assert sum(r["bccg_iters"] for r in ra) > 0
    scale = max(np.linalg.norm(pb), 1e-30)
    # the persistent kernel runs Algorithm 1 in four passes (alpha from p.Jp summed in real
    # space), the default path in three (alpha via Parseval): the FP32 roundings differ, and
    # over three load steps the two paths stay within 1e-4 (each solve is held to 1e-5 of
    # the oracle by test_persistent_phase_field_solve_parity_512 and tests/test_gpu_solvers.py)
    assert np.linalg.norm(pa - pb) / scale < 1e-4
    for x, y in zip(ra, rb):
        # FP32 solves stop at the rounding level of J v - b, where the iteration at which
        # the stopping tests fire depends on the summation order of the dot products
        assert abs(x["bccg_iters"] - y["bccg_iters"]) <= max(8, y["bccg_iters"] // 2), (x["bccg_iters"], y["bccg_iters"])
        np.testing.assert_allclose(x["eps_bar"], y["eps_bar"], rtol=1e-5, atol=1e-12)


def test_persistent_barrier_timeout_returns_status_and_handle_stays_usable(pff):
    # A one-cycle wait limit makes the first grid barrier of the persistent solve time out
    # (the first block to arrive is never released within it): the kernel sets the abort
    # flag, every block returns, and the call reports PFF_ERR_BARRIER_TIMEOUT with the
    # phase field unchanged.  With the default limit the same handle then solves normally.
    n, ell = 512, 4.0
    E = modulus_field(n, n, 32.0, 5)
    z = gaussian_field(n, n, 16.0, 6)
    phi0 = 0.5 * (z - z.min()) / (z.max() - z.min())
    em = eps_M(1.0, 0.2, 1.0, ell)
    eb = (0.0, 1.3 * em, 0.0)
    try:
        pff.set_persistent(True)
        p = pff.Problem(n, n, pff.MIXED, E=E, model=("AT1", "SPECTRAL", "CRACK_SET"),
                        params=dict(nu=0.2, ell=ell, pf_tol=1e-8))
        p.set_phase_field(phi0)
        p.set_strain(None, eb)
        pff.set_barrier_spin_limit(1)
        rep = pff.StepReport()
        rc = pff.lib.pff_solve_phase_field(p.h, ctypes.byref(rep))
        assert rc == pff.ERR_BARRIER_TIMEOUT, rc
        assert "timed out" in pff.lib.pff_last_error(p.h).decode()
        np.testing.assert_array_equal(p.get_fields(pff.FIELD_PHI), phi0.astype(np.float32).astype(np.float64))
        pff.set_barrier_spin_limit(0)
        rep_ok = p.solve_phase_field()
        phi_a = p.get_fields(pff.FIELD_PHI)
        p.close()
        pff.set_persistent(False)
        q = pff.Problem(n, n, pff.MIXED, E=E, model=("AT1", "SPECTRAL", "CRACK_SET"),
                        params=dict(nu=0.2, ell=ell, pf_tol=1e-8))
        q.set_phase_field(phi0)
        q.set_strain(None, eb)
        q.solve_phase_field()
        phi_b = q.get_fields(pff.FIELD_PHI)
        q.close()
    finally:
        pff.set_barrier_spin_limit(0)
        pff.set_persistent(False)
    assert rep_ok["bccg_iters"] > 0
    assert np.linalg.norm(phi_a - phi_b) / np.linalg.norm(phi_b) < 1e-5
