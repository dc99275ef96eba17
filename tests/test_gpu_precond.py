"""The preconditioned BCCG option (pff_params.pf_precondition = 1): the same
bound-constrained solution as Algorithm 1 (the oracle's), in fewer iterations,
for single solves at 64^2 and 512^2, over load steps, and on the benchmark's
batched workload (the optimality conditions re-evaluated by the oracle)."""
import numpy as np
import pytest

from oracle import constitutive as cm
from oracle import evolution as ev
from oracle import phasefield
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


def _state(n, ell, seed, amp):
    E = modulus_field(n, n, n / 16.0, seed)
    z = gaussian_field(n, n, n / 32.0, seed + 1)
    phi0 = amp * (z - z.min()) / (z.max() - z.min())
    return E, phi0


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "mixed"])
@pytest.mark.parametrize("n", [64, 512])
@pytest.mark.parametrize("fracture,irr,amp", [(AT1, CRACK_SET, 0.95), (AT2, DAMAGE, 0.6), (AT1, DAMAGE, 0.0)])
def test_preconditioned_solve_reaches_the_oracle_solution(pff, prec, n, fracture, irr, amp):
    ell = 2.0 if n == 64 else 4.0
    E, phi0 = _state(n, ell, 5, amp)
    em = eps_M(1.0, 0.2, 1.0, ell)
    par = Params(fracture=fracture, split=SPECTRAL, irreversibility=irr, ell=ell, pf_tol=1e-10, pf_atol=1e-14)
    eb = np.array([[0.0, 0.0], [0.0, 1.3 * em]])
    # any strain state is a valid input of the sub-problem: a smooth synthetic eps*
    z = gaussian_field(n, n, n / 16.0, 9)
    es = 0.05 * em * np.stack([np.stack([z, 0.3 * z], -1), np.stack([0.3 * z, -z], -1)], -2)
    lam, mu = cm.lame(E, 0.2)
    psi = cm.psi_plus(eb[None, None] + es, lam, mu, SPECTRAL)
    phi_ref, v_ref, info = phasefield.solve(phi0, psi, par)
    p = pff.Problem(n, n, prec, E=E)
    p.set_model(par.fracture, par.split, par.irreversibility)
    p.set_params(nu=0.2, ell=ell, pf_tol=1e-10, pf_atol=1e-14, pf_precondition=1)
    p.set_phase_field(phi0)
    p.set_strain(to3(es), bar3(eb))
    rep = p.solve_phase_field()
    phi = p.get_fields(pff.FIELD_PHI)
    err = rel_l2(phi, phi_ref)
    assert err < (1e-9 if prec == 0 else 1e-5), (err, rep["bccg_iters"], info["iters"])
    act = p.get_fields(pff.FIELD_ACTIVE) > 0.5
    mism = int(np.sum(act != info["active"]))
    assert mism == 0 if prec == 0 else mism <= max(2, act.size // 2000)
    assert rep["bccg_iters"] < info["iters"], (rep["bccg_iters"], info["iters"])
    p.close()


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "mixed"])
def test_preconditioned_load_steps_parity_32(pff, prec):
    n, ell = 32, 2.0
    em = eps_M(1.0, 0.2, 1.0, ell)
    E = modulus_field(n, n, 4.0, 11)
    par = Params(fracture=AT1, split=SPECTRAL, irreversibility=CRACK_SET, ell=ell, mech_tol=1e-10, pf_tol=1e-10,
                 pf_atol=1e-14, d_eps_bar=((0.0, 0.0), (0.0, em / 5)))
    st = ev.State.initial(E)
    p = pff.Problem(n, n, prec, E=E, model=("AT1", "SPECTRAL", "CRACK_SET"))
    p.set_params(nu=0.2, ell=ell, mech_tol=1e-10, pf_tol=1e-10, pf_atol=1e-14, d_eps_bar=(0.0, em / 5, 0.0),
                 pf_precondition=1)
    nsteps = 40
    reps = p.step_load(nsteps)
    for k in range(nsteps):
        r = ev.load_step(st, par)
        np.testing.assert_allclose(reps[k]["eps_bar"], bar3(r["eps_bar"]), rtol=1e-5 if prec else 1e-8, atol=1e-12)
        assert reps[k]["incremented"] == r["incremented"]
    assert rel_l2(p.get_fields(pff.FIELD_PHI), st.phi) < (1e-7 if prec == 0 else 1e-4)
    p.close()


def test_preconditioned_benchmark_workload_optimality(pff):
    import torch
    from tests.test_gpu_fullsize import _check_step
    n, ell = 512, 4.0
    em = eps_M(1.0, 0.2, 1.0, ell)
    models = [(f, s, i) for f in ("AT1", "AT2") for s in ("ISOTROPIC", "SPECTRAL") for i in ("CRACK_SET", "DAMAGE")]
    stream = torch.cuda.Stream()
    E = modulus_field(n, n, 32.0, 0)
    probs = []
    for m in models:
        p = pff.Problem(n, n, pff.MIXED, stream=stream.cuda_stream, E=E, model=m,
                        params=dict(nu=0.2, ell=ell, mech_tol=1e-8, pf_tol=1e-8, d_eps_bar=(0.0, em / 20, 0.0),
                                    pf_precondition=1))
        p.set_strain(None, (0.0, 0.95 * em, 0.0))
        probs.append(p)
    b = pff.create_batch(8, sum(pff.problem_bytes(n, n, pff.MIXED) for _ in probs), stream.cuda_stream)
    pff.batch_set_group_size(b, 1)
    for p in probs:
        assert pff.batch_admit(b, p.h) is not None
    pff.batch_step(b, 8, 1)
    phi_n = [p.get_fields(pff.FIELD_PHI) for p in probs]
    out = pff.batch_step(b, 8, 1)
    for i, p in enumerate(probs):
        _check_step(pff, p, E, models[i], ell, phi_n[i], out[i][0], mech_tol=5e-6, kkt_tol=1e-4)
    pff.destroy_batch(b)
    for p in probs:
        p.close()
