"""Full-size checks in the launch configuration the benchmark times (batched
simulations, one stream and CUDA-graph replays per simulation): after a load
step, the oracle re-evaluates in FP64, on the GPU's own output state, the
conditions that define the two sub-problem solutions at any size:
  * mechanics (Sec. 3.1.1, A7): ||P sigma(eps, phi_n)|| <= tol ||C_0 : eps_bar||
    for the returned strain (the rescale of Algorithm 4 scales eps, and P sigma
    is homogeneous of degree one in eps);
  * phase field (Algorithm 1, Sec. 3.1.2): the update v satisfies the
    bound-constrained conditions v >= v_con, r = J v - b ~ 0 where v > v_con and
    r >= 0 (up to the tolerance) where v = v_con.
Workloads: eight 512^2 variants (the benchmark), a 2048^2 AT2 spectral grid,
and a batch of 64 256^2 AT1 spectral crack-set microstructures (four sampled)."""
import numpy as np
import pytest

from oracle import constitutive as cm
from oracle import fourier, mechanics, phasefield
from oracle.params import AT1, AT2, CRACK_SET, DAMAGE, ISOTROPIC, SPECTRAL, Params
from paper_2203_16467_gb300.inputs import eps_M, modulus_field
from tests.helpers import bar22, from3

pytestmark = pytest.mark.gpu

_NAMES = {"AT1": AT1, "AT2": AT2, "ISOTROPIC": ISOTROPIC, "SPECTRAL": SPECTRAL, "CRACK_SET": CRACK_SET,
          "DAMAGE": DAMAGE}


@pytest.fixture(scope="module")
def env():
    import __graft_entry__
    __graft_entry__.build()
    import torch
    from paper_2203_16467_gb300 import pff
    return pff, torch


def _check_step(pff, p, E, model, ell, phi_n, rep, mech_tol, kkt_tol):
    par = Params(fracture=_NAMES[model[0]], split=_NAMES[model[1]], irreversibility=_NAMES[model[2]], ell=ell,
                 nu=0.2)
    eb = bar22(rep["eps_bar"])
    es = from3(p.get_fields(pff.FIELD_EPS_STAR))
    phi_new = p.get_fields(pff.FIELD_PHI)
    v = p.get_fields(pff.FIELD_UPDATE)
    # mechanics: the Newton stopping test at phi_n
    R = mechanics.residual(es, eb, phi_n, E, par)
    rel = np.sqrt(np.sum(R * R)) / mechanics.reference_norm(eb, E, par)
    assert rel < mech_tol, ("mechanics residual", rel)
    # phase field: bound-constrained conditions of the update
    lam, mu = cm.lame(E, par.nu)
    psi = cm.psi_plus(eb[None, None] + es, lam, mu, par.split)
    b = phasefield.minus_F_phi(phi_n, psi, par)
    vcon = phasefield.phi_con(phi_n, par) - phi_n
    r = phasefield.J_apply(v, psi, par) - b
    r0 = phasefield.J_apply(np.maximum(0.0, vcon), psi, par) - b
    scale = max(np.sqrt(np.sum(r0 * r0)), 1e-30)
    assert np.all(v >= vcon - 1e-6), ("bound", float((vcon - v).max()))
    bound = v <= vcon + 1e-6 * max(1.0, float(np.abs(vcon).max()))
    free = ~bound
    assert np.sqrt(np.sum(r[free] ** 2)) / scale < kkt_tol, ("free residual", np.sqrt(np.sum(r[free] ** 2)) / scale)
    if bound.any():
        assert r[bound].min() > -kkt_tol * scale, ("bound multiplier", float(r[bound].min()) / scale)
    np.testing.assert_allclose(phi_new, phi_n + v, atol=2e-7)
    assert rep["bccg_iters"] > 0 and rep["mech_cg_iters"] + rep["newton_iters"] > 0


def _run_batch(pff, torch, n, lc, ell, models, seeds, preload, steps=1, sample=None):
    stream = torch.cuda.Stream()
    em = eps_M(1.0, 0.2, 1.0, ell)
    probs, Es = [], []
    for m, s in zip(models, seeds):
        E = modulus_field(n, n, lc, s)
        p = pff.Problem(n, n, pff.MIXED, stream=stream.cuda_stream, E=E, model=m,
                        params=dict(nu=0.2, ell=ell, mech_tol=1e-8, pf_tol=1e-8, d_eps_bar=(0.0, em / 20, 0.0)))
        p.set_strain(None, (0.0, preload * em, 0.0))
        probs.append(p)
        Es.append(E)
    b = pff.create_batch(len(probs), sum(pff.problem_bytes(n, n, pff.MIXED) for _ in probs), stream.cuda_stream)
    for p in probs:
        assert pff.batch_admit(b, p.h) is not None
    for _ in range(steps - 1):
        pff.batch_step(b, len(probs), 1)
    idx = range(len(probs)) if sample is None else sample
    phi_n = {i: probs[i].get_fields(pff.FIELD_PHI) for i in idx}
    out = pff.batch_step(b, len(probs), 1)
    result = [(probs[i], Es[i], models[i], phi_n[i], out[i][0]) for i in idx]
    return b, probs, result


def test_benchmark_workload_512(env):
    pff, torch = env
    models = [(f, s, i) for f in ("AT1", "AT2") for s in ("ISOTROPIC", "SPECTRAL") for i in ("CRACK_SET", "DAMAGE")]
    b, probs, res = _run_batch(pff, torch, 512, 32.0, 4.0, models, [0] * 8, 0.95, steps=2)
    for p, E, m, phi_n, rep in res:
        _check_step(pff, p, E, m, 4.0, phi_n, rep, mech_tol=5e-6, kkt_tol=1e-4)
    pff.destroy_batch(b)
    for p in probs:
        p.close()


def test_single_2048_grid(env):
    pff, torch = env
    b, probs, res = _run_batch(pff, torch, 2048, 64.0, 2.0, [("AT2", "SPECTRAL", "CRACK_SET")], [3], 0.97)
    for p, E, m, phi_n, rep in res:
        _check_step(pff, p, E, m, 2.0, phi_n, rep, mech_tol=5e-6, kkt_tol=1e-4)
    pff.destroy_batch(b)
    for p in probs:
        p.close()


def test_batch_of_64_at_256(env):
    pff, torch = env
    models = [("AT1", "SPECTRAL", "CRACK_SET")] * 64
    b, probs, res = _run_batch(pff, torch, 256, 16.0, 2.0, models, list(range(64)), 1.0, sample=[0, 21, 42, 63])
    for p, E, m, phi_n, rep in res:
        _check_step(pff, p, E, m, 2.0, phi_n, rep, mech_tol=5e-6, kkt_tol=1e-4)
    pff.destroy_batch(b)
    for p in probs:
        p.close()
