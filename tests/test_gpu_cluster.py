"""The cluster mechanics solve of FP32 512 x 512 problems (one 16-CTA thread-block
cluster per problem, the Newton-CG solve of Sec. 3.1.1 in one launch) against the
per-kernel path (three kernels per CG iteration) and against the FP64 oracle."""
import numpy as np
import pytest

from oracle import constitutive as cm
from oracle import mechanics
from oracle.params import ISOTROPIC, SPECTRAL, SPECTRAL_STRESSFREE, SPECTRAL_VOLDEV, VOLDEV, Params
from paper_2203_16467_gb300.inputs import eps_M, gaussian_field, modulus_field
from tests.helpers import bar3, rel_l2, tensor_rel_l2, to3

pytestmark = pytest.mark.gpu
N = 512


@pytest.fixture(scope="module")
def pff():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2203_16467_gb300 import pff as m
    yield m
    m.set_cluster_mechanics(False)


def _state(seed=3, amp=0.9):
    E = modulus_field(N, N, 32.0, seed)
    z = gaussian_field(N, N, 16.0, seed + 1)
    phi = amp * (z - z.min()) / (z.max() - z.min())
    return E, phi


def _solve(pff, cluster, split, E, phi, eb, tol):
    pff.set_cluster_mechanics(cluster)
    p = pff.Problem(N, N, pff.MIXED, E=E)
    p.set_model(1, split, 0)
    p.set_params(nu=0.2, mech_tol=tol, mech_cg_rtol=1e-4)
    p.set_phase_field(phi)
    p.set_strain(None, bar3(eb))
    rep = p.solve_mechanics()
    eps = p.get_fields(pff.FIELD_STRAIN)
    p.close()
    return eps, rep


@pytest.mark.parametrize("split", [ISOTROPIC, SPECTRAL, SPECTRAL_STRESSFREE, VOLDEV, SPECTRAL_VOLDEV])
def test_cluster_mechanics_matches_per_kernel_path(pff, split):
    E, phi = _state()
    eb = np.array([[0.002, 0.001], [0.001, 0.01]])
    a, ra = _solve(pff, True, split, E, phi, eb, 1e-6)
    b, rb = _solve(pff, False, split, E, phi, eb, 1e-6)
    assert ra["mech_cg_iters"] > 0 and ra["status"] == 0
    assert tensor_rel_l2(a, b) < 1e-5, (tensor_rel_l2(a, b), ra["mech_cg_iters"], rb["mech_cg_iters"])
    # same stopping rules: the iteration counts agree up to the rounding of the step lengths
    assert abs(ra["mech_cg_iters"] - rb["mech_cg_iters"]) <= max(2, rb["mech_cg_iters"] // 20)
    assert ra["newton_iters"] == rb["newton_iters"]


@pytest.mark.parametrize("split", [ISOTROPIC, SPECTRAL])
def test_cluster_mechanics_matches_oracle(pff, split):
    # (h(phi) >= 0.16: the mixed path's mechanics floor of 1e-6 then gives errors below 1e-5)
    E, phi = _state(7, amp=0.6)
    eb = np.array([[0.0, 0.0], [0.0, 0.01]])
    par = Params(split=split, mech_tol=1e-8, mech_cg_rtol=1e-4)
    es_ref, info = mechanics.solve(np.zeros((N, N, 2, 2)), eb, phi, E, par)
    eps, rep = _solve(pff, True, split, E, phi, eb, 1e-6)
    err = tensor_rel_l2(eps, to3(eb[None, None] + es_ref))
    assert err < 1e-5, (err, rep["mech_cg_iters"], info)


def test_cluster_load_steps_match_per_kernel_path(pff):
    # eight variants in one batch, three load steps from 0.95 eps_M, both mechanics paths
    import torch
    ell = 4.0
    em = eps_M(1.0, 0.2, 1.0, ell)
    E = modulus_field(N, N, 32.0, 0)
    variants = [(f, s, i) for f in ("AT1", "AT2") for s in ("ISOTROPIC", "SPECTRAL") for i in ("CRACK_SET", "DAMAGE")]
    out = {}
    for cluster in (True, False):
        pff.set_cluster_mechanics(cluster)
        stream = torch.cuda.Stream()
        probs = []
        for v in variants:
            p = pff.Problem(N, N, pff.MIXED, stream=stream.cuda_stream, E=E, model=v,
                            params=dict(nu=0.2, ell=ell, mech_tol=1e-8, pf_tol=1e-8, d_eps_bar=(0.0, em / 20, 0.0)))
            p.set_strain(None, (0.0, 0.95 * em, 0.0))
            probs.append(p)
        b = pff.create_batch(len(probs), sum(pff.problem_bytes(N, N, pff.MIXED) for _ in probs), stream.cuda_stream)
        pff.batch_set_group_size(b, 0)
        for p in probs:
            pff.batch_admit(b, p.h)
        reps = pff.batch_step(b, len(probs), 3)
        out[cluster] = (reps, [p.get_fields(pff.FIELD_PHI) for p in probs],
                        [p.get_fields(pff.FIELD_STRAIN) for p in probs])
        pff.destroy_batch(b)
        for p in probs:
            p.close()
    pff.set_cluster_mechanics(False)
    (ra, pa, ea), (rb, pb, eb_) = out[True], out[False]
    for j in range(len(variants)):
        assert [r["incremented"] for r in ra[j]] == [r["incremented"] for r in rb[j]]
        for x, y in zip(ra[j], rb[j]):
            np.testing.assert_allclose(x["eps_bar"], y["eps_bar"], rtol=1e-5, atol=1e-12)
        assert tensor_rel_l2(ea[j], eb_[j]) < 1e-5
        sc = max(np.linalg.norm(pb[j]), 1e-30)
        assert np.linalg.norm(pa[j] - pb[j]) / sc < 1e-4, (variants[j], np.linalg.norm(pa[j] - pb[j]) / sc)
