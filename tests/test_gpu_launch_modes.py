"""Launch modes give bit-identical results: programmatic dependent launch on or
off, CUDA-graph replay with or without conditional nodes for the explicit BCCG
residual chain, or direct launches (every reduction has a fixed
summation order, so the mode must not change a single bit), on a non-square
grid (64 x 128)."""
import numpy as np
import pytest

from paper_2203_16467_gb300.inputs import eps_M, modulus_field

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import __graft_entry__
    __graft_entry__.build()
    import torch
    from paper_2203_16467_gb300 import pff
    return pff, torch


def _run(pff, torch, prec, model, pdl, graphs, steps=4):
    pff.set_pdl(pdl)
    pff.set_graphs(graphs)
    stream = torch.cuda.Stream()
    E = modulus_field(64, 128, 8.0, 11)
    em = eps_M(1.0, 0.2, 1.0, 2.0)
    p = pff.Problem(128, 64, prec, stream=stream.cuda_stream, E=E, model=model,
                    params=dict(nu=0.2, ell=2.0, mech_tol=1e-8, pf_tol=1e-8, d_eps_bar=(0.0, em / 20, 0.0)))
    p.set_strain(None, (0.0, 1.02 * em, 0.0))
    reps = p.step_load(steps)
    out = {f: p.get_fields(f) for f in (pff.FIELD_PHI, pff.FIELD_STRAIN)}
    p.close()
    return reps, out


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "mixed"])
@pytest.mark.parametrize("model", [("AT1", "SPECTRAL", "CRACK_SET"), ("AT2", "ISOTROPIC", "DAMAGE")])
def test_pdl_and_graphs_do_not_change_results(env, prec, model):
    pff, torch = env
    try:
        base = _run(pff, torch, prec, model, pdl=False, graphs=0)
        for pdl, graphs in ((True, 0), (True, 1), (False, 1), (False, 2)):
            reps, out = _run(pff, torch, prec, model, pdl, graphs)
            assert [r["bccg_iters"] for r in reps] == [r["bccg_iters"] for r in base[0]], (pdl, graphs)
            assert [r["mech_cg_iters"] for r in reps] == [r["mech_cg_iters"] for r in base[0]], (pdl, graphs)
            for f, a in out.items():
                np.testing.assert_array_equal(a, base[1][f], err_msg=f"pdl={pdl} graphs={graphs} field={f}")
        assert any(r["bccg_iters"] > 0 for r in base[0])
    finally:
        pff.set_pdl(True)
        pff.set_graphs(1)
