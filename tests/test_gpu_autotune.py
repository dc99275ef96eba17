"""The batch grouping autotuner: it runs ordinary load steps under each candidate
grouping, keeps one of the candidates, and leaves every simulation exactly where
the same number of load steps with a fixed grouping would (the grouping changes
no simulation's arithmetic)."""
import numpy as np
import pytest

from paper_2203_16467_gb300.inputs import eps_M, modulus_field

pytestmark = pytest.mark.gpu

MODELS = [("AT1", "SPECTRAL", "CRACK_SET"), ("AT2", "ISOTROPIC", "DAMAGE"), ("AT1", "ISOTROPIC", "DAMAGE"),
          ("AT2", "SPECTRAL", "CRACK_SET")]


@pytest.fixture(scope="module")
def env():
    import __graft_entry__
    __graft_entry__.build()
    import torch
    from paper_2203_16467_gb300 import pff
    return pff, torch


def _batch(pff, torch, n=64):
    stream = torch.cuda.Stream()
    em = eps_M(1.0, 0.2, 1.0, 2.0)
    probs = []
    for k, m in enumerate(MODELS):
        p = pff.Problem(n, n, pff.MIXED, stream=stream.cuda_stream, E=modulus_field(n, n, 8.0, k), model=m,
                        params=dict(nu=0.2, ell=2.0, mech_tol=1e-8, pf_tol=1e-8, d_eps_bar=(0.0, em / 10, 0.0)))
        p.set_strain(None, (0.0, 0.9 * em, 0.0))
        probs.append(p)
    b = pff.create_batch(len(probs), sum(pff.problem_bytes(n, n, pff.MIXED) for _ in probs), stream.cuda_stream)
    for p in probs:
        assert pff.batch_admit(b, p.h) is not None
    return b, probs


def test_autotune_picks_a_candidate_and_changes_no_result(env):
    pff, torch = env
    cands = (1, 2, 4)
    b, probs = _batch(pff, torch)
    chosen, reps = pff.batch_autotune(b, len(probs), cands, steps_each=1)
    assert chosen in cands
    assert all(len(r) == 2 * len(cands) for r in reps)
    tuned = [p.get_fields(pff.FIELD_PHI) for p in probs]
    more = pff.batch_step(b, len(probs), 1)            # the batch keeps working with the chosen grouping
    assert all(len(r) == 1 for r in more)
    pff.destroy_batch(b)
    for p in probs:
        p.close()
    b, probs = _batch(pff, torch)
    pff.batch_set_group_size(b, 1)
    fixed = pff.batch_step(b, len(probs), 2 * len(cands))
    for i, p in enumerate(probs):
        np.testing.assert_array_equal(p.get_fields(pff.FIELD_PHI), tuned[i])
        assert [r["bccg_iters"] for r in fixed[i]] == [r["bccg_iters"] for r in reps[i]]
    pff.destroy_batch(b)
    for p in probs:
        p.close()
