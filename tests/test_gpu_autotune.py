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


def test_kernel_variants_agree_and_tuner_keeps_a_candidate(env):
    # the column-pass shapes (4 or 2 columns per block) and the BCCG iteration structures (three
    # or four passes) compute the same method; fields after the same load steps agree to FP32
    # rounding, and the autotuner leaves one of its eight candidate combinations set
    pff, torch = env
    n = 512
    CS, BP = pff.VARIANT_COLUMN_SHAPE, pff.VARIANT_BCCG_PASSES
    out = {}
    try:
        for v in (0, 1):
            pff.set_kernel_variant(CS, n, 1, v)
            pff.set_kernel_variant(CS, n, 3, v)
            pff.set_kernel_variant(BP, 0, 1, v)
            assert pff.get_kernel_variant(CS, n, 1) == v and pff.get_kernel_variant(CS, n, 3) == v
            assert pff.get_kernel_variant(BP, 0, 1) == v
            b, probs = _batch(pff, torch, n)
            reps = pff.batch_step(b, len(probs), 3)
            out[v] = ([p.get_fields(pff.FIELD_PHI) for p in probs], [p.get_fields(pff.FIELD_STRAIN) for p in probs],
                      reps)
            pff.destroy_batch(b)
            for p in probs:
                p.close()
        for j in range(len(MODELS)):
            (pa, ea, ra), (pb, eb, rb) = [(o[0][j], o[1][j], o[2][j]) for o in (out[0], out[1])]
            assert [r["incremented"] for r in ra] == [r["incremented"] for r in rb]
            assert np.linalg.norm(ea - eb) / np.linalg.norm(eb) < 1e-5
            assert np.linalg.norm(pa - pb) / max(np.linalg.norm(pb), 1e-30) < 1e-4
        b, probs = _batch(pff, torch, n)
        chosen, scores, reps = pff.batch_autotune_kernels(b, len(probs), steps_each=1)
        assert all(c in (0, 1) for c in chosen) and len(scores) == 8
        assert all(s > 0 for s in scores)
        assert pff.get_kernel_variant(CS, n, 1) == chosen[0] and pff.get_kernel_variant(CS, n, 3) == chosen[1]
        assert pff.get_kernel_variant(BP, 0, 1) == chosen[2]
        assert all(len(r) == 16 for r in reps)   # one round: two steps per combination
        pff.destroy_batch(b)
        for p in probs:
            p.close()
    finally:
        pff.set_kernel_variant(CS, n, 1, 0)
        pff.set_kernel_variant(CS, n, 3, 0)
        pff.set_kernel_variant(BP, 0, 1, 0)
    with pytest.raises(pff.PffError):
        pff.set_kernel_variant(CS, 256, 1, 1)
