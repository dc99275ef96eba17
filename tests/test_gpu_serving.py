"""Continuous batching: admission by HBM budget, and each simulation's result is the
same alone and in a mix of other sizes and model variants that arrive while it runs."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def srv():
    import __graft_entry__
    __graft_entry__.build()
    import torch
    from paper_2203_16467_gb300 import pff, serving
    return pff, serving, torch


def _req(serving, pff, rid, n, fracture, split, irr, seed, arrival=0.0, prec=None, steps=25):
    return serving.Request(rid=rid, n=n, fracture=fracture, split=split, irreversibility=irr, seed=seed,
                           lc=8.0, ell=2.0, precision=pff.MIXED if prec is None else prec, max_steps=steps,
                           preload=0.97, arrival=arrival)


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "mixed"])
def test_result_same_alone_and_in_mix(srv, prec):
    pff, serving, torch = srv
    stream = torch.cuda.Stream()
    budget = 4 << 30
    a = lambda arr: _req(serving, pff, 0, 64, "AT1", "SPECTRAL", "CRACK_SET", 7, arrival=arr, prec=prec)
    alone = serving.Server(budget, max_slots=8, stream=stream.cuda_stream, keep_fields=True)
    alone.submit(a(0.0))
    alone.run()
    ref = alone.done[0]
    alone.close()
    mix = serving.Server(budget, max_slots=8, stream=stream.cuda_stream, keep_fields=True)
    mix.submit(_req(serving, pff, 1, 128, "AT2", "ISOTROPIC", "DAMAGE", 3, prec=prec))
    mix.submit(_req(serving, pff, 2, 64, "AT1", "ISOTROPIC", "DAMAGE", 4, prec=prec))
    mix.submit(_req(serving, pff, 3, 256, "AT2", "SPECTRAL", "CRACK_SET", 5, prec=prec, steps=10))
    mix.submit(a(0.0))
    mix.tick()                              # 0 is admitted with the others ...
    mix.submit(_req(serving, pff, 4, 64, "AT2", "SPECTRAL", "DAMAGE", 6, prec=prec))   # ... 4 arrives later
    mix.run()
    got = mix.done[0]
    mix.close()
    assert got["steps"] == ref["steps"]
    tol = 1e-12 if prec == 0 else 1e-6
    np.testing.assert_allclose(got["phi"], ref["phi"], atol=tol, rtol=0)
    for r1, r2 in zip(got["reports"], ref["reports"]):
        np.testing.assert_allclose(r1["eps_bar"], r2["eps_bar"], rtol=tol, atol=1e-15)
        assert r1["bccg_iters"] == r2["bccg_iters"] and r1["mech_cg_iters"] == r2["mech_cg_iters"]


def test_admission_respects_hbm_budget(srv):
    pff, serving, torch = srv
    one = pff.problem_bytes(128, 128, pff.MIXED)
    server = serving.Server(int(2.5 * one), max_slots=8)
    for i in range(5):
        server.submit(_req(serving, pff, i, 128, "AT1", "SPECTRAL", "CRACK_SET", i, steps=3))
    peak = 0
    while server.queue or server.active:
        server.tick()
        peak = max(peak, len(server.active))
    st = server.stats()
    server.close()
    assert peak == 2
    assert st["completed"] == 5
    assert st["step_latency_s"]["p99"] >= st["step_latency_s"]["p50"] > 0
