"""Continuous batching: admission by HBM budget, each simulation's result is the same alone
and in a mix of other sizes and model variants that arrive while it runs, and a request never
waits for a load step of another grid size."""
import threading
import time

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
    budget = 4 << 30
    a = lambda arr: _req(serving, pff, 0, 64, "AT1", "SPECTRAL", "CRACK_SET", 7, arrival=arr, prec=prec)
    alone = serving.Server(budget, max_slots=8, keep_fields=True)
    alone.submit(a(0.0))
    alone.run()
    ref = alone.done[0]
    alone.close()
    mix = serving.Server(budget, max_slots=8, keep_fields=True)
    mix.submit(_req(serving, pff, 1, 128, "AT2", "ISOTROPIC", "DAMAGE", 3, prec=prec))
    mix.submit(_req(serving, pff, 2, 64, "AT1", "ISOTROPIC", "DAMAGE", 4, prec=prec))
    mix.submit(_req(serving, pff, 3, 256, "AT2", "SPECTRAL", "CRACK_SET", 5, prec=prec, steps=10))
    mix.submit(a(0.0))
    # arrives while the others run: joins the 64x64 lane between two of its steps
    mix.submit(_req(serving, pff, 4, 64, "AT2", "SPECTRAL", "DAMAGE", 6, arrival=0.02, prec=prec))
    mix.run()
    got = mix.done[0]
    assert mix.done[4]["steps"] > 0
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
    st = server.run()
    server.close()
    assert st["peak_active"] == 2
    assert st["completed"] == 5
    assert st["step_latency_s"]["p99"] >= st["step_latency_s"]["p50"] > 0


def test_small_request_does_not_wait_for_a_large_step(srv):
    # a 64x64 request that arrives while a 1024x1024 simulation is inside a load step starts,
    # and finishes its first step, before that 1024x1024 step ends
    pff, serving, torch = srv
    server = serving.Server(8 << 30, max_slots=8)
    server.submit(_req(serving, pff, 0, 1024, "AT1", "SPECTRAL", "CRACK_SET", 1, steps=6))
    th = threading.Thread(target=server.run)
    th.start()
    key = (1024, pff.MIXED)
    t_end = time.time() + 120
    while time.time() < t_end and not (key in server.lanes and server.lanes[key].steps_log):
        time.sleep(0.001)
    arrival = server.now()
    server.submit(_req(serving, pff, 1, 64, "AT1", "SPECTRAL", "CRACK_SET", 2, arrival=arrival, steps=1))
    th.join()
    log = server.lanes[key].steps_log
    small = server.done[1]
    server.close()
    assert small["steps"] == 1 and server.done[0]["steps"] == 6
    # the large step running at (or, in a gap between steps, right after) the arrival
    end = next(e for s, e in log if e > arrival)
    first_start = arrival + small["start_latency"]
    assert first_start < end, (arrival, first_start, end, log)
    assert small["latency"] < end - arrival
