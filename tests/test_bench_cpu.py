"""The bench's roofline arithmetic on the CPU: the per-kernel algorithmic bytes per pixel add
up to the per-iteration figures of the design notes (FP32 storage, 512-pixel rows), FP64 doubles
every term, and the active-launch count follows the step reports (the explicit-residual chain
works only in the iterations that evaluate J v explicitly)."""
import pytest

import bench


def test_bytes_per_iteration_512():
    b = bench.bytes_per_px(4, 512)
    s = 8 * 257 / 512                                   # half-spectrum bytes per pixel per component
    assert b[(0, 1)] == pytest.approx(14 * 4 + 3 * s)  # 68.05: read p, r, eps*, phi, E; write p, S
    assert b[(1, 1)] == pytest.approx(15 * 4 + 3 * s)  # 72.05: read S, theta, r, p; write theta, r
    cg = b[(0, 1)] + b[(2, 1)] + b[(1, 1)]
    bccg = b[(0, 3)] + b[(2, 9)] + b[(1, 9)]
    explicit = b[(0, 4)] + b[(2, 6)] + b[(1, 5)]
    bccg4 = b[(0, 3)] + b[(2, 4)] + b[(1, 4)] + b[(3, 11)]   # the four-pass variant stores J p
    assert round(cg) == 164 and round(bccg) == 66 and round(explicit) == 50 and round(bccg4) == 82
    bi = bench.bytes_per_px(4, 512, iso=True)          # the isotropic tangent reads no strain
    assert round(bi[(0, 1)] + bi[(2, 1)] + bi[(1, 1)]) == 152
    b8 = bench.bytes_per_px(8, 512)
    for k in b:
        # FP64 doubles each value but the one-byte flag plane
        flags = {(0, 3): 1, (1, 9): 1, (1, 5): 2, (3, 11): 1}.get(k, 0)
        assert b8[k] == pytest.approx(2 * (b[k] - flags) + flags)


def test_active_launches_follow_the_reports():
    reps = [[{"mech_cg_iters": 10, "newton_iters": 2, "bccg_iters": 7, "bccg_full_iters": 3}],
            [{"mech_cg_iters": 4, "newton_iters": 1, "bccg_iters": 5, "bccg_full_iters": 1},
             {"mech_cg_iters": 0, "newton_iters": 0, "bccg_iters": 0, "bccg_full_iters": 0}]]
    a = bench.active_launches(reps)
    assert a[(0, 1)] == 14 and a[(2, 1)] == 14 and a[(1, 1)] == 14
    assert all(a[k] == 12 for k in ((0, 3), (2, 9), (1, 9)))
    assert all(a[k] == 4 for k in ((0, 4), (2, 6), (1, 5)))
    assert all(a[k] == 0 for k in bench.BCCG4)
    assert set(a) == set(bench.KERNEL_NAMES)
    a4 = bench.active_launches(reps, bccg4=True)     # the same iterations as four passes
    assert all(a4[k] == 12 for k in ((0, 3),) + bench.BCCG4) and all(a4[k] == 0 for k in bench.BCCG3)
    assert all(a4[k] == a[k] for k in ((0, 1), (2, 1), (1, 1), (0, 4), (2, 6), (1, 5)))


def test_kernel_table_and_roofline_of():
    # the per-kernel table and its roofline from fake event timings (the 2048^2 and 64 x 256^2
    # workloads report these; no GPU needed)
    class FakeTiming:
        VARIANT_BCCG_PASSES = 3

        @staticmethod
        def timing_read(stage, op):
            return (2.0 if (stage, op) == (1, 9) else 0.5), 12

        @staticmethod
        def get_kernel_variant(kind, n, ncomp):
            return 0

    reps = [[{"mech_cg_iters": 10, "newton_iters": 2, "bccg_iters": 7, "bccg_full_iters": 3}]]
    kern = bench.kernel_table(FakeTiming, reps, 512, 512)
    assert set(kern) == set(bench.KERNEL_NAMES.values())
    dom = bench.KERNEL_NAMES[(1, 9)]
    byts = bench.kernel_bytes(reps, [False], 4, 512, 512)[(1, 9)]
    assert kern[dom]["achieved_GBs"] == pytest.approx(byts / 2e-3 / 1e9)
    r = bench.roofline_of(kern)
    assert r["kernel"] == dom and r["frac"] == pytest.approx(kern[dom]["achieved_GBs"] / r["peak"])
