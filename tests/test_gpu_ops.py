"""Parity of single rows of the path (FFT operators, projection, constitutive model)
through the C ABI against the FP64 oracle."""
import numpy as np
import pytest

from oracle import constitutive as cm
from oracle import fourier
from oracle.params import ISOTROPIC, SPECTRAL, SPECTRAL_STRESSFREE, SPECTRAL_VOLDEV, VOLDEV
from paper_2203_16467_gb300.inputs import gaussian_field
from tests.helpers import from3, rel_l2, tensor_rel_l2, to3

pytestmark = pytest.mark.gpu

SIZES = [(16, 16), (64, 32), (32, 128), (256, 256), (512, 512), (64, 512), (512, 64), (2048, 2048)]


@pytest.fixture(scope="module")
def pff():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2203_16467_gb300 import pff as m
    return m


def _field(ny, nx, seed):
    rng = np.random.default_rng(seed)
    return gaussian_field(ny, nx, max(2.0, nx / 16), seed) + 0.3 * rng.standard_normal((ny, nx))


def _tol(prec, n):
    return 1e-12 if prec == 0 else (3e-6 if n <= 256 * 256 else 1e-5)


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "mixed"])
@pytest.mark.parametrize("ny,nx", SIZES)
def test_laplacian_parity(pff, prec, ny, nx):
    g = _field(ny, nx, 1)
    p = pff.Problem(nx, ny, prec)
    out = p.apply_laplacian(g)
    ref = fourier.laplacian(g)
    assert rel_l2(out, ref) < _tol(prec, nx * ny)
    p.close()


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "mixed"])
@pytest.mark.parametrize("ny,nx", SIZES)
def test_projection_parity(pff, prec, ny, nx):
    z = np.stack([_field(ny, nx, s) for s in (2, 3, 4)])
    p = pff.Problem(nx, ny, prec)
    out = p.apply_projection(z)
    ref = to3(fourier.project(from3(z)))
    assert tensor_rel_l2(out, ref) < _tol(prec, nx * ny)
    # idempotent on the device as well
    out2 = p.apply_projection(out)
    assert tensor_rel_l2(out2, out) < _tol(prec, nx * ny)
    p.close()


def _strains(ny, nx, seed):
    rng = np.random.default_rng(seed)
    e = 0.01 * rng.standard_normal((3, ny, nx))
    # special points: zero strain, equal principal strains (+/-), uniaxial, pure shear
    e[:, 0, 0] = 0.0
    e[:, 0, 1] = (0.004, 0.004, 0.0)
    e[:, 0, 2] = (-0.003, -0.003, 0.0)
    e[:, 0, 3] = (0.0, 0.01, 0.0)
    e[:, 0, 4] = (0.0, 0.0, 0.007)
    e[:, 0, 5] = (0.0, -0.01, 0.0)
    return e


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "mixed"])
@pytest.mark.parametrize("split", [ISOTROPIC, SPECTRAL, SPECTRAL_STRESSFREE, VOLDEV, SPECTRAL_VOLDEV])
def test_constitutive_parity(pff, prec, split):
    ny, nx = 32, 64
    rng = np.random.default_rng(9)
    E = np.exp(0.3 * rng.standard_normal((ny, nx)))
    phi = rng.uniform(0, 1, (ny, nx))
    eps = _strains(ny, nx, 10)
    pdir = 0.01 * rng.standard_normal((3, ny, nx))
    p = pff.Problem(nx, ny, prec, E=E)
    p.set_model(pff.AT1, split, pff.CRACK_SET)
    sig, psi, tang = p.constitutive(eps, phi, pdir)
    lam, mu = cm.lame(E, 0.2)
    et = from3(eps)
    sref = to3(cm.stress(et, phi, lam, mu, split))
    pref = cm.psi_plus(et, lam, mu, split)
    tref = to3(cm.Tangent(et, phi, lam, mu, split)(from3(pdir)))
    tol = 1e-12 if prec == 0 else 2e-6
    assert tensor_rel_l2(sig, sref) < tol
    assert rel_l2(psi, pref) < tol
    # the tangent differs only where principal strains coincide, a measure-zero set the
    # special points above probe: there both sides take the ramp derivative at e1
    assert tensor_rel_l2(tang, tref) < (1e-11 if prec == 0 else 2e-6)
    p.close()


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "mixed"])
def test_host_field_transfers(pff, prec):
    # fields in and out through host buffers (FP32 problems convert on the device through a
    # staging buffer): FP64 values come back exactly, FP32 ones as the FP32 rounding of the input,
    # into new arrays and into caller-provided (pinned) ones
    import torch
    nx, ny = 128, 64
    rng = np.random.default_rng(5)
    E = np.exp(0.3 * rng.standard_normal((ny, nx)))
    phi = rng.uniform(0.0, 0.9, (ny, nx))
    eps = 1e-3 * rng.standard_normal((3, ny, nx))
    rnd = (lambda a: a) if prec == 0 else (lambda a: a.astype(np.float32).astype(np.float64))
    p = pff.Problem(nx, ny, prec, E=E)
    p.set_phase_field(phi)
    p.set_strain(eps.reshape(3, -1), (0.0, 0.0, 0.0))
    assert np.array_equal(p.get_fields(pff.FIELD_MODULUS), rnd(E))
    assert np.array_equal(p.get_fields(pff.FIELD_PHI), rnd(phi))
    assert np.array_equal(p.get_fields(pff.FIELD_EPS_STAR), rnd(eps))
    pin = torch.empty(nx * ny, dtype=torch.float64, pin_memory=True)
    pin_np = pin.numpy()
    pin_np[:] = (2.0 * E).ravel()
    p.set_modulus_field(pin_np)
    out = torch.empty(nx * ny, dtype=torch.float64, pin_memory=True).numpy()
    got = p.get_fields(pff.FIELD_MODULUS, out=out)
    assert np.shares_memory(got, out) and np.array_equal(got, rnd(2.0 * E))
    p.set_modulus_field(2.0 * E)          # the same values again (sums unchanged)
    assert np.array_equal(p.get_fields(pff.FIELD_MODULUS), rnd(2.0 * E))
    with pytest.raises(ValueError):
        p.get_fields(pff.FIELD_PHI, out=np.empty(nx * ny - 1))
    with pytest.raises(pff.PffError):
        p.set_modulus_field(-E)           # rejected on the host, the stored field unchanged
    assert np.array_equal(p.get_fields(pff.FIELD_MODULUS), rnd(2.0 * E))
    p.close()


def test_host_transfers_from_concurrent_threads(pff):
    # handles are independent: eight FP32 problems on their own streams take fields in and out
    # from eight host threads at once (each through its own staging buffer)
    import torch
    from concurrent.futures import ThreadPoolExecutor
    n = 256
    rng = np.random.default_rng(11)
    fields = [np.exp(0.3 * rng.standard_normal((n, n))) for _ in range(8)]
    streams = [torch.cuda.Stream() for _ in range(8)]
    probs = [pff.Problem(n, n, pff.MIXED, stream=st.cuda_stream) for st in streams]

    def roundtrip(j):
        out = np.empty(n * n)
        for rep in range(4):
            probs[j].set_modulus_field(fields[j] * (rep + 1))
            probs[j].get_fields(pff.FIELD_MODULUS, out=out)
            if not np.array_equal(out.reshape(n, n), (fields[j] * (rep + 1)).astype(np.float32).astype(np.float64)):
                return False
        return True

    with ThreadPoolExecutor(max_workers=8) as ex:
        assert all(ex.map(roundtrip, range(8)))
    for p in probs:
        p.close()
