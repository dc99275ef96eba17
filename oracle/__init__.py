"""FP64 CPU oracle for the staggered phase-field fracture load step.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, obviously-correct
NumPy restatement of what the method of Andrews & Pastewka, "Crack-path
selection in phase-field models for brittle fracture" (arXiv:2203.16467),
computes on one periodic 2-D pixel grid.  Only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py`` (its ``cpu_baseline`` leg and its
``--impl reference`` arm) may import it.  The CUDA library never calls it and
shares no code with it: the only thing the two sides share are the seeded
synthetic inputs, which come from ``paper_2203_16467_gb300.inputs``.

Every function cites the section / equation / algorithm of the paper it
follows.  Tensors are stored as full 2x2 arrays on the last two axes
(shape ``(ny, nx, 2, 2)``); scalar fields have shape ``(ny, nx)`` with row
index y and column index x.  Library primitives used as single steps:
``numpy.fft.fft2/ifft2`` (the DFT of Sec. 3.1) and ``numpy.linalg.eigh``
(principal strains of Eq. strain_spectral_en).

Module map:
  fourier        grid, wavevectors, DFT operators, projection Gamma, Laplacian
  constitutive   Lame parameters, degradation, energy splits, stresses, tangent
  mechanics      Fourier-Galerkin residual and Newton-CG (Sec. 3.1.1)
  phasefield     driving force, Jacobian J, BCCG (Sec. 3.1.2, Algorithm 1)
  evolution      near-equilibrium load step (Algorithm 4), energies, reports;
                 alternating minimisation (Algorithm 2), time-dependent steps (Algorithm 3)
  structures     crack / void initial conditions, random and two-phase moduli (Sec. 3.3)
"""
from .params import Params, AT1, AT2, ISOTROPIC, SPECTRAL, SPECTRAL_STRESSFREE, VOLDEV, SPECTRAL_VOLDEV, CRACK_SET, DAMAGE  # noqa: F401
from . import fourier, constitutive, mechanics, phasefield, evolution, structures  # noqa: F401
