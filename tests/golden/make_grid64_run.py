"""Writes grid64_run.npz: the FP64 oracle's whole near-equilibrium run (Algorithm 4)
on the 64x64 workload -- E = exp(0.3 z)/mean with correlation length 8 px (seed 0),
nu = 0.2, G_c = 1, ell = 2 px, AT1, strain-spectral split, crack-set
irreversibility, Delta eps_bar_yy = eps_M/20, tolerances 1e-8 -- until
C_bar < C_broken.  Stores the final phase field, the run's step/increment counts,
and the solver state at the start of a few load steps (checkpoints) so that
single sub-problem solves on this workload can be compared without re-running
the oracle from the start.  Calls only oracle/ and the shared input generator.

    python tests/golden/make_grid64_run.py                       # grid64_run.npz
    python tests/golden/make_grid64_run.py --tolerance-family    # grid64_tol_family.npz
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import evolution as ev  # noqa: E402
from oracle.params import AT1, CRACK_SET, SPECTRAL, Params  # noqa: E402
from paper_2203_16467_gb300.inputs import eps_M, modulus_field  # noqa: E402

N, LC, ELL, SEED = 64, 8.0, 2.0, 0
CHECKPOINTS = (40, 150, 400, 700, 1000)


def params():
    em = eps_M(1.0, 0.2, 1.0, ELL)
    return Params(fracture=AT1, split=SPECTRAL, irreversibility=CRACK_SET, ell=ELL, nu=0.2,
                  d_eps_bar=((0.0, 0.0), (0.0, em / 20)), mech_tol=1e-8, pf_tol=1e-8)


def tolerance_family(tols=(1e-7, 1e-10)):
    """Final phase fields of the same run at neighbouring solver tolerances: the
    crack tail of this workload is decided at the tolerance level (two nearby
    crack tails exist), so whole-run comparisons use this family."""
    E = modulus_field(N, N, LC, SEED)
    out = {}
    for tol in tols:
        par = params()
        par.mech_tol = tol
        par.pf_tol = tol
        st, reps = ev.run(E, par, max_steps=5000)
        out[f"phi_final_tol{tol:.0e}"] = st.phi
        out[f"n_steps_tol{tol:.0e}"] = len(reps)
    np.savez_compressed(os.path.join(HERE, "grid64_tol_family.npz"), **out)
    print({k: v for k, v in out.items() if k.startswith("n_steps")})


def main():
    par = params()
    E = modulus_field(N, N, LC, SEED)
    st = ev.State.initial(E)
    ck = {}
    n_inc = 0
    for k in range(5000):
        if k in CHECKPOINTS:
            ck[k] = (st.phi.copy(), st.eps_star.copy(), st.eps_bar.copy(), st.flag)
        rep = ev.load_step(st, par)
        n_inc += int(rep["incremented"])
        if rep["broken"]:
            break
    out = {"phi_final": st.phi, "n_steps": k + 1, "n_increments": n_inc, "C_bar_final": rep["C_bar"],
           "checkpoints": np.array(sorted(ck))}
    for s, (phi, es, eb, flag) in ck.items():
        out[f"phi_{s}"] = phi
        out[f"eps_star_{s}"] = es
        out[f"eps_bar_{s}"] = eb
        out[f"flag_{s}"] = flag
    np.savez_compressed(os.path.join(HERE, "grid64_run.npz"), **out)
    print("steps", k + 1, "increments", n_inc, "cracked px", int((st.phi > 0.95).sum()))


if __name__ == "__main__":
    if "--tolerance-family" in sys.argv:
        tolerance_family()
    else:
        main()
