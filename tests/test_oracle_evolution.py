"""Pins of the oracle's near-equilibrium load step (Algorithm 4) and whole-run invariants."""
import numpy as np
import pytest

from oracle import constitutive as cm
from oracle import evolution as ev
from oracle import phasefield as pf
from oracle.params import AT1, AT2, CRACK_SET, DAMAGE, ISOTROPIC, SPECTRAL, SPECTRAL_STRESSFREE, Params
from paper_2203_16467_gb300.inputs import eps_M, modulus_field


def test_rescale_puts_max_driving_force_at_bound():
    # Lines 4-10 of Algorithm 4: after scaling eps by gamma, -F_phi(x*) = (-F_phi)_max
    # (psi_0^+ is degree-2 homogeneous).
    rng = np.random.default_rng(3)
    par = Params(fracture=AT1, split=SPECTRAL, ell=2.0)
    ny = nx = 16
    E = modulus_field(ny, nx, 4.0, 0)
    lam, mu = cm.lame(E, par.nu)
    y, x = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    phi = 0.3 * np.exp(-((x - 8.0) ** 2 + (y - 5.0) ** 2) / 8.0)      # smooth damage spot
    eps = np.zeros((ny, nx, 2, 2)); eps[..., 1, 1] = 1.5 + 0.3 * rng.standard_normal((ny, nx))
    eps_bar = np.array([[0.0, 0.0], [0.0, 1.5]])
    psi = cm.psi_plus(eps, lam, mu, par.split)
    lap = pf.laplacian(phi)
    gamma, flag, info = ev.rescale_factor(phi, psi, eps_bar, par, False, lap)
    assert flag and 0 < gamma < 1
    psi2 = cm.psi_plus(gamma * eps, lam, mu, par.split)
    mF = pf.minus_F_phi(phi, psi2, par, lap)
    assert mF.flat[info["istar"]] == pytest.approx(par.fmax(), rel=1e-12)


def test_no_rescale_below_threshold():
    par = Params(fracture=AT1, split=SPECTRAL, ell=2.0)
    phi = np.zeros((8, 8))
    psi = np.full((8, 8), 0.05)
    g, flag, _ = ev.rescale_factor(phi, psi, np.eye(2) * 0.1, par, False, pf.laplacian(phi))
    assert g == 1.0 and not flag


def test_homogeneous_run_breaks_near_elastic_limit():
    # Homogeneous modulus: the first phase-field evolution occurs once eps_bar_yy exceeds eps_M
    # (Sec. 3.3), and the run ends by the stiffness criterion C_bar < C_broken.
    ell = 2.0
    em = eps_M(1.0, 0.2, 1.0, ell)
    par = Params(fracture=AT1, split=SPECTRAL, irreversibility=CRACK_SET, ell=ell,
                 d_eps_bar=((0.0, 0.0), (0.0, em / 10)), mech_tol=1e-10, pf_tol=1e-10)
    E = np.ones((16, 16))
    # a one-pixel weak spot seeds the crack
    E[8, 8] = 0.9
    st, reps = ev.run(E, par, max_steps=400)
    first = next(r for r in reps if r["dphi_L1"] > 1e-8)
    assert first["eps_bar"][1, 1] >= 0.85 * em
    assert first["eps_bar"][1, 1] <= 1.1 * em
    assert reps[-1]["broken"]


@pytest.mark.parametrize("split,fracture,irr", [(SPECTRAL, AT1, CRACK_SET), (ISOTROPIC, AT2, DAMAGE),
                                                (SPECTRAL_STRESSFREE, AT1, DAMAGE)])
def test_short_run_invariants(split, fracture, irr):
    ell = 2.0
    em = eps_M(1.0, 0.2, 1.0, ell)
    par = Params(fracture=fracture, split=split, irreversibility=irr, ell=ell,
                 d_eps_bar=((0.0, 0.0), (0.0, em / 8)), mech_tol=1e-8, pf_tol=1e-8)
    E = modulus_field(24, 24, 4.0, 7)
    st = ev.State.initial(E)
    for _ in range(60):
        phi_old = st.phi.copy()
        rep = ev.load_step(st, par)
        assert np.all(st.phi >= pf.phi_con(phi_old, par) - 1e-12)    # Eq. irreversibility
        assert st.phi.min() >= -1e-12
        assert st.phi.max() <= 1.0 + 1e-6
        if rep["rescaled"]:
            assert rep["gamma"] < 1.0
        if rep["broken"]:
            break


def test_alternating_minimisation_increment():
    # Algorithm 2: the inner loop ends with ||dphi||_1 < Tol_AM, phi respects the increment's
    # constraint phi_con(phi_{s,0}), and the strain is in equilibrium with the final phase field.
    from oracle import mechanics
    ell = 2.0
    em = eps_M(1.0, 0.2, 1.0, ell)
    par = Params(fracture=AT1, split=SPECTRAL, irreversibility=DAMAGE, ell=ell,
                 d_eps_bar=((0.0, 0.0), (0.0, em / 8)), mech_tol=1e-10, pf_tol=1e-10)
    E = modulus_field(24, 24, 4.0, 7)
    st = ev.State.initial(E)
    st.eps_bar = np.array([[0.0, 0.0], [0.0, 0.95 * em]])
    for _ in range(3):
        phi0 = st.phi.copy()
        rep = ev.am_increment(st, par)
        assert rep["dphi_L1"] < 1e-3
        assert np.all(st.phi >= pf.phi_con(phi0, par) - 1e-12)
    assert rep["inner"] >= 1 and st.phi.max() > 0
    es, info = mechanics.solve(st.eps_star, st.eps_bar, st.phi, E, par)
    # one more mechanics solve after the last phase-field solve changes the strain only
    # by the last (small) phase-field update
    assert np.abs(es - st.eps_star).max() < 0.05 * np.abs(st.eps_bar).max()


def test_time_dependent_step_halves_and_recovers_dt():
    # Algorithm 3: above the elastic limit a full step (dt_max) evolves phi too much,
    # so dt is halved until ||dphi||_1 < (dphi)_max; easy steps double dt again.
    ell = 2.0
    em = eps_M(1.0, 0.2, 1.0, ell)
    par = Params(fracture=AT1, split=SPECTRAL, irreversibility=DAMAGE, ell=ell,
                 d_eps_bar=((0.0, 0.0), (0.0, em / 8)), mech_tol=1e-10, pf_tol=1e-10)
    E = modulus_field(24, 24, 4.0, 7)
    st = ev.State.initial(E)
    st.eps_bar = np.array([[0.0, 0.0], [0.0, 1.3 * em]])
    rep, dt = ev.td_step(st, par, 2.0 ** 16)
    assert rep["tries"] > 1 and rep["dphi_L1"] < 1.5
    assert not rep["incremented"]
    dts = [dt]
    for _ in range(30):
        rep, dt = ev.td_step(st, par, dt)
        dts.append(dt)
    assert max(dts) > min(dts)   # dt adapts
    assert np.all(st.phi >= -1e-12)


# ---------------------------------------------------------------------------
# energies() (Eq. Ff and the elastic energy of the contact model, Sec. 2.1)

@pytest.mark.parametrize("fracture", [AT1, AT2])
def test_energies_one_dimensional_crack_gives_Gc_per_length(fracture):
    # Eq. Ff is normalised by c_w so that an ideal crack dissipates G_c per unit length
    # (Sec. 2.1): the optimal 1-D profile (phase field held at 1 on one grid line, no
    # elastic drive) evaluated by energies() tends to G_c * (crack length) as ell/dx grows.
    # At the optimum the local and gradient parts contribute equally, so a wrong ell^2
    # factor or a wrong c_w moves the result away from G_c.
    ny, nx = 4, 256
    out = []
    for ell in (4.0, 8.0, 16.0):
        par = Params(fracture=fracture, ell=ell, Gc=1.7, irreversibility=CRACK_SET, pf_tol=1e-13, pf_atol=1e-14)
        phi = np.zeros((ny, nx))
        psi = np.zeros((ny, nx))
        b = pf.minus_F_phi(phi, psi, par)
        vcon = pf.phi_con(phi, par) - phi
        vcon[:, 0] = 1.0
        v, _ = pf.bccg(lambda x: pf.J_apply(x, psi, par), b, vcon, par.pf_tol, par.pf_atol, 50000)
        Fe, Ff = ev.energies(np.zeros((ny, nx, 2, 2)), v, np.ones((ny, nx)), par)
        assert Fe == 0.0
        out.append(Ff / (ny * par.dx) / par.Gc)
    assert abs(out[2] - 1.0) < 0.02
    assert abs(out[2] - 1.0) < abs(out[0] - 1.0) + 1e-12


def test_energies_fracture_term_of_a_cosine_mode():
    # a single Fourier mode phi = A cos(2 pi x / L) + B: sum phi^2 = N^2 (A^2/2 + B^2) and
    # sum |grad phi|^2 = N^2 A^2 (2 pi / L)^2 / 2 (dx = 1), so for AT2 (f = phi^2)
    # F_f = G_c/(2 ell) N^2 [A^2/2 + B^2 + ell^2 A^2 (2 pi/L)^2 / 2] exactly.
    n, A, B, ell = 16, 0.3, 0.4, 2.5
    par = Params(fracture=AT2, ell=ell, Gc=1.3)
    x = np.arange(n)
    phi = np.broadcast_to(A * np.cos(2 * np.pi * x / n) + B, (n, n)).copy()
    _, Ff = ev.energies(np.zeros((n, n, 2, 2)), phi, np.ones((n, n)), par)
    k = 2 * np.pi / n
    exact = par.Gc / (2.0 * ell) * n * n * (A * A / 2 + B * B + ell ** 2 * A * A * k * k / 2)
    assert Ff == pytest.approx(exact, rel=1e-12)


@pytest.mark.parametrize("split", [ISOTROPIC, SPECTRAL, SPECTRAL_STRESSFREE])
def test_energies_elastic_homogeneous_clapeyron(split):
    # Homogeneous grid, phi = 0: the elastic energy is half the work of the mean stress on the
    # applied strain, F_e = |Omega| sigma-bar : eps-bar / 2 (Clapeyron; psi is homogeneous of
    # degree 2 in eps for every split), with sigma-bar from the stress of the contact model.
    n, E0 = 8, 3.0
    par = Params(split=split, dx=0.5)
    E = np.full((n, n), E0)
    lam, mu = cm.lame(E, par.nu)
    for eb in (np.array([[0.01, 0.004], [0.004, -0.02]]), np.array([[-0.01, 0.0], [0.0, -0.03]]),
               np.array([[0.02, 0.01], [0.01, 0.005]])):
        eps = np.broadcast_to(eb, (n, n, 2, 2)).copy()
        Fe, Ff = ev.energies(eps, np.zeros((n, n)), E, par)
        sig = cm.stress(eps, np.zeros((n, n)), lam, mu, split).mean(axis=(0, 1))
        area = (n * par.dx) ** 2
        assert Fe == pytest.approx(0.5 * area * float(np.sum(sig * eb)), rel=1e-12)
        assert Ff == 0.0


def test_energies_elastic_of_broken_material_uses_the_contact_model():
    # phi = 1 everywhere (h = 0): only psi_0^- of the contact model remains (Sec. 2.1, Sec. 4.2.1).
    # Strain-spectral split: zero energy in tension, the full undamaged energy under
    # all-compressive principal strains; the stress-free contact model keeps no energy at all.
    n = 8
    E = np.full((n, n), 2.0)
    phi1, phi0 = np.ones((n, n)), np.zeros((n, n))
    tension = np.broadcast_to(np.array([[0.01, 0.002], [0.002, 0.02]]), (n, n, 2, 2)).copy()
    compression = -tension
    sp = Params(split=SPECTRAL)
    iso = Params(split=ISOTROPIC)
    sf = Params(split=SPECTRAL_STRESSFREE)
    assert ev.energies(tension, phi1, E, sp)[0] == 0.0
    full = ev.energies(compression, phi0, E, iso)[0]
    assert full > 0
    assert ev.energies(compression, phi1, E, sp)[0] == pytest.approx(full, rel=1e-12)
    assert ev.energies(compression, phi1, E, sf)[0] == 0.0
    assert ev.energies(tension, phi1, E, iso)[0] == 0.0
    # half-broken: h(1/2) = 1/4 of the isotropic energy
    assert ev.energies(tension, 0.5 * phi1, E, iso)[0] == pytest.approx(0.25 * ev.energies(tension, phi0, E, iso)[0],
                                                                        rel=1e-12)
