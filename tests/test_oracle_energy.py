"""Pins of the oracle's energy diagnostics and of the empirical constants'
sigma, each against something other than the oracle's own formula.

* Field energy 0.5 h^d sum_j |E(x~_j)|^2 of a density that is a single
  Fourier mode, built exactly on the regular nodes by particles sitting on
  them: the Poisson problem of Section 2 gives |E| = A / |k| in closed form,
  so the energy is A^2 L^d / (4 |k|^2).
* Time-centred kinetic energy KE^n = 0.5 sum_p m_p v^{n-1/2}.v^{n+1/2}: the
  leapfrog makes KE^{n+1} - KE^n equal, to rounding, the trapezoidal work
  0.5 sum_p q_p (E^n_p + E^{n+1}_p).(x^{n+1}_p - x^n_p) of the forces the push
  applied, for any field.  With a linear restoring external field and no
  self-field KE^n + 0.5 sum_p m_p w^2 (x_p - L/2)^2 is an exact invariant of
  the leapfrog.
* Field and kinetic energy together: a cold Langmuir oscillation
  (omega_p = 1) trades all of its energy between the two, and their sum
  stays constant to O((omega dt)^2).
* sigma of eq. empirical_constants = sqrt(|Q_e| max|rho~|) and of eq.
  particle_constant = sqrt((2/3)^d |Q_e| max|rho~|), in 2D and 3D, with the
  3D gamma of both constant sets on a single mode.

Each planted mistake (the 1/2 dropped, h in place of h^d, the uncentred
product v^{n+1/2}.v^{n+1/2}, the (2/3)^d factor in the empirical sigma)
fails at least one of these pins (the mutants are planted in subclasses of
the oracle, on the CPU).  CPU only.
"""
import math

import numpy as np
import pytest

from oracle import sgpic_oracle as O


# ---------------------------------------------------------------- helpers


def node_lattice_run(run_cls, L, n, mode, A, rho0=-1.0, tau=None):
    """One particle on every regular node, charge V (rho0 + A cos(k.x_j)):
    the CIC deposit puts all of it on that node, so the regular-grid density
    is exactly rho0 + A cos(k.x).  Returns (run, |k|^2)."""
    d = len(L)
    u = O.regular_node_positions(n, d)
    V = float(np.prod([L[m] / 2 ** n for m in range(d)]))
    k = [2 * math.pi * mode[m] / L[m] for m in range(d)]
    ph = sum(k[m] * u[:, m] * L[m] for m in range(d))
    q = V * (rho0 + A * np.cos(ph))
    v = np.zeros_like(u)
    run = run_cls(L, n, u, v, q, dt=0.05, tau=n if tau is None else tau)
    return run, sum(x * x for x in k)


def field_energy_closed_form_error(run_cls, L, n, mode, A):
    run, k2 = node_lattice_run(run_cls, L, n, mode, A)
    want = A * A * float(np.prod(L)) / (4.0 * k2)
    return abs(run.field_energy() - want) / want


def work_energy_error(run_cls, steps=6, eext_lin=(0.0, 0.0), seed=3):
    """Max over steps of |KE^{n+1} - KE^n - trapezoidal work| / |KE|, on a
    sparse-grid (tau = 1) Landau-type run with noise and an optional linear
    external field."""
    rng = np.random.default_rng(seed)
    Np, n = 600, 5
    L = (4 * math.pi, 3.0)
    u = rng.random((Np, 2))
    v = rng.normal(size=(Np, 2))
    q = -(L[0] * L[1] / Np) * (1.0 + 0.3 * np.cos(2 * math.pi * u[:, 0]))
    run = run_cls(L, n, u, v, q, dt=0.07, tau=1, eext_lin=eext_lin)
    E_prev = run.field_at(run.u)
    u_prev = run.u.copy()
    run.step(1)
    ke_prev = run.kinetic_energy
    worst = 0.0
    for _ in range(steps):
        E_now = run.field_at(run.u)
        du = run.u - u_prev
        du -= np.round(du)  # periodic: the displacement v dt is far below a box
        work = 0.0
        for m in range(2):
            work += 0.5 * float(np.sum(q * (E_prev[m] + E_now[m]) * du[:, m] * L[m]))
        u_prev = run.u.copy()
        E_prev = E_now
        run.step(1)
        ke = run.kinetic_energy
        worst = max(worst, abs((ke - ke_prev) - work) / abs(ke))
        ke_prev = ke
    return worst


def trap_invariant_spread(run_cls, steps=60):
    """KE^n + 0.5 sum m w^2 (x - L/2)^2 along a leapfrog orbit in the linear
    restoring field E = e (x - L/2) (q/m e = -w^2), charges too small for a
    self-field: its relative spread (zero in exact arithmetic)."""
    L = (10.0, 10.0)
    e = (0.8, 0.3)
    qm = -1.0
    u = np.array([[0.5 + 0.11, 0.5 - 0.07], [0.5 - 0.2, 0.5 + 0.05], [0.45, 0.62]])
    v = np.array([[0.3, -0.4], [-0.1, 0.2], [0.5, 0.0]])
    q = np.full(3, -1e-200)
    mass = q / qm
    run = run_cls(L, 4, u, v, q, dt=0.1, qm=qm, tau=1, eext_lin=e)
    vals = []
    for _ in range(steps):
        u_n = run.u.copy()
        run.step(1)
        pot = 0.0
        for m in range(2):
            w2 = -qm * e[m]
            pot += 0.5 * float(np.sum(mass * w2 * (u_n[:, m] * L[m] - 0.5 * L[m]) ** 2))
        vals.append(run.kinetic_energy + pot)
    vals = np.array(vals)
    return float((vals.max() - vals.min()) / abs(vals.mean()))


def langmuir_energy_spread(run_cls, steps=80, tau=5):
    """Cold plasma oscillation (omega_p = 1, k = 1): lattice particles
    displaced by delta sin(k x), at rest.  Returns the spread of
    KE^n + FE^n over the run divided by the largest field energy, and the
    largest KE divided by the largest FE (1 in theory)."""
    L = 2 * math.pi
    n = 5
    nx, ny = 64, 32  # two particles per cell along x, one row per cell along y: uniform CIC density
    UX, UY = np.meshgrid((np.arange(nx) + 0.5) / nx, (np.arange(ny) + 0.5) / ny, indexing="ij")
    delta = 0.02
    ux = UX.ravel() + delta * np.sin(2 * math.pi * UX.ravel()) / L
    u = np.stack([ux, UY.ravel()], axis=1)
    Np = u.shape[0]
    v = np.zeros((Np, 2))
    q = np.full(Np, -(L * L) / Np)
    run = run_cls((L, L), n, u, v, q, dt=0.05, tau=tau)
    tot, fe, ke = [], [], []
    for _ in range(steps):
        run.step(1)
        d = run.diagnostics()
        # after the step from n to n+1: kinetic_energy = KE^n, field_energy_prev = FE^n
        tot.append(d["kinetic_energy"] + d["field_energy_prev"])
        fe.append(d["field_energy_prev"])
        ke.append(d["kinetic_energy"])
    tot = np.array(tot)
    return float((tot.max() - tot.min()) / max(fe)), float(max(ke) / max(fe))


# ---------------------------------------------------------------- mutants


class HalfDropped(O.OracleRun):
    def field_energy(self):
        return 2.0 * super().field_energy()


class HInsteadOfHd(O.OracleRun):
    def field_energy(self):
        Ec = self.regular_field()
        h = self.L[0] / 2 ** self.n
        return 0.5 * h * float(sum(np.sum(e * e) for e in Ec))


class UncentredKE(O.OracleRun):
    """The oracle's step with KE = 0.5 sum m v^{n+1/2}.v^{n+1/2}."""

    def step(self, nsteps=1):
        for _ in range(nsteps):
            E = self.field_at(self.u)
            vnew = O.kick_rotate(self.v, E, self.qm, self.dt, self.B)
            mass = self.q / self.qm
            self.kinetic_energy = 0.5 * float(np.sum(mass * sum(vnew[m] * vnew[m] for m in range(self.d))))
            self.field_energy_prev = self.field_energy()
            self.v = vnew
            self.u = O.drift(self.u, self.v, self.dt, self.L)
            self._fields()
            self.step_count += 1


class KEHalfDropped(O.OracleRun):
    def step(self, nsteps=1):
        super().step(nsteps)
        self.kinetic_energy *= 2.0


# ---------------------------------------------------------------- field energy


@pytest.mark.parametrize("L,n,mode", [((2.0, 3.0), 5, (2, 1)), ((4 * math.pi, 4 * math.pi), 4, (1, 0)),
                                      ((1.0, 2.0, 3.0), 3, (1, 1, 1)), ((2.0, 2.0, 5.0), 3, (0, 2, 1))])
def test_field_energy_single_mode_closed_form(L, n, mode):
    assert field_energy_closed_form_error(O.OracleRun, L, n, mode, A=0.3) < 1e-12


def test_field_energy_sparse_grid_axis_mode():
    """An x-only mode at tau = 1: the combination reproduces an axis-aligned
    field exactly (the 2D coefficients telescope), so the same closed form
    holds on the sparse grid."""
    L, n = (2.0, 3.0), 5
    run, k2 = node_lattice_run(O.OracleRun, L, n, (3, 0), A=0.3, tau=1)
    want = 0.09 * L[0] * L[1] / (4.0 * k2)
    assert abs(run.field_energy() - want) < 1e-12 * want


@pytest.mark.parametrize("mutant", [HalfDropped, HInsteadOfHd])
def test_field_energy_pin_catches_planted_mistakes(mutant):
    assert field_energy_closed_form_error(mutant, (2.0, 3.0), 5, (2, 1), A=0.3) > 1e-3


# ---------------------------------------------------------------- kinetic energy


@pytest.mark.parametrize("eext", [(0.0, 0.0), (-0.4, 0.9)])
def test_kinetic_energy_work_identity(eext):
    assert work_energy_error(O.OracleRun, eext_lin=eext) < 1e-11


def test_kinetic_energy_trap_invariant():
    assert trap_invariant_spread(O.OracleRun) < 1e-12


@pytest.mark.parametrize("mutant", [UncentredKE, KEHalfDropped])
def test_kinetic_energy_pins_catch_planted_mistakes(mutant):
    assert work_energy_error(mutant) > 1e-4
    assert trap_invariant_spread(mutant) > 1e-4


# ---------------------------------------------------------------- both energies


@pytest.mark.parametrize("tau", [5, 1])
def test_langmuir_total_energy_conserved(tau):
    spread, ratio = langmuir_energy_spread(O.OracleRun, tau=tau)
    assert spread < 0.005  # leapfrog: O((omega dt)^2 / 4) = 6e-4
    assert ratio == pytest.approx(1.0, abs=0.03)


@pytest.mark.parametrize("mutant", [HalfDropped, HInsteadOfHd, UncentredKE, KEHalfDropped])
def test_langmuir_pin_catches_planted_mistakes(mutant):
    spread, ratio = langmuir_energy_spread(mutant, steps=80)
    assert spread > 0.02 or abs(ratio - 1.0) > 0.1


# ---------------------------------------------------------------- sigma and 3D constants


def single_mode_3d(n, L, mode, A, rho0):
    N = 2 ** n
    X = np.meshgrid(*[np.arange(N) * L / N] * 3, indexing="ij")
    k = [2 * math.pi * mode[m] / L for m in range(3)]
    rho = rho0 + A * np.cos(k[0] * X[0]) * np.cos(k[1] * X[1]) * np.cos(k[2] * X[2])
    return rho, k


def test_empirical_sigma_2d():
    """eq. empirical_constants: sigma = sqrt(|Q_e| max|rho~|), no (2/3)^d."""
    n, L = 6, 2.0
    N = 2 ** n
    X = np.meshgrid(np.arange(N) * L / N, np.arange(N) * L / N, indexing="ij")
    A, rho0, Qe = 0.2, -1.0, -4.0
    rho = rho0 + A * np.cos(2 * math.pi * X[0] / L)
    _, _, c = O.tau_estimator(rho, Np=1e6, L=L, alpha=0.01, pc_ref=5, Qe=Qe, constants="empirical")
    assert c["sigma"] == pytest.approx(math.sqrt(abs(Qe) * (abs(rho0) + A)), rel=1e-12)
    _, _, cp = O.tau_estimator(rho, Np=1e6, L=L, alpha=0.01, pc_ref=5, Qe=Qe, constants="paper")
    assert cp["sigma"] / c["sigma"] == pytest.approx(2.0 / 3.0, rel=1e-12)  # sqrt((2/3)^2)


def test_constants_3d_single_mode():
    """3D single mode A cos(kx x) cos(ky y) cos(kz z) on a background:
    eq. grid_constants kappa_m = k_m^2 A / 4, beta = k_a^2 k_b^2 A / 72,
    gamma = kx^2 ky^2 kz^2 A / 864 and sigma = sqrt((2/3)^3 |Q_e| max|rho|);
    eq. empirical_constants takes the amplitude A/8 of each of the 8 Fourier
    peaks times the same wavenumber products, and sigma without (2/3)^3."""
    n, L = 4, 3.0
    A, rho0, Qe = 0.25, -2.0, -7.0
    rho, k = single_mode_3d(n, L, (1, 2, 3), A, rho0)
    k2 = [x * x for x in k]
    _, _, c = O.tau_estimator(rho, Np=1e6, L=L, alpha=0.01, pc_ref=5, Qe=Qe, constants="paper")
    for m in range(3):
        assert c["kappa"][m] == pytest.approx(0.25 * k2[m] * A, rel=1e-9)
    assert c["beta"][0] == pytest.approx(k2[0] * k2[1] * A / 72, rel=1e-9)
    assert c["beta"][1] == pytest.approx(k2[1] * k2[2] * A / 72, rel=1e-9)
    assert c["beta"][2] == pytest.approx(k2[2] * k2[0] * A / 72, rel=1e-9)
    assert c["gamma"] == pytest.approx(k2[0] * k2[1] * k2[2] * A / 864, rel=1e-9)
    assert c["sigma"] == pytest.approx(math.sqrt((2 / 3) ** 3 * abs(Qe) * (abs(rho0) + A)), rel=1e-12)
    _, _, e = O.tau_estimator(rho, Np=1e6, L=L, alpha=0.01, pc_ref=5, Qe=Qe, constants="empirical")
    for m in range(3):
        assert e["kappa"][m] == pytest.approx(k2[m] * A / 8, rel=1e-9)
    assert e["beta"][0] == pytest.approx(k2[0] * k2[1] * A / 8, rel=1e-9)
    assert e["gamma"] == pytest.approx(k2[0] * k2[1] * k2[2] * A / 8, rel=1e-9)
    assert e["sigma"] == pytest.approx(math.sqrt(abs(Qe) * (abs(rho0) + A)), rel=1e-12)


def test_empirical_sigma_pin_catches_planted_mistake(monkeypatch):
    """Plant the eq. particle_constant factor (2/3)^d into the empirical
    sigma: the 2D pin above no longer holds."""
    real = O.tau_estimator

    def planted(rho_reg, Np, L, alpha, pc_ref, Qe, constants="paper"):
        tau, table, c = real(rho_reg, Np, L, alpha, pc_ref, Qe, constants)
        if constants == "empirical":
            c = dict(c, sigma=c["sigma"] * math.sqrt((2.0 / 3.0) ** np.ndim(rho_reg)))
        return tau, table, c

    monkeypatch.setattr(O, "tau_estimator", planted)
    with pytest.raises(AssertionError):
        test_empirical_sigma_2d()
