"""Physics pins of the whole oracle time loop (deposit -> solve -> gather ->
push): linear Landau damping and the cold two-stream growth rate, against
the textbook dispersion relations solved here with scipy.  A wrong sign in
the field, the push or the charge normalisation changes the frequency or
turns damping into growth, so these catch what the unit pins cannot.
"""
import math

import numpy as np
import pytest
from scipy.optimize import brentq
from scipy.special import erfinv, wofz

from oracle import sgpic_oracle as O


def landau_root(k, vth=1.0):
    """Root of 1 + (1/(k lambda_D)^2)[1 + zeta Z(zeta)] = 0, Z = i sqrt(pi) w."""
    def D(w):
        z = w / (math.sqrt(2.0) * k * vth)
        Z = 1j * math.sqrt(math.pi) * wofz(z)
        return 1.0 + (1.0 + z * Z) / (k * vth) ** 2

    w = 1.4 - 0.15j
    for _ in range(60):  # secant iterations on the complex plane
        w2 = w + 1e-6
        d1, d2 = D(w), D(w2)
        step = d1 * (w2 - w) / (d2 - d1)
        w = w - step
        if abs(step) < 1e-13:
            break
    return w


def mode_amplitude(run, k):
    Ec = O.combined_field_regular(run.comps, run.n, run.d)[0]
    N = 2 ** run.n
    x = np.arange(N) * run.L[0] / N
    return abs(np.sum(Ec * np.exp(-1j * k * x)[:, None])) / Ec.size


def quiet_landau(Np, L, alpha, k, seed, ny=4):
    """Quiet start: x on a uniform lattice (ny rows in y), v_x from normal
    quantiles in random order, cold in y; charge weights 1 + alpha cos(kx)."""
    rng = np.random.default_rng(seed)
    nx = Np // ny
    UX, UY = np.meshgrid((np.arange(nx) + 0.5) / nx, (np.arange(ny) + 0.5) / ny, indexing="ij")
    u = np.stack([UX.ravel(), UY.ravel()], axis=1)
    vx = math.sqrt(2.0) * erfinv(2.0 * ((rng.permutation(Np) + 0.5) / Np) - 1.0)
    v = np.stack([vx, np.zeros(Np)], axis=1)
    q = -(L * L / Np) * (1.0 + alpha * np.cos(k * u[:, 0] * L))
    return u, v, q


@pytest.mark.slow
def test_landau_damping_rate_and_frequency():
    """Peaks of the k = 0.5 field mode after the initial transient: spacing
    pi / omega_r and log-slope gamma (linear theory, alpha = 0.05)."""
    k, alpha = 0.5, 0.05
    L = 2 * math.pi / k
    u, v, q = quiet_landau(1 << 16, L, alpha, k, seed=1)
    run = O.OracleRun((L, L), 5, u, v, q, dt=0.05, tau=5)
    ts, amps = [], []
    for s in range(250):
        ts.append(run.step_count * run.dt)
        amps.append(mode_amplitude(run, k))
        run.step()
    ts, amps = np.array(ts), np.array(amps)
    peaks = [i for i in range(1, len(amps) - 1) if amps[i] > amps[i - 1] and amps[i] >= amps[i + 1]]
    peaks = [i for i in peaks if 2.0 < ts[i] < 12.0]
    assert len(peaks) >= 4
    tp, ap = ts[peaks], amps[peaks]
    gamma = np.polyfit(tp, np.log(ap), 1)[0]
    omega = math.pi / np.mean(np.diff(tp))
    root = landau_root(k)
    assert omega == pytest.approx(root.real, rel=0.04)
    assert gamma == pytest.approx(root.imag, rel=0.15)


def test_landau_root_textbook_value():
    """Known values for k lambda_D = 0.5: omega = 1.4156, gamma = -0.1533."""
    root = landau_root(0.5)
    assert root.real == pytest.approx(1.4156, abs=2e-4)
    assert root.imag == pytest.approx(-0.1533, abs=2e-4)


@pytest.mark.slow
def test_cold_two_stream_growth():
    """Two cold counter-streaming beams (each omega_p^2 / 2, drift +-v0):
    omega^2 = a^2 + 1/2 - sqrt(1 + 8 a^2)/2 with a = k v0; the unstable
    root grows at gamma = sqrt(-omega^2)."""
    k = 0.2
    a = 0.6
    v0 = a / k
    L = 2 * math.pi / k
    Np = 1 << 15
    ux = (np.arange(Np) // 2 + 0.5) / (Np // 2)
    uy = (np.arange(Np) % 64 + 0.5) / 64.0
    vx = np.where(np.arange(Np) % 2 == 0, v0, -v0)
    eps = 1e-4
    ux = ux + eps * np.sin(k * ux * L) / (k * L)
    u = np.stack([ux, uy], axis=1)
    v = np.stack([vx, np.zeros(Np)], axis=1)
    q = np.full(Np, -(L * L) / Np)
    run = O.OracleRun((L, L), 5, u, v, q, dt=0.05, tau=5)
    ts, amps = [], []
    for s in range(350):
        ts.append(run.step_count * run.dt)
        amps.append(mode_amplitude(run, k))
        run.step()
    ts, amps = np.array(ts), np.array(amps)
    w2 = a * a + 0.5 - 0.5 * math.sqrt(1 + 8 * a * a)
    gamma_th = math.sqrt(-w2)
    # after the stable roots have been outgrown, before saturation
    idx = np.where((ts >= 11.0) & (ts <= 17.0))[0]
    assert amps[idx[-1]] > 20 * amps[0]
    gamma = np.polyfit(ts[idx], np.log(amps[idx]), 1)[0]
    assert gamma == pytest.approx(gamma_th, rel=0.1)


def test_penning_axial_leapfrog_closed_form():
    """Penning trap (Section 5.2) with a vanishing charge: the axial motion is
    the harmonic oscillator z'' = (q/m) (30/L) (z - L/2), omega_z^2 = 1.5 for
    electrons.  Leapfrog started with the backward half kick reproduces the
    discrete cosine z_k - L/2 = a cos(k theta), cos theta = 1 - omega_z^2 dt^2 / 2,
    exactly; the radial coordinates of a particle on the axis stay put."""
    from paper_2008_09441_gb300 import workloads
    wl = workloads.penning3d(n_particles=3, n=3, seed=1)
    L = wl.L[0]
    a = 1.3
    u = np.array([[0.5, 0.5, 0.5 + a / L]] * 3)
    v = np.zeros((3, 3))
    q = np.full(3, 1e-200)  # no self-field worth the name
    run = O.OracleRun(wl.L, wl.n, u, v, q, wl.dt, qm=-1.0, tau=1, B=wl.B, eext_lin=wl.eext_lin)
    wz2 = 30.0 / L
    theta = np.arccos(1.0 - wz2 * wl.dt ** 2 / 2.0)
    for k in range(1, 40):
        run.step(1)
        z = run.u[0, 2] * L - L / 2
        assert abs(z - a * np.cos(k * theta)) < 1e-11, k
        assert abs(run.u[0, 0] - 0.5) < 1e-14 and abs(run.u[0, 1] - 0.5) < 1e-14
