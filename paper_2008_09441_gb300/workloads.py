"""Seeded synthetic inputs for the sparse-grid PIC workloads.

This module only draws initial particle states and run parameters; it holds
none of the method's arithmetic (no deposit, solve, combination or push).
The same arrays are handed to the CUDA path and to the FP64 oracle.

Positions are returned as fractions of the box (``u`` in [0, 1)^d),
velocities in physical units, charges per particle.  Seeds are
``2008094410 + workload index`` unless given.

Workloads (inputs stand in for the paper's synthetic plasma problems; no
dataset is involved):

* ``landau2d``   - 2D electrostatic Landau damping, periodic [0, 4 pi]^2,
  x, y uniform, charge q_p = -(Lx Ly / N_p) (1 + 0.05 cos(0.5 x_p))
  (uniform neutralising background of density 1), v ~ N(0, 1) per axis.
* ``twostream3d`` - 3D two-stream, periodic [0, 2 pi / 0.2]^3, two beams
  along x with drift +-3 and v_th = 0.3, charge weight 1 + 1e-3 cos(0.2 x).
* ``diocotron2d`` - 2D annulus r in [0.3, 0.4] L about the box centre,
  L = 1, uniform in area, charge weight 1 + 0.01 cos(3 theta), density
  magnitude 0.1 (omega_p^2 / omega_c^2 = 0.1 with B_z = 1), cold, initial
  velocity the E x B drift of the unperturbed annulus' analytic radial field.
* ``penning3d`` - 3D electrons in a Penning trap (Section 5.2): periodic
  [0, 20]^3, B = (0, 0, 5), quadrupole E_ext = (-15/L (x - L/2),
  -15/L (y - L/2), 30/L (z - L/2)), Gaussian positions about the centre with
  standard deviations (0.15, 0.05, 0.2) L (wrapped into the box), v ~ N(0, 1)
  per axis, total charge -1562.5 shared equally, dt = 0.05; the paper's
  estimator settings are (P_c)_ref = 1 and alpha = 0.005.
* ``diocotron_paper`` - the paper's 2D diocotron instability (Section 5.1):
  periodic [0, 22]^2, B = (0, 0, 5), no external E, total electron charge
  -400, dt = 0.02, T = 17.5; hollow profile
  f ~ exp(-|v|^2/2) exp(-(r - L/4)^2 / (2 (0.03 L)^2)) about the box
  centre.  ``sampling="gauss"``: r ~ N(L/4, 0.03 L), theta uniform,
  v ~ N(0, 1) per axis, equal charges; estimator settings (P_c)_ref = 5,
  alpha = 0.01.  ``sampling="uniform"``: x uniform in the box, v uniform in
  [-6, 6]^2, each particle's charge proportional to f at its phase-space
  point (normalised to the total charge), particles whose charge is below
  1e-9 in magnitude dropped; alpha = 0.03.  N_p = P_c 2^(2n) draws.
* ``serving_mix`` - parameters of independent runs (dimension, level,
  particle count, amplitude, wavenumber, arrival time).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 2008094410


@dataclass
class Workload:
    name: str
    dim: int
    L: tuple
    n: int
    tau: int
    u: np.ndarray          # (N_p, d) float64 in [0, 1)
    v: np.ndarray          # (N_p, d) float64
    q: np.ndarray          # (N_p,) float64
    dt: float
    qm: float = -1.0
    B: tuple = (0.0, 0.0, 0.0)
    eext_lin: tuple = (0.0, 0.0, 0.0)
    steps: int = 10
    extra: dict = field(default_factory=dict)

    @property
    def n_particles(self) -> int:
        return int(self.u.shape[0])


def landau2d(n_particles=65536, n=6, tau=1, amplitude=0.05, k=0.5, vth=1.0,
             dt=0.05, steps=10, seed=None, L=None):
    rng = np.random.default_rng(SEED_BASE + 0 if seed is None else seed)
    Lx = 2.0 * math.pi / k if L is None else L
    u = rng.random((n_particles, 2))
    x = u[:, 0] * Lx
    q = -(Lx * Lx / n_particles) * (1.0 + amplitude * np.cos(k * x))
    v = rng.normal(0.0, vth, (n_particles, 2))
    return Workload("landau2d", 2, (Lx, Lx), n, tau, u, v, q, dt, steps=steps,
                    extra={"amplitude": amplitude, "k": k, "vth": vth})


def twostream3d(n_particles=1 << 24, n=7, tau=1, amplitude=1e-3, k=0.2, drift=3.0,
                vth=0.3, dt=0.05, steps=10, seed=None):
    rng = np.random.default_rng(SEED_BASE + 2 if seed is None else seed)
    Lx = 2.0 * math.pi / k
    u = rng.random((n_particles, 3))
    x = u[:, 0] * Lx
    q = -(Lx ** 3 / n_particles) * (1.0 + amplitude * np.cos(k * x))
    v = rng.normal(0.0, vth, (n_particles, 3))
    sign = np.where(rng.random(n_particles) < 0.5, 1.0, -1.0)
    v[:, 0] += sign * drift
    return Workload("twostream3d", 3, (Lx, Lx, Lx), n, tau, u, v, q, dt, steps=steps,
                    extra={"amplitude": amplitude, "k": k, "drift": drift, "vth": vth})


def diocotron2d(n_particles=1 << 23, n=9, tau=1, r_in=0.3, r_out=0.4, amplitude=0.01,
                mode=3, density=0.1, Bz=1.0, dt=0.05, steps=1000, seed=None):
    rng = np.random.default_rng(SEED_BASE + 3 if seed is None else seed)
    L = 1.0
    r = np.sqrt(rng.uniform(r_in ** 2, r_out ** 2, n_particles)) * L
    th = rng.uniform(0.0, 2.0 * math.pi, n_particles)
    xc = 0.5 * L + r * np.cos(th)
    yc = 0.5 * L + r * np.sin(th)
    u = np.stack([xc / L, yc / L], axis=1)
    area = math.pi * (r_out ** 2 - r_in ** 2) * L * L
    Q = -density * area
    wgt = 1.0 + amplitude * np.cos(mode * th)
    q = Q / n_particles * wgt
    # Analytic radial field of the unperturbed annulus plus the uniform
    # background (Gauss's law in the plane, periodic images ignored): an
    # initial condition only.
    rho_a = -density
    rho_b = density * area / (L * L)
    enc = rho_a * (np.clip(r, r_in * L, r_out * L) ** 2 - (r_in * L) ** 2) / 2.0 + rho_b * r * r / 2.0
    Er = enc / np.maximum(r, 1e-12)
    Ex = Er * np.cos(th)
    Ey = Er * np.sin(th)
    v = np.stack([Ey / Bz, -Ex / Bz], axis=1)  # E x B / B^2 with B = Bz z
    return Workload("diocotron2d", 2, (L, L), n, tau, u, v, q, dt, B=(0.0, 0.0, Bz), steps=steps,
                    extra={"mode": mode, "amplitude": amplitude})


def diocotron_paper(n=9, pc=5, sampling="gauss", tau=1, Q=-400.0, Bz=5.0, dt=0.02, steps=875, seed=None):
    rng = np.random.default_rng(SEED_BASE + 6 if seed is None else seed)
    L = 22.0
    npart = int(pc) << (2 * n)
    r0, sr = 0.25 * L, 0.03 * L
    if sampling == "gauss":
        r = rng.normal(r0, sr, npart)
        th = rng.uniform(0.0, 2.0 * math.pi, npart)
        x = np.stack([0.5 * L + r * np.cos(th), 0.5 * L + r * np.sin(th)], axis=1)
        v = rng.normal(0.0, 1.0, (npart, 2))
        q = np.full(npart, Q / npart)
        alpha = 0.01
    elif sampling == "uniform":
        x = rng.uniform(0.0, L, (npart, 2))
        v = rng.uniform(-6.0, 6.0, (npart, 2))
        r = np.hypot(x[:, 0] - 0.5 * L, x[:, 1] - 0.5 * L)
        f = np.exp(-0.5 * np.sum(v * v, axis=1)) * np.exp(-((r - r0) ** 2) / (2.0 * sr * sr))
        q = Q * f / np.sum(f)
        keep = np.abs(q) >= 1e-9
        x, v, q = x[keep], v[keep], q[keep] * (Q / np.sum(q[keep]))
        alpha = 0.03
    else:
        raise ValueError("sampling must be 'gauss' or 'uniform'")
    u = x / L
    u = u - np.floor(u)
    u[u >= 1.0] = 0.0
    return Workload("diocotron_paper", 2, (L, L), n, tau, u, v, q, dt, B=(0.0, 0.0, Bz), steps=steps,
                    extra={"alpha": alpha, "pc_ref": 5.0, "sampling": sampling, "pc": pc})


def penning3d(n_particles=1 << 21, n=7, tau=1, Q=-1562.5, Bz=5.0, dt=0.05, steps=300, seed=None):
    rng = np.random.default_rng(SEED_BASE + 5 if seed is None else seed)
    L = 20.0
    sd = np.array([0.15, 0.05, 0.2]) * L
    x = rng.normal(0.5 * L, sd, size=(n_particles, 3))
    u = x / L
    u = u - np.floor(u)
    u[u >= 1.0] = 0.0
    v = rng.normal(0.0, 1.0, size=(n_particles, 3))
    q = np.full(n_particles, Q / n_particles)
    return Workload("penning3d", 3, (L, L, L), n, tau, u, v, q, dt, B=(0.0, 0.0, Bz),
                    eext_lin=(-15.0 / L, -15.0 / L, 30.0 / L), steps=steps,
                    extra={"alpha": 0.005, "pc_ref": 1.0})


WORKLOADS = {
    # name: (generator, kwargs) -- the five configurations of the benchmark
    "landau2d_n6_fp64": (landau2d, dict(n_particles=65536, n=6, tau=1, steps=10)),
    "landau2d_n10_fp32": (landau2d, dict(n_particles=4194304, n=10, tau=1, steps=200, seed=SEED_BASE + 1)),
    "twostream3d_n7_fp32": (twostream3d, dict(n_particles=16777216, n=7, tau=1, steps=10)),
    "diocotron2d_n9_fp32": (diocotron2d, dict(n_particles=8388608, n=9, tau=1, steps=1000)),
    "penning3d_n7_fp32": (penning3d, dict(n_particles=1 << 21, n=7, tau=1, steps=300)),
}


def make(name: str, **overrides) -> Workload:
    gen, kw = WORKLOADS[name]
    kw = dict(kw)
    kw.update(overrides)
    return gen(**kw)


def serving_mix(n_runs=512, seed=None, rate_per_s=None, max_log2_particles=23):
    """Parameters of independent Landau (2D) / two-stream (3D) runs.

    Level n uniform in 5..10 (2D) or 5..7 (3D); particle count log-uniform
    2^16..2^23; perturbation amplitude log-uniform 1e-3..0.1; wavenumber
    uniform 0.3..0.6; Poisson arrivals (exponential gaps) at ``rate_per_s``.
    """
    rng = np.random.default_rng(SEED_BASE + 4 if seed is None else seed)
    runs = []
    t = 0.0
    for i in range(n_runs):
        dim = 2 if rng.random() < 0.5 else 3
        n = int(rng.integers(5, 11)) if dim == 2 else int(rng.integers(5, 8))
        npart = int(round(2.0 ** rng.uniform(16, max_log2_particles)))
        amp = float(10.0 ** rng.uniform(-3, -1))
        k = float(rng.uniform(0.3, 0.6))
        if rate_per_s:
            t += float(rng.exponential(1.0 / rate_per_s))
        runs.append(dict(index=i, dim=dim, n=n, n_particles=npart, amplitude=amp, k=k,
                         arrival_s=t, seed=SEED_BASE + 100 + i, steps=100))
    return runs


def serving_run_workload(p) -> Workload:
    if p["dim"] == 2:
        return landau2d(n_particles=p["n_particles"], n=p["n"], tau=1, amplitude=p["amplitude"],
                        k=p["k"], steps=p["steps"], seed=p["seed"])
    return twostream3d(n_particles=p["n_particles"], n=p["n"], tau=1, amplitude=p["amplitude"],
                       k=p["k"], steps=p["steps"], seed=p["seed"])
