"""The benchmark workloads at full size, in the launch configuration
bench.py times (FP32 particles on the device, sort every 4 steps,
graph-launched steps), against the FP64 oracle: integer work bit for bit,
densities and fields in full or at sampled nodes, and the particles' first
step on a sample the oracle advances one by one.  Then the same
configurations over several steps on fewer particles, which the oracle
advances in full.  Workloads: 2D Landau damping (n = 10, tau = 1, 19
component grids, 4,194,304 particles), 3D two-stream (n = 7, tau = 1, 64
component grids, 16,777,216 particles) and the 2D diocotron annulus with the
Boris push (n = 9, tau = 1, 17 component grids, 8,388,608 particles)."""
import numpy as np
import pytest

from oracle import sgpic_oracle as O
from paper_2008_09441_gb300 import workloads
from test_gpu_parity import TOL, make_run, nrmse, nrmse_periodic, relerr, torch_cuda  # noqa: F401

pytestmark = pytest.mark.gpu

FULL = {"landau2d_n10_fp32": (4194304, 10, 19), "twostream3d_n7_fp32": (16777216, 7, 64),
        "diocotron2d_n9_fp32": (8388608, 9, 17)}


@pytest.mark.parametrize("name", list(FULL))
def test_fullsize_bench_configuration(torch_cuda, name):
    wl = workloads.make(name)
    n, d = wl.n, wl.dim
    assert (wl.n_particles, n, len(O.combination_grids(d, n, wl.tau))) == FULL[name] and wl.tau == 1
    run, (u64, v64, q64) = make_run(wl, "fp32", torch_cuda, sort_every=4)
    u64 = O.wrap_unit(u64)
    tol = TOL["fp32"]

    # cell keys and per-cell counts of the uploaded positions: bit-exact
    keys, counts = run.keys()
    k_ref = O.cell_keys(u64, n)
    assert np.array_equal(np.sort(keys), np.sort(k_ref))
    c_ref = np.bincount(k_ref.astype(np.int64), minlength=2 ** (n * d))
    assert np.array_equal(counts, c_ref)

    # the regular-grid density in full, every component density (R_i of it,
    # equal to the direct deposit by Proposition 1) and the combined field
    # at sampled regular nodes
    reg = O.deposit_cic(u64, q64, (n,) * d, wl.L)
    assert nrmse(run.regular_charge(), reg) < tol
    gq = run.grid_charges()
    comps = []
    for l, c in O.combination_grids(d, n, wl.tau):
        rho = O.restrict(reg, n, l)
        assert nrmse(gq[l], rho) < tol, l
        comps.append((l, c, rho, O.solve_poisson_spectral(rho, wl.L)))
    rng = np.random.default_rng(2008)
    idx = rng.integers(0, 1 << n, size=(4000, d))
    Eg = run.field()
    for m in range(d):
        ref = sum(c * O.prolong_at(E[m], n, l, idx) for l, c, rho, E in comps)
        assert nrmse(Eg[m][tuple(idx.T)], ref) < tol, m

    # first step on a sample: backward half kick at init, then kick and drift
    # with the initial field (both use E(x^0))
    s = np.sort(rng.choice(wl.n_particles, 8192, replace=False))
    us = u64[s]
    Ep = O.field_at_particles(comps, us, wl.L, wl.eext_lin)
    vs = [v64[s, m] for m in range(d)]
    vh = O.kick_rotate(vs, Ep, wl.qm, -0.5 * wl.dt, wl.B)
    v1 = O.kick_rotate(vh, Ep, wl.qm, wl.dt, wl.B)
    u1 = O.drift(us, v1, wl.dt, wl.L)
    run.step(1)
    ug, vg, _ = run.particles()
    assert nrmse_periodic(ug[s], u1) < tol
    assert nrmse(vg[s], np.stack(v1, axis=1)) < tol

    # three more steps end in a sort step (the push emits the tile keys): the
    # keys, the counts and the checksum of the GPU's own positions, bit-exact
    run.step(3)
    ug, _, _ = run.particles()
    ug64 = O.wrap_unit(ug.astype(np.float64))
    k4 = O.cell_keys(ug64, n)
    keys, counts = run.keys()
    assert np.array_equal(np.sort(keys), np.sort(k4))
    c4 = np.bincount(k4.astype(np.int64), minlength=2 ** (n * d))
    assert np.array_equal(counts, c4)
    assert run.diagnostics()["count_checksum"] == O.count_checksum(c4)
    run.close()


@pytest.mark.parametrize("name,n_particles,steps", [("landau2d_n10_fp32", 1 << 18, 10),
                                                    ("twostream3d_n7_fp32", 1 << 15, 5),
                                                    ("diocotron2d_n9_fp32", 1 << 18, 10)])
def test_bench_configuration_steps(torch_cuda, name, n_particles, steps):
    """Each benchmark configuration over several steps on fewer particles,
    which the oracle advances in full: the particle state after every step
    (the steps between sorts are the ones where particles have drifted since
    the last sort and the deposit's windows take their slow path), then the
    combined field, the component charges and the energies and charges of
    the diagnostics at the end."""
    wl = workloads.make(name, n_particles=n_particles, steps=steps)
    n, d = wl.n, wl.dim
    run, (u64, v64, q64) = make_run(wl, "fp32", torch_cuda, sort_every=4)
    ref = O.OracleRun(wl.L, n, u64, v64, q64, wl.dt, qm=wl.qm, tau=wl.tau, B=wl.B, eext_lin=wl.eext_lin)
    tol = TOL["fp32"]
    for s in range(steps):
        run.step(1)
        ref.step(1)
        ug, vg, _ = run.particles()
        e_u = nrmse_periodic(ug, ref.u)
        e_v = nrmse(vg, ref.velocities())
        assert e_u < tol and e_v < tol, (s, e_u, e_v)
    Ec = O.combined_field_regular(ref.comps, n, d)
    Eg = run.field()
    for m in range(d):
        assert nrmse(Eg[m], Ec[m]) < tol, m
    gq = run.grid_charges()
    for l, c, rho, E in ref.comps:
        assert nrmse(gq[l], rho) < tol, l
    dg, rd = run.diagnostics(), ref.diagnostics()
    assert dg["step"] == steps and dg["tau"] == 1
    for key in ("field_energy", "field_energy_prev", "kinetic_energy"):
        assert relerr(dg[key], rd[key]) <= tol, (key, dg[key], rd[key])
    assert relerr(dg["charge_combined"], rd["charge_combined"]) <= tol
    assert dg["charge_grid_max_abs_err"] <= tol * abs(rd["charge_total"])
    run.close()
