"""The paper's filter mode (eq. sparse_filter, Algorithm 2) and the adaptive
truncation parameter (Algorithm 1 every step) on the GPU, against the FP64
oracle on identical seeded inputs, through the C ABI."""
import numpy as np
import pytest

from oracle import sgpic_oracle as O
from paper_2008_09441_gb300 import workloads
from test_gpu_parity import TOL, make_run, nrmse, nrmse_periodic, relerr, torch_cuda  # noqa: F401

pytestmark = pytest.mark.gpu


def _wl(d, n, tau, np_, seed):
    if d == 2:
        return workloads.landau2d(n_particles=np_, n=n, tau=tau, seed=seed)
    return workloads.twostream3d(n_particles=np_, n=n, tau=tau, seed=seed)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("d,n,tau,np_", [(2, 6, 1, 3 * 2048 + 99), (2, 7, 3, 20000), (3, 4, 1, 9000),
                                         (3, 5, 2, 15000), (2, 10, 1, 20000)])
def test_filter_fields_at_init(torch_cuda, prec, d, n, tau, np_):
    """rho~, the component densities R_i rho~ and the field of the filtered
    density rho_f = sum_i c_i P_i R_i rho~ solved on the regular grid."""
    from paper_2008_09441_gb300 import SGError
    wl = _wl(d, n, tau, np_, 300 + n)
    run, (u64, v64, q64) = make_run(wl, prec, torch_cuda, mode="filter")
    tol = TOL[prec]
    u64 = O.wrap_unit(u64)
    rho, rho_f, E = O.filtered_field_regular(u64, q64, n, tau, wl.L)
    assert nrmse(run.regular_charge(), rho) < tol
    gq = run.grid_charges()
    for l, c in O.combination_grids(d, n, tau):
        assert nrmse(gq[l], O.restrict(rho, n, l)) < tol, l
    Eg = run.field()
    for m in range(d):
        assert nrmse(Eg[m], E[m]) < tol, m
    with pytest.raises(SGError):
        run.grid_fields()
    run.close()


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("d,n", [(2, 6), (3, 4)])
def test_filter_trajectory(torch_cuda, prec, d, n):
    """Five steps of Algorithm 2 with fixed tau: particle state every step,
    then the field, the energies and the charges."""
    wl = _wl(d, n, 1, 12000, 310 + d)
    run, (u64, v64, q64) = make_run(wl, prec, torch_cuda, mode="filter")
    ref = O.OracleRun(wl.L, n, u64, v64, q64, wl.dt, qm=wl.qm, tau=1, B=wl.B, eext_lin=wl.eext_lin,
                      mode="filter")
    tol = TOL[prec]
    for s in range(5):
        run.step(1)
        ref.step(1)
        ug, vg, _ = run.particles()
        e_u = nrmse_periodic(ug, ref.u)
        e_v = nrmse(vg, ref.velocities())
        assert e_u < tol and e_v < tol, (s, e_u, e_v)
    Eg = run.field()
    for m in range(d):
        assert nrmse(Eg[m], ref.E_regular[m]) < tol
    dg, rd = run.diagnostics(), ref.diagnostics()
    for key in ("field_energy", "field_energy_prev", "kinetic_energy"):
        assert relerr(dg[key], rd[key]) <= tol, (key, dg[key], rd[key])
    ctol = 1e-10 if prec == "fp64" else tol
    assert abs(dg["charge_combined"] - rd["charge_combined"]) <= ctol * abs(rd["charge_total"])
    run.close()


@pytest.mark.parametrize("mode", ["combine", "filter"])
def test_adaptive_tau_follows_oracle(torch_cuda, mode):
    """tau from Algorithm 1 before every field evaluation (at init and after
    every push), the diocotron annulus with the empirical constants: the
    chosen tau at every step and the particle state match the oracle."""
    from paper_2008_09441_gb300._lib import SG_TAU_ADAPTIVE
    wl = workloads.diocotron2d(n_particles=8000, n=7, tau=1, seed=41)
    run, (u64, v64, q64) = make_run(wl, "fp64", torch_cuda, tau=SG_TAU_ADAPTIVE, alpha=0.05,
                                    tau_constants="empirical", mode=mode)
    ref = O.OracleRun(wl.L, wl.n, u64, v64, q64, wl.dt, qm=wl.qm, B=wl.B, eext_lin=wl.eext_lin, tau="adaptive",
                      mode=mode, alpha=0.05, pc_ref=5.0, tau_constants="empirical")
    assert run.diagnostics()["tau"] == ref.tau_history[0]
    for s in range(3):
        run.step(1)
        ref.step(1)
        assert run.diagnostics()["tau"] == ref.tau_history[-1], s
        ug, vg, _ = run.particles()
        e_u = nrmse_periodic(ug, ref.u)
        e_v = nrmse(vg, ref.velocities())
        assert e_u < 1e-12 and e_v < 1e-12, (s, e_u, e_v)
    assert max(ref.tau_history) > 1  # the case exercises a tau other than the default
    run.close()


@pytest.mark.parametrize("mode", ["combine", "filter"])
def test_penning_adaptive_tau_follows_oracle(torch_cuda, mode):
    """The paper's 3D Penning trap (Section 5.2: B_z = 5, quadrupole E_ext,
    Gaussian bunch, (P_c)_ref = 1, alpha = 0.005) with Algorithm 1 before
    every field evaluation: tau sequence and particle state against the
    oracle (FP64)."""
    from paper_2008_09441_gb300._lib import SG_TAU_ADAPTIVE
    wl = workloads.penning3d(n_particles=20000, n=6, seed=61)
    run, (u64, v64, q64) = make_run(wl, "fp64", torch_cuda, tau=SG_TAU_ADAPTIVE, alpha=0.005, pc_ref=1.0,
                                    mode=mode)
    ref = O.OracleRun(wl.L, wl.n, u64, v64, q64, wl.dt, qm=wl.qm, B=wl.B, eext_lin=wl.eext_lin, tau="adaptive",
                      mode=mode, alpha=0.005, pc_ref=1.0, tau_constants="paper")
    assert run.diagnostics()["tau"] == ref.tau_history[0]
    for s in range(3):
        run.step(1)
        ref.step(1)
        assert run.diagnostics()["tau"] == ref.tau_history[-1], s
        ug, vg, _ = run.particles()
        e_u = nrmse_periodic(ug, ref.u)
        e_v = nrmse(vg, ref.velocities())
        assert e_u < 1e-12 and e_v < 1e-12, (s, e_u, e_v)
    run.close()


@pytest.mark.parametrize("centring", ["node", "cell"])
def test_penning_fp32_trajectory(torch_cuda, centring):
    """Penning trap, FP32 path, fixed tau = 2, five steps (Boris rotation with
    the quadrupole field) against the FP64 oracle."""
    wl = workloads.penning3d(n_particles=30000, n=6, tau=2, seed=62)
    run, (u64, v64, q64) = make_run(wl, "fp32", torch_cuda, centring=centring)
    ref = O.OracleRun(wl.L, wl.n, u64, v64, q64, wl.dt, qm=wl.qm, tau=2, B=wl.B, eext_lin=wl.eext_lin,
                      centring=centring)
    for s in range(5):
        run.step(1)
        ref.step(1)
        ug, vg, _ = run.particles()
        e_u = nrmse_periodic(ug, ref.u)
        e_v = nrmse(vg, ref.velocities())
        assert e_u < TOL["fp32"] and e_v < TOL["fp32"], (s, e_u, e_v)
    dg, rd = run.diagnostics(), ref.diagnostics()
    assert relerr(dg["field_energy"], rd["field_energy"]) <= TOL["fp32"]
    run.close()
