"""Cell-centred grids (sg_params.centring = SG_CELL_CENTRED; nodes at cell
centres, Section 4.3, with Appendix A's two-step densities) on the GPU
against the FP64 oracle on identical seeded inputs, through the C ABI."""
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
                                         (3, 5, 2, 15000), (2, 10, 1, 20000), (2, 4, 1, 3000), (3, 3, 1, 2000)])
def test_cell_fields_at_init(torch_cuda, prec, d, n, tau, np_):
    """The regular-grid deposit on cell centres, the two-step component
    densities R_i rho~ (Appendix A), their fields and the combined field
    sum_i c_i P_i E_i with the cell-centred P_i."""
    wl = _wl(d, n, tau, np_, 400 + n + tau)
    run, (u64, v64, q64) = make_run(wl, prec, torch_cuda, centring="cell")
    tol = TOL[prec]
    u64 = O.wrap_unit(u64)
    reg = O.deposit_cic(u64, q64, (n,) * d, wl.L, "cell")
    assert nrmse(run.regular_charge(), reg) < tol
    comps = O.component_fields(u64, q64, n, tau, wl.L, "cell")
    gq = run.grid_charges()
    gf = run.grid_fields()
    for l, c, rho, E in comps:
        assert nrmse(gq[l], rho) < tol, l
        for m in range(d):
            if np.max(np.abs(E[m])) > 0:
                assert nrmse(gf[l][m], E[m]) < tol, (l, m)
    Ec = O.combined_field_regular(comps, n, d, "cell")
    Eg = run.field()
    for m in range(d):
        assert nrmse(Eg[m], Ec[m]) < tol, m
    run.close()


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("d,n,tau,np_", [(2, 11, 2, 6000), (2, 12, 10, 3000), (3, 8, 6, 4000), (3, 2, 1, 500)])
def test_cell_line_lengths(torch_cuda, prec, d, n, tau, np_):
    """The longest and shortest lines the restriction and the combination
    take (2^12 and 2^2 values): component densities, and the combined field
    at sampled regular centres."""
    wl = _wl(d, n, tau, np_, 500 + n)
    run, (u64, v64, q64) = make_run(wl, prec, torch_cuda, centring="cell")
    u64 = O.wrap_unit(u64)
    comps = O.component_fields(u64, q64, n, tau, wl.L, "cell")
    gq = run.grid_charges()
    for l, c, rho, E in comps:
        assert nrmse(gq[l], rho) < TOL[prec], l
    rng = np.random.default_rng(1100 + n)
    idx = rng.integers(0, 1 << n, size=(2000, d))
    Eg = run.field()
    for m in range(d):
        ref = sum(c * O.prolong_at(E[m], n, l, idx, "cell") for l, c, rho, E in comps)
        got = Eg[m][tuple(idx[:, a] for a in range(d))]
        assert nrmse(got, ref) < TOL[prec], m
    run.close()


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("mode", ["combine", "filter"])
@pytest.mark.parametrize("d,n", [(2, 6), (3, 4)])
def test_cell_trajectory(torch_cuda, prec, mode, d, n):
    """Five steps with the two-step shape in both directions: particle state
    every step, then the field, the energies and the charges."""
    wl = _wl(d, n, 1, 12000, 520 + d)
    run, (u64, v64, q64) = make_run(wl, prec, torch_cuda, mode=mode, centring="cell")
    ref = O.OracleRun(wl.L, n, u64, v64, q64, wl.dt, qm=wl.qm, tau=1, B=wl.B, eext_lin=wl.eext_lin, mode=mode,
                      centring="cell")
    tol = TOL[prec]
    for s in range(5):
        run.step(1)
        ref.step(1)
        ug, vg, _ = run.particles()
        e_u = nrmse_periodic(ug, ref.u)
        e_v = nrmse(vg, ref.velocities())
        assert e_u < tol and e_v < tol, (s, e_u, e_v)
    Eg = run.field()
    Er = ref.regular_field()
    for m in range(d):
        assert nrmse(Eg[m], Er[m]) < tol
    gq = run.grid_charges()
    for l, c, rho, _ in ref.comps:
        assert nrmse(gq[l], rho) < tol, l
    dg, rd = run.diagnostics(), ref.diagnostics()
    for key in ("field_energy", "field_energy_prev", "kinetic_energy"):
        assert relerr(dg[key], rd[key]) <= tol, (key, dg[key], rd[key])
    ctol = 1e-10 if prec == "fp64" else tol
    assert abs(dg["charge_combined"] - rd["charge_combined"]) <= ctol * abs(rd["charge_total"])
    run.close()


def test_cell_boris_external_field(torch_cuda):
    """Diocotron annulus (uniform B, Boris rotation) on cell-centred grids, FP64."""
    wl = workloads.diocotron2d(n_particles=10000, n=7, tau=1, seed=531)
    run, (u64, v64, q64) = make_run(wl, "fp64", torch_cuda, centring="cell")
    ref = O.OracleRun(wl.L, wl.n, u64, v64, q64, wl.dt, qm=wl.qm, tau=1, B=wl.B, eext_lin=wl.eext_lin,
                      centring="cell")
    for s in range(3):
        run.step(1)
        ref.step(1)
    ug, vg, _ = run.particles()
    assert nrmse_periodic(ug, ref.u) < 1e-12 and nrmse(vg, ref.velocities()) < 1e-12
    run.close()


@pytest.mark.parametrize("mode", ["combine", "filter"])
def test_cell_adaptive_tau_follows_oracle(torch_cuda, mode):
    """Algorithm 1 on the cell-centred regular density before every field
    evaluation: the tau sequence and the particle state match the oracle."""
    from paper_2008_09441_gb300._lib import SG_TAU_ADAPTIVE
    wl = workloads.diocotron2d(n_particles=8000, n=7, tau=1, seed=41)
    run, (u64, v64, q64) = make_run(wl, "fp64", torch_cuda, tau=SG_TAU_ADAPTIVE, alpha=0.05,
                                    tau_constants="empirical", mode=mode, centring="cell")
    ref = O.OracleRun(wl.L, wl.n, u64, v64, q64, wl.dt, qm=wl.qm, B=wl.B, eext_lin=wl.eext_lin, tau="adaptive",
                      mode=mode, alpha=0.05, pc_ref=5.0, tau_constants="empirical", centring="cell")
    assert run.diagnostics()["tau"] == ref.tau_history[0]
    for s in range(3):
        run.step(1)
        ref.step(1)
        assert run.diagnostics()["tau"] == ref.tau_history[-1], s
        ug, vg, _ = run.particles()
        assert nrmse_periodic(ug, ref.u) < 1e-12 and nrmse(vg, ref.velocities()) < 1e-12, s
    run.close()


def test_cell_tau_n_is_shifted_node_run(torch_cuda):
    """tau = n: the cell-centred regular run of particles at u equals the
    node-centred run of particles at u - h/2, translated back (FP64)."""
    wl = workloads.landau2d(n_particles=6000, n=6, tau=6, seed=541)
    h = 0.5 / 2 ** wl.n
    run_c, (u64, v64, q64) = make_run(wl, "fp64", torch_cuda, centring="cell")
    wl.u = O.wrap_unit(wl.u - h)
    run_n, _ = make_run(wl, "fp64", torch_cuda)
    run_c.step(3)
    run_n.step(3)
    uc, vc, _ = run_c.particles()
    un, vn, _ = run_n.particles()
    du = (uc - O.wrap_unit(un + h) + 0.5) % 1.0 - 0.5
    assert np.max(np.abs(du)) < 1e-12 and nrmse(vc, vn) < 1e-12
    run_c.close()
    run_n.close()


def test_cell_invalid_centring_rejected(torch_cuda):
    from paper_2008_09441_gb300 import SGError
    wl = workloads.landau2d(n_particles=1000, n=5, tau=1, seed=551)
    with pytest.raises(SGError):
        make_run(wl, "fp64", torch_cuda, centring=7)


def test_cell_save_load_continues_and_rejects_other_centring(torch_cuda):
    from paper_2008_09441_gb300 import SGError
    wl = workloads.landau2d(n_particles=20000, n=6, tau=1, seed=561)
    a, _ = make_run(wl, "fp64", torch_cuda, centring="cell")
    a.step(3)
    blob = a.save()
    a.step(3)
    b, _ = make_run(wl, "fp64", torch_cuda, centring="cell")
    b.load(blob)
    b.step(3)
    for x, y in zip(a.particles(), b.particles()):
        assert nrmse(x, y) < 1e-13
    c, _ = make_run(wl, "fp64", torch_cuda)  # node-centred
    with pytest.raises(SGError):
        c.load(blob)
    for r in (a, b, c):
        r.close()
