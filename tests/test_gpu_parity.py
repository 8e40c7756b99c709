"""GPU path against the FP64 oracle on identical seeded inputs, through the
C ABI.  Integer work (keys, sort, counts, checksum) must match bit for bit;
floating-point results within NRMSE (eq. error_def) 1e-12 for the FP64 path
and 1e-5 for the FP32 path (FP32 inputs are handed to the oracle as the same
FP32 values widened to FP64)."""
import math

import numpy as np
import pytest

from oracle import sgpic_oracle as O
from paper_2008_09441_gb300 import workloads

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-5}


LIB_DEFAULT_SORT_EVERY = {2: 4, 3: 6}  # sg_params.sort_every = 0, by dimension


def nrmse(a, ref):
    a = np.asarray(a, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    den = np.sum(ref * ref)
    if den == 0:
        return float(np.sqrt(np.sum(a * a)))
    return float(np.sqrt(np.sum((a - ref) ** 2) / den))


def relerr(a, ref):
    """|a - ref| / |ref| of one scalar result (|a - ref| when ref is 0)."""
    a, ref = float(a), float(ref)
    return abs(a - ref) / abs(ref) if ref != 0.0 else abs(a - ref)


def nrmse_periodic(u, ref):
    du = np.asarray(u, np.float64) - np.asarray(ref, np.float64)
    du -= np.round(du)
    return float(np.sqrt(np.sum(du * du) / np.sum(np.asarray(ref, np.float64) ** 2)))


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available()
    torch.cuda.set_device(0)
    return torch


def cast(wl, prec):
    dt = np.float32 if prec == "fp32" else np.float64
    u = wl.u.astype(dt)
    v = wl.v.astype(dt)
    q = wl.q.astype(dt)
    return u, v, q, u.astype(np.float64), v.astype(np.float64), q.astype(np.float64)


def make_run(wl, prec, torch, device_inputs=True, **kw):
    from paper_2008_09441_gb300 import Run
    u, v, q, u64, v64, q64 = cast(wl, prec)
    if device_inputs:
        dev = torch.device("cuda:0")
        u_, v_, q_ = (torch.from_numpy(np.ascontiguousarray(x)).to(dev) for x in (u, v, q))
    else:
        u_, v_, q_ = u, v, q
    args = dict(tau=wl.tau, precision=prec, B=wl.B, eext_lin=wl.eext_lin)
    args.update(kw)
    run = Run(wl.L, wl.n, u_, v_, q_, wl.dt, **args)
    return run, (u64, v64, q64)


# ------------------------------------------------------------ keys, sort, counts


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("d,n,np_", [(2, 6, 3 * 4096 + 1234), (3, 5, 2 * 4096 + 77), (2, 10, 9001), (2, 2, 5)])
def test_cell_sort_bit_exact(torch_cuda, prec, d, n, np_):
    torch = torch_cuda
    from paper_2008_09441_gb300 import sg_cell_sort
    from paper_2008_09441_gb300._lib import SG_FP32, SG_FP64
    rng = np.random.default_rng(100 + d * 10 + n)
    dt = np.float32 if prec == "fp32" else np.float64
    u = rng.random((np_, d)).astype(dt)
    k = min(7, np_)
    u[:k] = (np.arange(k)[:, None] % (1 << n)) / float(1 << n)  # exact cell boundaries
    cols = [torch.from_numpy(np.ascontiguousarray(u[:, m])).cuda() for m in range(d)]
    keys, perm, counts = sg_cell_sort(cols, n, SG_FP32 if prec == "fp32" else SG_FP64)
    torch.cuda.synchronize()
    k_ref = O.cell_keys(u.astype(np.float64), n)
    p_ref, sk_ref, c_ref = O.sort_by_key(k_ref, n, d)
    assert np.array_equal(keys.cpu().numpy().view(np.uint32), sk_ref)
    assert np.array_equal(perm.cpu().numpy().view(np.uint32), p_ref)  # stable: unique permutation
    assert np.array_equal(counts.cpu().numpy().view(np.uint32), c_ref)


def test_cell_sort_empty(torch_cuda):
    torch = torch_cuda
    from paper_2008_09441_gb300 import sg_cell_sort
    cols = [torch.empty(0, dtype=torch.float32, device="cuda") for _ in range(2)]
    keys, perm, counts = sg_cell_sort(cols, 3)
    torch.cuda.synchronize()
    assert keys.numel() == 0 and int(counts.sum()) == 0


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_run_keys_counts_checksum(torch_cuda, prec):
    wl = workloads.landau2d(n_particles=3 * 4096 + 555, n=6, seed=11)
    run, (u64, v64, q64) = make_run(wl, prec, torch_cuda)
    keys, counts = run.keys()
    ug, _, _ = run.particles()
    # keys are of the current storage order; as a multiset they equal the oracle's
    k_ref = O.cell_keys(O.wrap_unit(u64), wl.n)
    assert np.array_equal(np.sort(keys), np.sort(k_ref))
    # the storage order is sorted by tile key (Morton key of the level-(n-s) cell)
    s = max(0, wl.n - 12 // 2)
    assert np.all(np.diff((keys >> (2 * s)).astype(np.int64)) >= 0)
    _, _, c_ref = O.sort_by_key(k_ref, wl.n, 2)
    assert np.array_equal(counts, c_ref)
    assert run.diagnostics()["count_checksum"] == O.count_checksum(c_ref)
    run.close()


# ------------------------------------------------------------ deposit, restriction, solve, combine


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("d,n,tau,np_", [(2, 6, 1, 3 * 2048 + 99), (2, 7, 3, 20000), (3, 4, 1, 9000), (3, 5, 2, 15000),
                                         (2, 8, 6, 30000), (3, 5, 4, 20000), (2, 10, 1, 20000)])
def test_fields_at_init(torch_cuda, prec, d, n, tau, np_):
    if d == 2:
        wl = workloads.landau2d(n_particles=np_, n=n, tau=tau, seed=5 + n)
    else:
        wl = workloads.twostream3d(n_particles=np_, n=n, tau=tau, seed=5 + n)
    run, (u64, v64, q64) = make_run(wl, prec, torch_cuda)
    tol = TOL[prec]
    u64 = O.wrap_unit(u64)
    # grid set
    assert sorted(run.grids()) == sorted(O.combination_grids(d, n, tau))
    # regular-grid density (Algorithm 1's input)
    reg = O.deposit_cic(u64, q64, (n,) * d, wl.L)
    assert nrmse(run.regular_charge(), reg) < tol
    # component densities: direct deposit (Proposition 1 makes the GPU's
    # regular-then-restrict route equal to it)
    comps = O.component_fields(u64, q64, n, tau, wl.L)
    gq = run.grid_charges()
    gf = run.grid_fields()
    for l, c, rho, E in comps:
        assert nrmse(gq[l], rho) < tol, l
        for m in range(d):
            if np.max(np.abs(E[m])) > 0:
                assert nrmse(gf[l][m], E[m]) < tol, (l, m)
            else:  # no E_m on this grid: only the paired inverse transform's rounding of the other component
                scale = max(np.max(np.abs(E[k])) for k in range(d))
                assert np.max(np.abs(gf[l][m])) <= tol * scale, (l, m)
    Ec = O.combined_field_regular(comps, n, d)
    Eg = run.field()
    for m in range(d):
        assert nrmse(Eg[m], Ec[m]) < tol
    run.close()


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("d,n,tau,np_", [(2, 11, 2, 6000), (2, 12, 10, 3000), (3, 8, 6, 4000), (3, 2, 1, 500)])
def test_restriction_line_lengths(torch_cuda, prec, d, n, tau, np_):
    """Component-grid charges against the direct deposit of Proposition 1
    and the combined field at sampled regular nodes, at the longest and
    shortest lines the restriction and the combination support (2^12 and
    2^2 values per line)."""
    if d == 2:
        wl = workloads.landau2d(n_particles=np_, n=n, tau=tau, seed=7 + n)
    else:
        wl = workloads.twostream3d(n_particles=np_, n=n, tau=tau, seed=7 + n)
    run, (u64, v64, q64) = make_run(wl, prec, torch_cuda)
    u64 = O.wrap_unit(u64)
    gq = run.grid_charges()
    for l, c in O.combination_grids(d, n, tau):
        ref = O.deposit_cic(u64, q64, l, wl.L)
        assert nrmse(gq[l], ref) < TOL[prec], l
    # combined field at sampled regular nodes: sum_i c_i (P_i E_i)(x_j)
    comps = O.component_fields(u64, q64, n, tau, wl.L)
    rng = np.random.default_rng(1000 + n)
    idx = rng.integers(0, 1 << n, size=(2000, d))
    ref = O.field_at_particles(comps, idx / float(1 << n), wl.L, (0.0, 0.0, 0.0))
    Eg = run.field()
    for m in range(d):
        got = Eg[m][tuple(idx[:, a] for a in range(d))]
        assert nrmse(got, ref[m]) < TOL[prec], m
    run.close()


# ------------------------------------------------------------ time stepping


def trajectory_check(wl, prec, torch, steps, tol_scale=1.0, **kw):
    run, (u64, v64, q64) = make_run(wl, prec, torch, **kw)
    ref = O.OracleRun(wl.L, wl.n, u64, v64, q64, wl.dt, qm=wl.qm, tau=wl.tau, B=wl.B, eext_lin=wl.eext_lin)
    tol = TOL[prec] * tol_scale
    period = kw.get("sort_every") or LIB_DEFAULT_SORT_EVERY[ref.d]
    # the oracle's checksum after every step (the GPU's is the one of its last
    # sort: init, then every `period` steps)
    k0 = O.cell_keys(O.wrap_unit(u64), ref.n)
    cks = {0: O.count_checksum(np.bincount(k0.astype(np.int64), minlength=2 ** (ref.n * ref.d)))}
    for s in range(steps):
        run.step(1)
        ref.step(1)
        keys_ref = O.cell_keys(ref.u, ref.n)
        cks[s + 1] = O.count_checksum(np.bincount(keys_ref.astype(np.int64), minlength=2 ** (ref.n * ref.d)))
        ug, vg, wg = run.particles()
        e_u = nrmse_periodic(ug, ref.u)
        e_v = nrmse(vg, ref.velocities())
        assert e_u < tol and e_v < tol, (s, e_u, e_v)
    d = run.diagnostics()
    rd = ref.diagnostics()
    Ec = O.combined_field_regular(ref.comps, ref.n, ref.d)
    Eg = run.field()
    for m in range(ref.d):
        assert nrmse(Eg[m], Ec[m]) < tol
    gq = run.grid_charges()
    for l, c, rho, E in ref.comps:
        assert nrmse(gq[l], rho) < tol
    assert d["step"] == steps and d["tau"] == wl.tau
    for key in ("field_energy", "field_energy_prev", "kinetic_energy"):
        assert relerr(d[key], rd[key]) <= tol, (key, d[key], rd[key])
    ctol = 1e-10 if prec == "fp64" else TOL[prec]
    assert abs(d["charge_combined"] - rd["charge_combined"]) <= ctol * abs(rd["charge_total"])
    assert d["charge_grid_max_abs_err"] <= (1e-10 if prec == "fp64" else 1e-5) * abs(rd["charge_total"])
    keys, counts = run.keys()
    last_sort = (steps // period) * period
    if prec == "fp64":
        assert d["count_checksum"] == cks[last_sort], (last_sort, d["count_checksum"], cks[last_sort])
    run.close()
    return d, rd


def test_landau_fp64_10_steps(torch_cuda):
    """Landau damping, FP64, 2D n = 6 (11 component grids), 65,536 particles, 10 steps."""
    wl = workloads.make("landau2d_n6_fp64")
    trajectory_check(wl, "fp64", torch_cuda, wl.steps)


def test_landau_fp32_10_steps(torch_cuda):
    wl = workloads.landau2d(n_particles=40000, n=7, tau=1, seed=21)
    trajectory_check(wl, "fp32", torch_cuda, 10)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_twostream3d_steps(torch_cuda, prec):
    wl = workloads.twostream3d(n_particles=12000, n=4, tau=1, seed=31)
    trajectory_check(wl, prec, torch_cuda, 5)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_diocotron_boris_steps(torch_cuda, prec):
    wl = workloads.diocotron2d(n_particles=20000, n=6, tau=1, seed=41)
    trajectory_check(wl, prec, torch_cuda, 5)


def test_boris_3d_and_external_field(torch_cuda):
    wl = workloads.twostream3d(n_particles=8000, n=4, tau=2, seed=51)
    wl.B = (0.3, -0.5, 1.0)
    wl.eext_lin = (-0.2, -0.1, 0.4)
    trajectory_check(wl, "fp64", torch_cuda, 4)


@pytest.mark.parametrize("sort_every", [1, 3, 1000])
def test_sort_period_does_not_change_results(torch_cuda, sort_every):
    wl = workloads.landau2d(n_particles=30000, n=6, tau=1, seed=61)
    trajectory_check(wl, "fp64", torch_cuda, 6, sort_every=sort_every)


@pytest.mark.parametrize("d,n", [(2, 10), (3, 6)])
def test_step_sort_orders_by_tile(torch_cuda, d, n):
    """After sort steps the storage order is sorted by tile key (bit-exact
    keys from the stored positions), every particle is still present once,
    and the per-cell counts equal the oracle's on the same positions."""
    if d == 2:
        wl = workloads.landau2d(n_particles=50000, n=n, tau=1, seed=171)
    else:
        wl = workloads.twostream3d(n_particles=50000, n=n, tau=1, seed=171)
    run, _ = make_run(wl, "fp32", torch_cuda, sort_every=2)
    run.step(4)
    keys, counts = run.keys()
    s = max(0, n - 12 // d)
    assert np.all(np.diff((keys >> (d * s)).astype(np.int64)) >= 0)
    ug, _, _ = run.particles()
    k_ref = O.cell_keys(ug.astype(np.float64), n)
    assert np.array_equal(np.sort(keys), np.sort(k_ref))
    _, _, c_ref = O.sort_by_key(k_ref, n, d)
    assert np.array_equal(counts, c_ref)
    assert run.diagnostics()["count_checksum"] == O.count_checksum(c_ref)
    run.close()


def test_regular_grid_identity_tau_n(torch_cuda):
    """tau = n: one component grid, the regular grid itself (Section 4.2)."""
    wl = workloads.landau2d(n_particles=20000, n=5, tau=5, seed=71)
    run, _ = make_run(wl, "fp64", torch_cuda)
    assert run.grids() == [((5, 5), 1)]
    run.close()
    trajectory_check(wl, "fp64", torch_cuda, 5)


def test_host_inputs_match_device_inputs(torch_cuda):
    wl = workloads.landau2d(n_particles=5000, n=5, tau=1, seed=81)
    r1, _ = make_run(wl, "fp64", torch_cuda, device_inputs=True)
    r2, _ = make_run(wl, "fp64", torch_cuda, device_inputs=False)
    r1.step(3)
    r2.step(3)
    a, b = r1.particles(), r2.particles()
    for x, y in zip(a, b):
        assert nrmse(x, y) < 1e-13
    r1.close()
    r2.close()


@pytest.mark.parametrize("np_", [1, 2, 33, 257])
def test_tiny_particle_counts(torch_cuda, np_):
    wl = workloads.landau2d(n_particles=np_, n=3, tau=1, seed=91)
    trajectory_check(wl, "fp64", torch_cuda, 3)


# ------------------------------------------------------------ tauEstimator


@pytest.mark.parametrize("constants", ["paper", "empirical"])
@pytest.mark.parametrize("d,n", [(2, 6), (3, 4)])
def test_select_tau_matches_oracle(torch_cuda, constants, d, n):
    if d == 2:
        wl = workloads.landau2d(n_particles=60000, n=n, tau=1, seed=101, amplitude=0.3)
    else:
        wl = workloads.twostream3d(n_particles=60000, n=n, tau=1, seed=101, amplitude=0.3)
    run, (u64, v64, q64) = make_run(wl, "fp64", torch_cuda, alpha=0.05, pc_ref=5.0, tau_constants=constants)
    tau, g, z = run.select_tau(cap=16)
    reg = O.deposit_cic(O.wrap_unit(u64), q64, (n,) * d, wl.L)
    t_ref, table, _ = O.tau_estimator(reg, Np=len(q64), L=wl.L[0], alpha=0.05, pc_ref=5.0,
                                      Qe=float(np.sum(q64)), constants=constants)
    for t, ge, ze in table:
        assert g[t - 1] == pytest.approx(ge, rel=1e-9)
        assert z[t - 1] == pytest.approx(ze, rel=1e-9)
    assert tau == t_ref
    run.close()


def test_select_tau_empty_range(torch_cuda):
    from paper_2008_09441_gb300 import SGError
    wl = workloads.landau2d(n_particles=1000, n=3, tau=1, seed=3)
    run, _ = make_run(wl, "fp64", torch_cuda)
    with pytest.raises(SGError, match="empty"):
        run.select_tau()
    run.close()


def test_set_tau_rebuilds_grids(torch_cuda):
    wl = workloads.landau2d(n_particles=20000, n=6, tau=1, seed=111)
    run, (u64, v64, q64) = make_run(wl, "fp64", torch_cuda)
    run.step(2)
    run.set_tau(3)
    ug, vg, wg = run.particles()
    assert sorted(run.grids()) == sorted(O.combination_grids(2, 6, 3))
    comps = O.component_fields(ug.astype(np.float64), wg.astype(np.float64), 6, 3, wl.L)
    gq = run.grid_charges()
    for l, c, rho, E in comps:
        assert nrmse(gq[l], rho) < 1e-12
    run.close()


def test_adaptive_tau_runs(torch_cuda):
    from paper_2008_09441_gb300._lib import SG_TAU_ADAPTIVE
    wl = workloads.landau2d(n_particles=50000, n=7, tau=1, seed=121, amplitude=0.3)
    run, _ = make_run(wl, "fp64", torch_cuda, tau=SG_TAU_ADAPTIVE, alpha=0.05)
    run.step(3)
    d = run.diagnostics()
    assert 1 <= d["tau"] <= 4
    # the last selection was made on the current positions (after the last
    # push): selecting again, and the oracle's Algorithm 1 on the GPU's
    # positions, give the same tau, or a tie within 1e-9 of the total
    t, g, z = run.select_tau()
    ug, _, wg = run.particles()
    reg = O.deposit_cic(O.wrap_unit(ug.astype(np.float64)), wg.astype(np.float64), (wl.n,) * 2, wl.L)
    t_ref, table, _ = O.tau_estimator(reg, Np=len(wg), L=wl.L[0], alpha=0.05, pc_ref=5.0,
                                      Qe=float(np.sum(wg.astype(np.float64))))
    tot = {tt: ge + ze for tt, ge, ze in table}

    def same(a, b):
        return a == b or abs(tot[a] - tot[b]) <= 1e-9 * tot[b]

    assert same(t, t_ref), (t, t_ref, tot)
    assert same(d["tau"], t_ref), (d["tau"], t_ref, tot)
    for tt, ge, ze in table:
        assert g[tt - 1] == pytest.approx(ge, rel=1e-9) and z[tt - 1] == pytest.approx(ze, rel=1e-9)
    run.close()


def test_pipelined_diagnostics(torch_cuda):
    """Records posted after every step and collected up to two steps later
    are the oracle's diagnostics at the step of their post; a full ring and
    an empty ring are refused; a record keeps the grid set of its post."""
    from paper_2008_09441_gb300._lib import SG_DIAG_RING, SG_ERR_STATE, SGError
    wl = workloads.landau2d(n_particles=9000, n=6, tau=1, seed=141)
    run, (u64, v64, q64) = make_run(wl, "fp64", torch_cuda)
    ref = O.OracleRun(wl.L, wl.n, u64, v64, q64, wl.dt, qm=wl.qm, tau=wl.tau, B=wl.B, eext_lin=wl.eext_lin)
    tol = TOL["fp64"]
    want, got = [], []
    for s in range(7):
        run.step(1)
        run.post_diagnostics()
        ref.step(1)
        want.append(ref.diagnostics())
        if s >= 2:
            got.append(run.collect_diagnostics())
    while len(got) < len(want):
        got.append(run.collect_diagnostics())
    for s, (d, rd) in enumerate(zip(got, want)):
        assert d["step"] == s + 1 and d["tau"] == wl.tau and d["t"] == pytest.approx((s + 1) * wl.dt)
        for key in ("field_energy", "field_energy_prev", "kinetic_energy"):
            assert relerr(d[key], rd[key]) <= tol, (s, key, d[key], rd[key])
        assert abs(d["charge_combined"] - rd["charge_combined"]) <= 1e-10 * abs(rd["charge_total"])
    for _ in range(SG_DIAG_RING):
        run.post_diagnostics()
    with pytest.raises(SGError) as e:
        run.post_diagnostics()
    assert e.value.status == SG_ERR_STATE
    for _ in range(SG_DIAG_RING):
        assert run.collect_diagnostics()["step"] == 7
    with pytest.raises(SGError) as e:
        run.collect_diagnostics()
    assert e.value.status == SG_ERR_STATE
    run.post_diagnostics()
    run.set_tau(3)
    run.post_diagnostics()
    d0, d1 = run.collect_diagnostics(), run.collect_diagnostics()
    assert d0["tau"] == 1 and d0["n_grids"] == len(O.combination_grids(2, 6, 1))
    assert d1["tau"] == 3 and d1["n_grids"] == len(O.combination_grids(2, 6, 3))
    sync = run.diagnostics()
    for key in ("field_energy", "charge_combined", "kinetic_energy"):
        assert relerr(sync[key], d1[key]) <= 1e-14, key
    run.close()


# ------------------------------------------------------------ checkpoint, errors


def test_save_load_continues(torch_cuda):
    wl = workloads.landau2d(n_particles=20000, n=6, tau=1, seed=131)
    a, _ = make_run(wl, "fp64", torch_cuda)
    a.step(4)
    blob = a.save()
    a.step(4)
    b, _ = make_run(wl, "fp64", torch_cuda)
    b.load(blob)
    assert b.diagnostics()["step"] == 4
    b.step(4)
    for x, y in zip(a.particles(), b.particles()):
        assert nrmse(x, y) < 1e-13
    da, db = a.diagnostics(), b.diagnostics()
    assert da["step"] == db["step"] == 8
    assert da["kinetic_energy"] == pytest.approx(db["kinetic_energy"], rel=1e-12)
    a.close()
    b.close()


def test_nonfinite_input_rejected(torch_cuda):
    from paper_2008_09441_gb300 import SGError
    wl = workloads.landau2d(n_particles=1000, n=4, tau=1, seed=141)
    wl.v[17, 0] = np.nan
    with pytest.raises(SGError, match="non-finite"):
        make_run(wl, "fp64", torch_cuda)


def test_invalid_arguments(torch_cuda):
    from paper_2008_09441_gb300 import SGError
    wl = workloads.landau2d(n_particles=100, n=4, tau=1, seed=1)
    with pytest.raises(SGError):
        make_run(wl, "fp64", torch_cuda, tau=9)
    wl3 = workloads.landau2d(n_particles=100, n=13, tau=1, seed=1)
    with pytest.raises(SGError):
        make_run(wl3, "fp64", torch_cuda)


def test_kernel_launch_count_reported(torch_cuda):
    wl = workloads.landau2d(n_particles=5000, n=5, tau=1, seed=151)
    run, _ = make_run(wl, "fp32", torch_cuda)
    c0 = run.kernel_launches()
    run.step(5)
    c1 = run.kernel_launches()
    assert c1 - c0 >= 5 * 6
    run.close()


def test_particle_tuner_record(torch_cuda):
    """The init-time particle-pass tuner picks among its candidates (push
    grids of half, one and two resident waves; deposit windows of 4096, 6144,
    8192 and 12288 nodes), reports positive timings, and a second run of the
    same shape takes the cached choice; both runs follow the oracle."""
    wl = workloads.landau2d(n_particles=150000, n=7, tau=1, seed=151)
    runs = []
    for _ in range(2):
        run, (u64, v64, q64) = make_run(wl, "fp32", torch_cuda)
        runs.append(run)
    t0, t1 = runs[0].tuning(), runs[1].tuning()
    wave = t0["push_wave_blocks"]
    assert t0["push_blocks"] in (max(1, wave // 2), wave, 2 * wave)
    assert t0["deposit_window_nodes"] in (4096, 6144, 8192, 12288)
    assert all(x > 0 for x in t0["push_ms_half_one_two_waves"] + t0["deposit_ms_4096_6144_8192_12288"])
    assert t1["particles_from_cache"] and (t1["push_blocks"], t1["deposit_window_nodes"]) == \
        (t0["push_blocks"], t0["deposit_window_nodes"])
    assert all(x == 0 for x in t0["deposit_ms_drifted"])  # not before the first sort step
    # past the first sort step (sort every 4): the window was timed again on
    # drifted particles, and a later run of the same shape starts from that
    ref = O.OracleRun(wl.L, wl.n, u64, v64, q64, wl.dt, qm=wl.qm, tau=wl.tau)
    ref.step(5)
    for run in runs:
        run.step(5)
        ug, vg, _ = run.particles()
        assert nrmse_periodic(ug, ref.u) < TOL["fp32"] and nrmse(vg, ref.velocities()) < TOL["fp32"]
    t0 = runs[0].tuning()
    assert all(x > 0 for x in t0["deposit_ms_drifted"])
    assert t0["deposit_window_nodes"] in (4096, 6144, 8192, 12288)
    run2, _ = make_run(wl, "fp32", torch_cuda)
    t2 = run2.tuning()
    assert t2["particles_from_cache"] and all(x > 0 for x in t2["deposit_ms_drifted"])
    assert t2["deposit_window_nodes"] == runs[1].tuning()["deposit_window_nodes"]
    run2.close()
    for run in runs:
        run.close()


def test_stage_profiling_mode_same_results(torch_cuda):
    wl = workloads.landau2d(n_particles=10000, n=5, tau=1, seed=161)
    r1, _ = make_run(wl, "fp64", torch_cuda)
    r2, _ = make_run(wl, "fp64", torch_cuda)
    r2.set_profiling(True)
    r1.step(3)
    r2.step(3)
    st = r2.stage_times()
    assert all(v >= 0 for v in st.values()) and st["deposit"] > 0
    for x, y in zip(r1.particles(), r2.particles()):
        assert nrmse(x, y) < 1e-13
    r1.close()
    r2.close()


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_fixed_solve_variants_agree(torch_cuda, prec):
    """Both solve variants, fixed through sg_pic_set_solve_variant, give the
    oracle's fields and the same trajectory; bad values are rejected."""
    from paper_2008_09441_gb300 import SGError
    wl = workloads.landau2d(n_particles=12000, n=7, tau=1, seed=171)
    runs = []
    for variant in ("passes", "one-block"):
        run, (u64, v64, q64) = make_run(wl, prec, torch_cuda)
        run.set_solve_variant(variant)
        assert run.tuning()["solve_variant"] == ("per-axis-passes" if variant == "passes" else "one-block-per-grid")
        run.step(3)
        runs.append(run)
    ref = O.OracleRun(wl.L, wl.n, u64, v64, q64, wl.dt, qm=wl.qm, tau=1)
    ref.step(3)
    for run in runs:
        ug, vg, _ = run.particles()
        assert nrmse_periodic(ug, ref.u) < TOL[prec] and nrmse(vg, ref.velocities()) < TOL[prec]
    with pytest.raises(SGError):
        runs[0].set_solve_variant(7)
    runs[0].set_solve_variant("auto")
    runs[0].step(1)
    for run in runs:
        run.close()


# ------------------------------------------------------------ combination accumulation (FP32 path)


@pytest.mark.parametrize("d,n,tau,np_,centring,mode", [
    (2, 7, 1, 20000, "node", "combine"), (3, 5, 1, 15000, "node", "combine"),
    (2, 6, 1, 12000, "cell", "combine"), (2, 6, 2, 12000, "node", "filter"),
    (2, 11, 2, 6000, "node", "combine"),  # lines of 2^11: the block-per-line kernel
])
def test_combine_fp64_accumulation(torch_cuda, d, n, tau, np_, centring, mode):
    """sg_params.combine = SG_COMBINE_FP64 on the FP32 path: the combined
    field (or the filter mode's field) equals the FP64 oracle within the FP32
    tolerance, and float-float and FP64 accumulation land within half of it
    of each other (both are limited by the FP32 component fields, not by
    the sum)."""
    if d == 2:
        wl = workloads.landau2d(n_particles=np_, n=n, tau=tau, seed=181 + n)
    else:
        wl = workloads.twostream3d(n_particles=np_, n=n, tau=tau, seed=181 + n)
    _, (u64, v64, q64) = make_run(wl, "fp32", torch_cuda, device_inputs=False, centring=centring, mode=mode)
    u64 = O.wrap_unit(u64)
    if mode == "filter":
        Eref = O.filtered_field_regular(u64, q64, n, tau, wl.L, centring)[2]
    else:
        Eref = O.combined_field_regular(O.component_fields(u64, q64, n, tau, wl.L, centring), n, d, centring)
    fields = {}
    for acc in ("float-float", "fp64"):
        run, _ = make_run(wl, "fp32", torch_cuda, centring=centring, mode=mode, combine=acc)
        fields[acc] = run.field()
        e = [nrmse(fields[acc][m], Eref[m]) for m in range(d)]
        assert max(e) < TOL["fp32"], (acc, e)
        run.close()
    for m in range(d):  # the runs differ only in the accumulation and the deposit's atomic order
        assert nrmse(fields["float-float"][m], fields["fp64"][m]) < 0.5 * TOL["fp32"]


def test_combine_fp64_trajectory(torch_cuda):
    """Ten FP32 steps with the FP64-accumulating combination against the
    oracle (the trajectory check of the float-float path)."""
    wl = workloads.landau2d(n_particles=40000, n=7, tau=1, seed=21)
    trajectory_check(wl, "fp32", torch_cuda, 10, combine="fp64")


def test_combine_invalid_value_rejected(torch_cuda):
    from paper_2008_09441_gb300 import SGError
    wl = workloads.landau2d(n_particles=100, n=4, tau=1, seed=1)
    with pytest.raises(SGError):
        make_run(wl, "fp32", torch_cuda, combine=7)
