"""Serving through the C ABI: independent runs admitted by memory footprint
and advanced together; each run's result is the same alone and in the mix
(within the FP32 tolerance), latency percentiles and admission behave."""
import numpy as np
import pytest

from paper_2008_09441_gb300 import workloads

pytestmark = pytest.mark.gpu


def nrmse(a, ref):
    a = np.asarray(a, np.float64)
    ref = np.asarray(ref, np.float64)
    return float(np.sqrt(np.sum((a - ref) ** 2) / np.sum(ref * ref)))


def mix_params():
    return [dict(dim=2, n=6, n_particles=20000, amplitude=0.05, k=0.5, seed=1, steps=6),
            dict(dim=3, n=5, n_particles=30000, amplitude=0.01, k=0.4, seed=2, steps=4),
            dict(dim=2, n=8, n_particles=65536, amplitude=0.02, k=0.3, seed=3, steps=5),
            dict(dim=3, n=4, n_particles=5000, amplitude=0.05, k=0.6, seed=4, steps=7),
            dict(dim=2, n=5, n_particles=3001, amplitude=0.1, k=0.45, seed=5, steps=3)]


def test_alone_equals_mix():
    import torch
    from paper_2008_09441_gb300 import Run
    from paper_2008_09441_gb300.sgpic import Server
    assert torch.cuda.is_available()
    params = mix_params()
    wls = [workloads.serving_run_workload(p) for p in params]
    srv = Server(hbm_budget_bytes=64 << 20, max_slots=3)
    tickets = []
    for p, wl in zip(params, wls):
        tickets.append(srv.submit(wl.L, wl.n, wl.u.astype(np.float32), wl.v.astype(np.float32),
                                  wl.q.astype(np.float32), wl.dt, p["steps"]))
    max_active = 0
    for _ in range(200):
        a = srv.tick()
        max_active = max(max_active, a)
        if all(srv.poll(t)[0] in (2, 3) for t in tickets):
            break
    assert max_active <= 3
    for t, p, wl in zip(tickets, params, wls):
        st, diag = srv.poll(t)
        assert st == 2, (t, st)
        assert diag["step"] == p["steps"]
        um, vm, wm = srv.result(t)
        run = Run(wl.L, wl.n, wl.u.astype(np.float32), wl.v.astype(np.float32), wl.q.astype(np.float32), wl.dt)
        run.step(p["steps"])
        ua, va, wa = run.particles()
        du = um.astype(np.float64) - ua
        du -= np.round(du)
        assert np.sqrt(np.sum(du ** 2) / np.sum(ua.astype(np.float64) ** 2)) < 1e-5
        assert nrmse(vm, va) < 1e-5
        run.close()
    s = srv.stats()
    assert s["steps"] == sum(p["steps"] for p in params)
    assert 0 < s["p50_ms"] <= s["p99_ms"]
    assert s["particle_steps_per_s"] > 0
    srv.close()


def test_admission_respects_budget():
    from paper_2008_09441_gb300.sgpic import Server
    from paper_2008_09441_gb300 import SGError
    wl = workloads.landau2d(n_particles=20000, n=6, seed=9)
    srv = Server(hbm_budget_bytes=8 << 20, max_slots=8)
    # a request larger than the whole budget is refused at submit
    big = workloads.landau2d(n_particles=1 << 20, n=10, seed=9)
    with pytest.raises(SGError):
        srv.submit(big.L, big.n, big.u.astype(np.float32), big.v.astype(np.float32), big.q.astype(np.float32),
                   big.dt, 2)
    ts = [srv.submit(wl.L, wl.n, wl.u.astype(np.float32), wl.v.astype(np.float32), wl.q.astype(np.float32),
                     wl.dt, 2) for _ in range(6)]
    seen = []
    for _ in range(50):
        seen.append(srv.tick())
        if all(srv.poll(t)[0] == 2 for t in ts):
            break
    assert all(srv.poll(t)[0] == 2 for t in ts)
    assert max(seen) < 6  # the budget kept some requests queued
    srv.close()


def test_modes_and_centrings_in_one_mix():
    """Runs in the combination and filter modes on node- and cell-centred
    grids share one batched server; each equals the same run alone."""
    import torch
    from paper_2008_09441_gb300 import Run
    from paper_2008_09441_gb300.sgpic import Server
    assert torch.cuda.is_available()
    params = mix_params()[:4]
    kinds = [("combine", "cell"), ("filter", "node"), ("filter", "cell"), ("combine", "node")]
    wls = [workloads.serving_run_workload(p) for p in params]
    srv = Server(hbm_budget_bytes=256 << 20, max_slots=4)
    tickets = []
    for p, wl, (mode, cen) in zip(params, wls, kinds):
        tickets.append(srv.submit(wl.L, wl.n, wl.u.astype(np.float32), wl.v.astype(np.float32),
                                  wl.q.astype(np.float32), wl.dt, p["steps"], mode=mode, centring=cen))
    for _ in range(200):
        srv.tick()
        if all(srv.poll(t)[0] in (2, 3) for t in tickets):
            break
    for t, p, wl, (mode, cen) in zip(tickets, params, wls, kinds):
        st, diag = srv.poll(t)
        assert st == 2 and diag["step"] == p["steps"], (t, st)
        um, vm, _ = srv.result(t)
        run = Run(wl.L, wl.n, wl.u.astype(np.float32), wl.v.astype(np.float32), wl.q.astype(np.float32), wl.dt,
                  mode=mode, centring=cen)
        run.step(p["steps"])
        ua, va, _ = run.particles()
        du = um.astype(np.float64) - ua
        du -= np.round(du)
        assert np.sqrt(np.sum(du ** 2) / np.sum(ua.astype(np.float64) ** 2)) < 1e-5, (mode, cen)
        assert nrmse(vm, va) < 1e-5, (mode, cen)
        run.close()
    srv.close()


@pytest.mark.parametrize("mode", ["batched", "plain"])
def test_served_runs_match_oracle(mode):
    """Runs served together (Poisson-style staggered submission, budget for
    two at a time) against the FP64 oracle advanced alone: particle state
    and field energy within the FP32 tolerance, in either serving mode."""
    from oracle import sgpic_oracle as O
    from paper_2008_09441_gb300.sgpic import Server
    params = [dict(dim=2, n=6, n_particles=12000, amplitude=0.05, k=0.5, seed=11, steps=5),
              dict(dim=3, n=4, n_particles=6000, amplitude=0.02, k=0.4, seed=12, steps=4),
              dict(dim=2, n=7, n_particles=9000, amplitude=0.1, k=0.3, seed=13, steps=6)]
    wls = [workloads.serving_run_workload(p) for p in params]
    srv = Server(hbm_budget_bytes=1 << 30, max_slots=2)
    srv.set_mode(mode)
    tickets = []
    for i in range(200):
        if len(tickets) < len(wls) and i % 2 == 0:  # a new request every second tick
            wl = wls[len(tickets)]
            tickets.append(srv.submit(wl.L, wl.n, wl.u.astype(np.float32), wl.v.astype(np.float32),
                                      wl.q.astype(np.float32), wl.dt, params[len(tickets)]["steps"]))
        srv.tick()
        if len(tickets) == len(wls) and all(srv.poll(t)[0] in (2, 3) for t in tickets):
            break
    for t, p, wl in zip(tickets, params, wls):
        st, diag = srv.poll(t)
        assert st == 2 and diag["step"] == p["steps"], (t, st)
        um, vm, _ = srv.result(t)
        u64 = wl.u.astype(np.float32).astype(np.float64)
        v64 = wl.v.astype(np.float32).astype(np.float64)
        q64 = wl.q.astype(np.float32).astype(np.float64)
        ref = O.OracleRun(wl.L, wl.n, u64, v64, q64, wl.dt, qm=wl.qm, tau=wl.tau)
        ref.step(p["steps"])
        du = um.astype(np.float64) - ref.u
        du -= np.round(du)
        assert np.sqrt(np.sum(du ** 2) / np.sum(ref.u ** 2)) < 1e-5
        assert nrmse(vm, ref.velocities()) < 1e-5
        fe = ref.diagnostics()["field_energy"]
        assert abs(diag["field_energy"] - fe) <= 1e-5 * abs(fe)
    ss = srv.solve_stats()
    if mode == "batched":  # every run here takes part in the cross-run solve
        assert ss["launches"] > 0 and ss["grids"] > ss["launches"]
    else:
        assert ss["launches"] == 0
    srv.close()


def test_cross_run_solve_mixed_runs():
    """Batched serving of runs that take part in the cross-run solve (FP32
    2D and 3D, and FP64: one launch per precision each tick) beside a
    filter-mode run, which replays its whole step graph: every run against
    the FP64 oracle advanced alone, at its precision's tolerance."""
    from oracle import sgpic_oracle as O
    from paper_2008_09441_gb300.sgpic import Server
    params = [dict(dim=2, n=6, n_particles=12000, amplitude=0.05, k=0.5, seed=21, steps=5),
              dict(dim=3, n=4, n_particles=6000, amplitude=0.02, k=0.4, seed=22, steps=5),
              dict(dim=2, n=5, n_particles=5000, amplitude=0.1, k=0.3, seed=23, steps=5),
              dict(dim=2, n=6, n_particles=8000, amplitude=0.1, k=0.5, seed=24, steps=5)]
    extra = [dict(), dict(), dict(precision="fp64"), dict(mode="filter")]
    wls = [workloads.serving_run_workload(p) for p in params]
    srv = Server(hbm_budget_bytes=1 << 30, max_slots=4)
    tickets = []
    for wl, p, x in zip(wls, params, extra):
        dt = np.float64 if x.get("precision") == "fp64" else np.float32
        tickets.append(srv.submit(wl.L, wl.n, wl.u.astype(dt), wl.v.astype(dt), wl.q.astype(dt), wl.dt,
                                  p["steps"], **x))
    for _ in range(20):
        srv.tick()
        if all(srv.poll(t)[0] in (2, 3) for t in tickets):
            break
    ss = srv.solve_stats()
    # five ticks, two precisions each, the filter run outside
    assert ss["launches"] == 10, ss
    for t, p, wl, x in zip(tickets, params, wls, extra):
        st, diag = srv.poll(t)
        assert st == 2 and diag["step"] == p["steps"], (t, st)
        um, vm, _ = srv.result(t)
        dt = np.float64 if x.get("precision") == "fp64" else np.float32
        tol = 1e-12 if x.get("precision") == "fp64" else 1e-5
        ref = O.OracleRun(wl.L, wl.n, *(a.astype(dt).astype(np.float64) for a in (wl.u, wl.v, wl.q)), wl.dt,
                          qm=wl.qm, tau=wl.tau, mode=x.get("mode", "combine"))
        ref.step(p["steps"])
        du = um.astype(np.float64) - ref.u
        du -= np.round(du)
        assert np.sqrt(np.sum(du ** 2) / np.sum(ref.u ** 2)) < tol, t
        assert nrmse(vm, ref.velocities()) < tol, t
        fe = ref.diagnostics()["field_energy"]
        assert abs(diag["field_energy"] - fe) <= tol * abs(fe), t
    srv.close()
