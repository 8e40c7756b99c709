"""Sharded runs on one GPU: a run's particles split over several handles
created with sg_pic_init_deferred, whose regular-grid densities are summed
between sg_pic_step_deposit and sg_pic_step_fields (the exchange a
multi-GPU run does with one all-reduce per step).  Two parts stepped in one
process, with the sum done by torch, must equal the whole run and the FP64
oracle within the stated tolerances."""
import numpy as np
import pytest

from oracle import sgpic_oracle as O
from paper_2008_09441_gb300 import workloads
from test_gpu_parity import TOL, nrmse, nrmse_periodic, relerr, torch_cuda  # noqa: F401

pytestmark = pytest.mark.gpu


def _parts(wl, prec, nparts, **kw):
    import torch
    from paper_2008_09441_gb300 import Run, shard
    dt = np.float32 if prec == "fp32" else np.float64
    tdt = torch.float32 if prec == "fp32" else torch.float64
    N = len(wl.q)
    runs, bounds = [], []
    for r in range(nparts):
        lo, hi = shard.partition(N, nparts, r)
        runs.append(Run(wl.L, wl.n, wl.u[lo:hi].astype(dt), wl.v[lo:hi].astype(dt), wl.q[lo:hi].astype(dt), wl.dt,
                        tau=wl.tau, precision=prec, B=wl.B, eext_lin=wl.eext_lin, deferred=True, **kw))
        bounds.append((lo, hi))
    q_total = float(np.sum(wl.q.astype(dt).astype(np.float64)))
    bufs = [torch.empty(1 << (wl.dim * wl.n), dtype=tdt, device="cuda") for _ in runs]

    def exchange():
        for run, b in zip(runs, bufs):
            run.density_copy(b, to_run=False)
        total = sum(bufs[1:], bufs[0].clone())
        for run in runs:
            run.density_copy(total, to_run=True)

    for run in runs:
        run.set_charge_total(q_total)
    exchange()
    for run in runs:
        run.start()

    def step():
        for run in runs:
            run.step_deposit()
        exchange()
        for run in runs:
            run.step_fields()

    return runs, bounds, step


def _gather(runs):
    parts = [run.particles() for run in runs]
    return (np.concatenate([p[0] for p in parts]), np.concatenate([p[1] for p in parts]),
            np.concatenate([p[2] for p in parts]))


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("nparts", [2, 3])
def test_parts_equal_oracle(torch_cuda, prec, nparts):
    """2D Landau, n = 7, tau = 1, six steps (a sort step among them): the
    parts' particles together and their common field against the FP64
    oracle of the whole run; field energy and grid charges of the whole run
    on every part, kinetic energy summed over the parts."""
    wl = workloads.landau2d(n_particles=30001, n=7, tau=1, seed=191)
    runs, bounds, step = _parts(wl, prec, nparts)
    dt = np.float32 if prec == "fp32" else np.float64
    ref = O.OracleRun(wl.L, wl.n, wl.u.astype(dt).astype(np.float64), wl.v.astype(dt).astype(np.float64),
                      wl.q.astype(dt).astype(np.float64), wl.dt, qm=wl.qm, tau=wl.tau)
    tol = TOL[prec]
    for s in range(6):
        step()
        ref.step(1)
        ug, vg, _ = _gather(runs)
        assert nrmse_periodic(ug, ref.u) < tol and nrmse(vg, ref.velocities()) < tol, s
    Ec = O.combined_field_regular(ref.comps, ref.n, ref.d)
    rd = ref.diagnostics()
    ke = 0.0
    for run in runs:
        Eg = run.field()
        for m in range(2):
            assert nrmse(Eg[m], Ec[m]) < tol
        d = run.diagnostics()
        assert d["step"] == 6
        assert relerr(d["field_energy"], rd["field_energy"]) <= tol
        assert relerr(d["charge_combined"], rd["charge_combined"]) <= tol
        ke += d["kinetic_energy"]
    assert relerr(ke, rd["kinetic_energy"]) <= tol
    for run in runs:
        run.close()


def test_sharded_run_one_rank_equals_run(torch_cuda):
    """ShardedRun without a process group is one part holding every
    particle: it equals the plain run to FP64 rounding."""
    from paper_2008_09441_gb300 import Run
    from paper_2008_09441_gb300.shard import ShardedRun
    wl = workloads.twostream3d(n_particles=9000, n=4, tau=1, seed=193)
    a = ShardedRun(wl.L, wl.n, wl.u, wl.v, wl.q, wl.dt, tau=1, precision="fp64")
    b = Run(wl.L, wl.n, wl.u, wl.v, wl.q, wl.dt, tau=1, precision="fp64")
    a.step(5)
    b.step(5)
    for x, y in zip(a.particles(), b.particles()):
        assert nrmse(x, y) < 1e-13
    da, db = a.diagnostics(), b.diagnostics()
    assert relerr(da["kinetic_energy"], db["kinetic_energy"]) < 1e-12
    assert relerr(da["field_energy"], db["field_energy"]) < 1e-12
    a.close()
    b.close()


def test_split_step_order_enforced(torch_cuda):
    from paper_2008_09441_gb300 import Run, SGError
    wl = workloads.landau2d(n_particles=2000, n=5, tau=1, seed=195)
    run = Run(wl.L, wl.n, wl.u, wl.v, wl.q, wl.dt, tau=1, precision="fp64", deferred=True)
    with pytest.raises(SGError, match="start"):
        run.step(1)
    with pytest.raises(SGError):
        run.step_deposit()
    run.start()
    with pytest.raises(SGError):
        run.start()
    with pytest.raises(SGError):
        run.step_fields()
    run.step_deposit()
    with pytest.raises(SGError):
        run.step(1)
    run.step_fields()
    run.step(1)
    assert run.diagnostics()["step"] == 2
    run.close()
    from paper_2008_09441_gb300._lib import SG_TAU_ADAPTIVE
    with pytest.raises(SGError):
        Run(wl.L, wl.n, wl.u, wl.v, wl.q, wl.dt, tau=SG_TAU_ADAPTIVE, precision="fp64", deferred=True)


def test_solve_tuning_cached(torch_cuda):
    """A second run of the same precision, dimension, level and tau takes the
    solve variant from the tuner's cache instead of timing it again."""
    from paper_2008_09441_gb300 import Run
    wl = workloads.landau2d(n_particles=3000, n=9, tau=2, seed=197)
    a = Run(wl.L, wl.n, wl.u, wl.v, wl.q, wl.dt, tau=2, precision="fp32")
    b = Run(wl.L, wl.n, wl.u, wl.v, wl.q, wl.dt, tau=2, precision="fp32")
    ta, tb = a.tuning(), b.tuning()
    assert tb["from_cache"] and tb["solve_variant"] == ta["solve_variant"]
    assert tb["passes_ms"] == ta["passes_ms"] and tb["one_block_ms"] == ta["one_block_ms"]
    a.close()
    b.close()
