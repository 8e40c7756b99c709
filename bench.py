"""Benchmark of the sparse-grid PIC hot path on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl {gb300,reference}]

One step = gather-push, cell-key sort (every --sort-every steps), deposit,
restriction to all component grids, batched spectral solves, FP64-grade
combination.  Workload: 2D Landau damping, level n = 10, tau = 1
(19 component grids), 4,194,304 FP32 particles (synthetic, seeded).

Prints one JSON line (rank 0).  Under torchrun each rank runs its own
replica of the workload (independent runs, no collective): weak scaling.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

# The oracle runs single-threaded wherever this file times it (the reference
# arm here, the CPU baseline in a child process): numpy's BLAS threads are
# pinned to one before numpy loads, so the reported core count is exact.
_SINGLE_THREAD_ENV = {"OPENBLAS_NUM_THREADS": "1", "OMP_NUM_THREADS": "1", "MKL_NUM_THREADS": "1"}
if "reference" in sys.argv:
    os.environ.update(_SINGLE_THREAD_ENV)

import numpy as np  # noqa: E402

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particle-steps/s and HBM-roofline fraction (deposit, gather); p50/p99 step latency"
UNIT = "particle-steps/s"
WORKLOAD = "landau2d_n10_fp32"
# --workload name -> registered workload (the first is the default line)
WORKLOAD_NAMES = {"landau": "landau2d_n10_fp32", "twostream3d": "twostream3d_n7_fp32",
                  "diocotron2d": "diocotron2d_n9_fp32", "penning3d": "penning3d_n7_fp32"}
DESCRIPTIONS = {"landau2d": "2D Landau damping", "twostream3d": "3D two-stream instability",
                "diocotron2d": "2D diocotron annulus (B_z = 1, Boris)",
                "penning3d": "3D Penning trap (B_z = 5, quadrupole E_ext, Boris)"}
L2_FLUSH_BYTES = 512 << 20


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def traffic_record(kernel):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, if the
    kernel's source has not changed since (else None)."""
    p = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    rec = d.get(kernel)
    if not rec:
        return None
    src = os.path.join(ROOT, rec["source"])
    if not os.path.exists(src) or hashlib.sha256(open(src, "rb").read()).hexdigest()[:16] != rec["sha256_16"]:
        return None
    return rec


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() and args.impl != "reference" else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
        pg = dist
    return world, rank, local, pg


def barrier(pg):
    if pg is not None:
        pg.barrier()


def max_over_ranks(pg, x):
    if pg is None:
        return x
    import torch
    dev = "cuda" if pg.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------- algorithmic bytes
def algorithmic_bytes(np_, n, d, real_bytes=4):
    """Bytes the method must move per step (sort excluded), per kernel.
    deposit: read u (d) + w; push: read u, v, w, write u, v; plus the
    combined field read once by the push (hi plane, d N^d floats)."""
    N = 1 << n
    dep = np_ * (d + 1) * real_bytes
    push = np_ * ((2 * d + 1) + 2 * d) * real_bytes + d * N ** d * real_bytes
    return {"deposit": dep, "push": push}


# Oracle sample per workload: particles and the wall-time bound of the
# CPU-baseline leg (the 3D oracle's regular-grid field alone is seconds).
CPU_SAMPLE = {"landau2d_n10_fp32": (1 << 18, 10.0), "twostream3d_n7_fp32": (1 << 15, 10.0),
              "diocotron2d_n9_fp32": (1 << 18, 10.0), "penning3d_n7_fp32": (1 << 15, 10.0)}


def cpu_baseline(workload=WORKLOAD, state_path=None, mode="combine", centring="node"):
    """cpu_baseline_sample in a child process with one BLAS thread.  With
    state_path the child also saves the oracle's final state there (positions,
    velocities, the field on the regular nodes), the reference of the
    precision comparison."""
    env = dict(os.environ, **_SINGLE_THREAD_ENV)
    sample, seconds = CPU_SAMPLE.get(workload, (1 << 16, 10.0))
    code = (f"import json, bench; print(json.dumps(bench.cpu_baseline_sample({workload!r}, {sample}, {seconds}, "
            f"state_path={state_path!r}, mode={mode!r}, centring={centring!r})))")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=900)
    if r.returncode != 0:
        raise RuntimeError("cpu baseline failed: " + r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def cpu_sample_workload(workload, sample_particles):
    from paper_2008_09441_gb300 import workloads
    return workloads.make(workload, n_particles=sample_particles)


def cpu_baseline_sample(workload=WORKLOAD, sample_particles=1 << 18, min_seconds=10.0, max_steps=50,
                        state_path=None, mode="combine", centring="node"):
    """The oracle as it stands on a bounded sample: steps of the sample
    until about min_seconds of CPU work (at most max_steps)."""
    from oracle import sgpic_oracle as O
    wl = cpu_sample_workload(workload, sample_particles)
    u = wl.u.astype(np.float32).astype(np.float64)
    v = wl.v.astype(np.float32).astype(np.float64)
    q = wl.q.astype(np.float32).astype(np.float64)
    run = O.OracleRun(wl.L, wl.n, u, v, q, wl.dt, qm=wl.qm, tau=wl.tau, B=wl.B, eext_lin=wl.eext_lin, mode=mode,
                      centring=centring)
    t0 = time.perf_counter()
    steps = 0
    while steps < max_steps and (steps == 0 or time.perf_counter() - t0 < min_seconds):
        run.step(1)
        steps += 1
    dt = time.perf_counter() - t0
    out = {"value": sample_particles * steps / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": f"{steps} step(s) of {sample_particles} particles of the {workload} workload "
                     f"(n={wl.n}, tau={wl.tau}, {mode} mode, {centring}-centred), FP64 numpy oracle, single "
                     f"thread, {dt:.1f} s",
           "steps": steps, "particles": sample_particles}
    if state_path:
        diag = run.diagnostics()
        E = run.regular_field()
        np.savez(state_path, u=run.u, v=run.velocities(), E=np.stack(E),
                 diag=np.array([diag["field_energy"], diag["kinetic_energy"], diag["charge_combined"],
                                diag["charge_total"]]))
    return out


def precision_vs_oracle(wname, cpu, state_path, stream, dev, mode="combine", centring="node"):
    """The FP32 GPU path on the CPU-baseline sample, advanced the same number
    of steps as the oracle there, against the oracle's final state: NRMSE
    (eq. error_def) of the positions (periodic difference), the velocities
    and the combined field on the regular nodes, and the relative error of
    the field energy, the kinetic energy and the combined charge; once with
    each accumulation of the combination."""
    import torch
    from paper_2008_09441_gb300 import Run
    ref = np.load(state_path)
    wl = cpu_sample_workload(wname, cpu["particles"])
    steps = cpu["steps"]
    d = wl.dim

    def nrmse(a, b):
        return float(np.sqrt(np.sum((np.asarray(a, np.float64) - b) ** 2) / np.sum(b * b)))

    out = {"reference": "FP64 oracle state at the end of the CPU-baseline sample", "steps": steps,
           "particles": cpu["particles"]}
    for acc in ("float-float", "fp64"):
        u = torch.from_numpy(wl.u.astype(np.float32)).to(dev)
        v = torch.from_numpy(wl.v.astype(np.float32)).to(dev)
        q = torch.from_numpy(wl.q.astype(np.float32)).to(dev)
        run = Run(wl.L, wl.n, u, v, q, wl.dt, tau=wl.tau, qm=wl.qm, B=wl.B, eext_lin=wl.eext_lin,
                  precision="fp32", stream=stream.cuda_stream, combine=acc, mode=mode, centring=centring)
        run.step(steps)
        ug, vg, _ = run.particles()
        E = run.field()
        dg = run.diagnostics()
        run.close()
        du = ug.astype(np.float64) - ref["u"]
        du -= np.round(du)
        fe, ke, qc, qt = (float(x) for x in ref["diag"])
        out[acc] = {"nrmse_u": float(np.sqrt(np.sum(du * du) / np.sum(ref["u"] ** 2))),
                    "nrmse_v": nrmse(vg, ref["v"]),
                    "nrmse_E": max(nrmse(E[m], ref["E"][m]) for m in range(d)),
                    "relerr_field_energy": abs(dg["field_energy"] - fe) / abs(fe),
                    "relerr_kinetic_energy": abs(dg["kinetic_energy"] - ke) / abs(ke),
                    "relerr_charge": abs(dg["charge_combined"] - qc) / abs(qt)}
    return out


def run_reference(args, world, rank, pg):
    """The oracle as it stands, on the host cores (the reference arm)."""
    if rank != 0:
        barrier(pg)
        return
    from oracle import sgpic_oracle as O
    from paper_2008_09441_gb300 import workloads
    sample = args.ref_particles
    wl = workloads.make(WORKLOAD, n_particles=sample)
    u = wl.u.astype(np.float32).astype(np.float64)
    v = wl.v.astype(np.float32).astype(np.float64)
    q = wl.q.astype(np.float32).astype(np.float64)
    run = O.OracleRun(wl.L, wl.n, u, v, q, wl.dt, tau=wl.tau)
    run.step(min(args.warmup, 1))
    times = []
    budget_s = args.ref_budget_s  # the oracle's per-step cost is seconds: bound the whole run
    for _ in range(args.steps):
        t0 = time.perf_counter()
        run.step(1)
        times.append(time.perf_counter() - t0)
        if sum(times) > budget_s:
            break
    tot = sum(times)
    val = sample * len(times) / tot
    out = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": world,
           "steps": len(times), "warmup": args.warmup, "ms_per_step": 1e3 * tot / len(times),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic",
           "config": {"workload": WORKLOAD, "particles": sample, "n": 10, "tau": 1, "grids": 19,
                      "note": "oracle timed on a bounded particle sample of the workload"},
           "cpu_baseline": {"value": val, "unit": UNIT, "cores": 1, "kind": "oracle",
                            "sample": f"{len(times)} of the {args.steps} requested steps (time budget "
                                      f"{budget_s:.0f} s) of {sample} particles, n=10, tau=1"},
           "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))
    sys.stdout.flush()
    barrier(pg)


def run_serving(args, world, rank, local):
    """Serving mix: independent 2D Landau / 3D two-stream runs with the
    serving configuration's parameter distribution (level n uniform in
    5..10 / 5..7, particles log-uniform 2^16..2^max, amplitude log-uniform
    1e-3..0.1, k uniform 0.3..0.6, `--steps` steps each), arriving as a
    Poisson process whose rate is set to about 80% of the batched server's
    measured capacity, admitted by memory footprint (8 GB budget, 16 slots).
    The same arrival stream is served batched (each run's cached graphs on
    its own stream, and one cross-run solve launch per tick for the runs of
    at most 2^20 particles) and plain (runs stepped in turn with direct
    launches, one solve launch per grid).
    Reports per mode: p50 / p99 per-step latency (device), particle-steps/s
    of device time and of wall time, the device's busy fraction, and p50 /
    p99 of the time from a request's arrival to its result."""
    import torch
    from paper_2008_09441_gb300 import workloads
    from paper_2008_09441_gb300.sgpic import Server
    torch.cuda.set_device(local)
    steps = max(1, args.steps)
    params = workloads.serving_mix(n_runs=args.serving_runs, max_log2_particles=args.serving_max_log2)
    wls = []
    for p in params:  # generated once, shared by both modes
        p["steps"] = steps
        wl = workloads.serving_run_workload(p)
        wls.append((wl.L, wl.n, wl.u.astype(np.float32), wl.v.astype(np.float32), wl.q.astype(np.float32), wl.dt))
    work = [p["n_particles"] * steps for p in params]
    budget, slots = 8 << 30, 16

    def serve(mode, arrivals):
        srv = Server(hbm_budget_bytes=budget, max_slots=slots)
        srv.set_mode(mode)
        tickets, done_at = [], {}
        t0 = time.perf_counter()
        i = 0
        while len(done_at) < len(arrivals):
            now = time.perf_counter() - t0
            while i < len(arrivals) and arrivals[i] <= now:
                L, n, u, v, q, dt = wls[i]
                tickets.append(srv.submit(L, n, u, v, q, dt, steps))
                i += 1
            if srv.tick() == 0 and i < len(arrivals):
                time.sleep(max(0.0, min(0.01, arrivals[i] - (time.perf_counter() - t0))))
            now = time.perf_counter() - t0
            for j, t in enumerate(tickets):
                if j not in done_at and srv.poll(t)[0] in (2, 3):
                    done_at[j] = now
        wall = time.perf_counter() - t0
        st = srv.stats()
        ok = sum(1 for t in tickets if srv.poll(t)[0] == 2)
        srv.close()
        resp = sorted(done_at[j] - arrivals[j] for j in done_at)
        total = sum(work[:len(arrivals)])
        return {"p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"], "particle_steps_per_s": st["particle_steps_per_s"],
                "wall_particle_steps_per_s": total / wall, "wall_s": wall, "steps_served": st["steps"],
                "runs_done": ok, "device_busy": (total / st["particle_steps_per_s"]) / wall
                if st["particle_steps_per_s"] > 0 else None,
                "response_p50_s": resp[len(resp) // 2], "response_p99_s": resp[min(len(resp) - 1,
                                                                                int(0.99 * len(resp)))]}

    # capacity of the batched server: the first runs, all arriving at once
    ncal = min(len(params), 24)
    cal = serve("batched", [0.0] * ncal)
    capacity = cal["wall_particle_steps_per_s"]
    rate = 0.8 * capacity / (sum(work) / len(work))
    rng = np.random.default_rng(workloads.SEED_BASE + 5)
    arrivals = list(np.cumsum(rng.exponential(1.0 / rate, size=len(params))) - 0.0)
    out = {"metric": "serving: p50/p99 step latency and particle-steps/s", "unit": UNIT, "n_gpus": world,
           "steps": steps, "runs": len(params), "data": "synthetic (seeded serving mix)",
           "config": {"workload": f"serving mix: {len(params)} runs (2D Landau n 5..10 / 3D two-stream n 5..7, "
                                  f"2^16..2^{args.serving_max_log2} FP32 particles, {steps} steps), Poisson "
                                  f"arrivals at {rate:.2f} runs/s (80% of the batched capacity "
                                  f"{capacity:.3g} particle-steps/s measured on {ncal} runs arriving at once)",
                      "budget_bytes": budget, "slots": slots},
           "modes": {}}
    for mode in ("batched", "plain"):
        out["modes"][mode] = serve(mode, arrivals)
    out["value"] = out["modes"]["batched"]["wall_particle_steps_per_s"]
    out["batched_over_plain"] = (out["modes"]["batched"]["wall_particle_steps_per_s"]
                                 / max(1e-30, out["modes"]["plain"]["wall_particle_steps_per_s"]))
    if rank == 0:
        print(json.dumps(out))


def run_diocotron_paper(args, world, rank, local):
    """The paper's Section 5.1 experiment on the GPU: the 2D diocotron
    instability (Gaussian or uniform weighted sampling) with tau chosen by
    Algorithm 1 every step, against regular PIC (tau = n) at the same
    particles per cell and fixed tau in Algorithm 1's range; the error of
    the charge density and of the field (eq. error_def, NRMSE over the
    regular nodes) at eight instants of [0, T] against the mean of an
    ensemble of regular-PIC runs with more particles per cell, and the tau
    history of the adaptive run."""
    import torch
    from paper_2008_09441_gb300 import Run, workloads
    from paper_2008_09441_gb300._lib import SG_TAU_ADAPTIVE
    torch.cuda.set_device(local)
    n, pc, smp = args.dio_n, args.dio_pc, args.dio_sampling
    steps = args.dio_steps
    wl = workloads.diocotron_paper(n=n, pc=pc, sampling=smp, steps=steps)
    marks = sorted(set(int(round(k * steps / 7)) for k in range(8)))
    kw = dict(precision="fp32", mode=args.mode, centring=args.centring, B=wl.B, alpha=wl.extra["alpha"],
              pc_ref=wl.extra["pc_ref"])

    def trajectory(w, tau, history=False):
        t0 = time.perf_counter()
        run = Run(w.L, w.n, w.u.astype(np.float32), w.v.astype(np.float32), w.q.astype(np.float32), w.dt, tau=tau,
                  **kw)
        rho, E, taus = {}, {}, []
        done = 0
        for m in marks:
            if history:
                for _ in range(m - done):
                    run.step(1)
                    taus.append(run.diagnostics()["tau"])
            else:
                run.step(m - done)
            done = m
            rho[m] = run.density()
            E[m] = run.field()
        run.close()
        return rho, E, taus, time.perf_counter() - t0

    def nrmse(a, ref):
        return float(np.sqrt(np.sum((a - ref) ** 2) / np.sum(ref * ref)))

    # reference: mean over an ensemble of regular-PIC runs (tau = n) with more particles per cell
    ref_rho = {m: 0.0 for m in marks}
    ref_E = {m: 0.0 for m in marks}
    t_ref = 0.0
    for i in range(args.dio_ensemble):
        w = workloads.diocotron_paper(n=n, pc=args.dio_pc_ref, sampling=smp, steps=steps,
                                      seed=workloads.SEED_BASE + 600 + i)
        r, e, _, t = trajectory(w, n)
        t_ref += t
        for m in marks:
            ref_rho[m] = ref_rho[m] + r[m] / args.dio_ensemble
            ref_E[m] = ref_E[m] + e[m] / args.dio_ensemble
    runs = {"adaptive": SG_TAU_ADAPTIVE, "regular": n}
    for t in range(1, n - 2):
        runs[f"tau={t}"] = t
    out_runs = {}
    for name, tau in runs.items():
        r, e, taus, t = trajectory(wl, tau, history=(name == "adaptive"))
        out_runs[name] = {"rho_error": [nrmse(r[m], ref_rho[m]) for m in marks],
                          "E_error": [nrmse(e[m], ref_E[m]) for m in marks], "seconds": t}
        if taus:
            hist = {}
            for x in taus:
                hist[x] = hist.get(x, 0) + 1
            changes = [(i + 1, taus[i]) for i in range(len(taus)) if i == 0 or taus[i] != taus[i - 1]]
            out_runs[name]["tau_histogram"] = {str(k): v for k, v in sorted(hist.items())}
            out_runs[name]["tau_changes"] = changes[:200]
    out = {"metric": "diocotron (Section 5.1): NRMSE of rho and E against a regular-PIC ensemble mean",
           "config": {"workload": f"diocotron_paper n={n} ({1 << n}^2), P_c={pc}, {smp} sampling, "
                                  f"{wl.n_particles} FP32 particles, dt={wl.dt}, {steps} steps (T={steps * wl.dt:g})",
                      "mode": args.mode, "centring": args.centring, "alpha": wl.extra["alpha"],
                      "pc_ref": wl.extra["pc_ref"],
                      "reference": f"mean of {args.dio_ensemble} regular-PIC runs (tau = n), P_c = {args.dio_pc_ref}, "
                                   "same mesh, independent seeds",
                      "instants_t": [m * wl.dt for m in marks]},
           "runs": out_runs, "reference_seconds": t_ref, "data": "synthetic (seeded)"}
    if rank == 0:
        print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--particles", type=int, default=0, help="0: the workload's own count")
    ap.add_argument("--sort-every", type=int, default=0)
    ap.add_argument("--mode", default="combine", choices=["combine", "filter"],
                    help="combine: solves on every component grid, fields combined (the default line); "
                         "filter: the paper's filter mode (eq. sparse_filter, Algorithm 2)")
    ap.add_argument("--centring", default="node", choices=["node", "cell"],
                    help="node: nodes at k h (the default line); cell: nodes at cell centres with the "
                         "two-step shape of Appendix A")
    ap.add_argument("--solve-variant", default="auto", choices=["auto", "passes", "one-block"],
                    help="component-grid solve: timed choice at init (default), or fixed; a profiler's "
                         "serialised launches distort the timed choice, so profile with the variant the "
                         "plain run chose")
    ap.add_argument("--combine", default="float-float", choices=["float-float", "fp64"],
                    help="accumulation of the signed combination on the FP32 path: float pairs (the default "
                         "line) or double")
    ap.add_argument("--ref-particles", type=int, default=1 << 16)
    ap.add_argument("--ref-budget-s", type=float, default=120.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--workload", default="landau", choices=list(WORKLOAD_NAMES) + ["serving", "diocotron-paper"],
                    help="landau: the 2D n=10 Landau run (the default line); twostream3d (3D, n=7, "
                         "16,777,216 particles), diocotron2d (n=9, 8,388,608, Boris), penning3d (n=7, "
                         "2,097,152, Boris + quadrupole field): the paper's other workloads; serving: the "
                         "serving mix")
    ap.add_argument("--dio-n", type=int, default=9, help="diocotron-paper: level n (mesh 2^n x 2^n)")
    ap.add_argument("--dio-pc", type=int, default=5, help="diocotron-paper: particles per cell")
    ap.add_argument("--dio-sampling", default="gauss", choices=["gauss", "uniform"])
    ap.add_argument("--dio-steps", type=int, default=875, help="diocotron-paper: steps (875 = T 17.5)")
    ap.add_argument("--dio-ensemble", type=int, default=4, help="diocotron-paper: regular-PIC reference runs")
    ap.add_argument("--dio-pc-ref", type=int, default=80, help="diocotron-paper: particles per cell of the reference")
    ap.add_argument("--serving-runs", type=int, default=128)
    ap.add_argument("--serving-max-log2", type=int, default=23)
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    world, rank, local, pg = dist_setup(args)
    if args.workload == "serving":
        run_serving(args, world, rank, local)
        return
    if args.workload == "diocotron-paper":
        run_diocotron_paper(args, world, rank, local)
        return
    if args.impl == "reference":
        run_reference(args, world, rank, pg)
        return

    import torch
    from paper_2008_09441_gb300 import Run, workloads
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    # A dedicated stream (torch's default stream has handle 0, which the
    # library reads as "create your own"): the library, the L2 flush and the
    # timing events all run on it.
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.set_stream(stream)
    wname = WORKLOAD_NAMES[args.workload]
    over = {"seed": workloads.SEED_BASE + 1 + rank}
    if args.particles > 0:
        over["n_particles"] = args.particles
    wl = workloads.make(wname, **over)
    d, n = wl.dim, wl.n
    u = torch.from_numpy(wl.u.astype(np.float32)).to(dev)
    v = torch.from_numpy(wl.v.astype(np.float32)).to(dev)
    q = torch.from_numpy(wl.q.astype(np.float32)).to(dev)
    sort_every = args.sort_every if args.sort_every > 0 else (6 if d == 3 else 4)  # the library default
    run = Run(wl.L, n, u, v, q, wl.dt, tau=wl.tau, qm=wl.qm, B=wl.B, eext_lin=wl.eext_lin, precision="fp32",
              sort_every=sort_every, stream=stream.cuda_stream, mode=args.mode, centring=args.centring,
              combine=args.combine)
    if args.solve_variant != "auto":
        run.set_solve_variant(args.solve_variant)
    run_grids = run.grids()
    del u, v, q
    # L2 flush between steps: write one buffer larger than L2, then read a
    # second one, so that each step starts with none of its data in L2 and no
    # dirty lines of the flush buffer left for the step's first kernel to
    # write back.
    flush_w = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    flush_r = torch.zeros(L2_FLUSH_BYTES // 8, dtype=torch.float32, device=dev)
    flush_acc = torch.zeros((), dtype=torch.float32, device=dev)

    def flush_l2():
        flush_w.zero_()
        torch.sum(flush_r, dim=0, out=flush_acc)
    np_ = wl.n_particles

    # warm-up (graph capture happens here)
    run.step(args.warmup)
    torch.cuda.synchronize()

    # ---- timed region: K graph-launched steps, L2 flushed before each
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    clocks = ClockSampler(local)
    barrier(pg)
    torch.cuda.synchronize()
    clocks.start()
    l0 = run.kernel_launches()
    wall0 = time.perf_counter()
    # An NVTX range marks the timed steps, so that a profiler's launch list can
    # be restricted to them (ncu --nvtx --nvtx-include "sg_timed_steps/").
    torch.cuda.nvtx.range_push("sg_timed_steps")
    for k in range(args.steps):
        flush_l2()
        starts[k].record(stream)
        run.step(1)
        ends[k].record(stream)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    barrier(pg)
    clk = clocks.stop()
    launches = run.kernel_launches() - l0
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    tot_ms = max_over_ranks(pg, sum(step_ms))
    value = world * np_ * args.steps / (tot_ms * 1e-3)

    # ---- per-kernel durations (events between stages, same workload, L2 flushed)
    run.set_profiling(True)
    stage = {k: 0.0 for k in ["push", "sort", "deposit", "restrict", "solve", "combine"]}
    for k in range(args.steps):
        flush_l2()
        run.step(1)
        for key, val in run.stage_times().items():
            stage[key] += val
    run.set_profiling(False)
    torch.cuda.synchronize()
    stage_avg = {k: v / args.steps for k, v in stage.items()}
    alg = algorithmic_bytes(np_, n, d)
    peak, peak_kind = measured_peaks()
    rl = {}
    for kern in ("deposit", "push"):
        ms = stage_avg[kern]
        ach = alg[kern] / (ms * 1e-3) / 1e9 if ms > 0 else 0.0
        rl[kern] = {"achieved": ach, "frac": ach / peak, "ms": ms, "alg_bytes": alg[kern]}
    dominant = max(("deposit", "push"), key=lambda k: stage_avg[k])
    tr = traffic_record({"deposit": "k_deposit", "push": "k_push"}[dominant])
    roofline = {"bound": "hbm", "kernel": dominant, "achieved": rl[dominant]["achieved"], "peak": peak,
                "peak_kind": peak_kind, "unit": "GB/s", "frac": rl[dominant]["frac"],
                "traffic": (tr["dram_bytes_per_launch"] * (np_ / tr["particles"]) if tr else None),
                "per_kernel": {k: {"achieved_gbs": rl[k]["achieved"], "frac": rl[k]["frac"],
                                   "ms": rl[k]["ms"], "alg_bytes": rl[k]["alg_bytes"]} for k in rl},
                "stage_ms": stage_avg, "autotune": run.tuning()}

    # ---- end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        hu = [torch.from_numpy(np.ascontiguousarray(wl.u[:, m], dtype=np.float32)).pin_memory() for m in range(d)]
        hv = [torch.from_numpy(np.ascontiguousarray(wl.v[:, m], dtype=np.float32)).pin_memory() for m in range(d)]
        hq = torch.from_numpy(wl.q.astype(np.float32)).pin_memory()
        ou = torch.empty((d, np_), dtype=torch.float32).pin_memory()
        ov = torch.empty((d, np_), dtype=torch.float32).pin_memory()
        ow = torch.empty(np_, dtype=torch.float32).pin_memory()
        run.close()
        torch.cuda.synchronize()
        barrier(pg)
        from paper_2008_09441_gb300 import _lib as L
        import ctypes as C
        t0 = time.perf_counter()
        r2 = Run(wl.L, n, hu, hv, hq, wl.dt, tau=wl.tau, qm=wl.qm, B=wl.B, eext_lin=wl.eext_lin, precision="fp32",
                 sort_every=sort_every, stream=stream.cuda_stream, mode=args.mode, centring=args.centring,
                 combine=args.combine)
        if args.solve_variant != "auto":
            r2.set_solve_variant(args.solve_variant)
        diag_bytes = 0
        for s in range(args.steps):
            # a user monitoring the run: every step's FP64 diagnostics read
            # back to the host, collected one step behind so that the host
            # waits for step s-1's record while step s runs
            r2.step(1)
            r2.post_diagnostics()
            if s >= 1:
                r2.collect_diagnostics()
            diag_bytes += C.sizeof(L.sg_diag)
        o = L.sg_particles_out()
        o.n = np_
        o.on_device = 0
        for m in range(d):
            o.u[m] = ou[m].data_ptr()
            o.v[m] = ov[m].data_ptr()
        o.w = ow.data_ptr()
        L.check(L.lib().sg_pic_get_particles(r2.h, C.byref(o)), "get_particles")
        diag = r2.collect_diagnostics() if args.steps else r2.diagnostics()
        e2e_s = max_over_ranks(pg, time.perf_counter() - t0)
        r2.close()
        h2d = np_ * (2 * d + 1) * 4
        d2h = np_ * (2 * d + 1) * 4 + diag_bytes
        e2e = {"value": world * np_ * args.steps / e2e_s, "unit": UNIT,
               "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps,
               "includes": "sg_pic_init from pinned host arrays (copy, sort, first solve), K x (one step + its FP64 "
                           "diagnostics read back to the host through sg_pic_diagnostics_post / _collect, "
                           "one step behind), particles back to pinned host memory",
               "field_energy": diag["field_energy"]}
    else:
        run.close()

    cpu = None
    precision = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import tempfile
        with tempfile.TemporaryDirectory() as td:
            state = os.path.join(td, "oracle_state.npz")
            cpu = cpu_baseline(wname, state_path=state, mode=args.mode, centring=args.centring)
            precision = precision_vs_oracle(wname, cpu, state, stream, dev, args.mode, args.centring)

    if rank == 0:
        srt = sorted(step_ms)
        p50 = srt[len(srt) // 2]
        p99 = srt[min(len(srt) - 1, int(math.ceil(0.99 * len(srt))) - 1)]
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": tot_ms / args.steps, "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": "f32",
               "data": f"synthetic (seeded {wl.name} particles)",
               "config": {"workload": f"{wname}: {DESCRIPTIONS[wl.name]}, n={n}, tau={wl.tau}, "
                                      f"{len(run_grids)} component grids, {np_} FP32 particles, dt={wl.dt}",
                          "particles_per_gpu": np_, "sort_every": sort_every, "l2": "flushed before every step (512 MB written, then a different 256 MB read)",
                          "mode": args.mode + (" (stage 'solve' = density filter, 'combine' = regular-grid solve)"
                                               if args.mode == "filter" else ""),
                          "centring": args.centring,
                          "combine": ("float-float (48-bit)" if args.combine == "float-float" else "FP64") +
                                     " accumulation, FP64 diagnostics",
                          "parallelism": f"{world} independent replicas"},
               "latency_ms": {"p50": p50, "p99": p99},
               "roofline": roofline, "cpu_baseline": cpu, "precision": precision, "e2e": e2e,
               "gpu_launches": launches,
               "clocks": clk, "wall_s_timed": wall}
        print(json.dumps(out))
        sys.stdout.flush()
    barrier(pg)


if __name__ == "__main__":
    main()
