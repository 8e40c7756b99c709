"""The paper's 2D diocotron workloads (Section 5.1: Gaussian and uniform
weighted sampling, B_z = 5, L = 22, dt = 0.02, (P_c)_ref = 5 with alpha 0.01
/ 0.03) with Algorithm 1 choosing tau before every field evaluation, in the
paper's filter mode on cell-centred grids and in the combination mode:
the tau sequence and the particle state against the FP64 oracle; and the
density the fields come from (sg_pic_get_density) against the oracle's
sum_i c_i P_i rho_i."""
import numpy as np
import pytest

from oracle import sgpic_oracle as O
from paper_2008_09441_gb300 import workloads
from test_gpu_parity import TOL, make_run, nrmse, nrmse_periodic, torch_cuda  # noqa: F401

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("sampling", ["gauss", "uniform"])
@pytest.mark.parametrize("mode,centring", [("filter", "cell"), ("combine", "node")])
def test_diocotron_paper_adaptive_follows_oracle(torch_cuda, sampling, mode, centring):
    from paper_2008_09441_gb300._lib import SG_TAU_ADAPTIVE
    wl = workloads.diocotron_paper(n=7, pc=2, sampling=sampling, seed=71)
    a, pr = wl.extra["alpha"], wl.extra["pc_ref"]
    run, (u64, v64, q64) = make_run(wl, "fp64", torch_cuda, tau=SG_TAU_ADAPTIVE, alpha=a, pc_ref=pr, mode=mode,
                                    centring=centring)
    ref = O.OracleRun(wl.L, wl.n, u64, v64, q64, wl.dt, qm=wl.qm, B=wl.B, tau="adaptive", mode=mode, alpha=a,
                      pc_ref=pr, centring=centring)
    assert run.diagnostics()["tau"] == ref.tau_history[0]
    for s in range(3):
        run.step(1)
        ref.step(1)
        assert run.diagnostics()["tau"] == ref.tau_history[-1], s
        ug, vg, _ = run.particles()
        assert nrmse_periodic(ug, ref.u) < TOL["fp64"] and nrmse(vg, ref.velocities()) < TOL["fp64"], s
    run.close()


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("mode,centring", [("filter", "cell"), ("filter", "node"), ("combine", "node"),
                                           ("combine", "cell")])
def test_density_matches_oracle(torch_cuda, prec, mode, centring):
    wl = workloads.diocotron_paper(n=7, pc=3, sampling="gauss", tau=2, seed=73)
    run, (u64, v64, q64) = make_run(wl, prec, torch_cuda, mode=mode, centring=centring)
    u64 = O.wrap_unit(u64)
    rho = O.deposit_cic(u64, q64, (wl.n,) * 2, wl.L, centring)
    ref = O.density_filter(rho, wl.n, wl.tau, wl.L, centring)
    assert nrmse(run.density(), ref) < TOL[prec]
    run.close()
