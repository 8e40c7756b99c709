"""Host logic of the library on the CPU (no GPU, no CUDA call): the grid set
the engine builds, against the oracle's (pinned to the paper's patterns),
argument checks, and the footprint estimate that serving admits by."""
import pytest

from oracle import sgpic_oracle as O


@pytest.fixture(scope="module")
def sg():
    from paper_2008_09441_gb300 import sgpic
    return sgpic


@pytest.mark.parametrize("d,nmax", [(2, 12), (3, 8)])
def test_library_grid_set_equals_oracle(sg, d, nmax):
    for n in range(2, nmax + 1):
        for tau in range(1, n + 1):
            got = sg.sg_combination_grids(d, n, tau)
            ref = O.combination_grids(d, n, tau)
            assert sorted(got) == sorted(ref), (d, n, tau)
            # the library's order: q ascending (coefficient pattern), then lexicographic
            assert [c for _, c in got] == [c for _, c in ref], (d, n, tau)
            assert got == sorted(got, key=lambda lc: (-sum(lc[0]), lc[0])), (d, n, tau)


def test_grid_set_argument_checks(sg):
    from paper_2008_09441_gb300 import SGError
    for args in ((1, 5, 1), (4, 5, 1), (2, 0, 1), (2, 5, 0), (2, 5, 6)):
        with pytest.raises(SGError):
            sg.sg_combination_grids(*args)


def test_grid_set_capacity(sg):
    import ctypes as C
    import numpy as np
    from paper_2008_09441_gb300 import _lib as L
    cnt = C.c_int()
    levels = np.zeros(3, dtype=np.int32)
    coeffs = np.zeros(1, dtype=np.int32)
    st = L.lib().sg_combination_grids(2, 10, 1, levels.ctypes.data, coeffs.ctypes.data, 1, C.byref(cnt))
    assert st == L.SG_ERR_SIZE and cnt.value == 19


def test_footprint_estimate(sg):
    from paper_2008_09441_gb300 import SGError
    a = sg.sg_estimate_footprint("fp32", 2, 10, 1, 1 << 20)
    b = sg.sg_estimate_footprint("fp32", 2, 10, 1, 1 << 22)
    c = sg.sg_estimate_footprint("fp64", 2, 10, 1, 1 << 22)
    assert 0 < a < b < c
    # at least both particle sets (u, v, w per particle) and the regular grid
    assert b >= 2 * (1 << 22) * 5 * 4 + (1 << 20) * 4
    with pytest.raises(SGError):
        sg.sg_estimate_footprint("fp32", 4, 10, 1, 1000)


def test_diocotron_paper_workload_generator():
    """Section 5.1's initial conditions: total charge -400; Gaussian sampling
    puts r about L/4 with spread 0.03 L and v ~ N(0, 1); uniform sampling
    weights each particle by f at its phase-space point and drops charges
    below 1e-9."""
    import math
    import numpy as np
    from paper_2008_09441_gb300 import workloads
    g = workloads.diocotron_paper(n=7, pc=4, sampling="gauss", seed=5)
    L = g.L[0]
    assert g.n_particles == 4 << 14 and abs(g.q.sum() + 400.0) < 1e-9
    r = np.hypot(g.u[:, 0] * L - L / 2, g.u[:, 1] * L - L / 2)
    assert abs(r.mean() - L / 4) < 0.01 and abs(r.std() - 0.03 * L) < 0.01
    assert abs(g.v.std() - 1.0) < 0.01 and g.B == (0.0, 0.0, 5.0) and g.dt == 0.02
    assert g.extra["alpha"] == 0.01 and g.extra["pc_ref"] == 5.0
    un = workloads.diocotron_paper(n=7, pc=4, sampling="uniform", seed=5)
    assert abs(un.q.sum() + 400.0) < 1e-9 and np.all(np.abs(un.q) >= 1e-9) and un.extra["alpha"] == 0.03
    x = un.u * L
    rr = np.hypot(x[:, 0] - L / 2, x[:, 1] - L / 2)
    f = np.exp(-0.5 * np.sum(un.v ** 2, axis=1)) * np.exp(-((rr - L / 4) ** 2) / (2 * (0.03 * L) ** 2))
    ratio = un.q / f
    assert np.allclose(ratio, ratio[0], rtol=1e-9)  # charge proportional to f
    assert np.all(np.abs(un.v) <= 6.0) and math.isclose(un.dt, 0.02)
