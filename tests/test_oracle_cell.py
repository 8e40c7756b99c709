"""Pins of the oracle's cell-centred grids (nodes at cell centres, the
paper's own choice in Section 4.3; Appendix A's two-step shape W_c).

Hand-computed weights, closed-form Fourier symbols of the transfer
operators, a library interpolation routine, the three shape-function
conditions of Appendix A, and translation invariance of the regular-grid
run.  CPU only.
"""
import math

import numpy as np
import pytest

from oracle import sgpic_oracle as O


# ---------------------------------------------------------------- deposit and gather


def test_cell_deposit_bruteforce_hand():
    """Level (2, 2), unit box: centres at 1/8, 3/8, 5/8, 7/8.  u = (0.3, 0.9):
    x lies 0.175 past centre 0 (weights 0.3 / 0.7 on nodes 0 / 1), y lies
    0.025 past centre 3 (0.9 on node 3, 0.1 on node 0 across the boundary).
    u = (0.05, 0.625): x is 0.075 left of centre 0 (0.7 on node 0, 0.3 on
    node 3), y exactly on centre 2."""
    V = 1.0 / 16
    rho = O.deposit_cic(np.array([[0.3, 0.9]]), np.array([2.0]), (2, 2), (1.0, 1.0), "cell")
    expect = np.zeros((4, 4))
    expect[0, 3], expect[1, 3], expect[0, 0], expect[1, 0] = 0.3 * 0.9, 0.7 * 0.9, 0.3 * 0.1, 0.7 * 0.1
    np.testing.assert_allclose(rho, 2.0 * expect / V, rtol=1e-14, atol=0)
    rho = O.deposit_cic(np.array([[0.05, 0.625]]), np.array([1.0]), (2, 2), (1.0, 1.0), "cell")
    expect = np.zeros((4, 4))
    expect[0, 2], expect[3, 2] = 0.7, 0.3
    np.testing.assert_allclose(rho, expect / V, rtol=1e-14, atol=1e-12)


def test_cell_grid_is_node_grid_shifted_by_half_a_cell():
    """Brute force: W(x_k - x_p) with x_k = (k + 1/2) h evaluated node by node
    equals the oracle's cell-centred deposit."""
    rng = np.random.default_rng(3)
    u = rng.random((40, 2))
    q = rng.standard_normal(40)
    l = (3, 2)
    rho = O.deposit_cic(u, q, l, (1.0, 1.0), "cell")
    ref = np.zeros((8, 4))
    for p in range(40):
        for kx in range(8):
            for ky in range(4):
                w = 1.0
                for m, k in ((0, kx), (1, ky)):
                    M = 2 ** l[m]
                    dist = abs(u[p, m] * M - (k + 0.5))
                    dist = min(dist, M - dist)
                    w *= max(0.0, 1.0 - dist)
                ref[kx, ky] += q[p] * w * 32
    np.testing.assert_allclose(rho, ref, rtol=1e-12, atol=1e-12)


def test_cell_gather_reproduces_linear_field_between_centres():
    """CIC interpolation is exact for a field linear between neighbouring
    centres: E = x on centres 0..3 of a level-2 axis sampled inside
    [1/8, 7/8]."""
    field = np.tile(((np.arange(4) + 0.5) / 4)[:, None], (1, 4))
    u = np.stack([np.linspace(0.13, 0.86, 9), np.full(9, 0.4)], axis=1)
    np.testing.assert_allclose(O.gather_cic(field, u, (2, 2), "cell"), u[:, 0], rtol=0, atol=1e-15)


# ---------------------------------------------------------------- transfer operators


def test_cell_restriction_taps_hand():
    """h_l = 2h: (1, 3, 3, 1) / 8 on fine cells 2k-1 .. 2k+2; h_l = 4h:
    (1, 3, 5, 7, 7, 5, 3, 1) / 32 on 4k-2 .. 4k+5 (hat of half-width h_l
    at half-integer offsets, times h / h_l)."""
    n = 4
    N = 16
    R2 = O.restriction_matrix_1d(n, n - 1, "cell")
    R4 = O.restriction_matrix_1d(n, n - 2, "cell")
    for k in range(8):
        row = np.zeros(N)
        for off, w in zip(range(-1, 3), (1, 3, 3, 1)):
            row[(2 * k + off) % N] = w / 8
        np.testing.assert_allclose(R2[k], row, rtol=0, atol=1e-16)
    for k in range(4):
        row = np.zeros(N)
        for off, w in zip(range(-2, 6), (1, 3, 5, 7, 7, 5, 3, 1)):
            row[(4 * k + off) % N] = w / 32
        np.testing.assert_allclose(R4[k], row, rtol=0, atol=1e-16)
    np.testing.assert_array_equal(O.restriction_matrix_1d(n, n, "cell"), np.eye(N))


@pytest.mark.parametrize("centring", ["node", "cell"])
def test_restriction_fourier_symbol(centring):
    """R is a symmetric filter followed by sampling, so a Fourier mode on the
    fine nodes maps to the same mode on the coarse nodes times the filter's
    symbol.  With theta = 2 pi m / N and r = h_l / h: node-centred
    (sin(r theta/2) / (r sin(theta/2)))^2 (a hat of half-width r at integer
    offsets: two r-point boxes); cell-centred the same times cos(theta/2)
    (half-integer offsets: one more two-point average)."""
    n = 6
    N = 2 ** n
    o = 0.5 if centring == "cell" else 0.0
    j = np.arange(N)
    for lev in range(1, n + 1):
        r = 2 ** (n - lev)
        k = np.arange(2 ** lev)
        R = O.restriction_matrix_1d(n, lev, centring)
        for m in (1, 2, 3, 5, 11, 31):
            th = 2 * math.pi * m / N
            box = 1.0 if r == 1 else math.sin(r * th / 2) / (r * math.sin(th / 2))
            sym = box * box * (math.cos(th / 2) if (centring == "cell" and r > 1) else 1.0)
            for phase in (0.0, 0.7):
                fine = np.cos(th * (j + o) + phase)
                coarse = np.cos(th * r * (k + o) + phase)
                np.testing.assert_allclose(R @ fine, sym * coarse, rtol=0, atol=1e-13)


@pytest.mark.parametrize("n,lev", [(4, 1), (4, 2), (5, 3), (6, 5), (5, 5)])
def test_cell_prolongation_is_periodic_linear_interpolation(n, lev):
    """P_i along one axis = piecewise-linear interpolation of the coarse
    centre values at the fine centres, periodic (numpy.interp with
    period 1)."""
    rng = np.random.default_rng(n * 10 + lev)
    E = rng.standard_normal(2 ** lev)
    xc = (np.arange(2 ** lev) + 0.5) / 2 ** lev
    xf = (np.arange(2 ** n) + 0.5) / 2 ** n
    ref = np.interp(xf, xc, E, period=1.0)
    np.testing.assert_allclose(O.prolongation_matrix_1d(n, lev, "cell") @ E, ref, rtol=0, atol=1e-14)


def test_cell_prolongation_weights_hand():
    """h_l = 2h: fine centre 2k sits h/2 left of coarse centre k, weights
    1/4 (k-1) and 3/4 (k); h_l = 4h: fine centres 4k .. 4k+3 take
    (3/8, 5/8), (1/8, 7/8) from k-1, k and (7/8, 1/8), (5/8, 3/8) from k, k+1."""
    P2 = O.prolongation_matrix_1d(3, 2, "cell")
    assert P2[4, 1] == 0.25 and P2[4, 2] == 0.75 and P2[5, 2] == 0.75 and P2[5, 3] == 0.25
    P4 = O.prolongation_matrix_1d(4, 2, "cell")
    k = 1
    assert (P4[4 * k, k - 1], P4[4 * k, k]) == (0.375, 0.625)
    assert (P4[4 * k + 1, k - 1], P4[4 * k + 1, k]) == (0.125, 0.875)
    assert (P4[4 * k + 2, k], P4[4 * k + 2, k + 1]) == (0.875, 0.125)
    assert (P4[4 * k + 3, k], P4[4 * k + 3, k + 1]) == (0.625, 0.375)
    assert P4[0, 3] == 0.375 and P4[0, 0] == 0.625  # periodic wrap


def test_cell_restriction_prolongation_adjoint():
    """eq. restriction holds for either centring: R = (h / h_l) P^T."""
    for n in (3, 5):
        for lev in range(1, n + 1):
            R = O.restriction_matrix_1d(n, lev, "cell")
            P = O.prolongation_matrix_1d(n, lev, "cell")
            np.testing.assert_allclose(R, P.T / 2 ** (n - lev), rtol=0, atol=1e-16)


# ---------------------------------------------------------------- Appendix A: the two-step shape W_c


def _two_step_shape(x, n, lev):
    """W_c(x_k - x) for all coarse centres k of a level-lev x axis: a
    particle at (x, centre of y row 3) deposited on the level-n regular
    grid, restricted along x only; rho_l = q W_c / (h_l h_y)."""
    N = 2 ** n
    y = (3 + 0.5) / N
    q = 1.0
    rho = O.deposit_cic(np.array([[x, y]]), np.array([q]), (n, n), (1.0, 1.0), "cell")
    rl = O.restrict(rho, n, (lev, n), "cell")
    return rl[:, 3] * (1.0 / 2 ** lev) * (1.0 / N) / q


@pytest.mark.parametrize("n,lev", [(5, 5), (5, 4), (5, 2), (6, 3)])
def test_appendix_a_two_step_shape_conditions(n, lev):
    """Appendix A's three conditions for W_c(zeta) = sum_j W_c(x_k - x~_j)
    W_f(x~_j - x): (1) even, (2) (1/h_c) integral = 1 (W_c is piecewise
    linear with kinks at fine centres, so the trapezoid rule on a grid that
    contains them is exact), (3) partition of unity."""
    N, M = 2 ** n, 2 ** lev
    rng = np.random.default_rng(n + lev)
    for x in rng.random(20):  # (3)
        assert abs(_two_step_shape(x, n, lev).sum() - 1.0) < 1e-13
    k = M // 2
    xk = (k + 0.5) / M
    for z in rng.random(10) * 1.5 / M:  # (1)
        a = _two_step_shape(xk + z, n, lev)[k]
        b = _two_step_shape(xk - z, n, lev)[k]
        assert abs(a - b) < 1e-13
    sub = 8  # (2): sample every 1/(8N), kinks at (j + 1/2)/N are sample points
    xs = (np.arange(N * sub) + 0.5 * sub) / (N * sub)
    vals = np.array([_two_step_shape(x, n, lev)[k] for x in xs])
    integral = vals.sum() / (N * sub)  # periodic trapezoid = mean x length
    assert abs(integral * M - 1.0) < 1e-12


def test_appendix_a_two_step_differs_from_direct_when_coarser():
    """Proposition 1's cell-centred remark: the two-step densities are not the
    direct deposit once h_l > h (kinks of the coarse hat fall between fine
    centres), and coincide at h_l = h."""
    rng = np.random.default_rng(9)
    u = rng.random((500, 2))
    q = rng.standard_normal(500)
    n = 5
    reg = O.deposit_cic(u, q, (n, n), (1.0, 1.0), "cell")
    same = O.restrict(reg, n, (n, n), "cell")
    np.testing.assert_allclose(same, O.deposit_cic(u, q, (n, n), (1.0, 1.0), "cell"), rtol=0, atol=1e-12)
    two = O.restrict(reg, n, (3, n), "cell")
    direct = O.deposit_cic(u, q, (3, n), (1.0, 1.0), "cell")
    assert np.max(np.abs(two - direct)) > 1e-3 * np.max(np.abs(direct))
    # both conserve the charge
    assert abs(two.sum() * (1 / 8) * (1 / 32) - q.sum()) < 1e-12 * np.abs(q).sum()


# ---------------------------------------------------------------- filter and runs


@pytest.mark.parametrize("d,n,tau", [(2, 6, 1), (2, 5, 2), (3, 4, 1)])
def test_cell_filter_invariants(d, n, tau):
    """Cell-centred filter: charge and constants preserved, symmetric in the
    grid inner product, identity at tau = n, one-axis densities pass, the
    checkerboard (symbol factor cos(pi/2) = 0) is removed."""
    rng = np.random.default_rng(40 + n + d)
    shape = (2 ** n,) * d
    L = [1.0] * d
    a = rng.standard_normal(shape)
    b = rng.standard_normal(shape)
    fa = O.density_filter(a, n, tau, L, "cell")
    assert abs(fa.sum() - a.sum()) < 1e-11 * np.abs(a).sum()
    assert np.allclose(O.density_filter(np.full(shape, 2.5), n, tau, L, "cell"), 2.5, rtol=0, atol=1e-13)
    lhs = float(np.sum(b * fa))
    rhs = float(np.sum(O.density_filter(b, n, tau, L, "cell") * a))
    assert abs(lhs - rhs) < 1e-12 * (abs(lhs) + 1.0)
    assert np.allclose(O.density_filter(a, n, n, L, "cell"), a, rtol=0, atol=1e-13)
    line = np.broadcast_to(rng.standard_normal(2 ** n).reshape((-1,) + (1,) * (d - 1)), shape).copy()
    assert np.allclose(O.density_filter(line, n, tau, L, "cell"), line, rtol=0, atol=1e-12)
    idx = np.indices(shape).sum(axis=0)
    chk = np.where(idx % 2 == 0, 1.0, -1.0)
    assert np.max(np.abs(O.density_filter(chk, n, tau, L, "cell"))) < 1e-13


@pytest.mark.parametrize("mode", ["combine", "filter"])
def test_cell_regular_run_is_shifted_node_run(mode):
    """tau = n leaves the regular grid alone, and a cell-centred regular grid
    is the node-centred one translated by h/2: a periodic run of particles at
    u on cell centres equals the node-centred run of particles at u - h/2,
    translated back."""
    rng = np.random.default_rng(17)
    npart, n = 2000, 5
    L = (4 * np.pi, 4 * np.pi)
    u = rng.random((npart, 2))
    v = rng.standard_normal((npart, 2))
    q = -np.full(npart, L[0] * L[1] / npart) * (1 + 0.3 * np.cos(2 * np.pi * u[:, 0]))
    h = 0.5 / 2 ** n
    a = O.OracleRun(L, n, u, v, q, 0.05, tau=n, mode=mode, centring="cell")
    b = O.OracleRun(L, n, O.wrap_unit(u - h), v, q, 0.05, tau=n, mode=mode, centring="node")
    for _ in range(3):
        a.step(1)
        b.step(1)
    du = (a.u - O.wrap_unit(b.u + h) + 0.5) % 1.0 - 0.5
    assert np.max(np.abs(du)) < 1e-12
    assert np.max(np.abs(a.velocities() - b.velocities())) < 1e-11
    assert abs(a.field_energy() - b.field_energy()) < 1e-11 * a.field_energy()


@pytest.mark.parametrize("d,n,tau", [(2, 5, 1), (3, 4, 1)])
def test_cell_run_conserves_charge_on_every_grid(d, n, tau):
    rng = np.random.default_rng(23 + d)
    npart = 1500
    L = (2.0, 3.0, 5.0)[:d]
    u = rng.random((npart, d))
    v = rng.standard_normal((npart, d))
    q = rng.normal(-1.0, 0.2, npart)
    run = O.OracleRun(L, n, u, v, q, 0.02, tau=tau, centring="cell")
    run.step(2)
    dg = run.diagnostics()
    assert dg["charge_grid_max_abs_err"] < 1e-11 * abs(dg["charge_total"])
    assert abs(dg["charge_combined"] - dg["charge_total"]) < 1e-11 * abs(dg["charge_total"])


@pytest.mark.parametrize("centring", ["node", "cell"])
def test_prolong_at_equals_prolong(centring):
    """prolong_at (rows of P at chosen regular nodes) == prolong, sampled."""
    rng = np.random.default_rng(61)
    n, l = 6, (3, 5)
    E = rng.standard_normal((8, 32))
    full = O.prolong(E, n, l, centring)
    idx = rng.integers(0, 64, size=(300, 2))
    np.testing.assert_allclose(O.prolong_at(E, n, l, idx, centring), full[idx[:, 0], idx[:, 1]], rtol=0, atol=1e-14)
