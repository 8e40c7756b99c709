"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test ties one oracle function to something other than itself: the
paper's printed patterns and closed forms, brute force on tiny inputs,
Proposition 1, invariants (charge conservation, |v| under rotation) and
textbook single-mode solutions.  CPU only.
"""
import itertools
import math

import numpy as np
import pytest

from oracle import sgpic_oracle as O

RNG = np.random.default_rng(12345)


# ---------------------------------------------------------------- grid set


@pytest.mark.parametrize("n", range(2, 11))
def test_combination_2d_pattern(n):
    for tau in range(1, n + 1):
        g = O.combination_grids(2, n, tau)
        plus = [l for l, c in g if c == 1]
        minus = [l for l, c in g if c == -1]
        assert len(g) == len(plus) + len(minus)
        # Section 4.3.1: n-(tau-1) grids with i+j = n+tau, (n-1)-(tau-1) with i+j = n+tau-1
        assert sorted(plus) == sorted((i, n + tau - i) for i in range(tau, n + 1))
        assert sorted(minus) == sorted((i, n + tau - 1 - i) for i in range(tau, n))
        assert len(plus) == n - tau + 1 and len(minus) == n - tau
        assert sum(c for _, c in g) == 1
    assert O.combination_grids(2, n, n) == [((n, n), 1)]  # tau = n: the regular grid


def test_combination_configs():
    g = O.combination_grids(2, 6, 1)
    assert len(g) == 11 and sum(2 ** sum(l) for l, _ in g) == 1088
    g = O.combination_grids(2, 10, 1)
    assert len(g) == 19 and sum(2 ** sum(l) for l, _ in g) == 29696
    g = O.combination_grids(2, 9, 1)
    assert len(g) == 17 and sum(2 ** sum(l) for l, _ in g) == 13312
    g = O.combination_grids(3, 7, 1)
    assert len(g) == 64 and sum(2 ** sum(l) for l, _ in g) == 21632
    by = {}
    for l, c in g:
        by.setdefault(sum(l), set()).add(c)
        assert all(1 <= x <= 7 for x in l)
    assert by == {9: {1}, 8: {-2}, 7: {1}}  # 3D binomial pattern +1, -2, +1


@pytest.mark.parametrize("n", range(3, 9))
def test_combination_3d_sum_and_regular(n):
    for tau in range(1, n + 1):
        g = O.combination_grids(3, n, tau)
        assert sum(c for _, c in g) == 1
        assert all(min(l) >= tau for l, _ in g)
    assert O.combination_grids(3, n, n) == [((n, n, n), 1)]


@pytest.mark.parametrize("d", [2, 3])
def test_estimator_brackets_follow_grid_set(d):
    """The printed noise and grid-error brackets (Section 4.3.1/4.3.2) equal
    sums over the grid set: noise counts each grid once, the mixed-derivative
    error term weights each grid by |c| (h_1..h_d products squared)."""
    L, Np, sigma = 3.7, 1e6, 1.3
    for n in range(4, 10):
        h = L / 2 ** n
        for tau in range(1, n + 1):
            g = O.combination_grids(d, n, tau)
            vols = [np.prod([L / 2 ** lm for lm in l]) for l, _ in g]
            noise_sum = sigma * sum(1.0 / math.sqrt(Np * V) for V in vols)
            noise = O.particle_noise_estimate(d, n, tau, L, Np, sigma)
            assert noise == pytest.approx(noise_sum, rel=1e-12)
            m = n - tau
            if d == 2:
                # grid term: h^2 beta L^2 2^{-2tau}[5m+1] == sum |c| (h_i h_j)^2
                mixed = sum(abs(c) * V * V for (l, c), V in zip(g, vols))
                assert h * h * L * L * 2.0 ** (-2 * tau) * (5 * m + 1) == pytest.approx(mixed, rel=1e-12)
            else:
                mixed = sum(abs(c) * V * V for (l, c), V in zip(g, vols))
                printed = h * h * L ** 4 * 2.0 ** (-(4 * tau + 1)) * (25 * m * m - 5 * m + 2)
                assert printed == pytest.approx(mixed, rel=1e-12)


@pytest.mark.parametrize("d", [2, 3])
def test_estimator_regular_grid_reduction(d):
    """tau = n recovers regular-PIC estimates (Section 4.3, Appendix B)."""
    L, Np, sigma = 2.0, 5e5, 0.7
    for n in range(3, 9):
        h = L / 2 ** n
        assert O.particle_noise_estimate(d, n, n, L, Np, sigma) == pytest.approx(
            sigma / math.sqrt(Np * h ** d), rel=1e-12)
        kap = [0.3, 0.5, 0.7][:d]
        beta = [1.1] if d == 2 else [1.1, 1.3, 1.7]
        gam = 0.0 if d == 2 else 1.9
        expect = h * h * sum(kap) + sum(beta) * h ** 4 + gam * h ** 6
        assert O.grid_error_estimate(d, n, n, L, kap, beta, gam) == pytest.approx(expect, rel=1e-12)


def test_tau_range():
    assert O.tau_range(2, 10) == list(range(1, 8))
    assert O.tau_range(3, 7) == list(range(1, 6))
    assert O.tau_range(2, 3) == []


# ---------------------------------------------------------------- keys, sort


def test_wrap_unit():
    u = np.array([[-1e-30, 0.5], [1.0, 2.25], [-0.25, 0.999999999]])
    w = O.wrap_unit(u)
    assert np.all((w >= 0) & (w < 1))
    assert w[0, 0] == 0.0 and w[1, 0] == 0.0 and w[1, 1] == 0.25 and w[2, 0] == 0.75


def test_morton_key_bruteforce():
    for d, n in [(2, 3), (3, 2), (2, 5)]:
        N = 2 ** n
        cells = list(itertools.product(range(N), repeat=d))
        u = np.array([[(c + 0.5) / N for c in cell] for cell in cells])
        keys = O.cell_keys(u, n)
        for cell, k in zip(cells, keys):
            expect = 0
            for b in range(n):
                for m in range(d):
                    if (cell[m] >> b) & 1:
                        expect += 2 ** (b * d + m)
            assert int(k) == expect
        assert sorted(int(k) for k in keys) == list(range(N ** d))  # bijection


def test_keys_at_cell_boundaries():
    n = 4
    u = np.array([[k / 16.0, (15 - k) / 16.0] for k in range(16)])
    idx = O.cell_index(u, n)
    assert np.array_equal(idx[:, 0], np.arange(16)) and np.array_equal(idx[:, 1], 15 - np.arange(16))


def test_stable_sort_and_counts():
    n, d = 4, 2
    u = RNG.random((5000, d))
    keys = O.cell_keys(u, n)
    perm, sk, counts = O.sort_by_key(keys, n, d)
    assert np.all(np.diff(sk.astype(np.int64)) >= 0)
    assert counts.sum() == 5000 and counts.size == 256
    # stability: equal keys keep increasing original index
    for k in np.unique(keys):
        idx = perm[sk == k]
        assert np.all(np.diff(idx.astype(np.int64)) > 0)
    assert O.count_checksum(counts) == int(np.sum(keys.astype(np.uint64) + 1))


# ---------------------------------------------------------------- deposit


def test_deposit_bruteforce_hand():
    """One particle at u = (0.3, 0.6) on levels (2, 1): s = (1.2, 1.2),
    weights 0.8/0.2 per axis; y-corner 2 wraps to node 0."""
    L = (2.0, 3.0)
    l = (2, 1)
    V = (2.0 / 4) * (3.0 / 2)
    rho = O.deposit_cic(np.array([[0.3, 0.6]]), np.array([1.5]), l, L)
    expect = np.zeros((4, 2))
    expect[1, 1] = 0.8 * 0.8
    expect[2, 1] = 0.2 * 0.8
    expect[1, 0] = 0.8 * 0.2
    expect[2, 0] = 0.2 * 0.2
    np.testing.assert_allclose(rho, 1.5 * expect / V, rtol=1e-15, atol=0)


def test_deposit_on_node_and_symmetry():
    L = (1.0, 1.0, 1.0)
    l = (3, 2, 1)
    # particle exactly on node (2, 1, 1): all charge on that node
    rho = O.deposit_cic(np.array([[2 / 8, 1 / 4, 1 / 2]]), np.array([2.0]), l, L)
    V = 1 / 8 * 1 / 4 * 1 / 2
    assert rho[2, 1, 1] == pytest.approx(2.0 / V) and np.count_nonzero(rho) == 1
    # mirror symmetry of the shape (Appendix A condition 1)
    a = O.deposit_cic(np.array([[0.5 + 0.03, 0.5]]), np.array([1.0]), (4, 4), (1, 1))
    b = O.deposit_cic(np.array([[0.5 - 0.03, 0.5]]), np.array([1.0]), (4, 4), (1, 1))
    np.testing.assert_allclose(a, b[::-1, :][np.r_[15, 0:15], :], rtol=1e-13)


@pytest.mark.parametrize("d", [2, 3])
def test_charge_conservation_every_grid(d):
    L = (4.0, 2.5, 1.5)[:d]
    u = RNG.random((3000, d))
    q = RNG.normal(-1.0, 0.3, 3000)
    for l, _ in O.combination_grids(d, 5 if d == 2 else 4, 1):
        rho = O.deposit_cic(u, q, l, L)
        assert float(np.sum(rho)) * O.cell_volume(l, L) == pytest.approx(float(np.sum(q)), rel=1e-13)


@pytest.mark.parametrize("d,n", [(2, 5), (3, 4)])
def test_proposition1_direct_equals_two_step(d, n):
    """Proposition 1 (node-centred, linear shapes): direct deposit on a
    component grid == deposit on the regular grid followed by R_i."""
    L = (2.0, 3.0, 5.0)[:d]
    u = RNG.random((2000, d))
    q = RNG.random(2000) - 1.3
    reg = O.deposit_cic(u, q, (n,) * d, L)
    for tau in (1, 2):
        for l, _ in O.combination_grids(d, n, tau):
            direct = O.deposit_cic(u, q, l, L)
            two = O.restrict(reg, n, l)
            scale = np.max(np.abs(direct))
            assert np.max(np.abs(direct - two)) <= 1e-13 * scale


def test_restriction_prolongation_adjoint():
    """eq. restriction: R_i = (h^d / V_i) P_i^T, one axis at a time."""
    for n in (3, 5):
        for l in range(1, n + 1):
            R = O.restriction_matrix_1d(n, l)
            P = O.prolongation_matrix_1d(n, l)
            np.testing.assert_allclose(R, P.T * (2 ** l / 2 ** n), rtol=0, atol=1e-15)
            np.testing.assert_allclose(P.sum(axis=1), 1.0, rtol=1e-15)  # partition of unity


# ---------------------------------------------------------------- solve


@pytest.mark.parametrize("shape,L,mode", [
    ((16, 8), (2.0, 3.0), (3, 2)),
    ((32, 2), (4 * math.pi, 4 * math.pi), (1, 0)),
    ((8, 8, 4), (1.0, 2.0, 3.0), (1, 3, 1)),
    ((64, 4), (5.0, 1.0), (-5, 1)),
])
def test_solve_single_mode(shape, L, mode):
    """rho = cos(k.x) gives phi = rho/|k|^2, E = k sin(k.x)/|k|^2 exactly."""
    d = len(shape)
    k = [2 * math.pi * mode[m] / L[m] for m in range(d)]
    X = np.meshgrid(*[np.arange(shape[m]) * L[m] / shape[m] for m in range(d)], indexing="ij")
    ph = sum(k[m] * X[m] for m in range(d))
    rho = np.cos(ph)
    k2 = sum(x * x for x in k)
    E = O.solve_poisson_spectral(rho, L)
    phi = O.potential_spectral(rho, L)
    np.testing.assert_allclose(phi, rho / k2, atol=1e-13)
    for m in range(d):
        np.testing.assert_allclose(E[m], k[m] * np.sin(ph) / k2, atol=1e-13)


def test_solve_nyquist_and_mean():
    L = (2.0, 2.0)
    j = np.arange(8)
    rho = np.cos(math.pi * j)[:, None] * np.ones((1, 4)) + 3.0  # Nyquist along x + mean
    E = O.solve_poisson_spectral(rho, L)
    np.testing.assert_allclose(E[0], 0.0, atol=1e-14)
    np.testing.assert_allclose(E[1], 0.0, atol=1e-14)
    phi = O.potential_spectral(rho, L)
    kn = math.pi * 8 / 2.0
    np.testing.assert_allclose(phi, (rho - 3.0) / kn ** 2, atol=1e-14)


# ---------------------------------------------------------------- combine / gather


@pytest.mark.parametrize("d,n,tau", [(2, 5, 1), (2, 5, 3), (3, 4, 1)])
def test_gather_dual_of_proposition1(d, n, tau):
    """sum_i c_i I_i[E_i](x_p) == CIC gather from sum_i c_i P_i E_i on the
    regular nodes (nested node-centred grids: a coarse multilinear
    interpolant is multilinear in every fine cell)."""
    L = (3.0, 2.0, 1.0)[:d]
    u = RNG.random((1500, d))
    q = RNG.random(1500) - 1.5
    comps = O.component_fields(u, q, n, tau, L)
    direct = O.field_at_particles(comps, u, L, (0, 0, 0))
    comb = O.combined_field_regular(comps, n, d)
    for m in range(d):
        via = O.gather_cic(comb[m], u, (n,) * d)
        assert np.max(np.abs(direct[m] - via)) <= 1e-12 * np.max(np.abs(direct[m]))


def test_axis_aligned_cancellation():
    """For an x-only density (uniform lattice in y), every grid with the same
    l_1 carries the same field, the +1/-1 pairs cancel and the combination
    equals the (n, tau) grid's field (the 2D coefficient pattern)."""
    n, tau = 6, 2
    L = (2.0, 2.0)
    nx = 4096
    ny = 2 ** n
    ux = (np.arange(nx) + 0.37) / nx
    uy = np.arange(ny) / ny
    UX, UY = np.meshgrid(ux, uy, indexing="ij")
    u = np.stack([UX.ravel(), UY.ravel()], axis=1)
    q = -(1.0 + 0.3 * np.cos(2 * math.pi * u[:, 0])) / u.shape[0]
    comps = O.component_fields(u, q, n, tau, L)
    comb = O.combined_field_regular(comps, n, 2)
    ref = [c for c in comps if c[0] == (n, tau)][0]
    for m in range(2):
        np.testing.assert_allclose(comb[m], O.prolong(ref[3][m], n, (n, tau)), atol=1e-12)


# ---------------------------------------------------------------- push


def test_free_streaming_exact():
    u = RNG.random((100, 2))
    v = [RNG.normal(size=100), RNG.normal(size=100)]
    E = [np.zeros(100), np.zeros(100)]
    v2 = O.kick_rotate(v, E, -1.0, 0.1, (0, 0, 0))
    assert all(np.array_equal(v[m], v2[m]) for m in range(2))
    u2 = O.drift(u, v2, 0.1, (2.0, 3.0))
    expect = np.stack([u[:, 0] + v[0] * 0.1 / 2.0, u[:, 1] + v[1] * 0.1 / 3.0], axis=1)
    np.testing.assert_array_equal(u2, O.wrap_unit(expect))


def test_boris_rotation_2d():
    """E = 0, uniform B_z: |v| conserved, rotation angle 2 atan(w_c dt / 2)."""
    qm, Bz, dt = -1.0, 5.0, 0.02
    v = [np.array([1.0, 0.3]), np.array([0.0, -2.0])]
    E = [np.zeros(2), np.zeros(2)]
    vn = O.kick_rotate(v, E, qm, dt, (0, 0, Bz))
    sp0 = np.hypot(v[0], v[1])
    sp1 = np.hypot(vn[0], vn[1])
    np.testing.assert_allclose(sp1, sp0, rtol=1e-15)
    ang = np.arctan2(vn[1], vn[0]) - np.arctan2(v[1], v[0])
    ang = (ang + math.pi) % (2 * math.pi) - math.pi
    wc = qm * Bz
    np.testing.assert_allclose(ang, -2 * math.atan(wc * dt / 2), rtol=1e-13)


def test_boris_rotation_3d():
    qm, B, dt = -1.0, (0.3, -1.1, 2.0), 0.05
    v = [RNG.normal(size=50) for _ in range(3)]
    E = [np.zeros(50)] * 3
    vn = O.kick_rotate(v, E, qm, dt, B)
    sp0 = np.sqrt(sum(x * x for x in v))
    sp1 = np.sqrt(sum(x * x for x in vn))
    np.testing.assert_allclose(sp1, sp0, rtol=1e-14)
    bn = np.array(B) / np.linalg.norm(B)
    par0 = sum(v[m] * bn[m] for m in range(3))
    par1 = sum(vn[m] * bn[m] for m in range(3))
    np.testing.assert_allclose(par1, par0, rtol=1e-13, atol=1e-15)


# ---------------------------------------------------------------- Appendix B


def test_appendix_b_second_moment():
    """Appendix B.1: the CIC-smoothed density is rho + (h^2/12) rho'' + ...
    Depositing a dense quadrature of cos(kx) gives cos(k x_j) times the
    CIC transfer factor; its h^2 coefficient is -k^2/12."""
    L = (1.0, 1.0)
    k = 2 * math.pi
    M = 1 << 15
    ratios = []
    for n in (4, 5, 6):
        ux = (np.arange(M) + 0.5) / M
        u = np.stack([ux, np.full(M, 0.25)], axis=1)
        q = np.cos(k * ux) / M
        rho = O.deposit_cic(u, q, (n, 1), L).sum(axis=1) * 0.5  # integrate out y (h_y = 1/2)
        xj = np.arange(2 ** n) / 2 ** n
        h = 1.0 / 2 ** n
        ratio = rho[0] / np.cos(k * xj[0])
        ratios.append((h, ratio))
    for h, r in ratios:
        c2 = (1.0 - r) / (k * k * h * h)
        assert c2 == pytest.approx(1.0 / 12.0, rel=0.02)


@pytest.mark.parametrize("d", [2, 3])
def test_appendix_b_noise_variance(d):
    """Appendix B.2: Var(rho~) = (2/3)^d Q rho / (N_p h^d) for independent
    uniform particles (exact finite-N_p form includes the -rho^2/N_p term)."""
    rng = np.random.default_rng(7 + d)
    n = 5 if d == 2 else 3
    Np = 200000
    L = (1.0,) * d
    Q = -2.0
    vals = []
    for _ in range(4):
        u = rng.random((Np, d))
        rho = O.deposit_cic(u, np.full(Np, Q / Np), (n,) * d, L)
        vals.append(rho.ravel())
    var = np.var(np.concatenate(vals))
    h = 1.0 / 2 ** n
    rho0 = Q
    expect = (2.0 / 3.0) ** d * Q * rho0 / (Np * h ** d) - rho0 ** 2 / Np
    assert var == pytest.approx(expect, rel=0.05)


# ---------------------------------------------------------------- estimator


def test_estimator_single_mode_constants():
    """Noise-free single mode: the eq. grid_constants norms have closed forms
    (kappa_x = 1/4 kx^2 A, beta = 1/72 kx^2 ky^2 A); the empirical form keeps
    the mode amplitude A/4 of each of the 4 Fourier peaks."""
    n, L = 6, 2.0
    N = 2 ** n
    kx, ky = 2 * math.pi * 2 / L, 2 * math.pi * 3 / L
    X = np.meshgrid(np.arange(N) * L / N, np.arange(N) * L / N, indexing="ij")
    A, rho0 = 0.2, -1.0
    rho = rho0 + A * np.cos(kx * X[0]) * np.cos(ky * X[1])
    tau, table, c = O.tau_estimator(rho, Np=1e6, L=L, alpha=0.01, pc_ref=5, Qe=-4.0, constants="paper")
    assert c["kappa"][0] == pytest.approx(0.25 * kx * kx * A, rel=1e-10)
    assert c["kappa"][1] == pytest.approx(0.25 * ky * ky * A, rel=1e-10)
    assert c["beta"][0] == pytest.approx(kx * kx * ky * ky * A / 72, rel=1e-10)
    assert c["sigma"] == pytest.approx(math.sqrt((4 / 9) * 4.0 * (1.0 + A)), rel=1e-12)
    tau2, table2, c2 = O.tau_estimator(rho, Np=1e6, L=L, alpha=0.01, pc_ref=5, Qe=-4.0, constants="empirical")
    assert c2["kappa"][0] == pytest.approx(kx * kx * A / 4, rel=1e-10)
    assert c2["beta"][0] == pytest.approx(kx * kx * ky * ky * A / 4, rel=1e-10)
    assert [t for t, _, _ in table] == list(range(1, n - 2))
    best = min(table, key=lambda r: (r[1] + r[2], r[0]))
    assert tau == best[0]


def test_estimator_threshold_drops_small_modes():
    n, L = 5, 1.0
    N = 2 ** n
    X = np.meshgrid(np.arange(N) / N, np.arange(N) / N, indexing="ij")
    big = np.cos(2 * math.pi * X[0])
    small = 1e-4 * np.cos(2 * math.pi * 7 * X[0]) * np.cos(2 * math.pi * 9 * X[1])
    _, _, c = O.tau_estimator(big + small - 2.0, Np=N * N * 5, L=L, alpha=0.01, pc_ref=5, Qe=-1.0)
    kx = 2 * math.pi
    # the small mixed mode (below eps) leaves no trace in beta
    assert c["beta"][0] == pytest.approx(0.0, abs=1e-9)
    assert c["kappa"][0] == pytest.approx(0.25 * kx * kx, rel=1e-10)


# ------------------------------------------------------------ filter mode (eq. sparse_filter, Algorithm 2)


@pytest.mark.parametrize("d,n", [(2, 5), (3, 3)])
def test_filter_tau_n_is_identity(d, n):
    """tau = n leaves the single regular grid: the filter is the identity."""
    rng = np.random.default_rng(70 + d)
    rho = rng.standard_normal((2 ** n,) * d)
    assert np.allclose(O.density_filter(rho, n, n, [1.0] * d), rho, rtol=0, atol=1e-13)


@pytest.mark.parametrize("d,n,tau", [(2, 6, 1), (2, 5, 2), (3, 4, 1)])
def test_filter_conserves_charge_and_constants(d, n, tau):
    """Every P_i R_i conserves h^d sum rho and the coefficients sum to 1, so
    the filter conserves the total charge and maps a constant to itself."""
    rng = np.random.default_rng(80 + n)
    rho = rng.standard_normal((2 ** n,) * d)
    rf = O.density_filter(rho, n, tau, [1.0] * d)
    assert abs(rf.sum() - rho.sum()) < 1e-11 * np.abs(rho).sum()
    const = np.full((2 ** n,) * d, 3.25)
    assert np.allclose(O.density_filter(const, n, tau, [1.0] * d), const, rtol=0, atol=1e-13)


@pytest.mark.parametrize("d,n,tau", [(2, 6, 1), (3, 4, 1)])
def test_filter_is_self_adjoint(d, n, tau):
    """R_i = (h^d / V_i) P_i^T makes each P_i R_i symmetric in the regular
    grid's inner product, hence the whole filter: <a, F b> = <F a, b>."""
    rng = np.random.default_rng(90 + d)
    a = rng.standard_normal((2 ** n,) * d)
    b = rng.standard_normal((2 ** n,) * d)
    lhs = float(np.sum(a * O.density_filter(b, n, tau, [1.0] * d)))
    rhs = float(np.sum(O.density_filter(a, n, tau, [1.0] * d) * b))
    assert abs(lhs - rhs) < 1e-12 * (abs(lhs) + 1.0)


@pytest.mark.parametrize("n,tau", [(6, 1), (7, 3)])
def test_filter_passes_single_axis_densities(n, tau):
    """2D: for rho(x) alone the y-restrictions are exact and the x parts
    telescope, sum over a of P R_a with +1 minus the same with -1 leaves the
    level-n term: a density varying along one axis passes unchanged."""
    rng = np.random.default_rng(100 + n)
    fx = rng.standard_normal(2 ** n)
    rho_x = np.repeat(fx[:, None], 2 ** n, axis=1)  # [i_x, i_y]
    rho_y = rho_x.T.copy()
    for r in (rho_x, rho_y):
        assert np.allclose(O.density_filter(r, n, tau, [1.0, 1.0]), r, rtol=0, atol=1e-12)


@pytest.mark.parametrize("d,n,tau", [(2, 6, 1), (2, 6, 4), (3, 4, 1)])
def test_filter_annihilates_the_checkerboard(d, n, tau):
    """Full weighting maps the Nyquist mode (-1)^i to zero, and every
    component grid is restricted along at least one axis unless tau = n:
    the (Nyquist, ..., Nyquist) checkerboard is filtered out entirely."""
    idx = np.indices((2 ** n,) * d).sum(axis=0)
    rho = np.where(idx % 2 == 0, 1.0, -1.0)
    assert np.max(np.abs(O.density_filter(rho, n, tau, [1.0] * d))) < 1e-13


def test_filter_mode_run_tau_n_equals_regular_pic():
    """tau = n: the filter mode is regular PIC, and so is the combination
    mode (one grid); the two runs must agree to rounding."""
    rng = np.random.default_rng(5)
    npart, n = 3000, 5
    u = rng.random((npart, 2))
    v = rng.standard_normal((npart, 2))
    q = -np.full(npart, (4 * np.pi) ** 2 / npart)
    a = O.OracleRun((4 * np.pi, 4 * np.pi), n, u, v, q, 0.05, tau=n, mode="combine")
    b = O.OracleRun((4 * np.pi, 4 * np.pi), n, u, v, q, 0.05, tau=n, mode="filter")
    a.step(3)
    b.step(3)
    assert np.max(np.abs(a.u - b.u)) < 1e-12
    assert abs(a.field_energy() - b.field_energy()) < 1e-12 * a.field_energy()


@pytest.mark.parametrize("d,n", [(2, 10), (3, 7)])
def test_morton_key_prefix_is_coarse_cell_key(d, n):
    """The step sort orders by tile key, the level-n key shifted right by
    d s bits: that is the Morton key of the level-(n - s) cell (the key's
    high bits interleave the cell index's high bits), so tiles are compact
    blocks of 2^s cells per axis."""
    rng = np.random.default_rng(77 + d)
    u = rng.random((5000, d))
    k = O.cell_keys(u, n).astype(np.int64)
    for s in range(0, n):
        np.testing.assert_array_equal(k >> (d * s), O.cell_keys(u, n - s).astype(np.int64))
