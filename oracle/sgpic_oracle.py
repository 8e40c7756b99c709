"""Plain FP64 CPU oracle for sparse-grid combination-technique PIC.

TEST INFRASTRUCTURE ONLY.  This module is the slow, obviously correct
statement of what the GPU path computes.  Only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline / reference leg
may import it.  The CUDA library never imports, links or calls it, and it
imports nothing from the GPU package; the two share only the seeded input
arrays that the tests hand to both.

Every function works in float64 and follows the paper
(Muralikrishnan, Cerfon, Frey, Ricketson, Adelmann, "Sparse grids based
adaptive noise reduction strategy for particle-in-cell schemes",
arXiv:2008.09441).  Section / equation names are the paper's.

State conventions (readings of the paper where it is silent):

* Domain: periodic box [0, L_1) x ... x [0, L_d) (Section 5 opening).
  Positions are carried as fractions of the box, ``u_m = x_m / L_m`` in
  [0, 1); velocities are physical.
* Grids are node-centred by default: node ``k`` of a level-``l`` axis sits
  at ``x_k = k L / 2^l`` (the case in which Proposition 1 is exact).  With
  ``centring="cell"`` node ``k`` sits at the cell centre
  ``x_k = (k + 1/2) L / 2^l`` (the paper's own choice, Section 4.3); then
  the component densities are the two-step ones, R_i applied to the
  regular-grid deposit, whose effective shape is Appendix A's W_c, and the
  field reaches the particles through the same two-step shape (P_i onto
  the regular grid, then the regular-grid CIC gather).
  Grid arrays are indexed ``[i_1, i_2(, i_3)]``, i.e. array axis m is
  coordinate axis m.
* Particle charge ``q_p`` is per particle (weighted particles); the mass is
  ``q_p / qm`` with ``qm = q/m`` (-1 in the paper).

Parity status: every function here is pinned by a test in
``tests/test_oracle_*.py`` against closed forms, brute force, invariants
or the paper's printed formulas.  No function is "parity unpinned".
"""
from __future__ import annotations

import itertools
from math import comb, sqrt

import numpy as np

# --------------------------------------------------------------------------
# Combination technique (Section 4.2, truncated combination technique)
# --------------------------------------------------------------------------


def combination_grids(d: int, n: int, tau: int):
    """Component grids and coefficients of the truncated combination technique.

    Section 4.2 (figure "truncated_comb" and its caption): for a 2^n-per-axis
    regular grid and truncation parameter tau, 2D uses the grids with
    l_1 + l_2 = n + tau (coefficient +1) and l_1 + l_2 = n + tau - 1
    (coefficient -1), every l_m >= tau (Section 4.3.1 error sum).  tau = 1 is
    the standard combination technique, tau = n the regular grid alone.  The
    d-dimensional form (3D is not printed in the paper) is the classical
    combination formula with the minimum level raised to tau:
    |l|_1 = n + (d-1) tau - q, coefficient (-1)^q C(d-1, q), q = 0..d-1.
    The 3D counts reproduce the paper's 3D noise and grid-error brackets
    (Section 4.3.1/4.3.2), which the tests check.

    Returns a list of ``(l, c)`` with ``l`` a tuple of d levels.
    """
    if d not in (2, 3):
        raise ValueError("dim must be 2 or 3")
    if not (1 <= tau <= n):
        raise ValueError("need 1 <= tau <= n")
    out = []
    for q in range(d):
        target = n + (d - 1) * tau - q
        coeff = (-1) ** q * comb(d - 1, q)
        for l in itertools.product(range(tau, n + 1), repeat=d):
            if sum(l) == target:
                out.append((tuple(l), coeff))
    return out


# --------------------------------------------------------------------------
# Positions, cell keys, sort (periodic box, Section 5 opening)
# --------------------------------------------------------------------------


def wrap_unit(u):
    """Map fractional positions into [0, 1): u - floor(u), and 1.0 -> 0.0
    (the subtraction can round up to exactly 1 for tiny negative u).  The
    periodic box of Section 5's test cases."""
    u = np.asarray(u, dtype=np.float64)
    w = u - np.floor(u)
    w[w >= 1.0] = 0.0
    return w


def cell_index(u, n):
    """Cell index floor(u_m 2^n) of every particle along every axis (N_p x d):
    the level-n cell that holds it (regular grid of Section 4.1)."""
    u = np.asarray(u, dtype=np.float64)
    return np.floor(u * float(2 ** n)).astype(np.int64)


def cell_keys(u, n):
    """Morton (Z-order) key of each particle's level-n cell.

    Bit b of the cell index along axis m goes to key bit b*d + m (x is the
    lowest bit).  Written as the plain bit loop.  The paper has no sort;
    this is the reference for the GPU path's cell-key sort, which orders
    particles by cell for the deposit."""
    idx = cell_index(u, n)
    d = idx.shape[1]
    key = np.zeros(idx.shape[0], dtype=np.int64)
    for b in range(n):
        for m in range(d):
            key |= ((idx[:, m] >> b) & 1) << (b * d + m)
    return key.astype(np.uint32)


def sort_by_key(keys, n, d):
    """Stable counting sort by cell key: returns (permutation, sorted keys,
    counts per cell).  Ties keep their previous order.  (No paper
    counterpart: the reference of the GPU path's stand-alone sort.)"""
    keys = np.asarray(keys, dtype=np.int64)
    perm = np.argsort(keys, kind="stable")
    counts = np.bincount(keys, minlength=2 ** (n * d)).astype(np.uint32)
    return perm.astype(np.uint32), keys[perm].astype(np.uint32), counts


def count_checksum(counts):
    """sum_k (k + 1) * count[k] modulo 2^64 (= sum over particles of key+1):
    an order-free integer fingerprint of the cell occupation (no paper
    counterpart; a diagnostic of the GPU path)."""
    c = np.asarray(counts, dtype=np.uint64)
    k = np.arange(1, c.size + 1, dtype=np.uint64)
    return int(np.sum(c * k, dtype=np.uint64))


# --------------------------------------------------------------------------
# CIC deposition (eq. rho_hf of Appendix A, tensor product in 2D/3D)
# --------------------------------------------------------------------------


def _node_offset(centring):
    """Position of node 0 in cells: 0 for node-centred grids, 1/2 for
    cell-centred ones."""
    if centring not in ("node", "cell"):
        raise ValueError("centring must be 'node' or 'cell'")
    return 0.5 if centring == "cell" else 0.0


def _cic_corners(u, l, centring="node"):
    """For each of the 2^d corners: (tuple of node-index arrays, weight array).

    W_m(zeta) = max(0, 1 - |zeta| / h_m) evaluated at the two nodes that
    bracket the particle along each axis (Section 4.1, eq. restriction).
    Node k of a level-l axis sits at (k + o) h_l, o = 0 (node-centred) or
    1/2 (cell-centred), periodically."""
    u = np.asarray(u, dtype=np.float64)
    d = u.shape[1]
    o = _node_offset(centring)
    s = [u[:, m] * float(2 ** l[m]) - o for m in range(d)]
    j = [np.floor(s[m]).astype(np.int64) for m in range(d)]
    f = [s[m] - j[m] for m in range(d)]
    out = []
    for corner in itertools.product((0, 1), repeat=d):
        idx = tuple((j[m] + corner[m]) % (2 ** l[m]) for m in range(d))
        w = np.ones_like(f[0])
        for m in range(d):
            w = w * (f[m] if corner[m] else 1.0 - f[m])
        out.append((idx, w))
    return out


def cell_volume(l, L):
    """V_i = prod_m L_m / 2^(l_m), the cell volume of component grid l
    (eq. restriction)."""
    return float(np.prod([L[m] / 2 ** l[m] for m in range(len(l))]))


def deposit_cic(u, q, l, L, centring="node"):
    """Direct CIC charge deposition onto a grid of levels ``l``.

    rho(x_k) = (1 / V) sum_p q_p prod_m W_m(x_{k,m} - x_{p,m}), V the cell
    volume: eq. rho_hf (Appendix A) generalised to d dimensions and to
    per-particle charges.  This is the sparse-PIC direct deposit onto a
    component grid (Section 4.1), and, at levels (n, ..., n), the regular-grid
    deposit of the two-step approach."""
    shape = tuple(2 ** lm for lm in l)
    rho = np.zeros(shape, dtype=np.float64)
    V = cell_volume(l, L)
    q = np.asarray(q, dtype=np.float64)
    for idx, w in _cic_corners(u, l, centring):
        np.add.at(rho, idx, q * w / V)
    return rho


def _periodic_distance(a, b, N):
    """|a - b| on a circle of circumference N (a, b in fine-cell units,
    scalars or broadcasting arrays)."""
    dist = np.mod(np.subtract(a, b), N)
    return np.minimum(dist, N - dist)


def _coarse_fine_distance(n, l, centring):
    """[k, j]: periodic distance, in level-n cells, between node k of level l
    at (k + o) h_l and node j of level n at (j + o) h (o = 0 or 1/2)."""
    N, M = 2 ** n, 2 ** l
    r = N // M
    o = _node_offset(centring)
    k = np.arange(M, dtype=np.float64)[:, None]
    j = np.arange(N, dtype=np.float64)[None, :]
    return _periodic_distance(j + o, (k + o) * r, N)


def restriction_matrix_1d(n, l, centring="node"):
    """R along one axis from the level-n grid to level l (eq. restriction):
    entry [k, j] = (h / h_l) W(x_k - x~_j) with periodic distance; node k of
    level l at (k + o) h_l, node j of level n at (j + o) h, o = 0 or 1/2."""
    r = 2 ** (n - l)  # regular cells per coarse cell
    return np.maximum(0.0, 1.0 - _coarse_fine_distance(n, l, centring) / r) / r


def restrict(rho_reg, n, l, centring="node"):
    """R_i rho~: transfer from the regular grid to component grid l using
    R_i = (h^d / V_i) prod_m W_m (eq. restriction).  The operator is a tensor
    product of 1D operators; applied axis by axis with a dense matrix."""
    out = np.asarray(rho_reg, dtype=np.float64)
    for m, lm in enumerate(l):
        if lm == n:
            continue  # R = identity along this axis
        R = restriction_matrix_1d(n, lm, centring)
        out = np.moveaxis(np.tensordot(R, np.moveaxis(out, m, 0), axes=(1, 0)), 0, m)
    return out


def prolongation_matrix_1d(n, l, centring="node"):
    """P along one axis from level l to the level-n nodes (eq. restriction):
    entry [j, k] = W(x~_j - x_k) with the coarse spacing h_l."""
    r = 2 ** (n - l)
    return np.maximum(0.0, 1.0 - _coarse_fine_distance(n, l, centring).T / r)


def prolong(field, n, l, centring="node"):
    """P_i: linear interpolation of a level-l nodal field onto the level-n
    nodes (eq. restriction), axis by axis."""
    out = np.asarray(field, dtype=np.float64)
    for m, lm in enumerate(l):
        if lm == n:
            continue  # P = identity along this axis
        P = prolongation_matrix_1d(n, lm, centring)
        out = np.moveaxis(np.tensordot(P, np.moveaxis(out, m, 0), axes=(1, 0)), 0, m)
    return out


def prolong_at(field, n, l, idx, centring="node"):
    """(P_i field)(x~_j) at the regular nodes j = idx[s] (an S x d integer
    array) only: the rows j of the per-axis P (eq. restriction), each with at
    most two non-zero entries (the bracketing coarse nodes)."""
    idx = np.asarray(idx)
    S, d = idx.shape
    ks, ws = [], []
    for m, lm in enumerate(l):
        rows = prolongation_matrix_1d(n, lm, centring)[idx[:, m]]  # S x 2^lm
        top = np.argsort(-rows, axis=1, kind="stable")[:, :2]
        ks.append(top)
        ws.append(np.take_along_axis(rows, top, axis=1))
    out = np.zeros(S)
    field = np.asarray(field, dtype=np.float64)
    for corner in itertools.product((0, 1), repeat=d):
        w = np.ones(S)
        for m in range(d):
            w = w * ws[m][:, corner[m]]
        out += w * field[tuple(ks[m][:, corner[m]] for m in range(d))]
    return out


# --------------------------------------------------------------------------
# Spectral Poisson solve (Section 2: -Laplace phi = rho, E = -grad phi)
# --------------------------------------------------------------------------


def wavenumbers(N, Lm):
    """k_m = 2 pi m / L for the DFT frequencies m in [-N/2, N/2-1] (the
    spectral solve of the Poisson problem of Section 2)."""
    return 2.0 * np.pi * np.fft.fftfreq(N, d=Lm / N)


def solve_poisson_spectral(rho, L):
    """Nodal E = -grad phi with -Laplace phi = rho on a periodic grid.

    Section 2 gives the continuous problem; the discretisation is spectral:
    phi^ = rho^ / |k|^2 with the k = 0 mode set to zero (the uniform
    neutralising background), E^_m = -i k_m phi^, and the Nyquist mode of
    axis m carries no E_m.  Returns a list of d real arrays."""
    rho = np.asarray(rho, dtype=np.float64)
    d = rho.ndim
    rh = np.fft.fftn(rho)
    ks = [wavenumbers(rho.shape[m], L[m]) for m in range(d)]
    grids = np.meshgrid(*ks, indexing="ij")
    k2 = sum(g * g for g in grids)
    phih = np.zeros_like(rh)
    nz = k2 != 0.0
    phih[nz] = rh[nz] / k2[nz]
    E = []
    for m in range(d):
        Nm = rho.shape[m]
        km = grids[m].copy()
        nyq = np.zeros(Nm, dtype=bool)
        nyq[Nm // 2] = True  # fftfreq index N/2 is frequency -N/2
        shape = [1] * d
        shape[m] = Nm
        km = np.where(nyq.reshape(shape), 0.0, km)
        E.append(np.real(np.fft.ifftn(-1j * km * phih)))
    return E


def potential_spectral(rho, L):
    """phi with -Laplace phi = rho (k = 0 mode zero), Section 2; used by the
    pins."""
    rho = np.asarray(rho, dtype=np.float64)
    d = rho.ndim
    rh = np.fft.fftn(rho)
    grids = np.meshgrid(*[wavenumbers(rho.shape[m], L[m]) for m in range(d)], indexing="ij")
    k2 = sum(g * g for g in grids)
    phih = np.zeros_like(rh)
    nz = k2 != 0.0
    phih[nz] = rh[nz] / k2[nz]
    return np.real(np.fft.ifftn(phih))


# --------------------------------------------------------------------------
# Gather (Section 2, step 3: same shape function as the deposit)
# --------------------------------------------------------------------------


def gather_cic(field, u, l, centring="node"):
    """CIC interpolation of a level-l nodal field to the particles: the
    field at the particles with the deposit's shape W (Section 2, the
    interpolation step; eq. restriction's hat function)."""
    out = np.zeros(np.asarray(u).shape[0], dtype=np.float64)
    for idx, w in _cic_corners(u, l, centring):
        out += w * field[idx]
    return out


def regular_node_positions(n, d, centring="node"):
    """Fractional positions (j + o) / 2^n of all level-n nodes, in array
    order (o = 0 node-centred, 1/2 cell-centred): the regular grid of
    Section 4.1."""
    N = 2 ** n
    o = _node_offset(centring)
    axes = np.meshgrid(*[(np.arange(N) + o) / N for _ in range(d)], indexing="ij")
    return np.stack([a.ravel() for a in axes], axis=1)


# --------------------------------------------------------------------------
# Push (Section 2, step 4; leapfrog, Boris rotation when B != 0)
# --------------------------------------------------------------------------


def external_field(u, L, eext_lin):
    """E_ext,m = eext_lin[m] (x_m - L_m/2): the linear (Penning-type) external
    field of Section 5.2, zero when eext_lin is zero."""
    u = np.asarray(u, dtype=np.float64)
    d = u.shape[1]
    return [eext_lin[m] * (u[:, m] * L[m] - 0.5 * L[m]) for m in range(d)]


def kick_rotate(v, E, qm, dt, B):
    """Velocity update over dt: half electric kick, magnetic rotation, half
    kick (Boris).  With B = 0 this is the plain leapfrog kick
    v + (q/m) E dt (Section 2, the push; the magnetised cases of Sections
    5.1-5.2 need the rotation).  ``v`` and ``E`` are lists of d arrays; in 2D
    only B_z acts (in-plane velocities)."""
    d = len(v)
    vm = [v[m] + qm * E[m] * (0.5 * dt) for m in range(d)]
    if d == 2:
        tz = qm * B[2] * 0.5 * dt
        if tz == 0.0:
            vp = vm
        else:
            s = 2.0 * tz / (1.0 + tz * tz)
            # v' = v- + v- x t ; v+ = v- + v' x s   (t = (0, 0, tz))
            vpx = vm[0] + vm[1] * tz
            vpy = vm[1] - vm[0] * tz
            vp = [vm[0] + vpy * s, vm[1] - vpx * s]
    else:
        t = [qm * B[m] * 0.5 * dt for m in range(3)]
        t2 = t[0] ** 2 + t[1] ** 2 + t[2] ** 2
        if t2 == 0.0:
            vp = vm
        else:
            s = [2.0 * t[m] / (1.0 + t2) for m in range(3)]
            cx = lambda a, b: [a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]]
            c1 = cx(vm, t)
            vprime = [vm[m] + c1[m] for m in range(3)]
            c2 = cx(vprime, s)
            vp = [vm[m] + c2[m] for m in range(3)]
    return [vp[m] + qm * E[m] * (0.5 * dt) for m in range(d)]


def drift(u, v, dt, L):
    """x^{n+1} = x^n + v^{n+1/2} dt, in fractional coordinates, wrapped into
    the periodic box (Section 2, the push)."""
    u = np.asarray(u, dtype=np.float64)
    out = np.empty_like(u)
    for m in range(u.shape[1]):
        out[:, m] = u[:, m] + v[m] * dt / L[m]
    return wrap_unit(out)


# --------------------------------------------------------------------------
# One sparse-PIC field evaluation and the time loop
# --------------------------------------------------------------------------


def component_fields(u, q, n, tau, L, centring="node"):
    """Component densities and fields (sparse PIC of Section 4.1 with the
    grid set of Section 4.2).  Node-centred: deposit directly on every
    component grid.  Cell-centred: the two-step densities R_i rho~ of the
    regular-grid deposit rho~ (Appendix A: their shape W_c is a shape
    function of its own, no longer the direct deposit).  Each density is
    solved on its grid.  Returns a list of (l, c, rho_l, [E_l,m])."""
    d = np.asarray(u).shape[1]
    out = []
    rho_reg = deposit_cic(u, q, (n,) * d, L, "cell") if centring == "cell" else None
    for l, c in combination_grids(d, n, tau):
        if centring == "cell":
            rho = restrict(rho_reg, n, l, "cell")
        else:
            rho = deposit_cic(u, q, l, L)
        E = solve_poisson_spectral(rho, L)
        out.append((l, c, rho, E))
    return out


def field_at_particles(comps, u, L, eext_lin, centring="node", n=None):
    """E(x_p) = sum_i c_i I_i[E_i](x_p) + E_ext(x_p).  Node-centred: each
    component field gathered with the CIC shape straight from its grid (no
    regular grid involved).  Cell-centred: the same two-step shape as the
    deposit, sum_k W_c(x_k - x_p) E_i(x_k) = regular-grid CIC gather of
    P_i E_i (Appendix A's W_c, used in both directions)."""
    d = np.asarray(u).shape[1]
    E = [np.zeros(np.asarray(u).shape[0]) for _ in range(d)]
    for l, c, _, El in comps:
        for m in range(d):
            if centring == "cell":
                E[m] += c * gather_cic(prolong(El[m], n, l, "cell"), u, (n,) * d, "cell")
            else:
                E[m] += c * gather_cic(El[m], u, l)
    Ee = external_field(u, L, eext_lin)
    return [E[m] + Ee[m] for m in range(d)]


def combined_field_regular(comps, n, d, centring="node"):
    """E_comb = sum_i c_i P_i E_i on the regular nodes (eq. sparse_filter with
    the same c_i and P_i, applied to the component fields)."""
    out = [np.zeros((2 ** n,) * d) for _ in range(d)]
    for l, c, _, El in comps:
        for m in range(d):
            out[m] += c * prolong(El[m], n, l, centring)
    return out


def density_filter(rho_reg, n, tau, L, centring="node"):
    """Sparse-grid filter of a regular-grid density (eq. sparse_filter,
    Algorithm 2): rho_f = sum_i c_i P_i R_i rho~, with R_i and P_i of eq.
    restriction and the grid set of Section 4.2."""
    d = np.asarray(rho_reg).ndim
    out = np.zeros_like(np.asarray(rho_reg, dtype=np.float64))
    for l, c in combination_grids(d, n, tau):
        out += c * prolong(restrict(rho_reg, n, l, centring), n, l, centring)
    return out


def filtered_field_regular(u, q, n, tau, L, centring="node"):
    """Field of the paper's filter mode on the regular nodes: deposit on the
    regular grid, filter the density (density_filter), one spectral solve
    on the regular grid (Algorithm 2's field step)."""
    d = np.asarray(u).shape[1]
    rho = deposit_cic(u, q, (n,) * d, L, centring)
    rho_f = density_filter(rho, n, tau, L, centring)
    return rho, rho_f, solve_poisson_spectral(rho_f, L)


class OracleRun:
    """Plain FP64 sparse-grid PIC run (deposit -> solve -> combine/gather ->
    push), the reference for the GPU hot path.

    Leapfrog start: v^{-1/2} from a backward half step at t = 0.
    Diagnostics: charge per grid and combined, field energy
    0.5 h^d sum |E|^2 over the regular nodes (current and previous step),
    time-centred kinetic energy, and the cell-count checksum.
    """

    def __init__(self, L, n, u, v, q, dt, qm=-1.0, tau=1, B=(0.0, 0.0, 0.0),
                 eext_lin=(0.0, 0.0, 0.0), mode="combine", alpha=0.01, pc_ref=5.0, tau_constants="paper",
                 centring="node"):
        # mode "combine": sparse PIC, fields solved per component grid and
        # combined (Section 4.1); "filter": the density is deposited on the
        # regular grid, filtered (eq. sparse_filter) and solved once there
        # (Algorithm 2).  tau = "adaptive": Algorithm 1 picks tau from the
        # regular-grid density before every field evaluation (alpha, pc_ref,
        # tau_constants are its parameters).  centring "node" | "cell": where
        # the grid nodes sit (module docstring).
        assert mode in ("combine", "filter")
        _node_offset(centring)
        self.mode = mode
        self.centring = centring
        self.adaptive = tau == "adaptive"
        self.alpha, self.pc_ref, self.tau_constants = float(alpha), float(pc_ref), tau_constants
        self.tau_history = []
        self.L = [float(x) for x in L]
        self.n = int(n)
        self.u = wrap_unit(np.array(u, dtype=np.float64))
        self.d = self.u.shape[1]
        self.v = [np.array(v[:, m], dtype=np.float64) for m in range(self.d)]
        self.q = np.array(q, dtype=np.float64)
        self.dt = float(dt)
        self.qm = float(qm)
        self.tau = 1 if self.adaptive else int(tau)
        self.B = [float(b) for b in B]
        self.eext = [float(e) for e in eext_lin]
        self.step_count = 0
        self.kinetic_energy = 0.0
        self.field_energy_prev = 0.0
        self._fields()
        E = self.field_at(self.u)
        self.v = kick_rotate(self.v, E, self.qm, -0.5 * self.dt, self.B)

    def _fields(self):
        """The field evaluation of one step: Algorithm 1 first when tau is
        adaptive, then the component fields (Section 4.1) or the filter
        mode's regular-grid field (Algorithm 2)."""
        if self.adaptive:
            rho = deposit_cic(self.u, self.q, (self.n,) * self.d, self.L, self.centring)
            self.tau = tau_estimator(rho, len(self.q), self.L[0], self.alpha, self.pc_ref,
                                     float(np.sum(self.q)), self.tau_constants)[0]
            self.tau_history.append(self.tau)
        if self.mode == "combine":
            self.comps = component_fields(self.u, self.q, self.n, self.tau, self.L, self.centring)
        else:  # component densities only (diagnostics), field on the regular grid
            self.comps = []
            rho, self.rho_filtered, self.E_regular = filtered_field_regular(self.u, self.q, self.n, self.tau,
                                                                            self.L, self.centring)
            for l, c in combination_grids(self.d, self.n, self.tau):
                self.comps.append((l, c, restrict(rho, self.n, l, self.centring), None))

    def field_at(self, u):
        """The field the push sees at positions u (plus E_ext)."""
        if self.mode == "combine":
            return field_at_particles(self.comps, u, self.L, self.eext, self.centring, self.n)
        Ee = external_field(u, self.L, self.eext)
        return [gather_cic(self.E_regular[m], u, (self.n,) * self.d, self.centring) + Ee[m] for m in range(self.d)]

    def regular_field(self):
        """The field on the regular nodes (combined, or the filter mode's)."""
        if self.mode == "combine":
            return combined_field_regular(self.comps, self.n, self.d, self.centring)
        return self.E_regular

    def field_energy(self):
        """0.5 h^d sum_j |E(x~_j)|^2 over the regular nodes."""
        Ec = self.regular_field()
        hd = float(np.prod([self.L[m] / 2 ** self.n for m in range(self.d)]))
        return 0.5 * hd * float(sum(np.sum(e * e) for e in Ec))

    def step(self, nsteps=1):
        """Leapfrog steps (Section 2): kick with the current field, drift,
        new field; the kinetic energy is time-centred over the kick."""
        for _ in range(nsteps):
            E = self.field_at(self.u)
            vnew = kick_rotate(self.v, E, self.qm, self.dt, self.B)
            mass = self.q / self.qm
            self.kinetic_energy = 0.5 * float(np.sum(mass * sum(self.v[m] * vnew[m] for m in range(self.d))))
            self.field_energy_prev = self.field_energy()
            self.v = vnew
            self.u = drift(self.u, self.v, self.dt, self.L)
            self._fields()
            self.step_count += 1

    def grid_charges(self):
        """V_i sum_k rho_i(x_k) per component grid: the charge each grid holds
        (the deposit's partition of unity keeps it equal to sum_p q_p)."""
        return [float(np.sum(rho)) * cell_volume(l, self.L) for l, _, rho, _ in self.comps]

    def diagnostics(self):
        """Charges per grid and combined (coefficients of Section 4.2), field
        and kinetic energies, tau, and the cell-occupation checksum."""
        qsum = float(np.sum(self.q))
        ch = self.grid_charges()
        coeffs = [c for _, c, _, _ in self.comps]
        keys = cell_keys(self.u, self.n)
        counts = np.bincount(keys.astype(np.int64), minlength=2 ** (self.n * self.d))
        return {
            "step": self.step_count,
            "t": self.step_count * self.dt,
            "tau": self.tau,
            "charge_total": qsum,
            "charge_combined": float(sum(c * x for c, x in zip(coeffs, ch))),
            "charge_grid_max_abs_err": float(max(abs(x - qsum) for x in ch)),
            "field_energy": self.field_energy(),
            "field_energy_prev": self.field_energy_prev,
            "kinetic_energy": self.kinetic_energy,
            "count_checksum": count_checksum(counts),
        }

    def velocities(self):
        """v^{n-1/2} as an (N_p, d) array."""
        return np.stack(self.v, axis=1)


# --------------------------------------------------------------------------
# tauEstimator (Algorithm 1, Section 4.3)
# --------------------------------------------------------------------------


def grid_error_estimate(d, n, tau, L, kappa, beta, gamma=0.0):
    """eq. 2D_grid_error / eq. 3D_grid_error with O(.) constants 1.
    kappa: d values; beta: 1 value (2D) or 3 values (3D)."""
    h = L / 2 ** n
    m = n - tau
    if d == 2:
        return h * h * (kappa[0] + kappa[1] + beta[0] * L * L * 2.0 ** (-2 * tau) * (5 * m + 1))
    return h * h * (sum(kappa) + sum(beta) * L * L * 2.0 ** (-2 * tau) * (5 * m + 1)
                    + gamma * L ** 4 * 2.0 ** (-(4 * tau + 1)) * (25 * m * m - 5 * m + 2))


def particle_noise_estimate(d, n, tau, L, Np, sigma):
    """eq. 2D_particle_noise / eq. 3D_particle_noise with O(.) constant 1."""
    h = L / 2 ** n
    m = n - tau
    if d == 2:
        return sigma * 2.0 ** (0.5 * (tau - 1)) * (m * (1 + sqrt(2.0)) + sqrt(2.0)) / sqrt(Np * h * L)
    return sigma * 2.0 ** (tau - 2) * ((3 + sqrt(2.0)) * m * m + (5 + sqrt(2.0)) * m + 4) / sqrt(Np * h * L * L)


def tau_range(d, n):
    """Admissible tau of Algorithm 1: [1, n-3] in 2D, [1, n-2] in 3D."""
    hi = n - 3 if d == 2 else n - 2
    return list(range(1, hi + 1))


def tau_estimator(rho_reg, Np, L, alpha, pc_ref, Qe, constants="paper"):
    """Algorithm 1 on the regular-grid density rho~ (indexed [i_1..i_d]).

    1. rho^ = F(rho~), normalised by 1/N_c (Fourier amplitudes).
    2. Hard threshold (eq. denoising) with eps = alpha sqrt(Pc_ref/Pc) max|rho^|
       (Section 5.1 parameter rule), Pc = Np / N_c.
    3. Constants: eq. grid_constants (spectral derivatives of the denoised
       density, inverse transform, max norm) and eq. particle_constant; or
       eq. empirical_constants (max over modes, no inverse transforms).
    4. For tau in the admissible range evaluate grid error + particle noise.
    5. Pick the tau with the smallest total (ties: the smallest tau).

    Returns (tau, list of (tau, grid, noise)).
    """
    rho = np.asarray(rho_reg, dtype=np.float64)
    d = rho.ndim
    N = rho.shape[0]
    n = int(round(np.log2(N)))
    Nc = rho.size
    rh = np.fft.fftn(rho) / Nc
    Pc = Np / Nc
    eps = alpha * sqrt(pc_ref / Pc) * float(np.max(np.abs(rh)))
    rh = np.where(np.abs(rh) >= eps, rh, 0.0)
    k = wavenumbers(N, L)
    K = np.meshgrid(*([k] * d), indexing="ij")
    K2 = [g * g for g in K]

    if constants == "paper":
        def dnorm(mult):
            return float(np.max(np.abs(np.real(np.fft.ifftn(mult * rh * Nc)))))
        # d^2/dx_m^2 <-> -k_m^2 ; d^4/dx^2dy^2 <-> k_x^2 k_y^2 ; d^6 <-> -k_x^2k_y^2k_z^2
        kappa = [0.25 * dnorm(-K2[m]) for m in range(d)]
        if d == 2:
            beta = [dnorm(K2[0] * K2[1]) / 72.0]
            gamma = 0.0
        else:
            beta = [dnorm(K2[0] * K2[1]) / 72.0, dnorm(K2[1] * K2[2]) / 72.0,
                    dnorm(K2[2] * K2[0]) / 72.0]
            gamma = dnorm(-K2[0] * K2[1] * K2[2]) / 864.0
        sigma = sqrt((2.0 / 3.0) ** d * abs(Qe) * float(np.max(np.abs(rho))))
    elif constants == "empirical":
        def mnorm(mult):
            return float(np.max(np.abs(mult * rh)))
        kappa = [mnorm(K2[m]) for m in range(d)]
        if d == 2:
            beta = [mnorm(K2[0] * K2[1])]
            gamma = 0.0
        else:
            beta = [mnorm(K2[0] * K2[1]), mnorm(K2[1] * K2[2]), mnorm(K2[0] * K2[2])]
            gamma = mnorm(K2[0] * K2[1] * K2[2])
        sigma = sqrt(abs(Qe) * float(np.max(np.abs(rho))))
    else:
        raise ValueError(constants)

    table = []
    for tau in tau_range(d, n):
        g = grid_error_estimate(d, n, tau, L, kappa, beta, gamma)
        z = particle_noise_estimate(d, n, tau, L, Np, sigma)
        table.append((tau, g, z))
    if not table:
        raise ValueError("empty tau range")
    best = min(table, key=lambda t: (t[1] + t[2], t[0]))
    return best[0], table, {"kappa": kappa, "beta": beta, "gamma": gamma, "sigma": sigma, "eps": eps}
