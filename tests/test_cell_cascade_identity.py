"""The identities the GPU's cell-centred transfer kernels rest on, checked on
the CPU against the oracle's dense cell-centred matrices (eq. restriction
between cell centres):

* restriction: R_l = FW_odd o FW^(n-l-1) o A, with A the average onto the
  faces a[t] = (x[t-1] + x[t]) / 2, FW full weighting at the even nodes and
  FW_odd full weighting evaluated at the odd nodes (R_n = identity);
* prolongation: linear interpolation through the level-l centres is the
  node-centred interpolant of the level-(l+1) line whose odd nodes hold the
  centre values and whose even nodes hold the midpoints, sampled at the
  regular centres, the midpoints of the level-n nodes.

These restate the kernels' arithmetic in numpy; the GPU parity tests check
the kernels themselves."""
import numpy as np
import pytest

from oracle import sgpic_oracle as O


def full_weighting_even(a):
    return 0.25 * np.roll(a, 1)[::2] + 0.5 * a[::2] + 0.25 * np.roll(a, -1)[::2]


def full_weighting_odd(a):
    return 0.25 * a[::2] + 0.5 * a[1::2] + 0.25 * np.roll(a, -2)[::2]


def cascade_restrict(x, n, lev):
    if lev == n:
        return x.copy()
    a = 0.5 * (np.roll(x, 1) + x)
    for _ in range(n - lev - 1):
        a = full_weighting_even(a)
    return full_weighting_odd(a)


def node_prolong_step(t):
    """Node-centred linear interpolation to the next finer level (periodic)."""
    out = np.empty(2 * t.size)
    out[::2] = t
    out[1::2] = 0.5 * (t + np.roll(t, -1))
    return out


def embed(E):
    """Centre values at the odd level-(l+1) nodes, midpoints at the even ones."""
    g = np.empty(2 * E.size)
    g[1::2] = E
    g[::2] = 0.5 * (np.roll(E, 1) + E)
    return g


def horner_cell_combination(fields, n):
    """sum_l c_l P_l E_l on the regular centres the way the combination kernel
    evaluates it: Horner over the node-centred levels with every grid entering
    one level higher, a final half step, then the level-n grids."""
    T = np.zeros(1)  # level 0: one node
    for L in range(1, n + 1):
        T = node_prolong_step(T)
        for lev, c, E in fields:
            if lev == L - 1:
                T = T + c * embed(E)
    out = 0.5 * (T + np.roll(T, -1))
    for lev, c, E in fields:
        if lev == n:
            out = out + c * E
    return out


@pytest.mark.parametrize("n", [2, 3, 5, 7])
def test_cell_restriction_cascade_equals_matrix(n):
    rng = np.random.default_rng(n)
    x = rng.standard_normal(2 ** n)
    for lev in range(1, n + 1):
        ref = O.restriction_matrix_1d(n, lev, "cell") @ x
        np.testing.assert_allclose(cascade_restrict(x, n, lev), ref, rtol=0, atol=1e-13)


@pytest.mark.parametrize("n", [2, 4, 6])
def test_cell_prolongation_horner_equals_matrix(n):
    rng = np.random.default_rng(10 + n)
    fields = [(lev, float(rng.choice([-2.0, -1.0, 1.0])), rng.standard_normal(2 ** lev)) for lev in range(1, n + 1)]
    ref = sum(c * (O.prolongation_matrix_1d(n, lev, "cell") @ E) for lev, c, E in fields)
    np.testing.assert_allclose(horner_cell_combination(fields, n), ref, rtol=0, atol=1e-12)


@pytest.mark.parametrize("n", [2, 4, 7])
def test_node_restriction_cascade_equals_matrix(n):
    """Node-centred: R_l is full weighting applied n - l times (the coarse hat
    is linear between fine nodes, Appendix A)."""
    rng = np.random.default_rng(20 + n)
    x = rng.standard_normal(2 ** n)
    for lev in range(1, n + 1):
        a = x.copy()
        for _ in range(n - lev):
            a = full_weighting_even(a)
        np.testing.assert_allclose(a, O.restriction_matrix_1d(n, lev) @ x, rtol=0, atol=1e-13)


@pytest.mark.parametrize("n", [2, 5])
def test_node_prolongation_horner_equals_matrix(n):
    """Node-centred: sum_l c_l P_l E_l by Horner's scheme (prolong one level,
    add the grids of that level)."""
    rng = np.random.default_rng(30 + n)
    fields = [(lev, float(rng.choice([-1.0, 1.0])), rng.standard_normal(2 ** lev)) for lev in range(1, n + 1)]
    T = np.zeros(1)
    for L in range(1, n + 1):
        T = node_prolong_step(T)
        for lev, c, E in fields:
            if lev == L:
                T = T + c * E
    ref = sum(c * (O.prolongation_matrix_1d(n, lev) @ E) for lev, c, E in fields)
    np.testing.assert_allclose(T, ref, rtol=0, atol=1e-12)


@pytest.mark.parametrize("centring", ["node", "cell"])
def test_transverse_bracket_equals_prolongation_rows(centring):
    """The combination's transverse interpolation (the kernels' integer
    bracket): node-centred k0 = y >> r, f = (y mod 2^r) / 2^r; cell-centred
    num = 2y + 1 - 2^r, k0 = num >> (r + 1) (an arithmetic shift: floor,
    -1 wraps), f = (num - k0 2^(r+1)) / 2^(r+1).  Weights 1 - f on k0 and f on
    k0 + 1 (periodic) must be the rows of the oracle's P."""
    for n in (3, 6):
        for lev in range(1, n + 1):
            P = O.prolongation_matrix_1d(n, lev, centring)
            r = n - lev
            nl = 1 << lev
            for y in range(1 << n):
                if centring == "node":
                    k0 = y >> r
                    f = (y & ((1 << r) - 1)) / (1 << r)
                else:
                    num = 2 * y + 1 - (1 << r)
                    fl = num >> (r + 1)  # Python's >> floors negative numbers like the kernels' shift
                    f = (num - fl * (2 << r)) / (2 << r)
                    k0 = fl & (nl - 1)
                k1 = (k0 + 1) & (nl - 1)
                row = np.zeros(nl)
                row[k0] += 1.0 - f
                row[k1] += f
                np.testing.assert_allclose(P[y], row, rtol=0, atol=1e-15)


@pytest.mark.parametrize("L", [6, 8, 10])
def test_lane_chunks_of_the_cell_embedding(L):
    """The combination kernel's per-lane form of the embedding at Horner level
    L (2^L = 32 K values, lane j holding K of them from x0 = j K): the lane
    reads its K/2 centre values from c0 = x0/2 and the one before,
    cm = (c0 - 1) mod 2^(L-1), and writes g[x0 + 2i + 1] = E[c0 + i],
    g[x0 + 2i] = (E[c0 + i - 1] + E[c0 + i]) / 2."""
    rng = np.random.default_rng(L)
    E = rng.standard_normal(1 << (L - 1))
    K = (1 << L) // 32
    H = K // 2
    nc = 1 << (L - 1)
    g = np.empty(1 << L)
    for lane in range(32):
        x0 = lane * K
        c0 = x0 >> 1
        cm = (c0 - 1) & (nc - 1)
        t = np.concatenate([[E[cm]], E[c0:c0 + H]])
        for i in range(H):
            g[x0 + 2 * i + 1] = t[i + 1]
            g[x0 + 2 * i] = 0.5 * (t[i] + t[i + 1])
    np.testing.assert_array_equal(g, embed(E))
