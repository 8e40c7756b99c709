"""The deposit kernel's window bookkeeping restated in numpy (CPU only):
per chunk of 2048 consecutive particles, the anchor cell of the chunk's
middle particle, the window origin (anchor - side/2, wrapped, along x rounded
down to a multiple of 4), the window index l = (c - origin) mod N of each
corner's node, the fast path when every l + 1 < side (else the corners go
straight to the grid), and the flush that adds window node x to global node
(origin + x) mod N.  Summed over chunks it must equal the oracle's deposit,
including grids smaller than the window (window entries alias nodes)."""
import numpy as np
import pytest

from oracle import sgpic_oracle as O

CHUNK = 2048


def window_deposit(u, q, n, L, side, shift=0.0):
    d = u.shape[1]
    N = 1 << n
    mask = N - 1
    V = float(np.prod([L[m] / N for m in range(d)]))
    rho = np.zeros((N,) * d)
    for c0 in range(0, u.shape[0], CHUNK):
        uc, qc = u[c0:c0 + CHUNK], q[c0:c0 + CHUNK]
        mid = min(c0 + CHUNK // 2, u.shape[0] - 1) - c0
        anchor = np.floor(uc[mid] * N).astype(np.int64)
        origin = (anchor - side // 2) & mask
        origin[0] &= ~3
        win = np.zeros((side,) * d)
        s = uc * N - shift
        c = np.floor(s).astype(np.int64)
        f = s - c
        l = (c - origin) & mask
        fast = np.all(l + 1 < side, axis=1)
        for corner in np.ndindex(*(2,) * d):
            w = qc / V
            for m in range(d):
                w = w * (f[:, m] if corner[m] else 1.0 - f[:, m])
            wi = tuple(l[fast, m] + corner[m] for m in range(d))
            np.add.at(win, wi, w[fast])
            gi = tuple((c[~fast, m] + corner[m]) & mask for m in range(d))
            np.add.at(rho, gi, w[~fast])
        # flush: window node x -> global node (origin + x) mod N
        idx = [((origin[m] + np.arange(side)) & mask) for m in range(d)]
        np.add.at(rho, np.ix_(*idx), win)
    return rho


@pytest.mark.parametrize("d,n,side,shift", [(2, 10, 128, 0.0), (2, 10, 128, 0.5), (2, 5, 128, 0.0),
                                            (2, 4, 128, 0.5), (3, 6, 24, 0.0), (3, 3, 24, 0.5)])
def test_window_deposit_equals_oracle(d, n, side, shift):
    rng = np.random.default_rng(n + d)
    npart = 3 * CHUNK + 517
    N = 1 << n
    u = rng.random((npart, d))
    # a sorted order (by cell key) as after the step sort, plus drift
    u = u[np.argsort(O.cell_keys(u, n), kind="stable")]
    u = O.wrap_unit(u + rng.normal(0.0, 6.0 / N, u.shape))
    q = rng.normal(-1.0, 0.1, npart)
    L = (2.0, 3.0, 5.0)[:d]
    got = window_deposit(u, q, n, L, side, shift)
    ref = O.deposit_cic(u, q, (n,) * d, L, "cell" if shift else "node")
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-10 * np.max(np.abs(ref)))


def flush_items(blo, bhi, threads, fixed):
    """The flush's enumeration of a touched box [blo, bhi] (window
    coordinates, x first): flat items f = thread, thread + threads, ...; item
    f is row r = f // nx and x = x0 + (f mod nx) * per, with x0 = blo_x
    rounded down to 4 and per = 4 nodes (fixed point) or x0 = blo_x and
    per = 1.  Returns the window nodes each item covers."""
    d = len(blo)
    per = 4 if fixed else 1
    x0 = (blo[0] & ~3) if fixed else blo[0]
    nx = (bhi[0] - x0) // per + 1
    ny = bhi[1] - blo[1] + 1
    nrows = ny if d == 2 else ny * (bhi[2] - blo[2] + 1)
    out = []
    for t in range(threads):
        for f in range(t, nrows * nx, threads):
            r, xi = divmod(f, nx)
            x = x0 + xi * per
            ly = blo[1] + (r if d == 2 else r % ny)
            lz = 0 if d == 2 else blo[2] + r // ny
            out.append([(x + k, ly, lz) for k in range(per)])
    return out


@pytest.mark.parametrize("d", [2, 3])
@pytest.mark.parametrize("fixed", [True, False])
def test_flush_items_cover_the_box_once(d, fixed):
    rng = np.random.default_rng(5 + d + 7 * fixed)
    side = 128 if d == 2 else 24
    for _ in range(50):
        lo = rng.integers(0, side - 1, d)
        hi = np.array([rng.integers(lo[m], side) for m in range(d)])  # hi <= side - 1: the fast path's bound
        items = flush_items(list(lo), list(hi), 512, fixed)
        nodes = [n for it in items for n in it]
        assert len(nodes) == len(set(nodes))  # no node twice
        want = {(x, y, z) for x in range(lo[0], hi[0] + 1) for y in range(lo[1], hi[1] + 1)
                for z in (range(lo[2], hi[2] + 1) if d == 3 else [0])}
        assert want <= set(nodes)  # every touched node flushed
        assert all(0 <= x < side for x, _, _ in nodes)  # 16-byte reads stay in the window row
        # the extra nodes are the quad padding along x of rows in the box
        assert all(lo[1] <= y <= hi[1] and (d == 2 or lo[2] <= z <= hi[2]) for _, y, z in nodes)
