"""Python face of the sparse-grid PIC library.

``sg_pic_init`` / ``sg_pic_step`` / ... mirror the C ABI one to one; the
``Run`` class wraps a handle.  Arrays may be numpy (host) or torch CUDA
tensors (device); torch is used only for device memory and the stream.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _lib as L
from ._lib import check, lib

_DT = {L.SG_FP32: np.float32, L.SG_FP64: np.float64}


def _is_torch(x):
    return type(x).__module__.startswith("torch")


def _columns(a, d, dtype):
    """(N, d) array or sequence of d 1-D arrays -> list of d contiguous columns."""
    if isinstance(a, (list, tuple)):
        cols = list(a)
    elif _is_torch(a):
        cols = [a[:, m] for m in range(d)]
    else:
        a = np.asarray(a)
        cols = [a[:, m] for m in range(d)]
    out = []
    for c in cols:
        if _is_torch(c):
            import torch
            tdt = torch.float32 if dtype == np.float32 else torch.float64
            out.append(c.to(tdt).contiguous())
        else:
            out.append(np.ascontiguousarray(c, dtype=dtype))
    return out


def _ptr(x):
    return C.c_void_p(x.data_ptr() if _is_torch(x) else x.ctypes.data)


def _on_device(x):
    return 1 if (_is_torch(x) and x.is_cuda) else 0


_MODES = {"combine": L.SG_MODE_COMBINE, "filter": L.SG_MODE_FILTER}
_CENTRINGS = {"node": L.SG_NODE_CENTRED, "cell": L.SG_CELL_CENTRED}
_COMBINES = {"float-float": L.SG_COMBINE_FLOAT_FLOAT, "fp64": L.SG_COMBINE_FP64}


def make_params(precision=L.SG_FP32, tau=1, dt=0.05, qm=-1.0, B=(0.0, 0.0, 0.0), eext_lin=(0.0, 0.0, 0.0),
                alpha=0.01, pc_ref=5.0, tau_constants=L.SG_TAU_CONST_PAPER, sort_every=0, stream=None,
                mode=L.SG_MODE_COMBINE, centring=L.SG_NODE_CENTRED, combine=L.SG_COMBINE_FLOAT_FLOAT):
    p = L.sg_params()
    p.precision = precision
    p.tau = tau
    p.dt = dt
    p.qm = qm
    for m in range(3):
        p.B[m] = B[m]
        p.Eext_lin[m] = eext_lin[m]
    p.alpha = alpha
    p.pc_ref = pc_ref
    p.tau_constants = tau_constants
    p.sort_every = sort_every
    p.stream = stream
    p.mode = _MODES.get(mode, mode)
    p.centring = _CENTRINGS.get(centring, centring)
    p.combine = _COMBINES.get(combine, combine)
    return p


# ------------------------------------------------------------------ raw ABI
def sg_pic_init(domain, level_n, dim, shape_order, particles, params):
    h = C.c_void_p()
    check(lib().sg_pic_init(C.byref(domain), level_n, dim, shape_order, C.byref(particles), C.byref(params),
                            C.byref(h)), "sg_pic_init")
    return h


def sg_pic_step(h, nsteps):
    return check(lib().sg_pic_step(h, nsteps), "sg_pic_step")


def sg_pic_diagnostics(h):
    d = L.sg_diag()
    check(lib().sg_pic_diagnostics(h, C.byref(d)), "sg_pic_diagnostics")
    return d.as_dict()


def sg_pic_diagnostics_post(h):
    return check(lib().sg_pic_diagnostics_post(h), "sg_pic_diagnostics_post")


def sg_pic_diagnostics_collect(h):
    d = L.sg_diag()
    check(lib().sg_pic_diagnostics_collect(h, C.byref(d)), "sg_pic_diagnostics_collect")
    return d.as_dict()


def sg_pic_select_tau(h, cap=32):
    t = C.c_int()
    g = np.zeros(cap)
    z = np.zeros(cap)
    check(lib().sg_pic_select_tau(h, C.byref(t), g.ctypes.data, z.ctypes.data, cap), "sg_pic_select_tau")
    return t.value, g, z


def sg_pic_set_tau(h, tau):
    return check(lib().sg_pic_set_tau(h, tau), "sg_pic_set_tau")


def sg_pic_destroy(h):
    if h:
        lib().sg_pic_destroy(h)


def sg_strerror(status):
    return lib().sg_strerror(status).decode()


def sg_last_error():
    return lib().sg_last_error().decode()


def sg_version():
    return lib().sg_version().decode()


def sg_combination_grids(dim, n, tau):
    """The library's grid set (host only): list of (levels tuple, coefficient)."""
    cnt = C.c_int()
    check(lib().sg_combination_grids(dim, n, tau, None, None, 0, C.byref(cnt)), "sg_combination_grids")
    levels = np.zeros(3 * cnt.value, dtype=np.int32)
    coeffs = np.zeros(cnt.value, dtype=np.int32)
    check(lib().sg_combination_grids(dim, n, tau, levels.ctypes.data, coeffs.ctypes.data, cnt.value,
                                     C.byref(cnt)), "sg_combination_grids")
    return [(tuple(int(x) for x in levels[3 * i:3 * i + dim]), int(coeffs[i])) for i in range(cnt.value)]


def sg_estimate_footprint(precision, dim, n, tau, n_particles):
    """Device bytes of a run of these sizes as the serving layer estimates them (host only)."""
    b = C.c_size_t()
    prec = L.SG_FP32 if precision in ("fp32", L.SG_FP32) else L.SG_FP64
    check(lib().sg_estimate_footprint(prec, dim, n, tau, int(n_particles), C.byref(b)), "sg_estimate_footprint")
    return int(b.value)


def sg_cell_sort(u_cols, level, precision=L.SG_FP32, stream=None):
    """Stand-alone cell-key sort of torch CUDA position columns.  Returns
    (sorted keys, permutation, counts) as torch uint32-in-int32 tensors."""
    import torch
    d = len(u_cols)
    n = int(u_cols[0].numel())
    dev = u_cols[0].device
    keys = torch.empty(n, dtype=torch.int32, device=dev)
    perm = torch.empty(n, dtype=torch.int32, device=dev)
    counts = torch.empty(1 << (d * level), dtype=torch.int32, device=dev)
    arr = (C.c_void_p * 3)(*[c.data_ptr() for c in u_cols] + [None] * (3 - d))
    s = C.c_void_p(stream if stream is not None else torch.cuda.current_stream().cuda_stream)
    check(lib().sg_cell_sort(precision, d, level, n, arr, C.c_void_p(keys.data_ptr()), C.c_void_p(perm.data_ptr()),
                             C.c_void_p(counts.data_ptr()), s), "sg_cell_sort")
    return keys, perm, counts


# ------------------------------------------------------------------ Run
class Run:
    """One sparse-grid PIC run on the GPU.

    u: positions as fractions of the box, shape (N, d) or d columns;
    v: velocities; w: per-particle charge.  numpy (host) or torch CUDA.
    """

    def __init__(self, L_box, n, u, v, w, dt, *, tau=1, qm=-1.0, precision="fp32", B=(0.0, 0.0, 0.0),
                 eext_lin=(0.0, 0.0, 0.0), alpha=0.01, pc_ref=5.0, tau_constants="paper", sort_every=0,
                 stream=None, mode="combine", centring="node", combine="float-float", deferred=False):
        self.d = len(L_box)
        self.n = n
        self.precision = L.SG_FP32 if precision in ("fp32", L.SG_FP32) else L.SG_FP64
        self.dtype = _DT[self.precision]
        self.L = tuple(float(x) for x in L_box)
        d = self.d
        ucols = _columns(u, d, self.dtype)
        vcols = _columns(v, d, self.dtype)
        wcol = _columns([w], 1, self.dtype)[0]
        self.np = int(ucols[0].shape[0])
        dom = L.sg_domain()
        dom.dim = d
        for m in range(3):
            dom.L[m] = self.L[m] if m < d else 1.0
        parts = L.sg_particles()
        parts.n = self.np
        parts.on_device = _on_device(ucols[0])
        for m in range(d):
            parts.u[m] = _ptr(ucols[m]).value
            parts.v[m] = _ptr(vcols[m]).value
        parts.w = _ptr(wcol).value
        tc = L.SG_TAU_CONST_PAPER if tau_constants == "paper" else L.SG_TAU_CONST_EMPIRICAL
        self.params = make_params(self.precision, tau, dt, qm, B, eext_lin, alpha, pc_ref, tc, sort_every,
                                  stream, mode, centring, combine)
        self._keep = (ucols, vcols, wcol)
        if deferred:  # a part of a sharded run: sg_pic_start after the density exchange
            h = C.c_void_p()
            check(lib().sg_pic_init_deferred(C.byref(dom), n, d, 1, C.byref(parts), C.byref(self.params),
                                             C.byref(h)), "sg_pic_init_deferred")
            self.h = h
        else:
            self.h = sg_pic_init(dom, n, d, 1, parts, self.params)
        self._keep = None

    def close(self):
        if getattr(self, "h", None):
            sg_pic_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, k=1):
        sg_pic_step(self.h, k)

    def diagnostics(self):
        return sg_pic_diagnostics(self.h)

    def post_diagnostics(self):
        """Enqueue the read-back of the current diagnostics (no wait)."""
        sg_pic_diagnostics_post(self.h)

    def collect_diagnostics(self):
        """Wait for the oldest posted diagnostics record and return it."""
        return sg_pic_diagnostics_collect(self.h)

    def select_tau(self, cap=32):
        return sg_pic_select_tau(self.h, cap)

    def set_tau(self, tau):
        sg_pic_set_tau(self.h, tau)

    def grids(self):
        ng = C.c_int()
        check(lib().sg_pic_get_grids(self.h, C.byref(ng), None, None, 0), "sg_pic_get_grids")
        lev = np.zeros((ng.value, 3), dtype=np.int32)
        co = np.zeros(ng.value, dtype=np.int32)
        check(lib().sg_pic_get_grids(self.h, C.byref(ng), lev.ctypes.data, co.ctypes.data, ng.value),
              "sg_pic_get_grids")
        return [(tuple(int(x) for x in lev[g, :self.d]), int(co[g])) for g in range(ng.value)]

    def particles(self):
        """(u, v, w) host arrays in the original particle order."""
        d, N = self.d, self.np
        u = np.empty((d, N), dtype=self.dtype)
        v = np.empty((d, N), dtype=self.dtype)
        w = np.empty(N, dtype=self.dtype)
        o = L.sg_particles_out()
        o.n = N
        o.on_device = 0
        for m in range(d):
            o.u[m] = u[m].ctypes.data
            o.v[m] = v[m].ctypes.data
        o.w = w.ctypes.data
        check(lib().sg_pic_get_particles(self.h, C.byref(o)), "sg_pic_get_particles")
        return u.T.copy(), v.T.copy(), w

    def particles_device(self, out_u, out_v, out_w):
        """Write particle states (original order) into torch CUDA tensors."""
        o = L.sg_particles_out()
        o.n = self.np
        o.on_device = 1
        for m in range(self.d):
            o.u[m] = out_u[m].data_ptr()
            o.v[m] = out_v[m].data_ptr()
        o.w = out_w.data_ptr()
        check(lib().sg_pic_get_particles(self.h, C.byref(o)), "sg_pic_get_particles")

    def keys(self):
        k = np.empty(self.np, dtype=np.uint32)
        c = np.empty(1 << (self.d * self.n), dtype=np.uint32)
        check(lib().sg_pic_get_keys(self.h, k.ctypes.data, c.ctypes.data, k.size, c.size), "sg_pic_get_keys")
        return k, c

    def field(self):
        """E_comb on the regular nodes, shape (d, 2^n, ..., 2^n) indexed [m, i_1, .., i_d]."""
        N = 1 << self.n
        e = np.empty(self.d * N ** self.d)
        check(lib().sg_pic_get_field(self.h, e.ctypes.data, e.size), "sg_pic_get_field")
        return _flat_to_axes(e.reshape(self.d, -1), [self.n] * self.d)

    def regular_charge(self):
        N = 1 << self.n
        e = np.empty(N ** self.d)
        check(lib().sg_pic_get_regular_charge(self.h, e.ctypes.data, e.size), "sg_pic_get_regular_charge")
        return _flat_to_axes(e[None], [self.n] * self.d)[0]

    def density(self):
        """sum_i c_i P_i rho_i on the regular nodes (the filter mode's rho_f), indexed [i_1, .., i_d]."""
        N = 1 << self.n
        e = np.empty(N ** self.d)
        check(lib().sg_pic_get_density(self.h, e.ctypes.data, e.size), "sg_pic_get_density")
        return _flat_to_axes(e[None], [self.n] * self.d)[0]

    def grid_charges(self):
        """{levels: rho array indexed [i_1, .., i_d]} of the component grids."""
        gs = self.grids()
        S = sum(1 << sum(l) for l, _ in gs)
        e = np.empty(S)
        check(lib().sg_pic_get_grid_charge(self.h, e.ctypes.data, e.size), "sg_pic_get_grid_charge")
        out, o = {}, 0
        for l, _ in gs:
            sz = 1 << sum(l)
            out[l] = _flat_to_axes(e[None, o:o + sz], list(l))[0]
            o += sz
        return out

    def grid_fields(self):
        gs = self.grids()
        S = sum(1 << sum(l) for l, _ in gs)
        e = np.empty(self.d * S)
        check(lib().sg_pic_get_grid_field(self.h, e.ctypes.data, e.size), "sg_pic_get_grid_field")
        out, o = {}, 0
        for l, _ in gs:
            sz = 1 << sum(l)
            out[l] = _flat_to_axes(e[o:o + self.d * sz].reshape(self.d, sz), list(l))
            o += self.d * sz
        return out

    def save(self):
        sz = C.c_size_t(0)
        check(lib().sg_pic_save(self.h, None, C.byref(sz)), "sg_pic_save")
        buf = (C.c_char * sz.value)()
        check(lib().sg_pic_save(self.h, buf, C.byref(sz)), "sg_pic_save")
        return bytes(buf)

    def load(self, blob: bytes):
        buf = C.create_string_buffer(blob, len(blob))
        check(lib().sg_pic_load(self.h, buf, len(blob)), "sg_pic_load")

    def kernel_launches(self):
        c = C.c_ulonglong()
        check(lib().sg_pic_kernel_launches(self.h, C.byref(c)), "sg_pic_kernel_launches")
        return c.value

    def set_profiling(self, on=True):
        check(lib().sg_pic_set_profiling(self.h, 1 if on else 0), "sg_pic_set_profiling")

    def set_solve_variant(self, variant="auto"):
        """'auto' (timed choice), 'passes' or 'one-block' (sg_pic_set_solve_variant)."""
        v = {"auto": L.SG_SOLVE_AUTO, "passes": L.SG_SOLVE_PASSES, "one-block": L.SG_SOLVE_ONE_BLOCK}.get(variant, variant)
        check(lib().sg_pic_set_solve_variant(self.h, v), "sg_pic_set_solve_variant")

    def stage_times(self):
        ms = np.zeros(6)
        check(lib().sg_pic_stage_times(self.h, ms.ctypes.data, 6), "sg_pic_stage_times")
        return dict(zip(["push", "sort", "deposit", "restrict", "solve", "combine"], ms.tolist()))

    def tuning(self):
        """Init-time autotuner record: solve variant, push grid and deposit
        window in use, and the timings (ms) they were chosen from."""
        ms = np.zeros(25)
        check(lib().sg_pic_stage_times(self.h, ms.ctypes.data, 25), "sg_pic_stage_times")
        return {"solve_variant": "one-block-per-grid" if ms[6] == 1 else "per-axis-passes",
                "passes_ms": float(ms[7]), "one_block_ms": float(ms[8]), "from_cache": bool(ms[9]),
                "push_blocks": int(ms[10]), "push_wave_blocks": int(ms[11]),
                "push_ms_half_one_two_waves": [float(x) for x in ms[12:15]],
                "deposit_window_nodes": int(ms[15]),
                "deposit_ms_4096_6144_8192_12288": [float(x) for x in ms[16:20]],
                "particles_from_cache": bool(ms[20]),
                "deposit_ms_drifted": [float(x) for x in ms[21:25]]}

    # ---- sharded runs (sg_pic_init_deferred / sg_pic_start / the split step)
    def start(self):
        check(lib().sg_pic_start(self.h), "sg_pic_start")

    def step_deposit(self):
        check(lib().sg_pic_step_deposit(self.h), "sg_pic_step_deposit")

    def step_fields(self):
        check(lib().sg_pic_step_fields(self.h), "sg_pic_step_fields")

    def set_charge_total(self, q_total):
        check(lib().sg_pic_set_charge_total(self.h, float(q_total)), "sg_pic_set_charge_total")

    def density_copy(self, buf, to_run):
        """Copy the regular-grid density into (to_run=False: out of the run) or
        from a torch CUDA tensor of 2^{dn} values of the run's precision."""
        check(lib().sg_pic_density_copy(self.h, C.c_void_p(buf.data_ptr()), int(buf.numel()), 1 if to_run else 0),
              "sg_pic_density_copy")

    def device_particles(self):
        o = L.sg_particles_out()
        check(lib().sg_pic_device_particles(self.h, C.byref(o)), "sg_pic_device_particles")
        return o


def _flat_to_axes(flat, levels):
    """Rows of x-fastest flat grid arrays -> arrays indexed [.., i_1, .., i_d]."""
    shape_rev = tuple(1 << l for l in reversed(levels))
    d = len(levels)
    out = flat.reshape((flat.shape[0],) + shape_rev)
    return np.ascontiguousarray(np.transpose(out, (0,) + tuple(range(d, 0, -1))))


# ------------------------------------------------------------------ serving
class Server:
    """Independent runs admitted by device-memory footprint and advanced
    together tick by tick (sg_serve_*)."""

    def __init__(self, hbm_budget_bytes, max_slots):
        self.h = C.c_void_p()
        check(lib().sg_serve_create(int(hbm_budget_bytes), int(max_slots), C.byref(self.h)), "sg_serve_create")
        self.meta = {}

    def submit(self, L_box, n, u, v, w, dt, nsteps, *, tau=1, qm=-1.0, precision="fp32", B=(0.0, 0.0, 0.0),
               eext_lin=(0.0, 0.0, 0.0), sort_every=0, mode="combine", centring="node", combine="float-float"):
        d = len(L_box)
        prec = L.SG_FP32 if precision in ("fp32", L.SG_FP32) else L.SG_FP64
        dt_np = _DT[prec]
        ucols = _columns(u, d, dt_np)
        vcols = _columns(v, d, dt_np)
        wcol = _columns([w], 1, dt_np)[0]
        req = L.sg_request()
        req.domain.dim = d
        for m in range(3):
            req.domain.L[m] = float(L_box[m]) if m < d else 1.0
        req.level_n = n
        req.dim = d
        req.particles.n = int(ucols[0].shape[0])
        req.particles.on_device = 0
        for m in range(d):
            req.particles.u[m] = _ptr(ucols[m]).value
            req.particles.v[m] = _ptr(vcols[m]).value
        req.particles.w = _ptr(wcol).value
        req.params = make_params(prec, tau, dt, qm, B, eext_lin, 0.01, 5.0, L.SG_TAU_CONST_PAPER, sort_every, None,
                                 mode, centring, combine)
        req.nsteps = int(nsteps)
        t = C.c_ulonglong()
        check(lib().sg_serve_submit(self.h, C.byref(req), C.byref(t)), "sg_serve_submit")
        self.meta[t.value] = (d, int(ucols[0].shape[0]), dt_np)
        return t.value

    def set_mode(self, mode):
        """"batched" (each run's cached graphs on its own stream, one cross-run solve launch per tick for
        the runs that take part) or "plain" (runs in turn, direct launches, one solve launch per grid)."""
        m = L.SG_SERVE_BATCHED if mode in ("batched", L.SG_SERVE_BATCHED) else L.SG_SERVE_PLAIN
        check(lib().sg_serve_set_mode(self.h, m), "sg_serve_set_mode")

    def tick(self):
        a = C.c_int()
        check(lib().sg_serve_tick(self.h, C.byref(a)), "sg_serve_tick")
        return a.value

    def poll(self, ticket):
        st = C.c_int()
        dg = L.sg_diag()
        check(lib().sg_serve_poll(self.h, ticket, C.byref(st), C.byref(dg)), "sg_serve_poll")
        return st.value, dg.as_dict()

    def result(self, ticket):
        d, N, dt_np = self.meta[ticket]
        u = np.empty((d, N), dtype=dt_np)
        v = np.empty((d, N), dtype=dt_np)
        w = np.empty(N, dtype=dt_np)
        o = L.sg_particles_out()
        o.n = N
        o.on_device = 0
        for m in range(d):
            o.u[m] = u[m].ctypes.data
            o.v[m] = v[m].ctypes.data
        o.w = w.ctypes.data
        check(lib().sg_serve_result(self.h, ticket, C.byref(o)), "sg_serve_result")
        return u.T.copy(), v.T.copy(), w

    def stats(self):
        p50, p99, pst = C.c_double(), C.c_double(), C.c_double()
        n = C.c_ulonglong()
        check(lib().sg_serve_stats(self.h, C.byref(p50), C.byref(p99), C.byref(pst), C.byref(n)), "sg_serve_stats")
        return {"p50_ms": p50.value, "p99_ms": p99.value, "particle_steps_per_s": pst.value, "steps": n.value}

    def solve_stats(self):
        """Cross-run solves of the batched mode: launches and grids solved."""
        a, b = C.c_ulonglong(), C.c_ulonglong()
        check(lib().sg_serve_solve_stats(self.h, C.byref(a), C.byref(b)), "sg_serve_solve_stats")
        return {"launches": a.value, "grids": b.value}

    def close(self):
        if getattr(self, "h", None):
            lib().sg_serve_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
