"""The allocation-free cell sort (sg_cell_sort_static) against the FP64
oracle's cell keys and stable sort, and against the allocating entry point
(sg_cell_sort), through the C ABI.

sg_cell_sort_static exists for callers that must not allocate device memory
(a device-memory budget owned by another allocator, or loops where an
allocation could synchronise the device); it keeps its scratch in a fixed
array inside the library.  Keys, permutation and counts are integer results,
so the two entry points must agree bit for bit.  Two calls in a row, the
second smaller and of the other precision, show that the contents the first
call leaves in the shared scratch do not leak into the second.
"""
import ctypes as C

import numpy as np
import pytest

from oracle import sgpic_oracle as O

pytestmark = pytest.mark.gpu


def _sort(fn, cols, level, precision):
    import torch
    d = len(cols)
    n = int(cols[0].numel())
    dev = cols[0].device
    keys = torch.empty(n, dtype=torch.int32, device=dev)
    perm = torch.empty(n, dtype=torch.int32, device=dev)
    counts = torch.empty(1 << (d * level), dtype=torch.int32, device=dev)
    arr = (C.c_void_p * 3)(*([c.data_ptr() for c in cols] + [None] * (3 - d)))
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    status = fn(precision, d, level, n, arr, C.c_void_p(keys.data_ptr()), C.c_void_p(perm.data_ptr()),
                C.c_void_p(counts.data_ptr()), stream)
    torch.cuda.synchronize()
    return status, keys.cpu().numpy(), perm.cpu().numpy(), counts.cpu().numpy()


def test_static_scratch_sort_matches_allocating_sort():
    import torch
    from paper_2008_09441_gb300 import _lib as L
    assert torch.cuda.is_available()
    lib = L.lib()
    rng = np.random.default_rng(20080944)
    cases = [(2, 8, 200000, L.SG_FP32, np.float32), (3, 5, 70001, L.SG_FP64, np.float64)]
    for d, level, n, prec, dt in cases:  # two calls in a row sharing the fixed scratch
        u = rng.random((n, d)).astype(dt)
        cols = [torch.from_numpy(np.ascontiguousarray(u[:, m])).cuda() for m in range(d)]
        sa, ka, pa, ca = _sort(lib.sg_cell_sort, cols, level, prec)
        sb, kb, pb, cb = _sort(lib.sg_cell_sort_static, cols, level, prec)
        assert sa == L.SG_OK and sb == L.SG_OK, lib.sg_last_error().decode()
        # the oracle's Morton keys of the same positions and its stable
        # counting sort: keys, permutation and counts are unique, bit for bit
        k_ref = O.cell_keys(u.astype(np.float64), level)
        p_ref, sk_ref, c_ref = O.sort_by_key(k_ref, level, d)
        assert np.array_equal(kb.view(np.uint32), sk_ref)
        assert np.array_equal(pb.view(np.uint32), p_ref)
        assert np.array_equal(cb.view(np.uint32), c_ref)
        assert np.array_equal(ka, kb)
        assert np.array_equal(pa, pb)
        assert np.array_equal(ca, cb)
        assert int(cb.sum()) == n


def test_static_scratch_rejects_oversize():
    import torch
    from paper_2008_09441_gb300 import _lib as L
    lib = L.lib()
    n = 262144 + 1  # SG_CELL_SORT_STATIC_MAX + 1
    cols = [torch.zeros(n, dtype=torch.float32, device="cuda") for _ in range(2)]
    status, _, _, _ = _sort(lib.sg_cell_sort_static, cols, 4, L.SG_FP32)
    assert status == L.SG_ERR_SIZE
    assert "fixed scratch capacity" in lib.sg_last_error().decode()
