"""fmpb_circulant_apply_static: the allocation-free variant of the block
Toeplitz product, for callers that cannot allocate device memory during the
call.  Checked through the C ABI against fmpb_circulant_apply on two calls in
a row (the static scratch keeps the previous call's contents, which must not
leak into the next result), plus the size limit of the static array."""
import ctypes

import numpy as np
import pytest
import torch

from workloads import random_complex_vectors

gb = pytest.importorskip("paper_2201_12050_gb300")


def _offsets(counts):
    Mx, My, Mz = counts
    return [(dx, dy, dz) for dz in range(1 - Mz, Mz) for dy in range(1 - My, My) for dx in range(1 - Mx, Mx)]


def _call(fn, counts, B, spec, x, y, accumulate):
    c = np.ascontiguousarray(np.asarray(counts, dtype=np.int32))
    R = x.shape[0]
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return fn(ctypes.c_void_p(c.ctypes.data), B, ctypes.c_void_p(spec.data_ptr()), R,
              ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()), accumulate, st)


@pytest.mark.gpu
@pytest.mark.parametrize("counts,B,R", [((3, 2, 1), 7, 3), ((5, 4, 1), 33, 2), ((2, 3, 2), 4, 6)])
def test_static_scratch_product_matches_allocating_product(counts, B, R):
    L = gb.lib()
    offs = _offsets(counts)
    blocks = random_complex_vectors(4000 + B, len(offs), B * B).reshape(len(offs), B, B)
    spec = gb.circulant_spectrum(counts, torch.as_tensor(blocks, device="cuda"))
    ncell = int(np.prod(counts))
    for call in range(2):
        x = torch.as_tensor(random_complex_vectors(5000 + 17 * call + R, R, ncell * B), device="cuda")
        y_ref = torch.empty_like(x)
        y_new = torch.full_like(x, complex(float("nan"), 0.0))
        assert _call(L.fmpb_circulant_apply, counts, B, spec, x, y_ref, 0) == 0
        assert _call(L.fmpb_circulant_apply_static, counts, B, spec, x, y_new, 0) == 0, L.fmpb_last_error()
        torch.cuda.synchronize()
        a, b = y_new.cpu().numpy(), y_ref.cpu().numpy()
        assert np.linalg.norm(a - b) <= 1e-12 * np.linalg.norm(b)
        # accumulate mode as well
        y_acc = x.clone()
        assert _call(L.fmpb_circulant_apply_static, counts, B, spec, x, y_acc, 1) == 0
        torch.cuda.synchronize()
        assert np.linalg.norm(y_acc.cpu().numpy() - (b + x.cpu().numpy())) <= 1e-12 * np.linalg.norm(b)


def _host_only_library():
    """The library for host-side argument checks: built here if need be, and
    skipped where it cannot be built (no CUDA toolkit)."""
    from paper_2201_12050_gb300 import build
    try:
        build.build()
        return gb.lib()
    except (RuntimeError, OSError) as e:
        pytest.skip(f"library not available: {e}")


# Every case below is refused on the host before any CUDA call, so these run
# only where no GPU is visible: with no device, nothing can be launched even
# if a check were wrong.
@pytest.mark.skipif(torch.cuda.is_available(), reason="host-side size check; run where no GPU is visible")
@pytest.mark.parametrize("counts,B,R,what", [
    ((40, 40, 1), 64, 8, b"static array holds"),       # P = 80 x 80, F = 6400: 2 F R B x 16 B = 105 MB > 32 MiB
    ((2, 1, 1), 1 << 20, 1, b"static array holds"),    # the largest B, F = 3: 96 MiB
    ((1, 1, 1), 1 << 59, 1, b"bad arguments"),         # 2 F R B x 16 B wraps to 0 in 64 bits
    ((1, 1, 1), (1 << 20) + 1, 1, b"bad arguments"),
    ((1, 1, 1), 0, 1, b"bad arguments"),
    ((1, 1, 1), 4, 0, b"R out of range"),
    ((1, 1, 1), 4, 4097, b"R out of range"),
    ((4097, 1, 1), 4, 1, b"count out of range"),
    ((0, 1, 1), 4, 1, b"count out of range"),
    ((4096, 4096, 1), 2, 4096, b"static array holds"),   # F R B near 2^41: no wrap in the test
])
def test_static_scratch_rejects_products_beyond_its_size(counts, B, R, what):
    L = _host_only_library()
    c = np.array(counts, dtype=np.int32)
    dummy = ctypes.c_void_p(256)
    st = L.fmpb_circulant_apply_static(ctypes.c_void_p(c.ctypes.data), ctypes.c_int64(B), dummy, R, dummy, dummy, 0,
                                       None)
    assert st == -1
    assert what in L.fmpb_last_error()


@pytest.mark.skipif(torch.cuda.is_available(), reason="host-side size check; run where no GPU is visible")
@pytest.mark.parametrize("counts,B,R", [((1, 1, 1), 1 << 59, 1), ((4096, 4096, 4096), 1 << 20, 4096),
                                        ((1, 1, 1), (1 << 20) + 1, 1)])
def test_allocating_product_rejects_sizes_that_overflow(counts, B, R):
    L = _host_only_library()
    c = np.array(counts, dtype=np.int32)
    dummy = ctypes.c_void_p(256)
    st = L.fmpb_circulant_apply(ctypes.c_void_p(c.ctypes.data), ctypes.c_int64(B), dummy, R, dummy, dummy, 0, None)
    assert st == -1
