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


@pytest.mark.skipif(torch.cuda.is_available(), reason="host-side size check; run where no GPU is visible")
def test_static_scratch_rejects_products_beyond_its_size():
    """The size check runs on the host before any CUDA call, so it is tested
    without a GPU: with no device visible, nothing can be launched."""
    from paper_2201_12050_gb300 import build
    build.build()
    L = gb.lib()
    counts = np.array([40, 40, 1], dtype=np.int32)      # P = 80 x 80, F = 6400
    B, R = 64, 8                                       # 2 F R B x 16 B = 105 MB > 32 MiB
    dummy = ctypes.c_void_p(256)
    st = L.fmpb_circulant_apply_static(ctypes.c_void_p(counts.ctypes.data), B, dummy, R, dummy, dummy, 0, None)
    assert st == -1
    assert b"static array holds" in L.fmpb_last_error()
