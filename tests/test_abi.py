"""The C ABI library loads and exports every entry point declared in
include/fmpb.h; host-only calls and argument checking work without a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "fmpb.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(fmpb_[a-z0-9_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def L():
    from paper_2201_12050_gb300 import build
    build.build()
    from paper_2201_12050_gb300 import lib
    return lib()


def test_every_declared_symbol_is_exported_and_bound(L):
    from paper_2201_12050_gb300._lib import SIGNATURES
    names = _declared()
    assert len(names) >= 15
    for n in names:
        assert hasattr(L, n), n
    assert sorted(SIGNATURES) == names


def test_every_declared_call_has_a_binding_of_the_same_name(L):
    # the Python binding calls every entry point of the header
    # (fmpb_last_error feeds its exceptions)
    import paper_2201_12050_gb300 as gb
    api_src = open(os.path.join(ROOT, "paper_2201_12050_gb300", "api.py")).read()
    for n in _declared():
        if n != "fmpb_last_error":
            assert re.search(rf"(lib\(\)|self\._lib)\.{n}\b", api_src), n
    assert gb.version() == (0, 1)
    # device vectors must be complex128 CUDA tensors: refused before any call
    import torch
    x = torch.zeros(4, dtype=torch.complex128)
    with pytest.raises(TypeError):
        gb.circulant_apply_static([2, 1, 1], torch.zeros((3, 2, 2), dtype=torch.complex128), x)


def test_host_only_calls(L):
    from paper_2201_12050_gb300 import circulant_shape, FmpbError
    assert L.fmpb_version() == (0 << 16) | 1
    # smallest 2,3,5,7-smooth P >= 2M - 1 (Sec. 2.4 embedding; any P >= 2M-1 is exact)
    assert circulant_shape([3, 20, 1]) == ([5, 40, 1], 200)
    assert circulant_shape([32, 32]) == ([63, 63, 1], 3969)
    assert circulant_shape([16, 16, 4]) == ([32, 32, 7], 7168)
    assert circulant_shape([6]) == ([12, 1, 1], 12)      # 11 is not smooth
    with pytest.raises(FmpbError) as e:
        circulant_shape([0, 1, 1])
    assert e.value.name == "FMPB_EINVAL"


def test_padded_lengths_are_the_smallest_smooth_embedding_for_every_count(L):
    # every count the library accepts: P = 1 for one cell, else the smallest
    # 2,3,5,7-smooth P >= 2M - 1 (found here by trial division); F = P0 P1 P2
    from paper_2201_12050_gb300 import circulant_shape, FmpbError

    def smooth(n):
        for f in (2, 3, 5, 7):
            while n % f == 0:
                n //= f
        return n == 1

    for M in range(1, 4097):
        P = 1
        if M > 1:
            P = 2 * M - 1
            while not smooth(P):
                P += 1
        got, F = circulant_shape([1, M, 1])
        assert got == [1, P, 1] and F == P, M
    assert circulant_shape([4096, 4096, 4096])[1] == 8192 ** 3
    with pytest.raises(FmpbError):
        circulant_shape([4097, 1, 1])


def test_spectrum_holds_at_least_the_printed_number_of_blocks(L):
    # the spectrum of Sec. 2.4 holds (2M_x-1)(2M_y-1) blocks
    # (tests/golden/paper_storage_counts.txt); the library pads each length
    # to a 2,3,5,7-smooth P >= 2M - 1, so it holds exactly that many where
    # 2M - 1 is smooth and more elsewhere
    from paper_2201_12050_gb300 import circulant_shape
    line = next(l for l in open(os.path.join(ROOT, "tests", "golden", "paper_storage_counts.txt"))
                if l.startswith("spectrum_blocks"))
    expr = line.split("|")[1].strip()
    assert re.fullmatch(r"[0-9MxMy*()+\- ]+", expr)
    for Mx, My in ((5, 5), (5, 10), (5, 100), (3, 20), (2, 3)):
        printed = eval(expr, {"__builtins__": {}}, {"Mx": Mx, "My": My})
        P, F = circulant_shape([Mx, My, 1])
        assert F >= printed
        assert (F == printed) == (P[0] == 2 * Mx - 1 and P[1] == 2 * My - 1)


def test_argument_errors_are_statuses_not_crashes(L):
    h = ctypes.c_void_p()
    st = L.fmpb_operator_create(None, 0, None, 0, None, 1.0, None, None, None)
    assert st == -1 and b"NULL" in L.fmpb_last_error()
    st = L.fmpb_operator_create(None, 0, None, 0, None, -1.0, None, None, ctypes.byref(h))
    assert st == -1 and b"wavenumber" in L.fmpb_last_error()
    assert L.fmpb_matvec(None, 1, None, None, None) == -1
    L.fmpb_operator_destroy(None)


def test_plan_overrides_check_their_range(L):
    # the tile-variant and DFT-plan overrides are host-side settings: valid
    # values (and -1, back to the autotuners) are accepted without a GPU, the
    # rest are FMPB_EINVAL with a message
    for kind in (0, 1, 2, -1):
        assert L.fmpb_set_dft_plan(kind) == 0
    for bad in (3, -2):
        assert L.fmpb_set_dft_plan(bad) == -1 and b"plan kind" in L.fmpb_last_error()
    for v in (0, 3, -1):
        assert L.fmpb_set_tile_variant(v) == 0
    assert L.fmpb_set_tile_variant(4) == -1


def test_product_sizes_are_checked_before_device_calls(L):
    # sizes whose device copies would not be addressable are refused on the
    # host, before any device call; the dummy pointers are never touched, so
    # the check runs only where no GPU is visible
    import torch
    if torch.cuda.is_available():
        pytest.skip("host-only check")
    dummy = ctypes.c_void_p(256)
    big = (ctypes.c_int32 * 3)(4096, 4096, 4096)
    one = (ctypes.c_int32 * 3)(1, 1, 1)
    off = (ctypes.c_int32 * 3)(0, 0, 0)
    # 2^36 cells x 4096 right-hand sides x 2^21 BF16 values wraps in 64 bits
    assert L.fmpb_offset_gemm_bf16(big, 1, off, 64, 1 << 20, dummy, 4096, dummy, ctypes.c_void_p(512), 0,
                                   None) == -1
    assert b"launch limit" in L.fmpb_last_error()
    assert L.fmpb_offset_gemm2_bf16(big, 1, off, 64, 64, dummy, 1, dummy, 64, dummy, dummy,
                                    ctypes.c_void_p(512), 0, None) == -1
    assert b"launch limit" in L.fmpb_last_error()
    # one column tile too many: 65,535 x 128 + 1 columns
    cols = (ctypes.c_int32 * 3)(65535 * 128 // 4096 + 1, 1, 1)
    assert L.fmpb_offset_gemm_bf16(cols, 1, off, 64, 64, dummy, 4096, dummy, ctypes.c_void_p(512), 0,
                                   None) == -1
    # B^2 x 16 bytes wraps for B = 2^32; too many cells for the offset list
    for counts, B in ((one, 1 << 32), (one, (1 << 20) + 1), (big, 4)):
        assert L.fmpb_circulant_spectrum(counts, B, dummy, ctypes.c_void_p(512), None) == -1
        assert b"circulant_spectrum" in L.fmpb_last_error()


def test_server_reports_missing_device_as_status(L):
    import torch
    if torch.cuda.is_available():
        pytest.skip("host-only check")
    from paper_2201_12050_gb300._lib import ServerOpts
    h = ctypes.c_void_p()
    st = L.fmpb_server_create(ctypes.byref(ServerOpts()), ctypes.byref(h))
    assert st in (-8, -2) and not h.value
    assert L.fmpb_server_submit(None, None, None, None) == -1


def test_element_and_pressure_order_checks_are_host_side(L):
    # combinations refused before any device work, so the checks run on any host
    from paper_2201_12050_gb300._lib import OperatorOpts, Lattice
    lat = Lattice()
    for a in range(3):
        lat.counts[a] = 1
        lat.vectors[a][a] = 1.0
    h = ctypes.c_void_p()

    def create(**kw):
        o = OperatorOpts()
        for name, v in kw.items():
            setattr(o, name, v)
        return L.fmpb_operator_create(None, 0, None, 0, ctypes.byref(lat), 2.0, ctypes.byref(o), None, ctypes.byref(h))

    cases = [dict(element=2),                                   # no such element
             dict(pressure_order=1),                            # higher orders take quadrilaterals
             dict(element=1, pressure_order=3),                 # no such order
             dict(element=1, form=2, pressure_order=1),         # FMPBEM2: constant pressure only
             dict(element=1, form=2, precision=1),              # FMPBEM2 runs FP64
             dict(element=1, precision=2),                      # no BF16 tables on quadrilaterals
             dict(element=1, form=0, precision=3)]              # the FMM form: FP64 or FP32
    for kw in cases:
        assert create(**kw) == -1, kw
    assert not h.value
    st = L.fmpb_build_blocks_q9p(None, 0, None, 0, 3, ctypes.byref(lat), 2.0, 0.0, 0.0, 1,
                                 (ctypes.c_int32 * 3)(0, 0, 0), ctypes.c_void_p(1), None)
    assert st == -1 and b"order" in L.fmpb_last_error()
