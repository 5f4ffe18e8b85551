"""Thin Python binding of the C ABI (include/fmpb.h), same names, argument
marshalling only.  Device vectors are torch.complex128 CUDA tensors (the
interleaved layout of fmpb_c64); host arrays are numpy.  Work is enqueued on
torch's current CUDA stream.
"""
import ctypes

import numpy as np
import torch

from ._lib import (lib, check, Lattice, OperatorOpts, OperatorInfo, Incident, C64, SolveOpts, SolveInfo, FmpbError, ServerOpts,
                   Request, Result, ServerStats, STATUS)

FORM_AUTO, FORM_FMM, FORM_PBEM, FORM_FMM2 = -1, 0, 1, 2
FORM_NAMES = {FORM_FMM: "fmm", FORM_PBEM: "pbem", FORM_FMM2: "fmm2"}
FP64, FP32, BF16, MIXED = 0, 1, 2, 3
ELEM_TRI3, ELEM_QUAD9 = 0, 1
PRECISION_NAMES = {FP64: "fp64", FP32: "fp32", BF16: "bf16", MIXED: "mixed"}


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(a) -> ctypes.c_void_p:
    if isinstance(a, torch.Tensor):
        return ctypes.c_void_p(a.data_ptr())
    return ctypes.c_void_p(a.ctypes.data)


def _host(a, dtype):
    return np.ascontiguousarray(np.asarray(a, dtype=dtype))


def _lattice(counts, vectors) -> Lattice:
    L = Lattice()
    c = list(counts) + [1] * (3 - len(counts))
    for a in range(3):
        L.counts[a] = int(c[a])
    V = np.asarray(vectors, dtype=np.float64).reshape(3, 3)
    for a in range(3):
        for d in range(3):
            L.vectors[a][d] = float(V[a, d])
    return L


def _cvec(x, N, name):
    if not (isinstance(x, torch.Tensor) and x.is_cuda and x.dtype == torch.complex128):
        raise TypeError(f"{name} must be a complex128 CUDA tensor")
    if not x.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if x.numel() % N:
        raise ValueError(f"{name} has {x.numel()} entries, not a multiple of N = {N}")
    return x.numel() // N


class Operator:
    """fmpb_operator: the tables of one (unit-cell mesh, lattice, k); beta is
    the surface's uniform normalised admittance (0: rigid); plane =
    (axis, offset, R_p) makes it a half-space operator (None: full space).
    tris with nine columns are nine-node quadrilaterals (FMPB_ELEM_QUAD9),
    whose discontinuous pressure has order pressure_order (0, 1 or 2)."""

    def __init__(self, verts, tris, counts, vectors, k, form=FORM_AUTO, n_t=0, precision=FP64, beta=0.0,
                 plane=None, n_t_near=0, near_levels=0, pressure_order=0):
        self._lib = lib()
        v = _host(verts, np.float64)
        t = _host(tris, np.int32)
        self._lat = _lattice(counts, vectors)
        beta = complex(beta)
        opts = OperatorOpts(int(form), int(n_t), int(precision), beta.real, beta.imag)
        opts.n_t_near, opts.near_levels = int(n_t_near), int(near_levels)
        if t.ndim == 2 and t.shape[1] == 9:
            opts.element = ELEM_QUAD9
        opts.pressure_order = int(pressure_order)
        if plane is not None:
            axis, offset, Rp = plane
            Rp = complex(Rp)
            opts.halfspace, opts.plane_axis, opts.plane_offset = 1, int(axis), float(offset)
            opts.Rp_re, opts.Rp_im = Rp.real, Rp.imag
        h = ctypes.c_void_p()
        check(self._lib.fmpb_operator_create(_ptr(v), len(v), _ptr(t), len(t), ctypes.byref(self._lat),
                                             float(k), ctypes.byref(opts), _stream(), ctypes.byref(h)))
        self._h = h
        self.k = float(k)
        info = OperatorInfo()
        check(self._lib.fmpb_operator_get_info(self._h, ctypes.byref(info)))
        self.info = {f: (list(getattr(info, f)) if f == "P" else getattr(info, f)) for f, _ in info._fields_}
        self.info["form_name"] = FORM_NAMES[self.info["form"]]
        self.info["precision_name"] = PRECISION_NAMES.get(self.info["precision"], "?")
        self.N = self.info["N"]

    def close(self):
        if getattr(self, "_h", None):
            self._lib.fmpb_operator_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def rhs_plane_wave(self, dirs, amps=None, out=None):
        d = _host(dirs, np.float64).reshape(-1, 3)
        R = len(d)
        a = None if amps is None else _host(np.asarray(amps, dtype=np.complex128).reshape(R), np.complex128)
        b = out if out is not None else torch.empty((R, self.N), dtype=torch.complex128, device="cuda")
        check(self._lib.fmpb_rhs_plane_wave(self._h, R, _ptr(d), None if a is None else _ptr(a), _ptr(b), _stream()))
        return b

    def rhs_incident(self, incidents, out=None):
        """fmpb_rhs_incident: incidents = [(kind, vec, amp)], kind "plane"
        (vec = unit direction) or "monopole" (vec = source position)."""
        inc = _incidents(incidents)
        R = len(inc)
        b = out if out is not None else torch.empty((R, self.N), dtype=torch.complex128, device="cuda")
        check(self._lib.fmpb_rhs_incident(self._h, R, ctypes.cast(inc, ctypes.c_void_p), _ptr(b), _stream()))
        return b

    def field_incident(self, p, incidents, pts):
        """fmpb_field_incident: total pressure at pts for incident fields of any kind."""
        R = _cvec(p, self.N, "p")
        inc = _incidents(incidents)
        if len(inc) != R:
            raise ValueError("one incident field per right-hand side")
        if not (isinstance(pts, torch.Tensor) and pts.is_cuda and pts.dtype == torch.float64):
            pts = torch.as_tensor(np.asarray(pts, dtype=np.float64), device="cuda")
        pts = pts.contiguous()
        npts = pts.numel() // 3
        out = torch.empty((R, npts), dtype=torch.complex128, device="cuda")
        check(self._lib.fmpb_field_incident(self._h, R, _ptr(p), ctypes.cast(inc, ctypes.c_void_p), npts, _ptr(pts),
                                            _ptr(out), _stream()))
        return out

    def insertion_loss(self, p, incidents, pts):
        """fmpb_insertion_loss: Eq. (insertionloss) in dB for the solutions p of the incident fields."""
        R = _cvec(p, self.N, "p")
        inc = _incidents(incidents)
        if len(inc) != R:
            raise ValueError("one incident field per right-hand side")
        if not (isinstance(pts, torch.Tensor) and pts.is_cuda and pts.dtype == torch.float64):
            pts = torch.as_tensor(np.asarray(pts, dtype=np.float64), device="cuda")
        pts = pts.contiguous()
        il = ctypes.c_double()
        check(self._lib.fmpb_insertion_loss(self._h, R, _ptr(p), ctypes.cast(inc, ctypes.c_void_p), pts.numel() // 3,
                                            _ptr(pts), ctypes.byref(il), _stream()))
        return il.value

    def matvec(self, x, out=None):
        R = _cvec(x, self.N, "x")
        y = out if out is not None else torch.empty_like(x)
        check(self._lib.fmpb_matvec(self._h, R, _ptr(x), _ptr(y), _stream()))
        return y

    def solve(self, b, tol=1e-8, restart=30, maxit=1000, timeout_ms=0, out=None, raise_on_noconv=True,
              inner_tol=0.0):
        R = _cvec(b, self.N, "b")
        p = out if out is not None else torch.empty_like(b)
        opts = SolveOpts(float(tol), int(restart), int(maxit), int(timeout_ms), float(inner_tol))
        infos = (SolveInfo * R)()
        st = self._lib.fmpb_solve(self._h, R, _ptr(b), _ptr(p), ctypes.byref(opts), ctypes.cast(infos, ctypes.c_void_p),
                                  _stream())
        info = [{"iters": i.iters, "converged": bool(i.converged), "relres_est": i.relres_est,
                 "relres_true": i.relres_true, "refinements": i.refinements} for i in infos]
        if st != 0 and (raise_on_noconv or st not in (-5, -6)):
            check(st)
        return p, info

    def check(self):
        """fmpb_operator_check: raises FmpbError if a tensor-core wait of this operator gave up."""
        check(self._lib.fmpb_operator_check(self._h, _stream()))

    def field(self, p, dirs, pts, amps=None):
        R = _cvec(p, self.N, "p")
        d = _host(dirs, np.float64).reshape(R, 3)
        a = None if amps is None else _host(np.asarray(amps, dtype=np.complex128).reshape(R), np.complex128)
        if not (isinstance(pts, torch.Tensor) and pts.is_cuda and pts.dtype == torch.float64):
            pts = torch.as_tensor(np.asarray(pts, dtype=np.float64), device="cuda")
        pts = pts.contiguous()
        npts = pts.numel() // 3
        out = torch.empty((R, npts), dtype=torch.complex128, device="cuda")
        check(self._lib.fmpb_field(self._h, R, _ptr(p), _ptr(d), None if a is None else _ptr(a), npts, _ptr(pts),
                                   _ptr(out), _stream()))
        return out


def solve_batch(ops, b, tol=1e-8, restart=30, maxit=1000, timeout_ms=0, out=None, raise_on_noconv=True,
                inner_tol=0.0):
    """fmpb_solve_batch: the systems of several operators with one N in one GMRES.

    b: (n_ops, R, N) complex128 CUDA; returns (p of the same shape, info as a
    list of n_ops lists of R dicts)."""
    n_ops = len(ops)
    if not (isinstance(b, torch.Tensor) and b.is_cuda and b.dtype == torch.complex128 and b.is_contiguous()):
        raise TypeError("b must be a contiguous complex128 CUDA tensor")
    N = ops[0].N
    if b.dim() != 3 or b.shape[0] != n_ops or b.shape[2] != N:
        raise ValueError(f"b must have shape (n_ops, R, N) = ({n_ops}, R, {N})")
    R = b.shape[1]
    p = out if out is not None else torch.empty_like(b)
    handles = (ctypes.c_void_p * n_ops)(*[op._h.value for op in ops])
    opts = SolveOpts(float(tol), int(restart), int(maxit), int(timeout_ms), float(inner_tol))
    infos = (SolveInfo * (n_ops * R))()
    st = lib().fmpb_solve_batch(ctypes.cast(handles, ctypes.c_void_p), n_ops, R, _ptr(b), _ptr(p), ctypes.byref(opts),
                                ctypes.cast(infos, ctypes.c_void_p), _stream())
    info = [[{"iters": i.iters, "converged": bool(i.converged), "relres_est": i.relres_est,
              "relres_true": i.relres_true, "refinements": i.refinements} for i in infos[o * R:(o + 1) * R]]
            for o in range(n_ops)]
    if st != 0 and (raise_on_noconv or st not in (-5, -6)):
        check(st)
    return p, info


def build_blocks(verts, tris, counts, vectors, k, offsets):
    """fmpb_build_blocks: T_delta for each offset, (n_off, n, n) on the device."""
    v = _host(verts, np.float64)
    t = _host(tris, np.int32)
    off = _host(offsets, np.int32).reshape(-1, 3)
    lat = _lattice(counts, vectors)
    out = torch.empty((len(off), len(t), len(t)), dtype=torch.complex128, device="cuda")
    check(lib().fmpb_build_blocks(_ptr(v), len(v), _ptr(t), len(t), ctypes.byref(lat), float(k), len(off), _ptr(off),
                                  _ptr(out), _stream()))
    return out


def _incidents(incidents):
    kinds = {"plane": 0, "monopole": 1}
    arr = (Incident * len(incidents))()
    for i, (kind, vec, amp) in enumerate(incidents):
        a = complex(amp)
        arr[i].kind = kinds[kind]
        for d in range(3):
            arr[i].vec[d] = float(vec[d])
        arr[i].amp = C64(a.real, a.imag)
    return arr


def halfspace_plan(verts, tris, counts, vectors, plane_axis, plane_offset):
    """fmpb_halfspace_plan, or fmpb_halfspace_plan_q9 for nine-column elements
    (host only): (perpendicular axis, near image offsets, nearest far image)."""
    v = _host(verts, np.float64)
    t = _host(tris, np.int32)
    lat = _lattice(counts, vectors)
    h, nn, dmin = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_double()
    fn = lib().fmpb_halfspace_plan_q9 if t.ndim == 2 and t.shape[1] == 9 else lib().fmpb_halfspace_plan
    check(fn(_ptr(v), len(v), _ptr(t), len(t), ctypes.byref(lat), int(plane_axis), float(plane_offset),
             ctypes.byref(h), ctypes.byref(nn), ctypes.byref(dmin)))
    return h.value, nn.value, dmin.value


def near2_plan_counts(verts, tris, counts, vectors, near_levels=0, n_t_near=0):
    """fmpb_near2_plan_counts, or fmpb_near2_plan_counts_q9 for nine-column
    elements (host only): (levels, M2L pairs, exact entries, translations)."""
    v = _host(verts, np.float64)
    t = _host(tris, np.int32)
    lat = _lattice(counts, vectors)
    lv = ctypes.c_int32()
    a, b, c = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    fn = lib().fmpb_near2_plan_counts_q9 if t.ndim == 2 and t.shape[1] == 9 else lib().fmpb_near2_plan_counts
    check(fn(_ptr(v), len(v), _ptr(t), len(t), ctypes.byref(lat), int(near_levels), int(n_t_near), ctypes.byref(lv),
             ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
    return lv.value, a.value, b.value, c.value


def build_blocks_admittance(verts, tris, counts, vectors, k, beta, offsets):
    """fmpb_build_blocks_admittance: T_delta of a surface of admittance beta."""
    v = _host(verts, np.float64)
    t = _host(tris, np.int32)
    off = _host(offsets, np.int32).reshape(-1, 3)
    lat = _lattice(counts, vectors)
    beta = complex(beta)
    out = torch.empty((len(off), len(t), len(t)), dtype=torch.complex128, device="cuda")
    check(lib().fmpb_build_blocks_admittance(_ptr(v), len(v), _ptr(t), len(t), ctypes.byref(lat), float(k),
                                             beta.real, beta.imag, len(off), _ptr(off), _ptr(out), _stream()))
    return out


def build_blocks_q9(nodes, elems, counts, vectors, k, offsets, beta=0.0, pressure_order=0):
    """fmpb_build_blocks_q9 (pressure_order 0) or fmpb_build_blocks_q9p (1, 2):
    T_delta on nine-node quadrilaterals (elems n x 9), (n_off, N, N) with
    N = n x (1, 4, 8)[pressure_order]."""
    v = _host(nodes, np.float64)
    t = _host(elems, np.int32).reshape(-1, 9)
    off = _host(offsets, np.int32).reshape(-1, 3)
    lat = _lattice(counts, vectors)
    beta = complex(beta)
    order = int(pressure_order)
    N = len(t) * {0: 1, 1: 4, 2: 8}.get(order, 1)
    out = torch.empty((len(off), N, N), dtype=torch.complex128, device="cuda")
    if order == 0:
        check(lib().fmpb_build_blocks_q9(_ptr(v), len(v), _ptr(t), len(t), ctypes.byref(lat), float(k), beta.real,
                                         beta.imag, len(off), _ptr(off), _ptr(out), _stream()))
    else:
        check(lib().fmpb_build_blocks_q9p(_ptr(v), len(v), _ptr(t), len(t), order, ctypes.byref(lat), float(k),
                                          beta.real, beta.imag, len(off), _ptr(off), _ptr(out), _stream()))
    return out


def multipole_tables_admittance(verts, tris, k, beta, n_t):
    """fmpb_multipole_tables_admittance: (V_0, U_0) of a surface of admittance beta."""
    v = _host(verts, np.float64)
    t = _host(tris, np.int32)
    B = (n_t + 1) ** 2
    beta = complex(beta)
    V0 = torch.empty((B, len(t)), dtype=torch.complex128, device="cuda")
    U0 = torch.empty((len(t), B), dtype=torch.complex128, device="cuda")
    check(lib().fmpb_multipole_tables_admittance(_ptr(v), len(v), _ptr(t), len(t), float(k), beta.real, beta.imag,
                                                 int(n_t), _ptr(V0), _ptr(U0), _stream()))
    return V0, U0


def multipole_tables(verts, tris, k, n_t):
    """fmpb_multipole_tables: (V_0 (B, n), U_0 (n, B)) on the device."""
    v = _host(verts, np.float64)
    t = _host(tris, np.int32)
    B = (n_t + 1) ** 2
    V0 = torch.empty((B, len(t)), dtype=torch.complex128, device="cuda")
    U0 = torch.empty((len(t), B), dtype=torch.complex128, device="cuda")
    check(lib().fmpb_multipole_tables(_ptr(v), len(v), _ptr(t), len(t), float(k), int(n_t), _ptr(V0), _ptr(U0),
                                      _stream()))
    return V0, U0


def m2l_blocks(k, n_t, dvecs):
    """fmpb_m2l_blocks: K(d) for each translation, (n_d, B, B)."""
    d = _host(dvecs, np.float64).reshape(-1, 3)
    B = (n_t + 1) ** 2
    out = torch.empty((len(d), B, B), dtype=torch.complex128, device="cuda")
    check(lib().fmpb_m2l_blocks(float(k), int(n_t), len(d), _ptr(d), _ptr(out), _stream()))
    return out


def offset_gemm_bf16(counts, offsets, T, x, out=None, accumulate=False):
    """fmpb_offset_gemm_bf16: y[r, c] (+)= sum_o T[o] x[r, c - delta_o] on the tensor cores.

    T: (n_off, m, k) complex128 CUDA; x: (R, n_cells * k); returns (R, n_cells * m)."""
    c = _host(list(counts) + [1] * (3 - len(counts)), np.int32)
    off = _host(offsets, np.int32).reshape(-1, 3)
    n_off, m, k = T.shape
    ncell = int(np.prod(c))
    R = _cvec(x, ncell * k, "x")
    y = out if out is not None else torch.empty((R, ncell * m), dtype=torch.complex128, device="cuda")
    check(lib().fmpb_offset_gemm_bf16(_ptr(c), int(n_off), _ptr(off), int(m), int(k), _ptr(T.contiguous()), R,
                                      _ptr(x), _ptr(y), 1 if accumulate else 0, _stream()))
    return y


def offset_gemm2_bf16(counts, offsets, T, x, T2, x2, out=None, accumulate=False):
    """fmpb_offset_gemm2_bf16: y[r, c] (+)= sum_o T[o] x[r, c - delta_o] + T2 x2[r, c]
    in one tensor-core accumulation.

    T: (n_off, m, k), T2: (m, k2) complex128 CUDA; x: (R, n_cells * k),
    x2: (R, n_cells * k2); returns (R, n_cells * m)."""
    c = _host(list(counts) + [1] * (3 - len(counts)), np.int32)
    off = _host(offsets, np.int32).reshape(-1, 3)
    n_off, m, k = T.shape
    m2, k2 = T2.shape
    if m2 != m:
        raise ValueError(f"T2 has {m2} rows, T has {m}")
    ncell = int(np.prod(c))
    R = _cvec(x, ncell * k, "x")
    if _cvec(x2, ncell * k2, "x2") != R:
        raise ValueError("x and x2 hold different numbers of right-hand sides")
    y = out if out is not None else torch.empty((R, ncell * m), dtype=torch.complex128, device="cuda")
    check(lib().fmpb_offset_gemm2_bf16(_ptr(c), int(n_off), _ptr(off), int(m), int(k), _ptr(T.contiguous()), R,
                                       _ptr(x), int(k2), _ptr(T2.contiguous()), _ptr(x2), _ptr(y),
                                       1 if accumulate else 0, _stream()))
    return y


def circulant_shape(counts):
    c = _host(list(counts) + [1] * (3 - len(counts)), np.int32)
    P = np.zeros(3, dtype=np.int32)
    F = ctypes.c_int64()
    check(lib().fmpb_circulant_shape(_ptr(c), _ptr(P), ctypes.byref(F)))
    return P.tolist(), F.value


def circulant_spectrum(counts, blocks):
    """fmpb_circulant_spectrum: blocks (n_off, B, B) complex128 CUDA -> (F, B, B)."""
    c = _host(list(counts) + [1] * (3 - len(counts)), np.int32)
    B = blocks.shape[-1]
    _, F = circulant_shape(counts)
    spec = torch.empty((F, B, B), dtype=torch.complex128, device="cuda")
    check(lib().fmpb_circulant_spectrum(_ptr(c), B, _ptr(blocks.contiguous()), _ptr(spec), _stream()))
    return spec


def circulant_apply(counts, spec, x, out=None, accumulate=False):
    """fmpb_circulant_apply: y (+)= T x for x of shape (R, n_cells * B)."""
    c = _host(list(counts) + [1] * (3 - len(counts)), np.int32)
    B = spec.shape[-1]
    ncell = int(np.prod(c))
    R = _cvec(x, ncell * B, "x")
    y = out if out is not None else torch.empty_like(x)
    check(lib().fmpb_circulant_apply(_ptr(c), B, _ptr(spec), R, _ptr(x), _ptr(y), 1 if accumulate else 0, _stream()))
    return y


def circulant_apply_static(counts, spec, x, out=None, accumulate=False):
    """fmpb_circulant_apply_static: circulant_apply without device allocation
    (its scratch is the library's fixed static array; larger products raise
    FMPB_EINVAL).  out must be given by callers that cannot allocate either."""
    c = _host(list(counts) + [1] * (3 - len(counts)), np.int32)
    B = spec.shape[-1]
    ncell = int(np.prod(c))
    R = _cvec(x, ncell * B, "x")
    y = out if out is not None else torch.empty_like(x)
    check(lib().fmpb_circulant_apply_static(_ptr(c), B, _ptr(spec), R, _ptr(x), _ptr(y), 1 if accumulate else 0,
                                            _stream()))
    return y


def circulant_apply_f32(counts, spec, x, out=None, accumulate=False):
    """fmpb_circulant_apply_f32: the circulant product in complex FP32 (spectrum, DFT passes, products)."""
    c = _host(list(counts) + [1] * (3 - len(counts)), np.int32)
    B = spec.shape[-1]
    ncell = int(np.prod(c))
    R = _cvec(x, ncell * B, "x")
    y = out if out is not None else torch.empty_like(x)
    check(lib().fmpb_circulant_apply_f32(_ptr(c), B, _ptr(spec.contiguous()), R, _ptr(x), _ptr(y),
                                         1 if accumulate else 0, _stream()))
    return y


def circulant_apply_bf16(counts, spec, x, out=None, accumulate=False):
    """fmpb_circulant_apply_bf16: the circulant product with BF16 tensor-core frequency products."""
    c = _host(list(counts) + [1] * (3 - len(counts)), np.int32)
    B = spec.shape[-1]
    ncell = int(np.prod(c))
    R = _cvec(x, ncell * B, "x")
    y = out if out is not None else torch.empty_like(x)
    check(lib().fmpb_circulant_apply_bf16(_ptr(c), B, _ptr(spec.contiguous()), R, _ptr(x), _ptr(y),
                                          1 if accumulate else 0, _stream()))
    return y


def version():
    """fmpb_version: (major, minor) of the library."""
    v = lib().fmpb_version()
    return v >> 16, v & 0xFFFF


def kernel_launches() -> int:
    """fmpb_kernel_launches: kernels launched by the library in this process."""
    return int(lib().fmpb_kernel_launches())


def profile_enable(on: bool = True):
    lib().fmpb_profile_enable(1 if on else 0)


def profile_reset():
    check(lib().fmpb_profile_reset())


def profile_summary() -> dict:
    """Per-kernel {name: (launches, total_ms)} of the recorded launches."""
    import json
    buf = ctypes.create_string_buffer(1 << 16)
    check(lib().fmpb_profile_summary(buf, len(buf)))
    return {k: (int(v[0]), float(v[1])) for k, v in json.loads(buf.value.decode()).items()}


def set_tile_variant(variant: int):
    """fmpb_set_tile_variant: force a tensor-core tile variant (0..3) or autotune (-1)."""
    check(lib().fmpb_set_tile_variant(int(variant)))


def set_dft_plan(kind: int):
    """fmpb_set_dft_plan: force a DFT plan kind (0 direct, 1 two-factor, 2 radix-2) or autotune (-1)."""
    check(lib().fmpb_set_dft_plan(int(kind)))


def tuning_summary() -> list:
    """fmpb_tuning_summary: tile shapes chosen by the tensor-core autotuner."""
    import json
    buf = ctypes.create_string_buffer(1 << 16)
    check(lib().fmpb_tuning_summary(buf, len(buf)))
    return json.loads(buf.value.decode())


class Server:
    """fmpb_server: queued solves of many (mesh, lattice, k) problems."""

    def __init__(self, hbm_budget_bytes=0, max_batch_rhs=64, cache_entries=8, precision=FP64, tol=1e-8,
                 restart=200, maxit=3000):
        self._lib = lib()
        o = ServerOpts(int(hbm_budget_bytes), int(max_batch_rhs), int(cache_entries), int(precision), float(tol),
                       int(restart), int(maxit))
        h = ctypes.c_void_p()
        check(self._lib.fmpb_server_create(ctypes.byref(o), ctypes.byref(h)))
        self._h = h
        self._pending = {}

    def submit(self, verts, tris, counts, vectors, k, dirs, amps=None, form=FORM_AUTO, n_t=0):
        """Queues a request; returns a ticket.  The result array is kept alive here."""
        v = _host(verts, np.float64)
        t = _host(tris, np.int32)
        d = _host(dirs, np.float64).reshape(-1, 3)
        R = len(d)
        a = None if amps is None else _host(np.asarray(amps, dtype=np.complex128).reshape(R), np.complex128)
        ncell = int(np.prod(list(counts) + [1] * (3 - len(counts))))
        out = np.zeros((R, len(t) * ncell), dtype=np.complex128)
        req = Request(_ptr(v), len(v), _ptr(t), len(t), _lattice(counts, vectors), float(k), int(form), int(n_t), R,
                      _ptr(d), None if a is None else _ptr(a))
        tk = ctypes.c_uint64()
        check(self._lib.fmpb_server_submit(self._h, ctypes.byref(req), _ptr(out), ctypes.byref(tk)))
        self._pending[tk.value] = (out, v, t, d, a)
        return tk.value

    def wait(self, ticket, timeout_ms=0):
        """(result dict, surface pressure R x N numpy array)."""
        r = Result()
        check(self._lib.fmpb_server_wait(self._h, ctypes.c_uint64(ticket), int(timeout_ms), ctypes.byref(r)))
        out = self._pending.pop(ticket)[0]
        res = {f: getattr(r, f) for f, _ in r._fields_}
        res["status_name"] = STATUS.get(res["status"], str(res["status"]))
        return res, out

    def stats(self):
        s = ServerStats()
        check(self._lib.fmpb_server_get_stats(self._h, ctypes.byref(s)))
        return {f: getattr(s, f) for f, _ in s._fields_}

    def close(self):
        if getattr(self, "_h", None):
            self._lib.fmpb_server_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
