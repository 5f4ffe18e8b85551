// Internal declarations shared by the library's translation units.
#pragma once
#include <mutex>
#include <vector>
#include <algorithm>

#include "common.cuh"
#include "ff.cuh"
#include "quad9.cuh"

namespace fmpb {

// Source-element geometry in float-float for the far-class quadrature.
struct FfElem {
  ff w0[3];      // v0 - centroid
  ff ba[3];      // v1 - v0
  ff cb[3];      // v2 - v1
  ff ny[3];      // unit normal
  ff c[3];       // centroid (collocation point of a target element)
  ff two_area;
  float hmax;
  float pad;
};
constexpr int NTAY = 9;   // Taylor terms of cos and sin in the float-float exponential
struct FfConst {
  ff s[Q_FAR], t[Q_FAR];
  ff W[Q_FAR * Q_FAR];    // s_a w_a w_b of the collapsed far rule
  ff ccos[NTAY], csin[NTAY];
  ff inv4pi;
};

// Float-float helpers of the far-class quadrature (quadrature.cu, quad9.cu).
__device__ __forceinline__ ff ff_dot3(const ff a[3], const ff b[3]) {
  return ff_add(ff_add(ff_mul(a[0], b[0]), ff_mul(a[1], b[1])), ff_mul(a[2], b[2]));
}

// e^{i psi} for |psi| <= 0.75 * 2^m
__device__ __forceinline__ ffc expi_ff(ff psi, int m, const FfConst& C) {
  const float sc = ldexpf(1.f, -m);
  const ff p = {psi.h * sc, psi.l * sc};    // exact scaling by a power of two
  const ff z = ff_mul(p, p);
  ff c = C.ccos[NTAY - 1], s = C.csin[NTAY - 1];
#pragma unroll
  for (int k = NTAY - 2; k >= 0; --k) {
    c = ff_add(C.ccos[k], ff_mul(z, c));
    s = ff_add(C.csin[k], ff_mul(z, s));
  }
  s = ff_mul(p, s);
  for (int i = 0; i < m; ++i) {
    const ff cs = ff_mul(c, s);
    c = ff_sub(ff_mul(c, c), ff_mul(s, s));
    s = {2.f * cs.h, 2.f * cs.l};
  }
  return {c, s};
}

// 2 pi split into two doubles (2 pi = TWO_PI_HI + TWO_PI_LO to ~1e-32)
constexpr double TWO_PI_HI = 6.283185307179586;
constexpr double TWO_PI_LO = 2.4492935982947064e-16;

// Fills the Taylor coefficients and 1/(4 pi) of C (every other field untouched).
__device__ inline void ff_const_series(FfConst& C) {
  double f = 1.0;   // (2k)! and (2k+1)!, exact in FP64 up to 17!
  for (int k = 0; k < NTAY; ++k) {
    const double f2k = f;
    const double f2k1 = f * (2 * k + 1);
    const double sgn = (k & 1) ? -1.0 : 1.0;
    C.ccos[k] = ff_from_d(sgn / f2k);
    C.csin[k] = ff_from_d(sgn / f2k1);
    f = f2k1 * (2 * k + 2);
  }
  C.inv4pi = ff_from_d(0.25 / PI);
}

// Gauss-Legendre node i (ascending) and weight of order q on [0, 1]
// (Newton's method on P_q).
__host__ __device__ void gl_node(int q, int i, double* t, double* w);

// T = -(D + (i/k) H)
__host__ __device__ __forceinline__ cd bm_entry(cd D, cd H, double k) {
  return mkc(-D.x + H.y / k, -D.y - H.x / k);
}

// T = -(D + b H) - i k beta (S + b K), b = i/k: the admittance condition
// dp/dn_m = -i k beta p turns the dp/dn terms of the Burton-Miller equation
// into -i k beta S + beta K.
__host__ __device__ __forceinline__ cd bm_entry_adm(cd D, cd H, cd S, cd K, double k, cd beta) {
  const cd t = mkc(K.x + k * S.y, K.y - k * S.x);   // K - i k S
  return cadd(bm_entry(D, H, k), cmul(beta, t));
}

// The same with rk = 1 / k given (no division per entry).
__host__ __device__ __forceinline__ cd bm_entry_rk(cd D, cd H, double rk) {
  return mkc(-D.x + H.y * rk, -D.y - H.x * rk);
}
__host__ __device__ __forceinline__ cd bm_entry_adm_rk(cd D, cd H, cd S, cd K, double k, double rk, cd beta) {
  const cd t = mkc(K.x + k * S.y, K.y - k * S.x);   // K - i k S
  return cadd(bm_entry_rk(D, H, rk), cmul(beta, t));
}

// How a block kernel stores an entry: out = v, or out (+)= scale v (image
// blocks of a half-space operator: R_p times the entries, added to the
// full-space blocks when both share one block Toeplitz pattern).
struct BlockWrite {
  cd scale;
  int scaled, accumulate;
  __device__ __forceinline__ void put(cd* dst, cd v) const {
    if (scaled) v = cmul(scale, v);
    *dst = accumulate ? cadd(*dst, v) : v;
  }
};

// Finite cell grid (Sec. 2.2): counts M[a] along lattice vectors L[a].
struct CellGrid {
  int M[3];
  double L[3][3];
  int ncells;
  __host__ __device__ void cell_index(int c, int idx[3]) const {
    idx[0] = c % M[0];
    idx[1] = (c / M[0]) % M[1];
    idx[2] = c / (M[0] * M[1]);
  }
  __host__ __device__ void cell_position(int c, double pos[3]) const {
    int id[3];
    cell_index(c, id);
    for (int d = 0; d < 3; ++d) pos[d] = id[0] * L[0][d] + id[1] * L[1][d] + id[2] * L[2][d];
  }
};

// Circulant embedding shape: padded lengths P[a] >= 2 M[a] - 1 (Sec. 2.4).
struct CircShape {
  int M[3];
  int P[3];
  int64_t F;
  int64_t ncells;
};
int padded_length(int M);
CircShape make_shape(const int M[3]);
// Flat slot of offset delta in the padded grid: ((dz mod Pz) Py + (dy mod Py)) Px + (dx mod Px).
int64_t offset_slot(const CircShape& s, int dx, int dy, int dz);

struct DeviceMesh {
  int n = 0;
  Elem* el = nullptr;
  QuadRules* qr_dev = nullptr;
  QuadRules qr;
  FfElem* ffel = nullptr;
  FfConst* fc_dev = nullptr;
  FfConst fc;
  double radius = 0.0;   // max |vertex| about the origin (expansion centre)
  // Nine-node quadrilaterals (nodes = 9; el then holds each element's centre,
  // normal, chord and area for the collocation points): the elements and
  // their class-rule points, the far rule point-major and field-major
  // (q9_far[(p 7 + f) n + e], f: y, n_y, w|J|) for coalesced loads across
  // source elements, the near and very-near rules element-major
  // (q9_near[(e 320 + p) 8 + f]) for a warp sharing one element.
  // With pressure of order q9_order = 1 or 2 (nb = 4 or 8 nodes per element)
  // n counts the q9_ne nb dofs (dof e nb + a) and el holds each dof's
  // collocation point and normal.
  int nodes = 3;
  int q9_order = 0;
  int q9_ne = 0;
  Q9Elem* q9 = nullptr;
  double* q9_far = nullptr;
  // the far rule again in float-float pairs relative to the element centre
  // (u = y - c, n_y, w|J|; q9_farff[(p 7 + f) n + e]) for the float-float
  // far class of constant-pressure elements
  float2* q9_farff = nullptr;
  double* q9_near = nullptr;
  Q9Rules q9r;
};

fmpb_status upload_mesh(const double* verts, int64_t nv, const int32_t* tris, int64_t ntri, DeviceMesh& m,
                        cudaStream_t st);
void free_mesh(DeviceMesh& m);
// Nine-node quadrilateral mesh: nodes nn x 3, elems n x 9 node indices
// (node (i, j) of the element's 3 x 3 grid at 3 j + i, i along xi,
// y_xi x y_eta into the fluid).
fmpb_status upload_mesh_q9(const double* nodes, int64_t nn, const int32_t* elems, int64_t n, DeviceMesh& m,
                           cudaStream_t st);
// build_entries for a nine-node mesh with constant pressure (quad9.cu).
fmpb_status build_entries_q9(const DeviceMesh& m, const CellGrid& g, double k, cd beta, int n_off,
                             const int32_t* offsets, const int64_t* list, int64_t count, const int64_t* self_slot,
                             cd* out, cudaStream_t st);
// The same with discontinuous pressure of order 1 or 2 (quad9p.cu).
fmpb_status upload_mesh_q9p(const double* nodes, int64_t nn, const int32_t* elems, int64_t n, int order,
                            DeviceMesh& m, cudaStream_t st);
struct ImageBlocks;
// With img (every order, 0 included): the image blocks of m's collocation
// points against the mirrored cell img->source (nodes R Y in their order).
fmpb_status build_blocks_q9p(const DeviceMesh& m, const CellGrid& g, double k, cd beta, int n_off,
                             const int32_t* offsets, const int64_t* dest_host, cd* out, cudaStream_t st,
                             const ImageBlocks* img = nullptr);
// out[r][p] += the scattered pressure of the surface solution surf at the
// points (nine-node meshes of any pressure order; with pl.on also R_p times
// the part of the mirrored cell refl).
struct PlaneDev;
fmpb_status field_scattered_q9(const DeviceMesh& m, const DeviceMesh* refl, const PlaneDev& pl, const CellGrid& g,
                               double k, cd beta, int R, const cd* surf, int64_t npts, const double* pts, cd* out,
                               cudaStream_t st);
// build_blocks for a nine-node mesh (full space only).
fmpb_status build_blocks_q9(const DeviceMesh& m, const CellGrid& g, double k, cd beta, int n_off,
                            const int32_t* offsets, const int64_t* dest_host, cd* out, cudaStream_t st);
// Image blocks of a half-space operator (Sec. 2.3): per offset the shift of
// the reflected unit cell (3 doubles, host), the factor R_p, and whether the
// entries are added to out (the full-space blocks of the same pattern).
struct ImageBlocks {
  const DeviceMesh* source;   // the reflected unit cell (elements); targets stay in m
  const double* shifts;
  cd scale;
  bool accumulate;
};
// Builds n_off collocation blocks; block o is written at out + dest[o] * n * n.
// beta: uniform normalised admittance of the surface (0: rigid).  img: the
// image blocks of m's collocation points against the reflected cell (no self
// terms), else the full-space blocks at shifts -delta . lattice.
fmpb_status build_blocks(const DeviceMesh& m, const CellGrid& g, double k, cd beta, int n_off,
                         const int32_t* offsets, const int64_t* dest_host, cd* out, cudaStream_t st,
                         const ImageBlocks* img = nullptr);

// The truncation rule (truncation.cu): the smallest n_t in 4..MAX_NT whose
// U_0 K(d) V_0 reproduces the exact block of the nearest far cell d on four
// probe vectors to 1e-6 relative; met = false (nt = MAX_NT) when none does;
// err: the relative probe error at the chosen n_t.  Grids without far cell
// pairs take 4.
bool nearest_far_offset(const CellGrid& g, int32_t d[3]);
fmpb_status auto_truncation(const DeviceMesh& mesh, const CellGrid& g, double k, cd beta, int* nt, bool* met,
                            double* err, cudaStream_t st);

// Listed entries of n_off blocks (list: device, count indices
// (o n + i) n + j, o indexing offsets), written to out[e]; self_slot (device,
// n entries, -1 where absent): the position in out of entry (i, i) of the
// zero offset, filled with the singular self term.
fmpb_status build_entries(const DeviceMesh& m, const CellGrid& g, double k, cd beta, int n_off,
                          const int32_t* offsets, const int64_t* list, int64_t count, const int64_t* self_slot,
                          cd* out, cudaStream_t st);

// One incident field on the device (kind 0: plane wave, v = direction;
// kind 1: monopole, v = source position) and the symmetry plane of a
// half-space operator (on = 0: full space).
struct IncDev {
  int kind;
  double v[3];
  cd amp;
};
struct PlaneDev {
  int on;
  int axis;
  double offset;
  cd Rp;
};
fmpb_status rhs_incident(const DeviceMesh& m, const CellGrid& g, double k, int R, const fmpb_incident* inc,
                         const PlaneDev& pl, cd* b, cudaStream_t st);
fmpb_status field_incident(const DeviceMesh& m, const DeviceMesh* refl, const CellGrid& g, double k, cd beta,
                           const PlaneDev& pl, int R, const cd* surf, const fmpb_incident* inc, int64_t npts,
                           const double* pts, cd* out, cudaStream_t st);
// Eq. (insertionloss) over the points for the R solutions surf together.
fmpb_status insertion_loss(const DeviceMesh& m, const DeviceMesh* refl, const CellGrid& g, double k, cd beta,
                           const PlaneDev& pl, int R, const cd* surf, const fmpb_incident* inc, int64_t npts,
                           const double* pts, double* il, cudaStream_t st);

// P x: cells reversed along lattice axis h for every right-hand side (16- or
// 8-byte elements, n per cell); a * s in place.
fmpb_status reverse_cells(const void* in, void* out, size_t elem_bytes, int R, const int M[3], int n, int h,
                          cudaStream_t st);
fmpb_status scale_inplace(cd* a, size_t n, cd s, cudaStream_t st);

// Raises a kernel's dynamic shared-memory limit to `bytes` once per process
// (thread-safe; later calls return the first call's status).  Operators are
// built and applied from several host threads at once, so the limit is never
// changed while another thread may be launching the kernel.
// One instance (and one flag) per kernel: the kernel is a template argument.
template <auto Kernel>
inline cudaError_t smem_limit_once(int bytes) {
  static std::once_flag once;
  static cudaError_t status = cudaSuccess;
  std::call_once(once, [&] { status = cudaFuncSetAttribute(Kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes); });
  return status;
}

// Pruned DFT passes (dft.cu): storage formats of the values a pass reads and
// writes (complex double, float-float pairs, complex FP32).
enum DftFormat { DFT_CD = 0, DFT_FF = 1, DFT_F32 = 2, DFT_BF16R = 3 };
// DFT_BF16R (output only, FP32 passes): the values as the BF16 rows of the
// tensor-core products, value e = row B + b at pair b of row `row`
// (row_kh pairs per row; pairs b >= B are left untouched).
// True if an axis of padded length P splits into two factors of at most 16
// (every P up to 256 of the 2,3,5,7-smooth lengths the engine uses except a
// few, such as 245).
bool dft_supported(int P);
// One pass along an axis (see dft.cu): ff_arith selects float-float or FP32
// arithmetic; in place needs in == out with equal strides and Pin = Pout = P.
// Appends the DFT autotuner's choices as JSON objects (comma-separated) to out.
void dft_tuning_summary(std::string& out);
// Forces one plan kind of every DFT pass (0 direct, 1 two-factor, 2 radix-2)
// where the pass has it, or restores the autotuner (-1).
fmpb_status dft_force_plan(int kind);
fmpb_status dft_pass(const char* name, bool ff_arith, int in_fmt, int out_fmt, const void* in, void* out, int O1,
                     int O2, int64_t I, int64_t a1, int64_t a2, int64_t aj, int64_t b1, int64_t b2, int64_t bf,
                     int Pin, int Pout, int P, int sign, double scale, bool accumulate, cudaStream_t st,
                     int64_t row_b = 0, int row_kh = 0);
// True if an FP32 pass of length P with Pin inputs can write DFT_BF16R rows
// (the direct or the radix-2 form).
bool dft_rows_ok(int P, int Pin);

// Circulant engine (circulant.cu)
// In-place forward DFT over the padded grid of F slots, each holding `inner`
// complex doubles; leaves the result as float-float pairs (16 bytes each).
fmpb_status grid_fft_inplace(const CircShape& s, int64_t inner, cd* grid, cudaStream_t st);
// y (+)= T x through pruned FFT, block product, pruned inverse FFT.
// scratch: 2 * F * R * B complex values.
// Storage formats of a spectrum: complex double, float-float pairs (16 bytes,
// FP64-class accuracy) or complex FP32 (8 bytes, the low-precision half of the
// mixed-precision operator).
// SPEC_BF16: the spectrum as realified BF16 tiles (tc_realify_ff layout),
// applied on the tensor cores; needs tc_rows (F R tc_depth(B) BF16 values of
// scratch) and the error word tc_err of the tensor-core kernels.
enum SpecFormat { SPEC_CD = 0, SPEC_FF = 1, SPEC_F32 = 2, SPEC_BF16 = 3 };
fmpb_status circulant_apply(const CircShape& s, int64_t B, const cd* spec, int R, const cd* x, cd* y,
                            bool accumulate, cd* scratch, cudaStream_t st, int spec_format = SPEC_CD,
                            void* tc_rows = nullptr, unsigned* tc_err = nullptr, bool ff_io = false,
                            bool f32_passes = false, const void* const* spec_batch = nullptr, int n_ops = 1,
                            const int* batch_blk = nullptr, int n_blocks = 0, void* y_rows = nullptr);
// y_rows (FP32 passes, not accumulating): the result as the BF16 rows of a
// tensor-core product instead of y, row r Nc + c holding the B values of
// cell c of right-hand side r (tc_depth(B) / 2 pairs per row, the padding
// untouched); y is then not written.
// spec_batch: the products of several operators of one shape in one pass
// sequence (BF16 spectra only).  R counts the right-hand sides of n_blocks
// operator blocks (R / n_blocks each, block b's after those of b - 1); the
// per-frequency products run for the n_ops operators listed, operator q's
// spectrum spec_batch[q] acting on block batch_blk[q] (null: q; n_blocks 0:
// n_ops).  The DFT passes run over all blocks.
// ff_io: x and y are float-float vectors (float4 per value, passed as cd*;
// same 16 bytes) instead of complex double; accumulate must be false.
// f32_passes: the DFT passes and the frequency-domain values in complex FP32
// (8 bytes per value) instead of float-float; for the FP32 and BF16 spectra
// only (SPEC_F32, SPEC_BF16), and only where circulant_f32_ok(s) holds.
bool circulant_f32_ok(const CircShape& s);
// float-float spectrum -> complex FP32 (out has n float2 entries)
fmpb_status spectrum_ff_to_f32(const cd* in, void* out, size_t n, cudaStream_t st);
// In-place conversion of n complex doubles to float-float pairs (re_hi, re_lo, im_hi, im_lo).
fmpb_status spectrum_to_ff(cd* spec, size_t n, cudaStream_t st);
// Out-of-place conversion of n complex doubles to float-float pairs.
fmpb_status vector_to_ff(const cd* x, float4* y, size_t n, cudaStream_t st);
// Out-of-place rounding of n complex doubles to complex FP32.
fmpb_status vector_to_f32(const cd* x, float2* y, size_t n, cudaStream_t st);
size_t circulant_scratch_elems(const CircShape& s, int64_t B, int R);

}  // namespace fmpb
