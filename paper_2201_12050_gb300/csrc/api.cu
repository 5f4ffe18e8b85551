// C ABI of the library (include/fmpb.h): argument checking, the operator
// object and the composition of the kernels into the FMPBEM and PBEM
// products (Sec. 3.5, Eq. (FMPBEMsystem); Sec. 2.4).
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>

#include "common.cuh"
#include "internal.cuh"
#include "multipole.cuh"
#include "nearfield.cuh"
#include "gmres.cuh"
#include "tc_gemm.cuh"
#include "fmm2.cuh"

namespace fmpb {

static thread_local std::string g_error = "no error";

void set_error(const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_error = buf;
}

const char* take_failed_launch();

fmpb_status cuda_status(cudaError_t e, const char* what) {
  const char* k = take_failed_launch();
  if (k)
    set_error("CUDA error in %s: %s (refused launch of %s)", what, cudaGetErrorString(e), k);
  else
    set_error("CUDA error in %s: %s", what, cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? FMPB_ENOMEM : FMPB_ECUDA;
}

fmpb_status circulant_spectrum_from_blocks(const CircShape& s, int64_t B, const cd* blocks, cd* spec, cudaStream_t st);

static fmpb_status make_grid(const fmpb_lattice* lat, CellGrid& g) {
  if (!lat) {
    set_error("lattice is NULL");
    return FMPB_EINVAL;
  }
  int64_t nc = 1;
  for (int a = 0; a < 3; ++a) {
    if (lat->counts[a] < 1 || lat->counts[a] > 4096) {
      set_error("lattice count %d out of range 1..4096", lat->counts[a]);
      return FMPB_EINVAL;
    }
    g.M[a] = lat->counts[a];
    nc *= lat->counts[a];
    for (int d = 0; d < 3; ++d) {
      g.L[a][d] = lat->vectors[a][d];
      if (!std::isfinite(g.L[a][d])) {
        set_error("lattice vector is not finite");
        return FMPB_EINVAL;
      }
    }
  }
  if (nc > (1 << 24)) {
    set_error("too many cells (%lld)", (long long)nc);
    return FMPB_EINVAL;
  }
  g.ncells = (int)nc;
  return FMPB_OK;
}

template <typename T>
static fmpb_status dev_alloc(T** p, size_t count, size_t& bytes) {
  if (count > SIZE_MAX / sizeof(T)) {
    set_error("cannot allocate %zu elements of %zu bytes on the device", count, sizeof(T));
    return FMPB_ENOMEM;
  }
  cudaError_t e = cudaMalloc((void**)p, sizeof(T) * (count ? count : 1));
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_error("cannot allocate %zu bytes on the device", sizeof(T) * count);
    return FMPB_ENOMEM;
  }
  bytes += sizeof(T) * count;
  return FMPB_OK;
}

}  // namespace fmpb


namespace fmpb {

// Offsets of the (2M-1)^d block Toeplitz pattern (delta_x fastest) split into
// near (|delta|_inf <= 1) and far, and the form to build: AUTO picks FMM when
// the nearest far translation is at least 3 cell radii (two-centre expansion
// ratio 2 rho / |d| <= 2/3), else PBEM; FMM forced with |d| <= 2 rho is refused.
fmpb_status decide_form(const CellGrid& g, double rho, int requested, int* form, std::vector<int32_t>* all_off,
                        std::vector<int32_t>* near_off, std::vector<int32_t>* far_off) {
  double dmin = 1e300;
  for (int dz = 1 - g.M[2]; dz < g.M[2]; ++dz)
    for (int dy = 1 - g.M[1]; dy < g.M[1]; ++dy)
      for (int dx = 1 - g.M[0]; dx < g.M[0]; ++dx) {
        const int32_t dl[3] = {dx, dy, dz};
        const bool near = abs(dx) <= 1 && abs(dy) <= 1 && abs(dz) <= 1;
        if (all_off) all_off->insert(all_off->end(), dl, dl + 3);
        std::vector<int32_t>* dst = near ? near_off : far_off;
        if (dst) dst->insert(dst->end(), dl, dl + 3);
        if (!near) {
          double d2 = 0.0;
          for (int c = 0; c < 3; ++c) {
            const double v = dx * g.L[0][c] + dy * g.L[1][c] + dz * g.L[2][c];
            d2 += v * v;
          }
          dmin = fmin(dmin, sqrt(d2));
        }
      }
  int f = requested;
  if (f == FMPB_FORM_AUTO) f = (dmin >= 3.0 * rho) ? FMPB_FORM_FMM : FMPB_FORM_PBEM;
  if ((f == FMPB_FORM_FMM || f == FMPB_FORM_FMM2) && !(dmin > 2.0 * rho)) {
    set_error("operator_create: FMM form not admissible (nearest far cell at %.4g, cell radius %.4g)", dmin, rho);
    return FMPB_EADMISS;
  }
  *form = f;
  return FMPB_OK;
}

// Form, circulant block size and spectrum length, and the device bytes an
// operator will hold, computed on the host without building it (admission).
fmpb_status plan_operator(const double* verts, int64_t nv, const int32_t* tris, int64_t ntri,
                          const fmpb_lattice* lattice, const fmpb_operator_opts* opts, int* form, int64_t* B,
                          int64_t* F, size_t* bytes) {
  CellGrid g;
  FMPB_TRY(make_grid(lattice, g));
  double rho = 0.0;
  for (int64_t t = 0; t < 3 * ntri; ++t) {
    const int32_t v = tris[t];
    if (v < 0 || v >= nv) {
      set_error("plan: triangle index out of range");
      return FMPB_EMESH;
    }
    const double* p = verts + 3 * v;
    rho = fmax(rho, sqrt(p[0] * p[0] + p[1] * p[1] + p[2] * p[2]));
  }
  FMPB_TRY(decide_form(g, rho, opts->form, form, nullptr, nullptr, nullptr));
  const CircShape sh = make_shape(g.M);
  // the truncation rule (n_t = 0) needs device work; admission plans with
  // n_t = 12, above what the rule picks for the cells it was tried on (10-11)
  const int nt = opts->n_t > 0 ? opts->n_t : 12;
  const int64_t n = ntri;
  const int64_t b = *form == FMPB_FORM_PBEM ? n : (int64_t)(nt + 1) * (nt + 1);
  const int dim = (g.M[0] > 1) + (g.M[1] > 1) + (g.M[2] > 1);
  int nnear = 1;
  for (int i = 0; i < dim; ++i) nnear *= 3;
  size_t per = 16;   // float-float spectrum
  if (opts->precision == FMPB_FP32) per = 8;
  if (opts->precision == FMPB_MIXED && *form == FMPB_FORM_PBEM) per = 24;
  size_t total = per * (size_t)sh.F * b * b;
  // realified BF16 spectrum of BF16 operators and of MIXED operators in the FMM form
  const size_t spec_bf16 = 2 * (size_t)sh.F * tc_rows(b) * tc_depth(b);
  if (*form == FMPB_FORM_FMM && opts->precision == FMPB_BF16) total = spec_bf16;
  if (*form == FMPB_FORM_FMM && opts->precision == FMPB_MIXED) total += spec_bf16;
  const size_t tc_bytes = 2 * ((size_t)nnear * tc_rows(n) * tc_depth(n) + (size_t)tc_rows(b) * tc_depth(n) +
                               (size_t)tc_rows(n) * tc_depth(b));
  if (*form == FMPB_FORM_FMM && opts->precision == FMPB_BF16)
    total += tc_bytes;
  else if (*form == FMPB_FORM_FMM)
    total += 16 * ((size_t)nnear * n * n + 2 * (size_t)b * n) + (opts->precision == FMPB_MIXED ? tc_bytes : 0);
  *B = b;
  *F = sh.F;
  *bytes = total;
  return FMPB_OK;
}

}  // namespace fmpb

using namespace fmpb;

struct fmpb_operator {
  int device = 0;
  DeviceMesh mesh;
  CellGrid grid;
  CircShape shape;
  double k = 0.0;
  cd beta = {0.0, 0.0};     // uniform normalised admittance (0: rigid)
  int form = FMPB_FORM_PBEM;
  int nt = 0;
  double nt_rule_err = -1.0;   // relative probe error of the truncation rule's n_t (-1: n_t given)
  int64_t B = 0;
  int dim = 0;
  cd* spec = nullptr;      // F x B x B, float-float pairs (re_hi, re_lo, im_hi, im_lo) per entry
  void* spec32 = nullptr;  // F x B x B complex FP32 (FP32 operators, MIXED in the PBEM form)
  __nv_bfloat16* specb = nullptr;  // F x tc_rows(B) x tc_depth(B) realified BF16 (BF16, MIXED FMM)
  int precision = FMPB_FP64;
  cd* S = nullptr;         // n_near x n x n (FMM form), float-float pairs
  int* near_offs = nullptr;
  int n_near = 0;
  cd* V0 = nullptr;        // B x n, float-float pairs
  cd* U0 = nullptr;        // n x B, float-float pairs
  // BF16 operators: S, V_0, U_0 as realified BF16 tiles for the tensor cores
  __nv_bfloat16* Sb = nullptr;    // n_near x tc_rows(n) x tc_depth(n)
  __nv_bfloat16* V0b = nullptr;   // tc_rows(B) x tc_depth(n)
  __nv_bfloat16* U0b = nullptr;   // tc_rows(n) x tc_depth(B)
  TcOffsets near_tc{};
  unsigned* tc_err = nullptr;     // set by a tensor-core kernel whose wait gave up
  // half-space image part (Sec. 2.3, Sec. 3.4)
  PlaneDev plane{0, 0, 0.0, {0.0, 0.0}};
  int hankel = -1;                // lattice axis perpendicular to the plane
  bool img_sep = false;           // image part with its own tables and products
  DeviceMesh refl;                // reflected unit cell (R v, reversed winding)
  cd* spec_img = nullptr;         // image spectrum (PBEM blocks or FMM M2L), float-float
  void* spec32_img = nullptr;     // the same in complex FP32
  cd* S_img = nullptr;            // n_near_img x n x n image near blocks (FMM)
  int* near_offs_img = nullptr;
  int n_near_img = 0;
  cd* V0_img = nullptr;           // R_p x P2M table of the reflected cell (FMM)
  Near2* near2 = nullptr;         // multilevel near field (FMPBEM2 form)
  size_t bytes = 0;
  // scratch, grown on demand (calls on one operator are stream-ordered)
  cd* scratch = nullptr;
  size_t scratch_elems = 0;

  ~fmpb_operator() {
    cudaDeviceSynchronize();
    free_mesh(mesh);
    cudaFree(spec);
    cudaFree(spec32);
    cudaFree(specb);
    cudaFree(S);
    cudaFree(near_offs);
    cudaFree(V0);
    cudaFree(U0);
    cudaFree(Sb);
    cudaFree(V0b);
    cudaFree(U0b);
    cudaFree(tc_err);
    cudaFree(scratch);
    free_mesh(refl);
    cudaFree(spec_img);
    cudaFree(spec32_img);
    cudaFree(S_img);
    cudaFree(near_offs_img);
    cudaFree(V0_img);
    delete near2;
  }

  fmpb_status ensure_scratch(size_t elems) {
    if (elems <= scratch_elems) return FMPB_OK;
    cudaFree(scratch);
    scratch = nullptr;
    scratch_elems = 0;
    size_t dummy = 0;
    FMPB_TRY(dev_alloc(&scratch, elems, dummy));
    scratch_elems = elems;
    return FMPB_OK;
  }

  // The PBEM-form product of an FP64 operator on float-float vectors.
  bool has_ff_matvec() const { return form == FMPB_FORM_PBEM && spec != nullptr && !img_sep; }
  fmpb_status matvec_ff(int R, const float4* x, float4* y, cudaStream_t st) {
    FMPB_TRY(ensure_scratch(circulant_scratch_elems(shape, B, R)));
    return circulant_apply(shape, B, spec, R, reinterpret_cast<const cd*>(x), reinterpret_cast<cd*>(y), false,
                           scratch, st, SPEC_FF, nullptr, nullptr, true);
  }

  // The BF16 tensor-core product of the FMM form (BF16 operators and the
  // inner products of MIXED FMM operators) on complex double (x_f32, y_f32
  // false) or complex FP32 vectors: P2M, M2L through the circulant engine,
  // then the near field with the L2P term as the tail of the same
  // tensor-core accumulation, y = sum S_d x + U_0 L.
  bool has_tc_matvec() const { return form == FMPB_FORM_FMM && !near2 && Sb != nullptr; }
  fmpb_status matvec_tc(int R, const void* x, bool x_f32, void* y, bool y_f32, cudaStream_t st) {
    const int64_t Nc = shape.ncells;
    const int n = mesh.n;
    const size_t circ = circulant_scratch_elems(shape, B, R);
    const size_t mom = (size_t)R * Nc * B;
    const size_t xb_elems = (size_t)R * Nc * tc_depth(n), lb_elems = (size_t)R * Nc * tc_depth(B);
    const size_t fb_elems = (size_t)shape.F * R * tc_depth(B);
    const size_t extra = (2 * (xb_elems + lb_elems + fb_elems) + sizeof(cd) - 1) / sizeof(cd);
    FMPB_TRY(ensure_scratch(circ + 2 * mom + extra));
    cd* Mom = scratch + circ;
    cd* Loc = Mom + mom;
    __nv_bfloat16* xb = reinterpret_cast<__nv_bfloat16*>(Loc + mom);
    __nv_bfloat16* lb = xb + xb_elems;
    __nv_bfloat16* fb = lb + lb_elems;
    TcOffsets zero{};
    zero.n = 1;
    if (x_f32)
      FMPB_TRY(tc_rows_from_f32(reinterpret_cast<const float2*>(x), (int64_t)R * Nc, n, xb, st));
    else
      FMPB_TRY(tc_rows_to_bf16(reinterpret_cast<const cd*>(x), (int64_t)R * Nc, n, xb, st));
    FMPB_TRY(tc_offset_gemm(V0b, zero, B, n, shape.M, R, xb, Mom, false, tc_err, st));
    // local expansions straight into the BF16 rows of the L2P tail where the
    // FP32 passes can write them
    const bool p32 = circulant_f32_ok(shape);
    const bool lrows = p32 && dft_rows_ok(shape.P[0], shape.P[0]);
    FMPB_TRY(circulant_apply(shape, B, reinterpret_cast<const cd*>(specb), R, Mom, Loc, false, scratch, st,
                             SPEC_BF16, fb, tc_err, false, p32, nullptr, 1, nullptr, 0, lrows ? lb : nullptr));
    if (!lrows) FMPB_TRY(tc_rows_to_bf16(Loc, (int64_t)R * Nc, B, lb, st));
    const __nv_bfloat16* sb1[1] = {Sb};
    const __nv_bfloat16* ub1[1] = {U0b};
    return tc_offset_gemm_batch(sb1, 1, near_tc, n, n, shape.M, R, xb, y, false, tc_err, st, nullptr, ub1, B, lb,
                                y_f32);
  }

  // low: the inner product of a MIXED operator (PBEM form: the FP32 spectrum;
  // FMM form: the BF16 tensor-core path of BF16 operators)
  fmpb_status matvec(int R, const cd* x, cd* y, cudaStream_t st, bool low = false) {
    const int64_t Nc = shape.ncells;
    const bool f32 = precision == FMPB_FP32 || (precision == FMPB_MIXED && low);
    const cd* sp = f32 ? reinterpret_cast<const cd*>(spec32) : spec;
    const int fmt = f32 ? SPEC_F32 : SPEC_FF;
    // low-precision spectra take FP32 DFT passes (8-byte frequency values)
    const bool p32 = f32 && circulant_f32_ok(shape);
    if (form == FMPB_FORM_PBEM) {
      const size_t circ = circulant_scratch_elems(shape, B, R);
      FMPB_TRY(ensure_scratch(circ + (img_sep ? (size_t)R * Nc * B : 0)));
      FMPB_TRY(circulant_apply(shape, B, sp, R, x, y, false, scratch, st, fmt, nullptr, nullptr, false, p32));
      if (img_sep) {
        // the block Hankel image part: (T^ P)(P x) (Sec. 2.4)
        cd* q = scratch + circ;
        FMPB_TRY(reverse_cells(x, q, sizeof(cd), R, shape.M, mesh.n, hankel, st));
        const cd* spi = f32 ? reinterpret_cast<const cd*>(spec32_img) : spec_img;
        FMPB_TRY(circulant_apply(shape, B, spi, R, q, y, true, scratch, st, fmt, nullptr, nullptr, false, p32));
      }
      return FMPB_OK;
    }
    const size_t circ = circulant_scratch_elems(shape, B, R);
    const size_t mom = (size_t)R * Nc * B;
    const size_t nvec = (size_t)R * Nc * mesh.n;
    if (near2) {
      // FMPBEM2: the multilevel near field in FP64, then the cell-level far field
      const size_t n2 = near2_scratch_elems(*near2, (int64_t)R * Nc);
      FMPB_TRY(ensure_scratch(circ + 2 * mom + nvec + n2));
      cd* Mom2 = scratch + circ;
      cd* Loc2 = Mom2 + mom;
      float4* xf2 = reinterpret_cast<float4*>(Loc2 + mom);
      FMPB_TRY(vector_to_ff(x, xf2, nvec, st));
      FMPB_TRY(near2_apply(*near2, shape.M, R, x, xf2, y, reinterpret_cast<cd*>(xf2 + nvec), st));
      FMPB_TRY(p2m_apply(reinterpret_cast<const float4*>(V0), mesh.n, (int)B, (int64_t)R * Nc, xf2, Mom2, st));
      FMPB_TRY(circulant_apply(shape, B, spec, R, Mom2, Loc2, false, scratch, st, SPEC_FF));
      FMPB_TRY(l2p_apply(reinterpret_cast<const float4*>(U0), mesh.n, (int)B, (int64_t)R * Nc, Loc2, y, st));
      return FMPB_OK;
    }
    FMPB_TRY(ensure_scratch(circ + 2 * mom + (img_sep ? 2 : 1) * nvec));
    cd* Mom = scratch + circ;
    cd* Loc = Mom + mom;
    float4* xff = reinterpret_cast<float4*>(Loc + mom);
    if (precision == FMPB_BF16 || (precision == FMPB_MIXED && low)) return matvec_tc(R, x, false, y, false, st);
    // the image part of a half-space operator (Eq. (2dPeriodicFMM_halfspace)):
    // near blocks S^ and P2M table V^ of the mirrored cell act on q = P x, its
    // M2L spectrum adds to the same local expansions (U^ = U)
    const cd* spi = f32 ? reinterpret_cast<const cd*>(spec32_img) : spec_img;
    if (precision == FMPB_FP32) {
      float2* x32 = reinterpret_cast<float2*>(Loc + mom);
      FMPB_TRY(vector_to_f32(x, x32, nvec, st));
      FMPB_TRY(near_apply_f32(reinterpret_cast<const float2*>(S), near_offs, n_near, mesh.n, shape.M, R, x32, y, false,
                              st));
      FMPB_TRY(p2m_apply_f32(reinterpret_cast<const float2*>(V0), mesh.n, (int)B, (int64_t)R * Nc, x32, Mom, st));
      FMPB_TRY(circulant_apply(shape, B, sp, R, Mom, Loc, false, scratch, st, fmt, nullptr, nullptr, false, p32));
      if (img_sep) {
        float2* q32 = x32;
        if (hankel >= 0) {
          q32 = x32 + nvec;
          FMPB_TRY(reverse_cells(x32, q32, sizeof(float2), R, shape.M, mesh.n, hankel, st));
        }
        FMPB_TRY(near_apply_f32(reinterpret_cast<const float2*>(S_img), near_offs_img, n_near_img, mesh.n, shape.M, R,
                                q32, y, true, st));
        FMPB_TRY(p2m_apply_f32(reinterpret_cast<const float2*>(V0_img), mesh.n, (int)B, (int64_t)R * Nc, q32, Mom, st));
        FMPB_TRY(circulant_apply(shape, B, spi, R, Mom, Loc, true, scratch, st, fmt, nullptr, nullptr, false, p32));
      }
      FMPB_TRY(l2p_apply_f32(reinterpret_cast<const float2*>(U0), mesh.n, (int)B, (int64_t)R * Nc, Loc, y, st));
      return FMPB_OK;
    }
    FMPB_TRY(vector_to_ff(x, xff, nvec, st));
    FMPB_TRY(near_apply(reinterpret_cast<const float4*>(S), near_offs, n_near, mesh.n, shape.M, R, xff, y, false, st));
    FMPB_TRY(p2m_apply(reinterpret_cast<const float4*>(V0), mesh.n, (int)B, (int64_t)R * Nc, xff, Mom, st));
    FMPB_TRY(circulant_apply(shape, B, sp, R, Mom, Loc, false, scratch, st, fmt));
    if (img_sep) {
      float4* qff = xff;
      if (hankel >= 0) {
        qff = xff + nvec;
        FMPB_TRY(reverse_cells(xff, qff, sizeof(float4), R, shape.M, mesh.n, hankel, st));
      }
      FMPB_TRY(near_apply(reinterpret_cast<const float4*>(S_img), near_offs_img, n_near_img, mesh.n, shape.M, R, qff, y,
                          true, st));
      FMPB_TRY(p2m_apply(reinterpret_cast<const float4*>(V0_img), mesh.n, (int)B, (int64_t)R * Nc, qff, Mom, st));
      FMPB_TRY(circulant_apply(shape, B, spi, R, Mom, Loc, true, scratch, st, fmt));
    }
    FMPB_TRY(l2p_apply(reinterpret_cast<const float4*>(U0), mesh.n, (int)B, (int64_t)R * Nc, Loc, y, st));
    return FMPB_OK;
  }
};

#define CHECK_ARG(cond, ...)      \
  do {                            \
    if (!(cond)) {                \
      set_error(__VA_ARGS__);     \
      return FMPB_EINVAL;         \
    }                             \
  } while (0)

namespace fmpb {

// Half-space set-up (Sec. 2.3): checks the plane and the role of every
// lattice axis (parallel to the plane, or perpendicular to it: at most one),
// checks that every cell lies on one side of the plane, and uploads the
// reflected unit cell (R v, reversed winding, so that its element normals are
// R n and the quadrature rules apply unchanged).
// npe: nodes per element (3: triangles, the centroid; 9: nine-node
// quadrilaterals, the centre node 4).
static fmpb_status halfspace_check(const CellGrid& g, const fmpb_operator_opts& o, const double* verts, int64_t nv,
                                   const int32_t* tris, int64_t ntri, int* hankel, int npe = 3) {
  const int ax = o.plane_axis;
  if (ax < 0 || ax > 2 || !std::isfinite(o.plane_offset) || !std::isfinite(o.Rp_re) || !std::isfinite(o.Rp_im)) {
    set_error("operator_create: half-space needs plane_axis 0..2 and finite plane_offset, R_p");
    return FMPB_EINVAL;
  }
  int h = -1;
  for (int a = 0; a < 3; ++a) {
    if (g.M[a] <= 1) continue;
    const double n = sqrt(g.L[a][0] * g.L[a][0] + g.L[a][1] * g.L[a][1] + g.L[a][2] * g.L[a][2]);
    const double along = fabs(g.L[a][ax]);
    if (along <= 1e-12 * n) continue;
    if (fabs(along - n) <= 1e-12 * n && h < 0) {
      h = a;
      continue;
    }
    set_error("operator_create: lattice vector %d is neither parallel nor perpendicular to the plane "
              "(or a second perpendicular axis)", a);
    return FMPB_EINVAL;
  }
  // extent of the cells' positions along the plane normal (corners of the grid)
  double pmin = 1e300, pmax = -1e300;
  for (int corner = 0; corner < 8; ++corner) {
    double p = 0.0;
    for (int a = 0; a < 3; ++a) p += ((corner >> a) & 1) * (g.M[a] - 1) * g.L[a][ax];
    pmin = fmin(pmin, p);
    pmax = fmax(pmax, p);
  }
  double vmin = 1e300, vmax = -1e300, cmin = 1e300, cmax = -1e300, scale = fabs(o.plane_offset);
  for (int64_t v = 0; v < nv; ++v) {
    vmin = fmin(vmin, verts[3 * v + ax]);
    vmax = fmax(vmax, verts[3 * v + ax]);
    scale = fmax(scale, fabs(verts[3 * v + ax]));
  }
  for (int64_t t = 0; t < ntri; ++t) {
    const double c = npe == 9 ? verts[3 * (int64_t)tris[9 * t + 4] + ax]
                              : (verts[3 * (int64_t)tris[3 * t] + ax] + verts[3 * (int64_t)tris[3 * t + 1] + ax] +
                                 verts[3 * (int64_t)tris[3 * t + 2] + ax]) / 3.0;
    cmin = fmin(cmin, c);
    cmax = fmax(cmax, c);
  }
  scale = fmax(scale, fmax(fabs(pmin), fabs(pmax)));
  const double tol = 1e-12 * scale;
  const bool above = vmin + pmin - o.plane_offset >= -tol && cmin + pmin - o.plane_offset > tol;
  const bool below = vmax + pmax - o.plane_offset <= tol && cmax + pmax - o.plane_offset < -tol;
  if (!above && !below) {
    set_error("operator_create: the cells do not lie on one side of the plane x[%d] = %.6g", ax, o.plane_offset);
    return FMPB_EMESH;
  }
  *hankel = h;
  return FMPB_OK;
}

static fmpb_status setup_halfspace(fmpb_operator* op, const fmpb_operator_opts& o, const double* verts, int64_t nv,
                                   const int32_t* tris, int64_t ntri, cudaStream_t st) {
  int h = -1;
  const bool quad9 = o.element == FMPB_ELEM_QUAD9;
  FMPB_TRY(halfspace_check(op->grid, o, verts, nv, tris, ntri, &h, quad9 ? 9 : 3));
  const int ax = o.plane_axis;
  std::vector<double> rv(verts, verts + 3 * nv);
  for (int64_t v = 0; v < nv; ++v) rv[3 * v + ax] = -rv[3 * v + ax];
  if (quad9) {
    // nine-node cells keep their node order (the shapes keep their
    // parameters); the image kernels change the sign of D and H instead
    FMPB_TRY(upload_mesh_q9p(rv.data(), nv, tris, ntri, o.pressure_order, op->refl, st));
    op->plane = PlaneDev{1, ax, o.plane_offset, mkc(o.Rp_re, o.Rp_im)};
    op->hankel = h;
    return FMPB_OK;
  }
  std::vector<int32_t> rt(3 * ntri);
  for (int64_t t = 0; t < ntri; ++t) {
    rt[3 * t] = tris[3 * t];
    rt[3 * t + 1] = tris[3 * t + 2];
    rt[3 * t + 2] = tris[3 * t + 1];
  }
  FMPB_TRY(upload_mesh(rv.data(), nv, rt.data(), ntri, op->refl, st));
  op->plane = PlaneDev{1, ax, o.plane_offset, mkc(o.Rp_re, o.Rp_im)};
  op->hankel = h;
  return FMPB_OK;
}

// shift(delta~) = -delta~ . L - (M_h - 1) L_h + 2 offset e: where the
// reflected unit cell sits for the image block delta~ (x_c - y^_c = -shift).
static std::vector<double> image_shifts(const CellGrid& g, int hankel, int axis, double offset,
                                        const std::vector<int32_t>& offs) {
  const size_t n = offs.size() / 3;
  std::vector<double> sh(3 * n);
  for (size_t o = 0; o < n; ++o)
    for (int d = 0; d < 3; ++d) {
      double v = 0.0;
      for (int a = 0; a < 3; ++a) v -= offs[3 * o + a] * g.L[a][d];
      if (hankel >= 0) v -= (g.M[hankel] - 1) * g.L[hankel][d];
      if (d == axis) v += 2.0 * offset;
      sh[3 * o + d] = v;
    }
  return sh;
}
static std::vector<double> image_shifts(const fmpb_operator* op, const std::vector<int32_t>& offs) {
  return image_shifts(op->grid, op->hankel, op->plane.axis, op->plane.offset, offs);
}

// r of the mirrored admissibility criterion: the longest lattice vector
// among the axes with more than one cell.
static double image_r(const CellGrid& g) {
  double r = 0.0, rall = 0.0;
  for (int a = 0; a < 3; ++a) {
    const double n = sqrt(g.L[a][0] * g.L[a][0] + g.L[a][1] * g.L[a][1] + g.L[a][2] * g.L[a][2]);
    rall = fmax(rall, n);
    if (g.M[a] > 1) r = fmax(r, n);
  }
  return r > 0.0 ? r : rall;
}

}  // namespace fmpb

extern "C" {

const char* fmpb_last_error(void) { return g_error.c_str(); }

int fmpb_version(void) { return (FMPB_VERSION_MAJOR << 16) | FMPB_VERSION_MINOR; }

fmpb_status fmpb_circulant_shape(const int32_t counts[3], int32_t P[3], int64_t* F) {
  CHECK_ARG(counts && P && F, "circulant_shape: NULL argument");
  int M[3];
  for (int a = 0; a < 3; ++a) {
    CHECK_ARG(counts[a] >= 1 && counts[a] <= 4096, "circulant_shape: count out of range");
    M[a] = counts[a];
  }
  CircShape s = make_shape(M);
  for (int a = 0; a < 3; ++a) P[a] = s.P[a];
  *F = s.F;
  return FMPB_OK;
}

fmpb_status fmpb_operator_create(const double* verts, int64_t nv, const int32_t* tris, int64_t ntri,
                                 const fmpb_lattice* lattice, double k, const fmpb_operator_opts* opts, void* stream,
                                 fmpb_operator** out) {
  CHECK_ARG(out, "operator_create: out is NULL");
  CHECK_ARG(k > 0.0 && std::isfinite(k), "operator_create: wavenumber must be positive");
  fmpb_operator_opts o = opts ? *opts : fmpb_operator_opts{FMPB_FORM_AUTO, 0, FMPB_FP64};
  CHECK_ARG(o.form >= -1 && o.form <= 2, "operator_create: bad form %d", o.form);
  CHECK_ARG(o.form != FMPB_FORM_FMM2 || (o.precision == FMPB_FP64 && !o.halfspace),
            "operator_create: the FMPBEM2 form runs FMPB_FP64 in full space");
  CHECK_ARG(o.n_t_near >= 0 && o.n_t_near <= MAX_NT && o.near_levels >= 0 && o.near_levels <= 10,
            "operator_create: n_t_near must be 0..%d and near_levels 0..10", MAX_NT);
  CHECK_ARG(o.precision == FMPB_FP64 || o.precision == FMPB_FP32 || o.precision == FMPB_BF16 ||
                o.precision == FMPB_MIXED,
            "operator_create: precision must be FMPB_FP64, FMPB_FP32, FMPB_BF16 or FMPB_MIXED");
  CHECK_ARG(o.n_t >= 0 && o.n_t <= MAX_NT, "operator_create: n_t must be 0 (the truncation rule) or 1..%d", MAX_NT);
  int nt = o.n_t;
  CHECK_ARG(std::isfinite(o.beta_re) && std::isfinite(o.beta_im), "operator_create: admittance must be finite");
  CHECK_ARG(o.element == FMPB_ELEM_TRI3 || o.element == FMPB_ELEM_QUAD9,
            "operator_create: element must be FMPB_ELEM_TRI3 or FMPB_ELEM_QUAD9");
  const bool quad9 = o.element == FMPB_ELEM_QUAD9;
  CHECK_ARG(o.pressure_order == 0 || (quad9 && (o.pressure_order == 1 || o.pressure_order == 2)),
            "operator_create: pressure of order 1 or 2 takes FMPB_ELEM_QUAD9 elements");
  CHECK_ARG(!quad9 || ((o.form != FMPB_FORM_FMM2 || o.pressure_order == 0) && o.precision != FMPB_BF16 &&
                       !(o.form == FMPB_FORM_FMM && o.precision == FMPB_MIXED)),
            "operator_create: nine-node quadrilaterals run the PBEM form (FP64, FP32 or MIXED), the FMM form "
            "(FP64 or FP32) or, with constant pressure, the FMPBEM2 form");
  const cd beta = mkc(o.beta_re, o.beta_im);
  cudaStream_t st = (cudaStream_t)stream;
  fmpb_operator* op = new (std::nothrow) fmpb_operator();
  if (!op) {
    set_error("operator_create: host allocation failed");
    return FMPB_ENOMEM;
  }
  auto fail = [&](fmpb_status s) {
    delete op;
    return s;
  };
  cudaGetDevice(&op->device);
  op->k = k;
  op->beta = beta;
  fmpb_status s = make_grid(lattice, op->grid);
  if (s != FMPB_OK) return fail(s);
  s = quad9 ? upload_mesh_q9p(verts, nv, tris, ntri, o.pressure_order, op->mesh, st)
            : upload_mesh(verts, nv, tris, ntri, op->mesh, st);
  if (s != FMPB_OK) return fail(s);
  op->shape = make_shape(op->grid.M);
  const CircShape& sh = op->shape;
  op->dim = (sh.M[0] > 1) + (sh.M[1] > 1) + (sh.M[2] > 1);
  const int n = op->mesh.n;
  std::vector<int32_t> all_off, far_off, near_off;
  int form = 0;
  s = decide_form(op->grid, op->mesh.radius, quad9 && o.form == FMPB_FORM_AUTO ? FMPB_FORM_PBEM : o.form, &form,
                  &all_off, &near_off, &far_off);
  if (s != FMPB_OK) return fail(s);
  if (form == FMPB_FORM_PBEM && o.precision == FMPB_BF16) {
    set_error("operator_create: BF16 runs the near-field, P2M and L2P products of the FMM form on the tensor cores; "
              "this lattice needs the PBEM form, which has none (use FMPB_FP32 or FMPB_MIXED)");
    return fail(FMPB_EINVAL);
  }
  // half-space: the image offsets delta~ over the same pattern; in the FMM
  // form those whose mirrored cell is within 2 r (Eq. (admissibilityMirror))
  // are near, the others must admit the expansion about the mirrored centre
  std::vector<int32_t> near_img, far_img;
  std::vector<double> far_img_t;
  if (o.halfspace) {
    s = setup_halfspace(op, o, verts, nv, tris, ntri, st);
    if (s != FMPB_OK) return fail(s);
    const std::vector<double> shifts = image_shifts(op, all_off);
    const double r2 = 2.0 * image_r(op->grid) * (1.0 - 1e-9);
    double dmin_img = 1e300;
    for (size_t i = 0; i < all_off.size() / 3; ++i) {
      const double* t = &shifts[3 * i];
      const double d = sqrt(t[0] * t[0] + t[1] * t[1] + t[2] * t[2]);
      std::vector<int32_t>& dst = d < r2 ? near_img : far_img;
      dst.insert(dst.end(), &all_off[3 * i], &all_off[3 * i] + 3);
      if (d >= r2) {
        for (int c = 0; c < 3; ++c) far_img_t.push_back(-t[c]);
        dmin_img = fmin(dmin_img, d);
      }
    }
    const double rho = op->mesh.radius;
    if (o.form == FMPB_FORM_AUTO && form == FMPB_FORM_FMM && !(dmin_img >= 3.0 * rho)) form = FMPB_FORM_PBEM;
    if (o.form == FMPB_FORM_FMM && !(dmin_img > 2.0 * rho)) {
      set_error("operator_create: FMM form not admissible for the mirrored cells (nearest far image at %.4g, "
                "cell radius %.4g)", dmin_img, rho);
      return fail(FMPB_EADMISS);
    }
    if (o.precision == FMPB_BF16 || (o.precision == FMPB_MIXED && form == FMPB_FORM_FMM)) {
      set_error("operator_create: half-space operators run FMPB_FP64, FMPB_FP32 or (PBEM form) FMPB_MIXED");
      return fail(FMPB_EINVAL);
    }
    op->img_sep = form == FMPB_FORM_FMM || op->hankel >= 0;
  }
  // n_t = 0: the truncation rule on the cell itself; an AUTO form whose far
  // blocks no n_t up to MAX_NT reproduces to the rule's tolerance falls back
  // to the exact PBEM form
  if (form != FMPB_FORM_PBEM && nt == 0) {
    bool met = false;
    double terr = 0.0;
    s = auto_truncation(op->mesh, op->grid, k, beta, &nt, &met, &terr, st);
    if (s != FMPB_OK) return fail(s);
    op->nt_rule_err = terr;
    if (!met && o.form == FMPB_FORM_AUTO) {
      form = FMPB_FORM_PBEM;
      nt = 0;
      if (op->plane.on) op->img_sep = op->hankel >= 0;
    }
  }
  op->form = form;
  if (form == FMPB_FORM_PBEM) {
    op->B = n;
    const size_t elems = (size_t)sh.F * n * n;
    s = dev_alloc(&op->spec, elems, op->bytes);
    if (s != FMPB_OK) return fail(s);
    if (cudaMemsetAsync(op->spec, 0, sizeof(cd) * elems, st) != cudaSuccess) return fail(cuda_status(cudaGetLastError(), "memset"));
    const int n_off = (int)(all_off.size() / 3);
    std::vector<int64_t> dest(n_off);
    for (int i = 0; i < n_off; ++i) dest[i] = offset_slot(sh, all_off[3 * i], all_off[3 * i + 1], all_off[3 * i + 2]);
    s = build_blocks(op->mesh, op->grid, k, beta, n_off, all_off.data(), dest.data(), op->spec, st);
    if (s != FMPB_OK) return fail(s);
    if (op->plane.on) {
      // image blocks R_p T^(delta~): added to the same pattern when the
      // lattice is parallel to the plane, else a second (block Hankel) spectrum
      const std::vector<double> shifts = image_shifts(op, all_off);
      cd* dst = op->spec;
      if (op->img_sep) {
        s = dev_alloc(&op->spec_img, elems, op->bytes);
        if (s != FMPB_OK) return fail(s);
        if (cudaMemsetAsync(op->spec_img, 0, sizeof(cd) * elems, st) != cudaSuccess)
          return fail(cuda_status(cudaGetLastError(), "memset"));
        dst = op->spec_img;
      }
      const ImageBlocks ib{&op->refl, shifts.data(), op->plane.Rp, !op->img_sep};
      s = build_blocks(op->mesh, op->grid, k, beta, n_off, all_off.data(), dest.data(), dst, st, &ib);
      if (s == FMPB_OK && op->img_sep) s = grid_fft_inplace(sh, (int64_t)n * n, op->spec_img, st);
      if (s != FMPB_OK) return fail(s);
    }
    s = grid_fft_inplace(sh, (int64_t)n * n, op->spec, st);   // leaves float-float pairs
    if (s != FMPB_OK) return fail(s);
  } else {
    op->nt = nt;
    op->B = (int64_t)(nt + 1) * (nt + 1);
    const int64_t B = op->B;
    op->n_near = form == FMPB_FORM_FMM2 ? 0 : (int)(near_off.size() / 3);
    s = dev_alloc(&op->S, (size_t)op->n_near * n * n, op->bytes);
    if (s == FMPB_OK) s = dev_alloc(&op->near_offs, near_off.size(), op->bytes);
    if (s == FMPB_OK) s = dev_alloc(&op->V0, (size_t)B * n, op->bytes);
    if (s == FMPB_OK) s = dev_alloc(&op->U0, (size_t)B * n, op->bytes);
    if (s == FMPB_OK) s = dev_alloc(&op->spec, (size_t)sh.F * B * B, op->bytes);
    if (s != FMPB_OK) return fail(s);
    if (cudaMemcpyAsync(op->near_offs, near_off.data(), sizeof(int) * near_off.size(), cudaMemcpyHostToDevice, st) !=
            cudaSuccess ||
        cudaMemsetAsync(op->spec, 0, sizeof(cd) * (size_t)sh.F * B * B, st) != cudaSuccess)
      return fail(cuda_status(cudaGetLastError(), "operator_create copies"));
    std::vector<int64_t> dnear(op->n_near);
    for (int i = 0; i < op->n_near; ++i) dnear[i] = i;
    if (form == FMPB_FORM_FMM2) {
      // FMPBEM2 (Sec. 3.3): the near blocks as a multilevel FMM over the cell's octree
      op->near2 = new (std::nothrow) Near2();
      if (!op->near2) return fail(FMPB_ENOMEM);
      s = near2_build(op->mesh, op->grid, verts, tris, k, beta, o.near_levels, o.n_t_near > 0 ? o.n_t_near : 6,
                      near_off, *op->near2, st);
      op->bytes += op->near2->bytes;
    } else {
      s = build_blocks(op->mesh, op->grid, k, beta, op->n_near, near_off.data(), dnear.data(), op->S, st);
    }
    if (s == FMPB_OK) s = multipole_tables(op->mesh, k, beta, nt, op->V0, op->U0, st);
    // the products read the near blocks and the P2M/L2P tables as float-float
    // pairs, or as complex FP32 for FP32 operators (8 bytes per entry)
    if (o.precision == FMPB_BF16 || o.precision == FMPB_MIXED) {
      if (s == FMPB_OK) s = dev_alloc(&op->Sb, (size_t)op->n_near * tc_rows(n) * tc_depth(n), op->bytes);
      if (s == FMPB_OK) s = dev_alloc(&op->V0b, (size_t)tc_rows(B) * tc_depth(n), op->bytes);
      if (s == FMPB_OK) s = dev_alloc(&op->U0b, (size_t)tc_rows(n) * tc_depth(B), op->bytes);
      if (s == FMPB_OK) s = dev_alloc(&op->tc_err, 1, op->bytes);
      if (s == FMPB_OK && cudaMemsetAsync(op->tc_err, 0, sizeof(unsigned), st) != cudaSuccess)
        s = cuda_status(cudaGetLastError(), "memset");
      if (s == FMPB_OK) s = tc_realify(op->S, op->n_near, n, n, op->Sb, st);
      if (s == FMPB_OK) s = tc_realify(op->V0, 1, B, n, op->V0b, st);
      if (s == FMPB_OK) s = tc_realify(op->U0, 1, n, B, op->U0b, st);
      if (s == FMPB_OK && cudaStreamSynchronize(st) != cudaSuccess) s = cuda_status(cudaGetLastError(), "tables");
      if (s == FMPB_OK) {
        op->near_tc.n = op->n_near;
        for (int i = 0; i < op->n_near; ++i)
          for (int c = 0; c < 3; ++c) op->near_tc.d[i][c] = near_off[3 * i + c];
      }
    }
    if (o.precision == FMPB_BF16) {
      if (s == FMPB_OK) {
        for (cd** t : {&op->S, &op->V0, &op->U0}) {
          cudaFree(*t);
          *t = nullptr;
        }
        op->bytes -= sizeof(cd) * ((size_t)op->n_near * n * n + 2 * (size_t)B * n);
      }
    } else if (o.precision == FMPB_FP32) {
      for (cd** t : {&op->S, &op->V0, &op->U0}) {
        const size_t ne = (t == &op->S) ? (size_t)op->n_near * n * n : (size_t)B * n;
        float2* f32 = nullptr;
        if (s == FMPB_OK) s = dev_alloc(&f32, ne, op->bytes);
        if (s == FMPB_OK) s = vector_to_f32(*t, f32, ne, st);
        if (s == FMPB_OK && cudaStreamSynchronize(st) != cudaSuccess) s = cuda_status(cudaGetLastError(), "tables");
        if (s == FMPB_OK) {
          cudaFree(*t);
          op->bytes -= sizeof(cd) * ne;
          *t = reinterpret_cast<cd*>(f32);
        } else if (f32) {
          cudaFree(f32);
        }
      }
    } else {
      if (s == FMPB_OK && op->n_near > 0) s = spectrum_to_ff(op->S, (size_t)op->n_near * n * n, st);
      if (s == FMPB_OK) s = spectrum_to_ff(op->V0, (size_t)B * n, st);
      if (s == FMPB_OK) s = spectrum_to_ff(op->U0, (size_t)B * n, st);
    }
    if (s != FMPB_OK) return fail(s);
    const int n_far = (int)(far_off.size() / 3);
    std::vector<double> dvec(3 * (size_t)n_far);
    std::vector<int64_t> dfar(n_far);
    for (int i = 0; i < n_far; ++i) {
      const int32_t* dl = &far_off[3 * i];
      for (int c = 0; c < 3; ++c)
        dvec[3 * i + c] = dl[0] * op->grid.L[0][c] + dl[1] * op->grid.L[1][c] + dl[2] * op->grid.L[2][c];
      dfar[i] = offset_slot(sh, dl[0], dl[1], dl[2]);
    }
    s = m2l_blocks(nt, k, n_far, dvec.data(), dfar.data(), op->spec, st);
    if (s == FMPB_OK) s = grid_fft_inplace(sh, B * B, op->spec, st);   // leaves float-float pairs
    if (s != FMPB_OK) return fail(s);
    if (op->img_sep) {
      // image part (Eq. (2dPeriodicFMM_halfspace)): R_p S^ at the near image
      // offsets, V^ = R_p x the P2M table of the reflected cell, and the M2L
      // blocks of the translations x_c - y^_c of the far image offsets
      op->n_near_img = (int)(near_img.size() / 3);
      const std::vector<double> shn = image_shifts(op, near_img);
      std::vector<int64_t> dn(op->n_near_img);
      for (int i = 0; i < op->n_near_img; ++i) dn[i] = i;
      s = dev_alloc(&op->S_img, (size_t)op->n_near_img * n * n, op->bytes);
      if (s == FMPB_OK) s = dev_alloc(&op->near_offs_img, near_img.size(), op->bytes);
      if (s == FMPB_OK) s = dev_alloc(&op->V0_img, (size_t)B * n, op->bytes);
      if (s == FMPB_OK) s = dev_alloc(&op->spec_img, (size_t)sh.F * B * B, op->bytes);
      if (s != FMPB_OK) return fail(s);
      if ((near_img.size() && cudaMemcpyAsync(op->near_offs_img, near_img.data(), sizeof(int) * near_img.size(),
                                              cudaMemcpyHostToDevice, st) != cudaSuccess) ||
          cudaMemsetAsync(op->spec_img, 0, sizeof(cd) * (size_t)sh.F * B * B, st) != cudaSuccess)
        return fail(cuda_status(cudaGetLastError(), "operator_create copies"));
      const ImageBlocks ib{&op->refl, shn.data(), op->plane.Rp, false};
      if (op->n_near_img > 0)
        s = build_blocks(op->mesh, op->grid, k, beta, op->n_near_img, near_img.data(), dn.data(), op->S_img, st, &ib);
      if (s == FMPB_OK)
        s = multipole_tables(op->refl, k, beta, nt, op->V0_img, nullptr, st, nullptr, op->refl.nodes == 9 ? -1.0 : 1.0);
      if (s == FMPB_OK) s = scale_inplace(op->V0_img, (size_t)B * n, op->plane.Rp, st);
      const int n_far_img = (int)(far_img.size() / 3);
      std::vector<int64_t> dfi(n_far_img);
      for (int i = 0; i < n_far_img; ++i) dfi[i] = offset_slot(sh, far_img[3 * i], far_img[3 * i + 1], far_img[3 * i + 2]);
      if (s == FMPB_OK && n_far_img > 0) s = m2l_blocks(nt, k, n_far_img, far_img_t.data(), dfi.data(), op->spec_img, st);
      if (s == FMPB_OK) s = grid_fft_inplace(sh, B * B, op->spec_img, st);
      if (o.precision == FMPB_FP32) {
        for (cd** t : {&op->S_img, &op->V0_img}) {
          const size_t ne = (t == &op->S_img) ? (size_t)op->n_near_img * n * n : (size_t)B * n;
          float2* f32 = nullptr;
          if (s == FMPB_OK) s = dev_alloc(&f32, ne, op->bytes);
          if (s == FMPB_OK) s = vector_to_f32(*t, f32, ne, st);
          if (s == FMPB_OK && cudaStreamSynchronize(st) != cudaSuccess) s = cuda_status(cudaGetLastError(), "tables");
          if (s == FMPB_OK) {
            cudaFree(*t);
            op->bytes -= sizeof(cd) * ne;
            *t = reinterpret_cast<cd*>(f32);
          } else if (f32) {
            cudaFree(f32);
          }
        }
      } else {
        if (s == FMPB_OK) s = spectrum_to_ff(op->S_img, (size_t)op->n_near_img * n * n, st);
        if (s == FMPB_OK) s = spectrum_to_ff(op->V0_img, (size_t)B * n, st);
      }
      if (s != FMPB_OK) return fail(s);
    }
  }
  op->precision = o.precision;
  const size_t ne = (size_t)sh.F * op->B * op->B;
  const bool want32 = o.precision == FMPB_FP32 || (o.precision == FMPB_MIXED && form == FMPB_FORM_PBEM);
  const bool wantb = o.precision == FMPB_BF16 || (o.precision == FMPB_MIXED && form == FMPB_FORM_FMM);
  if (want32) {
    s = dev_alloc(reinterpret_cast<float2**>(&op->spec32), ne, op->bytes);
    if (s == FMPB_OK) s = spectrum_ff_to_f32(op->spec, op->spec32, ne, st);
    if (s == FMPB_OK && op->spec_img) s = dev_alloc(reinterpret_cast<float2**>(&op->spec32_img), ne, op->bytes);
    if (s == FMPB_OK && op->spec_img) s = spectrum_ff_to_f32(op->spec_img, op->spec32_img, ne, st);
    if (s != FMPB_OK) return fail(s);
  }
  if (wantb) {
    s = dev_alloc(&op->specb, (size_t)sh.F * tc_rows(op->B) * tc_depth(op->B), op->bytes);
    if (s == FMPB_OK)
      s = tc_realify_ff(reinterpret_cast<const float4*>(op->spec), (int)sh.F, op->B, op->B, op->specb, st);
    if (s != FMPB_OK) return fail(s);
  }
  if (o.precision == FMPB_FP32 || o.precision == FMPB_BF16) {
    if (cudaStreamSynchronize(st) != cudaSuccess) return fail(cuda_status(cudaGetLastError(), "operator_create"));
    cudaFree(op->spec);
    op->spec = nullptr;
    op->bytes -= sizeof(cd) * ne;
    if (op->spec_img) {
      cudaFree(op->spec_img);
      op->spec_img = nullptr;
      op->bytes -= sizeof(cd) * ne;
    }
  }
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail(cuda_status(e, "operator_create"));
  *out = op;
  return FMPB_OK;
}

fmpb_status fmpb_operator_get_info(const fmpb_operator* op, fmpb_operator_info* info) {
  CHECK_ARG(op && info, "operator_get_info: NULL argument");
  info->n = op->mesh.n;
  info->n_cells = op->shape.ncells;
  info->N = (int64_t)op->mesh.n * op->shape.ncells;
  info->dim = op->dim;
  info->form = op->form;
  info->n_t = op->nt;
  info->B = op->B;
  for (int a = 0; a < 3; ++a) info->P[a] = op->shape.P[a];
  info->F = op->shape.F;
  info->n_near = op->n_near;
  info->bytes_device = op->bytes;
  info->precision = op->precision;
  info->beta_re = op->beta.x;
  info->beta_im = op->beta.y;
  info->halfspace = op->plane.on;
  info->hankel_axis = op->hankel;
  info->n_near_image = op->n_near_img;
  info->image_separate = op->img_sep ? 1 : 0;
  info->near_levels = op->near2 ? op->near2->L : 0;
  info->n_m2l_near = op->near2 ? op->near2->n_m2l : 0;
  info->n_p2p_near = op->near2 ? op->near2->n_p2p : 0;
  info->element = op->mesh.nodes == 9 ? FMPB_ELEM_QUAD9 : FMPB_ELEM_TRI3;
  info->pressure_order = op->mesh.q9_order;
  info->n_t_rule_err = op->nt_rule_err;
  return FMPB_OK;
}

void fmpb_operator_destroy(fmpb_operator* op) { delete op; }

fmpb_status fmpb_rhs_plane_wave(const fmpb_operator* op, int R, const double* dirs, const fmpb_c64* amps,
                                fmpb_c64* b, void* stream) {
  CHECK_ARG(op && dirs && b, "rhs_plane_wave: NULL argument");
  CHECK_ARG(R >= 1 && R <= 65535, "rhs_plane_wave: R out of range");
  std::vector<fmpb_incident> inc(R);
  for (int r = 0; r < R; ++r) {
    inc[r].kind = FMPB_INC_PLANE;
    for (int d = 0; d < 3; ++d) inc[r].vec[d] = dirs[3 * r + d];
    inc[r].amp = amps ? amps[r] : fmpb_c64{1.0, 0.0};
  }
  return rhs_incident(op->mesh, op->grid, op->k, R, inc.data(), op->plane, (cd*)b, (cudaStream_t)stream);
}

fmpb_status fmpb_rhs_incident(const fmpb_operator* op, int R, const fmpb_incident* inc, fmpb_c64* b, void* stream) {
  CHECK_ARG(op && inc && b, "rhs_incident: NULL argument");
  CHECK_ARG(R >= 1 && R <= 65535, "rhs_incident: R out of range");
  return rhs_incident(op->mesh, op->grid, op->k, R, inc, op->plane, (cd*)b, (cudaStream_t)stream);
}

fmpb_status fmpb_matvec(const fmpb_operator* op, int R, const fmpb_c64* x, fmpb_c64* y, void* stream) {
  CHECK_ARG(op && x && y, "matvec: NULL argument");
  CHECK_ARG(R >= 1 && R <= 4096, "matvec: R out of range");
  CHECK_ARG((const void*)x != (const void*)y, "matvec: x and y must not alias");
  return const_cast<fmpb_operator*>(op)->matvec(R, (const cd*)x, (cd*)y, (cudaStream_t)stream);
}

fmpb_status fmpb_solve(const fmpb_operator* op, int R, const fmpb_c64* b, fmpb_c64* p, const fmpb_solve_opts* opts,
                       fmpb_solve_info* info, void* stream) {
  CHECK_ARG(op && b && p, "solve: NULL argument");
  CHECK_ARG(R >= 1 && R <= 4096, "solve: R out of range");
  CHECK_ARG((const void*)b != (const void*)p, "solve: b and p must not alias");
  fmpb_solve_opts o = opts ? *opts : fmpb_solve_opts{0.0, 0, 0, 0, 0.0};
  fmpb_operator* mop = const_cast<fmpb_operator*>(op);
  MatvecFn A = [mop](int r, const cd* x, cd* y, cudaStream_t st) { return mop->matvec(r, x, y, st); };
  const int64_t N = (int64_t)op->mesh.n * op->shape.ncells;
  fmpb_status s;
  // BF16 tensor-core products (BF16 operators, the inner solves of MIXED FMM
  // operators) iterate on an FP32 Krylov basis
  const MatvecF32Fn A32 = [mop](int r, const float2* x, float2* y, cudaStream_t st) {
    return mop->matvec_tc(r, x, true, y, true, st);
  };
  if (op->precision == FMPB_MIXED) {
    MatvecFn Alow = [mop](int r, const cd* x, cd* y, cudaStream_t st) { return mop->matvec(r, x, y, st, true); };
    s = gmres_refined(A, Alow, R, N, (const cd*)b, (cd*)p, o, info, (cudaStream_t)stream,
                      mop->has_tc_matvec() ? &A32 : nullptr);
  } else {
    const MatvecFfFn Aff = [mop](int r, const float4* x, float4* y, cudaStream_t st) {
      return mop->matvec_ff(r, x, y, st);
    };
    const bool tc = op->precision == FMPB_BF16 && mop->has_tc_matvec();
    s = gmres_solve(A, R, N, (const cd*)b, (cd*)p, o, info, (cudaStream_t)stream,
                    mop->has_ff_matvec() && op->precision == FMPB_FP64 ? &Aff : nullptr, nullptr,
                    tc ? &A32 : nullptr);
  }
  if (s != FMPB_OK && s != FMPB_ENOCONV) return s;
  const fmpb_status c = fmpb_operator_check(op, stream);
  return c != FMPB_OK ? c : s;
}

// ------------------------------------------------ batched solves -------
// Device scratch of a batched solve, grown on demand and freed with it.
struct BatchScratch {
  cd* p = nullptr;
  size_t elems = 0;
  ~BatchScratch() { cudaFree(p); }
  fmpb_status ensure(size_t e) {
    if (e <= elems) return FMPB_OK;
    cudaFree(p);
    p = nullptr;
    elems = 0;
    if (cudaMalloc((void**)&p, sizeof(cd) * e) != cudaSuccess) {
      cudaGetLastError();
      set_error("solve_batch: cannot allocate %zu bytes of scratch", sizeof(cd) * e);
      return FMPB_ENOMEM;
    }
    elems = e;
    return FMPB_OK;
  }
};

// Operators whose products can run as one sequence of tensor-core launches:
// the FMM form on the tensor cores (BF16 operators; MIXED ones for their
// inner products), one shape (mesh size, lattice, block size), full space,
// no multilevel near field, on one device.
static bool tc_batchable(const fmpb_operator* const* ops, int n_ops, bool low) {
  if (n_ops < 2 || n_ops > TC_MAX_BATCH) return false;
  const fmpb_operator* a = ops[0];
  for (int q = 0; q < n_ops; ++q) {
    const fmpb_operator* b = ops[q];
    if (b->form != FMPB_FORM_FMM || b->near2 || b->plane.on) return false;
    if (!(b->precision == FMPB_BF16 || (b->precision == FMPB_MIXED && low))) return false;
    if (!b->Sb || !b->V0b || !b->U0b || !b->specb || !b->tc_err) return false;
    if (b->device != a->device || b->mesh.n != a->mesh.n || b->B != a->B || b->shape.F != a->shape.F ||
        b->n_near != a->n_near)
      return false;
    for (int c = 0; c < 3; ++c)
      if (b->shape.M[c] != a->shape.M[c]) return false;
    for (int i = 0; i < a->n_near; ++i)
      for (int c = 0; c < 3; ++c)
        if (b->near_tc.d[i][c] != a->near_tc.d[i][c]) return false;
  }
  return true;
}

// y = A_o x for every operator o at once (R right-hand sides each, operator
// o's R N values after those of o - 1): each step of the FMM product (near
// field, P2M, DFT passes, per-frequency M2L products, L2P) is one launch over
// all operators.  Tensor-core waits report to the first operator's flag.
// active (host, n_ops R entries, may be null): systems still iterating; an
// operator none of whose systems iterates is left out of the tensor-core
// products (its outputs are not read), the DFT passes still run over all.
// x, y: complex double, or with x_f32 / y_f32 complex FP32 (float2).
static fmpb_status batch_matvec_tc(const fmpb_operator* const* ops, int n_ops, int R, const void* x, void* y,
                                   cudaStream_t st, BatchScratch& sc, const int* active = nullptr,
                                   bool x_f32 = false, bool y_f32 = false) {
  const fmpb_operator* a = ops[0];
  const int Rt = n_ops * R;
  const int64_t Nc = a->shape.ncells, n = a->mesh.n, B = a->B, F = a->shape.F;
  const size_t circ = circulant_scratch_elems(a->shape, B, Rt);
  const size_t mom = (size_t)Rt * Nc * B;
  const size_t xb_elems = (size_t)Rt * Nc * tc_depth(n), lb_elems = (size_t)Rt * Nc * tc_depth(B);
  const size_t fb_elems = (size_t)F * Rt * tc_depth(B);
  const size_t extra = (2 * (xb_elems + lb_elems + fb_elems) + sizeof(cd) - 1) / sizeof(cd);
  FMPB_TRY(sc.ensure(circ + 2 * mom + extra));
  cd* Mom = sc.p + circ;
  cd* Loc = Mom + mom;
  __nv_bfloat16* xb = reinterpret_cast<__nv_bfloat16*>(Loc + mom);
  __nv_bfloat16* lb = xb + xb_elems;
  __nv_bfloat16* fb = lb + lb_elems;
  const __nv_bfloat16 *Sb[TC_MAX_BATCH], *V0b[TC_MAX_BATCH], *U0b[TC_MAX_BATCH];
  const void* sp[TC_MAX_BATCH];
  int blk[TC_MAX_BATCH];
  int na = 0;
  for (int q = 0; q < n_ops; ++q) {
    bool on = !active;
    for (int r = 0; active && r < R && !on; ++r) on = active[q * R + r] != 0;
    if (!on) continue;
    Sb[na] = ops[q]->Sb;
    V0b[na] = ops[q]->V0b;
    U0b[na] = ops[q]->U0b;
    sp[na] = ops[q]->specb;
    blk[na] = q;
    ++na;
  }
  if (na == 0) return FMPB_OK;
  TcOffsets zero{};
  zero.n = 1;
  unsigned* err = a->tc_err;
  if (x_f32)
    FMPB_TRY(tc_rows_from_f32(reinterpret_cast<const float2*>(x), (int64_t)Rt * Nc, n, xb, st));
  else
    FMPB_TRY(tc_rows_to_bf16(reinterpret_cast<const cd*>(x), (int64_t)Rt * Nc, n, xb, st));
  FMPB_TRY(tc_offset_gemm_batch(V0b, na, zero, B, n, a->shape.M, R, xb, Mom, false, err, st, blk));
  const bool p32 = circulant_f32_ok(a->shape);
  const bool lrows = p32 && dft_rows_ok(a->shape.P[0], a->shape.P[0]);
  FMPB_TRY(circulant_apply(a->shape, B, nullptr, Rt, Mom, Loc, false, sc.p, st, SPEC_BF16, fb, err, false, p32, sp,
                           na, blk, n_ops, lrows ? lb : nullptr));
  if (!lrows) FMPB_TRY(tc_rows_to_bf16(Loc, (int64_t)Rt * Nc, B, lb, st));
  FMPB_TRY(tc_offset_gemm_batch(Sb, na, a->near_tc, n, n, a->shape.M, R, xb, y, false, err, st, blk, U0b, B, lb,
                                y_f32));
  return FMPB_OK;
}

fmpb_status fmpb_solve_batch(const fmpb_operator* const* ops, int n_ops, int R, const fmpb_c64* b, fmpb_c64* p,
                             const fmpb_solve_opts* opts, fmpb_solve_info* info, void* stream) {
  CHECK_ARG(ops && b && p, "solve_batch: NULL argument");
  CHECK_ARG(n_ops >= 1 && n_ops <= TC_MAX_BATCH, "solve_batch: 1..%d operators", TC_MAX_BATCH);
  CHECK_ARG(R >= 1 && (int64_t)R * n_ops <= 4096, "solve_batch: R x operators must be 1..4096");
  CHECK_ARG((const void*)b != (const void*)p, "solve_batch: b and p must not alias");
  for (int q = 0; q < n_ops; ++q) CHECK_ARG(ops[q], "solve_batch: operator %d is NULL", q);
  const int64_t N = (int64_t)ops[0]->mesh.n * ops[0]->shape.ncells;
  const bool mixed = ops[0]->precision == FMPB_MIXED;
  bool ff = true;
  for (int q = 0; q < n_ops; ++q) {
    const fmpb_operator* op = ops[q];
    CHECK_ARG((int64_t)op->mesh.n * op->shape.ncells == N, "solve_batch: operator %d has another size", q);
    CHECK_ARG((op->precision == FMPB_MIXED) == mixed, "solve_batch: MIXED operators batch only with MIXED ones");
    ff = ff && op->has_ff_matvec() && op->precision == FMPB_FP64;
  }
  fmpb_solve_opts o = opts ? *opts : fmpb_solve_opts{0.0, 0, 0, 0, 0.0};
  cudaStream_t st = (cudaStream_t)stream;
  BatchScratch sc;
  const int64_t RN = (int64_t)R * N;
  auto loop = [&](bool low, const cd* x, cd* y, cudaStream_t s) -> fmpb_status {
    for (int q = 0; q < n_ops; ++q)
      FMPB_TRY(const_cast<fmpb_operator*>(ops[q])->matvec(R, x + q * RN, y + q * RN, s, low));
    return FMPB_OK;
  };
  const bool fused = tc_batchable(ops, n_ops, false), fused_low = tc_batchable(ops, n_ops, true);
  // systems still iterating (published by the GMRES driver at every poll of
  // its convergence flags): operators whose systems have all stopped are
  // left out of the products
  std::vector<int> act((size_t)n_ops * R, 1);
  MatvecFn A = [&](int, const cd* x, cd* y, cudaStream_t s) -> fmpb_status {
    if (fused) return batch_matvec_tc(ops, n_ops, R, x, y, s, sc, act.data());
    for (int q = 0; q < n_ops; ++q) {
      bool on = false;
      for (int r = 0; r < R && !on; ++r) on = act[(size_t)q * R + r] != 0;
      if (on) FMPB_TRY(const_cast<fmpb_operator*>(ops[q])->matvec(R, x + q * RN, y + q * RN, s, false));
    }
    return FMPB_OK;
  };
  fmpb_status s;
  // fused BF16 tensor-core products iterate on an FP32 Krylov basis
  const MatvecF32Fn Alow32 = [&](int, const float2* x, float2* y, cudaStream_t s2) -> fmpb_status {
    return batch_matvec_tc(ops, n_ops, R, x, y, s2, sc, nullptr, true, true);
  };
  const MatvecF32Fn A32 = [&](int, const float2* x, float2* y, cudaStream_t s2) -> fmpb_status {
    return batch_matvec_tc(ops, n_ops, R, x, y, s2, sc, act.data(), true, true);
  };
  if (mixed) {
    MatvecFn Alow = [&](int, const cd* x, cd* y, cudaStream_t s2) -> fmpb_status {
      return fused_low ? batch_matvec_tc(ops, n_ops, R, x, y, s2, sc) : loop(true, x, y, s2);
    };
    s = gmres_refined(A, Alow, n_ops * R, N, (const cd*)b, (cd*)p, o, info, st, fused_low ? &Alow32 : nullptr);
  } else if (fused) {
    s = gmres_solve(A, n_ops * R, N, (const cd*)b, (cd*)p, o, info, st, nullptr, act.data(), &A32);
  } else {
    const MatvecFfFn Aff = [&](int, const float4* x, float4* y, cudaStream_t s2) -> fmpb_status {
      for (int q = 0; q < n_ops; ++q) {
        bool on = false;
        for (int r = 0; r < R && !on; ++r) on = act[(size_t)q * R + r] != 0;
        if (on) FMPB_TRY(const_cast<fmpb_operator*>(ops[q])->matvec_ff(R, x + q * RN, y + q * RN, s2));
      }
      return FMPB_OK;
    };
    s = gmres_solve(A, n_ops * R, N, (const cd*)b, (cd*)p, o, info, st, ff ? &Aff : nullptr, act.data());
  }
  if (s != FMPB_OK && s != FMPB_ENOCONV) return s;
  for (int q = 0; q < n_ops; ++q) {
    const fmpb_status c = fmpb_operator_check(ops[q], stream);
    if (c != FMPB_OK) return c;
  }
  return s;
}

fmpb_status fmpb_operator_check(const fmpb_operator* op, void* stream) {
  CHECK_ARG(op, "operator_check: NULL operator");
  cudaStream_t st = (cudaStream_t)stream;
  FMPB_CUDA(cudaStreamSynchronize(st));
  if (!op->tc_err) return FMPB_OK;
  unsigned flag = 0;
  FMPB_CUDA(cudaMemcpyAsync(&flag, op->tc_err, sizeof(flag), cudaMemcpyDeviceToHost, st));
  FMPB_CUDA(cudaStreamSynchronize(st));
  if (flag) {
    set_error("a tensor-core product gave up waiting for its MMAs (results of this operator are invalid)");
    return FMPB_ECUDA;
  }
  return FMPB_OK;
}

fmpb_status fmpb_field(const fmpb_operator* op, int R, const fmpb_c64* p, const double* dirs, const fmpb_c64* amps,
                       int64_t npts, const double* pts, fmpb_c64* out, void* stream) {
  CHECK_ARG(op && p && dirs && pts && out, "field: NULL argument");
  CHECK_ARG(R >= 1 && R <= 65535 && npts >= 1, "field: R or npts out of range");
  std::vector<fmpb_incident> inc(R);
  for (int r = 0; r < R; ++r) {
    inc[r].kind = FMPB_INC_PLANE;
    for (int d = 0; d < 3; ++d) inc[r].vec[d] = dirs[3 * r + d];
    inc[r].amp = amps ? amps[r] : fmpb_c64{1.0, 0.0};
  }
  return fmpb_field_incident(op, R, p, inc.data(), npts, pts, out, stream);
}

fmpb_status fmpb_field_incident(const fmpb_operator* op, int R, const fmpb_c64* p, const fmpb_incident* inc,
                                int64_t npts, const double* pts, fmpb_c64* out, void* stream) {
  CHECK_ARG(op && p && inc && pts && out, "field: NULL argument");
  CHECK_ARG(R >= 1 && R <= 65535 && npts >= 1, "field: R or npts out of range");
  return field_incident(op->mesh, op->plane.on ? &op->refl : nullptr, op->grid, op->k, op->beta, op->plane, R,
                        (const cd*)p, inc, npts, pts, (cd*)out, (cudaStream_t)stream);
}

fmpb_status fmpb_insertion_loss(const fmpb_operator* op, int R, const fmpb_c64* p, const fmpb_incident* inc,
                                int64_t npts, const double* pts, double* il, void* stream) {
  CHECK_ARG(op && p && inc && pts && il, "insertion_loss: NULL argument");
  CHECK_ARG(R >= 1 && R <= 65535 && npts >= 1, "insertion_loss: R or npts out of range");
  return insertion_loss(op->mesh, op->plane.on ? &op->refl : nullptr, op->grid, op->k, op->beta, op->plane, R,
                        (const cd*)p, inc, npts, pts, il, (cudaStream_t)stream);
}

static fmpb_status halfspace_plan_npe(const double* verts, int64_t nv, const int32_t* tris, int64_t ntri, int npe,
                                      const fmpb_lattice* lattice, int plane_axis, double plane_offset,
                                      int32_t* hankel_axis, int32_t* n_near_image, double* dmin_far_image) {
  CHECK_ARG(verts && tris && nv >= npe && ntri >= 1, "halfspace_plan: bad mesh");
  CHECK_ARG(hankel_axis && n_near_image && dmin_far_image, "halfspace_plan: NULL output");
  for (int64_t e = 0; e < npe * ntri; ++e)
    CHECK_ARG(tris[e] >= 0 && tris[e] < nv, "halfspace_plan: node index out of range");
  CellGrid g;
  FMPB_TRY(make_grid(lattice, g));
  fmpb_operator_opts o{};
  o.halfspace = 1;
  o.plane_axis = plane_axis;
  o.plane_offset = plane_offset;
  o.Rp_re = 1.0;
  int h = -1;
  FMPB_TRY(halfspace_check(g, o, verts, nv, tris, ntri, &h, npe));
  std::vector<int32_t> offs;
  for (int dz = 1 - g.M[2]; dz < g.M[2]; ++dz)
    for (int dy = 1 - g.M[1]; dy < g.M[1]; ++dy)
      for (int dx = 1 - g.M[0]; dx < g.M[0]; ++dx) offs.insert(offs.end(), {dx, dy, dz});
  const std::vector<double> sh = image_shifts(g, h, plane_axis, plane_offset, offs);
  const double r2 = 2.0 * image_r(g) * (1.0 - 1e-9);
  int near = 0;
  double dmin = 1e300;
  for (size_t i = 0; i < offs.size() / 3; ++i) {
    const double d = sqrt(sh[3 * i] * sh[3 * i] + sh[3 * i + 1] * sh[3 * i + 1] + sh[3 * i + 2] * sh[3 * i + 2]);
    if (d < r2)
      ++near;
    else
      dmin = fmin(dmin, d);
  }
  *hankel_axis = h;
  *n_near_image = near;
  *dmin_far_image = dmin;
  return FMPB_OK;
}

fmpb_status fmpb_halfspace_plan(const double* verts, int64_t nv, const int32_t* tris, int64_t ntri,
                                const fmpb_lattice* lattice, int plane_axis, double plane_offset,
                                int32_t* hankel_axis, int32_t* n_near_image, double* dmin_far_image) {
  return halfspace_plan_npe(verts, nv, tris, ntri, 3, lattice, plane_axis, plane_offset, hankel_axis, n_near_image,
                            dmin_far_image);
}

fmpb_status fmpb_halfspace_plan_q9(const double* nodes, int64_t nn, const int32_t* elems, int64_t n,
                                   const fmpb_lattice* lattice, int plane_axis, double plane_offset,
                                   int32_t* hankel_axis, int32_t* n_near_image, double* dmin_far_image) {
  return halfspace_plan_npe(nodes, nn, elems, n, 9, lattice, plane_axis, plane_offset, hankel_axis, n_near_image,
                            dmin_far_image);
}

static fmpb_status near2_counts(const double* verts, int64_t nv, const int32_t* idx, int64_t n, int npe,
                                const fmpb_lattice* lattice, int near_levels, int n_t_near, int32_t* levels_out,
                                int64_t* n_m2l, int64_t* n_p2p, int64_t* n_translations) {
  CHECK_ARG(verts && idx && nv >= npe && n >= 1 && n <= (1 << 20), "near2_plan: bad mesh");
  CHECK_ARG(levels_out && n_m2l && n_p2p && n_translations, "near2_plan: NULL output");
  CHECK_ARG(near_levels >= 0 && near_levels <= 10, "near2_plan: near_levels must be 0..10");
  for (int64_t e = 0; e < npe * n; ++e)
    CHECK_ARG(idx[e] >= 0 && idx[e] < nv, "near2_plan: node index out of range");
  CellGrid g;
  FMPB_TRY(make_grid(lattice, g));
  std::vector<int32_t> near_off;
  for (int dz = 1 - g.M[2]; dz < g.M[2]; ++dz)
    for (int dy = 1 - g.M[1]; dy < g.M[1]; ++dy)
      for (int dx = 1 - g.M[0]; dx < g.M[0]; ++dx)
        if (abs(dx) <= 1 && abs(dy) <= 1 && abs(dz) <= 1) near_off.insert(near_off.end(), {dx, dy, dz});
  Near2 t;
  Near2Host h;
  FMPB_TRY(near2_plan(verts, idx, (int)n, g, near_levels, n_t_near > 0 ? n_t_near : 6, near_off, t, h, npe));
  *levels_out = t.L;
  *n_m2l = t.n_m2l;
  *n_p2p = t.n_p2p;
  *n_translations = t.n_k;
  return FMPB_OK;
}

fmpb_status fmpb_near2_plan_counts(const double* verts, int64_t nv, const int32_t* tris, int64_t ntri,
                                   const fmpb_lattice* lattice, int near_levels, int n_t_near, int32_t* levels_out,
                                   int64_t* n_m2l, int64_t* n_p2p, int64_t* n_translations) {
  return near2_counts(verts, nv, tris, ntri, 3, lattice, near_levels, n_t_near, levels_out, n_m2l, n_p2p,
                      n_translations);
}

fmpb_status fmpb_near2_plan_counts_q9(const double* nodes, int64_t nn, const int32_t* elems, int64_t n,
                                      const fmpb_lattice* lattice, int near_levels, int n_t_near, int32_t* levels_out,
                                      int64_t* n_m2l, int64_t* n_p2p, int64_t* n_translations) {
  return near2_counts(nodes, nn, elems, n, 9, lattice, near_levels, n_t_near, levels_out, n_m2l, n_p2p,
                      n_translations);
}

fmpb_status fmpb_build_blocks(const double* verts, int64_t nv, const int32_t* tris, int64_t ntri,
                              const fmpb_lattice* lattice, double k, int n_off, const int32_t* offsets, fmpb_c64* out,
                              void* stream) {
  return fmpb_build_blocks_admittance(verts, nv, tris, ntri, lattice, k, 0.0, 0.0, n_off, offsets, out, stream);
}

fmpb_status fmpb_build_blocks_admittance(const double* verts, int64_t nv, const int32_t* tris, int64_t ntri,
                                         const fmpb_lattice* lattice, double k, double beta_re, double beta_im,
                                         int n_off, const int32_t* offsets, fmpb_c64* out, void* stream) {
  CHECK_ARG(offsets && out && n_off >= 1, "build_blocks: bad offsets or output");
  CHECK_ARG(k > 0.0 && std::isfinite(k), "build_blocks: wavenumber must be positive");
  CHECK_ARG(std::isfinite(beta_re) && std::isfinite(beta_im), "build_blocks: admittance must be finite");
  CellGrid g;
  FMPB_TRY(make_grid(lattice, g));
  DeviceMesh m;
  cudaStream_t st = (cudaStream_t)stream;
  FMPB_TRY(upload_mesh(verts, nv, tris, ntri, m, st));
  std::vector<int64_t> dest(n_off);
  for (int i = 0; i < n_off; ++i) dest[i] = i;
  fmpb_status s = build_blocks(m, g, k, mkc(beta_re, beta_im), n_off, offsets, dest.data(), (cd*)out, st);
  free_mesh(m);
  return s;
}

fmpb_status fmpb_build_blocks_q9(const double* nodes, int64_t nn, const int32_t* elems, int64_t n,
                                 const fmpb_lattice* lattice, double k, double beta_re, double beta_im, int n_off,
                                 const int32_t* offsets, fmpb_c64* out, void* stream) {
  CHECK_ARG(offsets && out && n_off >= 1, "build_blocks_q9: bad offsets or output");
  CHECK_ARG(k > 0.0 && std::isfinite(k), "build_blocks_q9: wavenumber must be positive");
  CHECK_ARG(std::isfinite(beta_re) && std::isfinite(beta_im), "build_blocks_q9: admittance must be finite");
  CellGrid g;
  FMPB_TRY(make_grid(lattice, g));
  DeviceMesh m;
  cudaStream_t st = (cudaStream_t)stream;
  fmpb_status s = upload_mesh_q9(nodes, nn, elems, n, m, st);
  if (s == FMPB_OK) {
    std::vector<int64_t> dest(n_off);
    for (int i = 0; i < n_off; ++i) dest[i] = i;
    s = build_blocks_q9(m, g, k, mkc(beta_re, beta_im), n_off, offsets, dest.data(), (cd*)out, st);
  }
  free_mesh(m);
  return s;
}

fmpb_status fmpb_build_blocks_q9p(const double* nodes, int64_t nn, const int32_t* elems, int64_t n, int order,
                                  const fmpb_lattice* lattice, double k, double beta_re, double beta_im, int n_off,
                                  const int32_t* offsets, fmpb_c64* out, void* stream) {
  CHECK_ARG(offsets && out && n_off >= 1, "build_blocks_q9p: bad offsets or output");
  CHECK_ARG(order == 1 || order == 2, "build_blocks_q9p: pressure order must be 1 or 2");
  CHECK_ARG(k > 0.0 && std::isfinite(k), "build_blocks_q9p: wavenumber must be positive");
  CHECK_ARG(std::isfinite(beta_re) && std::isfinite(beta_im), "build_blocks_q9p: admittance must be finite");
  CellGrid g;
  FMPB_TRY(make_grid(lattice, g));
  DeviceMesh m;
  cudaStream_t st = (cudaStream_t)stream;
  fmpb_status s = upload_mesh_q9p(nodes, nn, elems, n, order, m, st);
  if (s == FMPB_OK) {
    std::vector<int64_t> dest(n_off);
    for (int i = 0; i < n_off; ++i) dest[i] = i;
    s = build_blocks_q9p(m, g, k, mkc(beta_re, beta_im), n_off, offsets, dest.data(), (cd*)out, st);
  }
  free_mesh(m);
  return s;
}

fmpb_status fmpb_multipole_tables(const double* verts, int64_t nv, const int32_t* tris, int64_t ntri, double k,
                                  int n_t, fmpb_c64* V0, fmpb_c64* U0, void* stream) {
  return fmpb_multipole_tables_admittance(verts, nv, tris, ntri, k, 0.0, 0.0, n_t, V0, U0, stream);
}

fmpb_status fmpb_multipole_tables_admittance(const double* verts, int64_t nv, const int32_t* tris, int64_t ntri,
                                             double k, double beta_re, double beta_im, int n_t, fmpb_c64* V0,
                                             fmpb_c64* U0, void* stream) {
  CHECK_ARG(k > 0.0 && std::isfinite(k), "multipole_tables: wavenumber must be positive");
  CHECK_ARG(std::isfinite(beta_re) && std::isfinite(beta_im), "multipole_tables: admittance must be finite");
  CHECK_ARG(n_t >= 1 && n_t <= MAX_NT, "multipole_tables: n_t must be 1..%d", MAX_NT);
  DeviceMesh m;
  cudaStream_t st = (cudaStream_t)stream;
  FMPB_TRY(upload_mesh(verts, nv, tris, ntri, m, st));
  fmpb_status s = multipole_tables(m, k, mkc(beta_re, beta_im), n_t, (cd*)V0, (cd*)U0, st);
  if (s == FMPB_OK && cudaStreamSynchronize(st) != cudaSuccess) s = cuda_status(cudaGetLastError(), "multipole_tables");
  free_mesh(m);
  return s;
}

fmpb_status fmpb_m2l_blocks(double k, int n_t, int n_d, const double* dvecs, fmpb_c64* out, void* stream) {
  CHECK_ARG(k > 0.0 && std::isfinite(k), "m2l_blocks: wavenumber must be positive");
  CHECK_ARG(n_t >= 1 && n_t <= MAX_NT, "m2l_blocks: n_t must be 1..%d", MAX_NT);
  CHECK_ARG(n_d >= 1 && dvecs && out, "m2l_blocks: bad translations or output");
  for (int i = 0; i < n_d; ++i) {
    double r2 = dvecs[3 * i] * dvecs[3 * i] + dvecs[3 * i + 1] * dvecs[3 * i + 1] + dvecs[3 * i + 2] * dvecs[3 * i + 2];
    CHECK_ARG(r2 > 0.0 && std::isfinite(r2), "m2l_blocks: translation %d is zero or not finite", i);
  }
  std::vector<int64_t> dest(n_d);
  for (int i = 0; i < n_d; ++i) dest[i] = i;
  return m2l_blocks(n_t, k, n_d, dvecs, dest.data(), (cd*)out, (cudaStream_t)stream);
}

fmpb_status fmpb_circulant_spectrum(const int32_t counts[3], int64_t B, const fmpb_c64* blocks, fmpb_c64* spec,
                                    void* stream) {
  CHECK_ARG(counts && blocks && spec && B >= 1 && B <= (1 << 20), "circulant_spectrum: bad arguments");
  int M[3];
  int64_t nc = 1;
  for (int a = 0; a < 3; ++a) {
    CHECK_ARG(counts[a] >= 1 && counts[a] <= 4096, "circulant_spectrum: count out of range");
    M[a] = counts[a];
    nc *= M[a];
  }
  // (2M-1)^3 <= 8 x cells offsets are listed on the host; the F B^2 spectrum
  // values must be addressable in bytes
  CHECK_ARG(nc <= (1 << 24), "circulant_spectrum: too many cells (%lld)", (long long)nc);
  const CircShape sh = make_shape(M);
  CHECK_ARG((size_t)sh.F * (size_t)B <= ((size_t)1 << 59) / (size_t)B,
            "circulant_spectrum: %lld frequencies x B^2 = %lld^2 is too large", (long long)sh.F, (long long)B);
  return circulant_spectrum_from_blocks(sh, B, (const cd*)blocks, (cd*)spec, (cudaStream_t)stream);
}

fmpb_status fmpb_tuning_summary(char* buf, size_t len) {
  CHECK_ARG(buf && len >= 3, "tuning_summary: buffer too small");
  std::string out, dft;
  FMPB_TRY(tc_tuning_summary(out));   // "[...]"
  dft_tuning_summary(dft);
  if (!dft.empty()) {
    out.pop_back();
    if (out.size() > 1) out += ", ";
    out += dft + "]";
  }
  CHECK_ARG(out.size() + 1 <= len, "tuning_summary: buffer of %zu bytes too small (%zu needed)", len, out.size() + 1);
  memcpy(buf, out.c_str(), out.size() + 1);
  return FMPB_OK;
}

fmpb_status fmpb_set_tile_variant(int variant) { return tc_force_variant(variant); }

fmpb_status fmpb_set_dft_plan(int kind) { return dft_force_plan(kind); }

namespace {
fmpb_status offset_gemm_bf16(const int32_t counts[3], int n_off, const int32_t* offsets, int64_t m, int64_t k,
                             const fmpb_c64* T, int R, const fmpb_c64* x, int64_t k2, const fmpb_c64* T2,
                             const fmpb_c64* x2, fmpb_c64* y, int accumulate, void* stream) {
  CHECK_ARG(counts && offsets && T && x && y, "offset_gemm_bf16: NULL argument");
  CHECK_ARG(n_off >= 1 && n_off <= TC_MAX_OFF, "offset_gemm_bf16: n_off must be 1..%d", TC_MAX_OFF);
  CHECK_ARG(m >= 1 && m <= (1 << 20) && k >= 1 && k <= (1 << 20), "offset_gemm_bf16: m or k out of range");
  CHECK_ARG(R >= 1 && R <= 4096, "offset_gemm_bf16: R out of range");
  CHECK_ARG((const void*)x != (const void*)y, "offset_gemm_bf16: x and y must not alias");
  const bool tail = T2 != nullptr;
  if (tail) {
    CHECK_ARG(x2 && k2 >= 1 && k2 <= (1 << 20), "offset_gemm2_bf16: x2 NULL or k2 out of range");
    CHECK_ARG((const void*)x2 != (const void*)y, "offset_gemm2_bf16: x2 and y must not alias");
  }
  int M[3];
  int64_t Nc = 1;
  for (int a = 0; a < 3; ++a) {
    CHECK_ARG(counts[a] >= 1 && counts[a] <= 4096, "offset_gemm_bf16: count out of range");
    M[a] = counts[a];
    Nc *= M[a];
  }
  // the launch limits of the tensor-core product, checked before the sizes
  // of the device copies below are formed: at most 2^30 cells and 65,535
  // column tiles of 128 (cells x right-hand sides)
  CHECK_ARG(Nc <= (1 << 30) && (Nc * R + 127) / 128 <= 65535,
            "offset_gemm_bf16: %lld cells x %d right-hand sides exceed the launch limit", (long long)Nc, R);
  TcOffsets offs{};
  offs.n = n_off;
  for (int i = 0; i < n_off; ++i)
    for (int c = 0; c < 3; ++c) offs.d[i][c] = offsets[3 * i + c];
  cudaStream_t st = (cudaStream_t)stream;
  const size_t a_elems = (size_t)n_off * tc_rows(m) * tc_depth(k);
  const size_t x_elems = (size_t)R * Nc * tc_depth(k);
  __nv_bfloat16 *Ab = nullptr, *Xb = nullptr, *A2b = nullptr, *X2b = nullptr;
  unsigned* err = nullptr;
  size_t bytes = 0;
  fmpb_status s = dev_alloc(&Ab, a_elems, bytes);
  if (s == FMPB_OK) s = dev_alloc(&Xb, x_elems, bytes);
  if (s == FMPB_OK && tail) s = dev_alloc(&A2b, (size_t)tc_rows(m) * tc_depth(k2), bytes);
  if (s == FMPB_OK && tail) s = dev_alloc(&X2b, (size_t)R * Nc * tc_depth(k2), bytes);
  if (s == FMPB_OK) s = dev_alloc(&err, 1, bytes);
  if (s == FMPB_OK && cudaMemsetAsync(err, 0, sizeof(unsigned), st) != cudaSuccess)
    s = cuda_status(cudaGetLastError(), "memset");
  if (s == FMPB_OK) s = tc_realify((const cd*)T, n_off, m, k, Ab, st);
  if (s == FMPB_OK) s = tc_rows_to_bf16((const cd*)x, (int64_t)R * Nc, k, Xb, st);
  if (s == FMPB_OK && tail) s = tc_realify((const cd*)T2, 1, m, k2, A2b, st);
  if (s == FMPB_OK && tail) s = tc_rows_to_bf16((const cd*)x2, (int64_t)R * Nc, k2, X2b, st);
  if (s == FMPB_OK) {
    const __nv_bfloat16* a1[1] = {Ab};
    const __nv_bfloat16* a2[1] = {A2b};
    s = tc_offset_gemm_batch(a1, 1, offs, m, k, M, R, Xb, (cd*)y, accumulate != 0, err, st, nullptr,
                             tail ? a2 : nullptr, tail ? k2 : 0, X2b);
  }
  unsigned flag = 0;
  if (s == FMPB_OK && cudaMemcpyAsync(&flag, err, sizeof(flag), cudaMemcpyDeviceToHost, st) != cudaSuccess)
    s = cuda_status(cudaGetLastError(), "offset_gemm_bf16");
  if (s == FMPB_OK && cudaStreamSynchronize(st) != cudaSuccess) s = cuda_status(cudaGetLastError(), "offset_gemm_bf16");
  if (s == FMPB_OK && flag) {
    set_error("offset_gemm_bf16: a tensor-core wait gave up");
    s = FMPB_ECUDA;
  }
  cudaStreamSynchronize(st);
  cudaFree(Ab);
  cudaFree(Xb);
  cudaFree(A2b);
  cudaFree(X2b);
  cudaFree(err);
  return s;
}
}  // namespace

fmpb_status fmpb_offset_gemm_bf16(const int32_t counts[3], int n_off, const int32_t* offsets, int64_t m, int64_t k,
                                  const fmpb_c64* T, int R, const fmpb_c64* x, fmpb_c64* y, int accumulate,
                                  void* stream) {
  return offset_gemm_bf16(counts, n_off, offsets, m, k, T, R, x, 0, nullptr, nullptr, y, accumulate, stream);
}

fmpb_status fmpb_offset_gemm2_bf16(const int32_t counts[3], int n_off, const int32_t* offsets, int64_t m, int64_t k,
                                   const fmpb_c64* T, int R, const fmpb_c64* x, int64_t k2, const fmpb_c64* T2,
                                   const fmpb_c64* x2, fmpb_c64* y, int accumulate, void* stream) {
  CHECK_ARG(T2, "offset_gemm2_bf16: NULL argument");
  return offset_gemm_bf16(counts, n_off, offsets, m, k, T, R, x, k2, T2, x2, y, accumulate, stream);
}

fmpb_status fmpb_circulant_apply_bf16(const int32_t counts[3], int64_t B, const fmpb_c64* spec, int R,
                                     const fmpb_c64* x, fmpb_c64* y, int accumulate, void* stream) {
  CHECK_ARG(counts && spec && x && y && B >= 1 && B <= (1 << 20), "circulant_apply_bf16: bad arguments");
  CHECK_ARG(R >= 1 && R <= 4096, "circulant_apply_bf16: R out of range");
  CHECK_ARG((const void*)x != (const void*)y, "circulant_apply_bf16: x and y must not alias");
  int M[3];
  for (int a = 0; a < 3; ++a) {
    CHECK_ARG(counts[a] >= 1 && counts[a] <= 4096, "circulant_apply_bf16: count out of range");
    M[a] = counts[a];
  }
  const CircShape sh = make_shape(M);
  CHECK_ARG(sh.F <= 65535, "circulant_apply_bf16: %lld frequencies exceed the launch limit", (long long)sh.F);
  cudaStream_t st = (cudaStream_t)stream;
  __nv_bfloat16 *Ab = nullptr, *rows = nullptr;
  cd* scratch = nullptr;
  unsigned* err = nullptr;
  size_t bytes = 0;
  fmpb_status s = dev_alloc(&Ab, (size_t)sh.F * tc_rows(B) * tc_depth(B), bytes);
  if (s == FMPB_OK) s = dev_alloc(&rows, (size_t)sh.F * R * tc_depth(B), bytes);
  if (s == FMPB_OK) s = dev_alloc(&scratch, circulant_scratch_elems(sh, B, R), bytes);
  if (s == FMPB_OK) s = dev_alloc(&err, 1, bytes);
  if (s == FMPB_OK && cudaMemsetAsync(err, 0, sizeof(unsigned), st) != cudaSuccess)
    s = cuda_status(cudaGetLastError(), "memset");
  if (s == FMPB_OK) s = tc_realify((const cd*)spec, (int)sh.F, B, B, Ab, st);
  if (s == FMPB_OK)
    s = circulant_apply(sh, B, reinterpret_cast<const cd*>(Ab), R, (const cd*)x, (cd*)y, accumulate != 0, scratch,
                        st, SPEC_BF16, rows, err);
  unsigned flag = 0;
  if (s == FMPB_OK && cudaMemcpyAsync(&flag, err, sizeof(flag), cudaMemcpyDeviceToHost, st) != cudaSuccess)
    s = cuda_status(cudaGetLastError(), "circulant_apply_bf16");
  if (s == FMPB_OK && cudaStreamSynchronize(st) != cudaSuccess)
    s = cuda_status(cudaGetLastError(), "circulant_apply_bf16");
  if (s == FMPB_OK && flag) {
    set_error("circulant_apply_bf16: a tensor-core wait gave up");
    s = FMPB_ECUDA;
  }
  cudaStreamSynchronize(st);
  cudaFree(Ab);
  cudaFree(rows);
  cudaFree(scratch);
  cudaFree(err);
  return s;
}

fmpb_status fmpb_circulant_apply_f32(const int32_t counts[3], int64_t B, const fmpb_c64* spec, int R,
                                     const fmpb_c64* x, fmpb_c64* y, int accumulate, void* stream) {
  CHECK_ARG(counts && spec && x && y && B >= 1 && B <= (1 << 20), "circulant_apply_f32: bad arguments");
  CHECK_ARG(R >= 1 && R <= 4096, "circulant_apply_f32: R out of range");
  CHECK_ARG((const void*)x != (const void*)y, "circulant_apply_f32: x and y must not alias");
  int M[3];
  for (int a = 0; a < 3; ++a) {
    CHECK_ARG(counts[a] >= 1 && counts[a] <= 4096, "circulant_apply_f32: count out of range");
    M[a] = counts[a];
  }
  const CircShape sh = make_shape(M);
  CHECK_ARG(circulant_f32_ok(sh), "circulant_apply_f32: padded lengths %d x %d x %d do not all split into two "
            "factors of at most 16", sh.P[0], sh.P[1], sh.P[2]);
  CHECK_ARG((size_t)sh.F * (size_t)R <= ((size_t)1 << 59) / (size_t)B && (size_t)sh.F * B <= ((size_t)1 << 59) / B,
            "circulant_apply_f32: product too large");
  cudaStream_t st = (cudaStream_t)stream;
  float2* spec32 = nullptr;
  cd* scratch = nullptr;
  size_t bytes = 0;
  fmpb_status s = dev_alloc(&spec32, (size_t)sh.F * B * B, bytes);
  if (s == FMPB_OK) s = dev_alloc(&scratch, circulant_scratch_elems(sh, B, R) / 2 + 1, bytes);
  if (s == FMPB_OK) s = vector_to_f32((const cd*)spec, spec32, (size_t)sh.F * B * B, st);
  if (s == FMPB_OK)
    s = circulant_apply(sh, B, reinterpret_cast<const cd*>(spec32), R, (const cd*)x, (cd*)y, accumulate != 0,
                        scratch, st, SPEC_F32, nullptr, nullptr, false, true);
  cudaStreamSynchronize(st);
  cudaFree(spec32);
  cudaFree(scratch);
  return s;
}

fmpb_status fmpb_circulant_apply(const int32_t counts[3], int64_t B, const fmpb_c64* spec, int R, const fmpb_c64* x,
                                 fmpb_c64* y, int accumulate, void* stream) {
  CHECK_ARG(counts && spec && x && y && B >= 1 && B <= (1 << 20), "circulant_apply: bad arguments");
  CHECK_ARG(R >= 1 && R <= 4096, "circulant_apply: R out of range");
  int M[3];
  for (int a = 0; a < 3; ++a) {
    CHECK_ARG(counts[a] >= 1 && counts[a] <= 4096, "circulant_apply: count out of range");
    M[a] = counts[a];
  }
  CircShape sh = make_shape(M);
  // 2 F R B complex values must be addressable: F < 2^40, R <= 4096 and
  // B <= 2^20 keep 2 F R B 16 below 2^64 only while F R B stays below 2^59
  CHECK_ARG((size_t)sh.F * (size_t)R <= ((size_t)1 << 59) / (size_t)B,
            "circulant_apply: %lld frequencies x %d right-hand sides x B = %lld is too large", (long long)sh.F, R,
            (long long)B);
  cudaStream_t st = (cudaStream_t)stream;
  cd* scratch = nullptr;
  FMPB_CUDA(cudaMallocAsync(&scratch, sizeof(cd) * circulant_scratch_elems(sh, B, R), st));
  fmpb_status s = circulant_apply(sh, B, (const cd*)spec, R, (const cd*)x, (cd*)y, accumulate != 0, scratch, st);
  cudaFreeAsync(scratch, st);
  return s;
}

}  // extern "C"
