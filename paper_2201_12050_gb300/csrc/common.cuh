// Shared device/host definitions of the FMPBEM library (complex arithmetic,
// element geometry, status handling).  Internal header: the public C ABI is
// include/fmpb.h.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <cmath>
#include <string>

#include "../../include/fmpb.h"

namespace fmpb {

// ----------------------------------------------------------- complex ------
typedef double2 cd;   // interleaved (re, im), the layout of fmpb_c64

__host__ __device__ __forceinline__ cd mkc(double r, double i) { return make_double2(r, i); }
__host__ __device__ __forceinline__ cd cadd(cd a, cd b) { return mkc(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ cd csub(cd a, cd b) { return mkc(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ cd cmul(cd a, cd b) { return mkc(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__host__ __device__ __forceinline__ cd cmulr(cd a, double s) { return mkc(a.x * s, a.y * s); }
__host__ __device__ __forceinline__ cd cconj(cd a) { return mkc(a.x, -a.y); }
// a += b * c
__host__ __device__ __forceinline__ cd cfma(cd b, cd c, cd a) {
  return mkc(fma(b.x, c.x, fma(-b.y, c.y, a.x)), fma(b.x, c.y, fma(b.y, c.x, a.y)));
}
// a += conj(b) * c
__host__ __device__ __forceinline__ cd cfma_conj(cd b, cd c, cd a) {
  return mkc(fma(b.x, c.x, fma(b.y, c.y, a.x)), fma(b.x, c.y, fma(-b.y, c.x, a.y)));
}

// ------------------------------------------------------ element geometry --
// One flat triangle, packed for the quadrature kernels (18 doubles).
struct Elem {
  double v[3][3];   // vertices in mesh order
  double c[3];      // centroid (collocation point)
  double nrm[3];    // unit normal, into the fluid
  double area;
  double hmax;      // longest edge
};

// Gauss-Legendre rules on [0, 1] for the orders the operator uses.
constexpr int Q_FAR = 3;
constexpr int Q_NEAR = 8;
constexpr int Q_SELF = 8;
struct QuadRules {
  double t3[Q_FAR], w3[Q_FAR];
  double t8[Q_NEAR], w8[Q_NEAR];
};

// Class thresholds on d/h, scaled by (1 + 1e-9) so that exact ties (which
// regular meshes produce) go to the more accurate class on every machine.
constexpr double TIE = 1e-9;
constexpr double FAR_RATIO = 4.0 * (1.0 + TIE);
constexpr double NEAR_RATIO = 1.5 * (1.0 + TIE);
constexpr double PI = 3.14159265358979323846;

// ----------------------------------------------------------- status ------
void set_error(const char* fmt, ...);
fmpb_status cuda_status(cudaError_t e, const char* what);

#define FMPB_CUDA(call)                                               \
  do {                                                                \
    cudaError_t _e = (call);                                          \
    if (_e != cudaSuccess) return ::fmpb::cuda_status(_e, #call);     \
  } while (0)

#define FMPB_TRY(call)                                                \
  do {                                                                \
    fmpb_status _s = (call);                                          \
    if (_s != FMPB_OK) return _s;                                     \
  } while (0)

inline unsigned grid_for(size_t n, unsigned block) {
  size_t g = (n + block - 1) / block;
  return (unsigned)(g == 0 ? 1 : g);
}

}  // namespace fmpb
