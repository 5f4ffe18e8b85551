// fmpb_circulant_apply_static: the block Toeplitz product of
// fmpb_circulant_apply with its scratch in a fixed device array instead of
// memory allocated per call.
//
// Some callers cannot allocate device memory while they run: a host program
// whose device memory is owned by another runtime's pool, a plug-in called
// from inside such a runtime, or a latency-bound loop that cannot afford the
// device-wide synchronisation an allocation may imply.  For them this entry
// point takes only the caller's inputs and outputs and draws every temporary
// from one statically sized array that the library declares at file scope.
#include <mutex>

#include "common.cuh"
#include "internal.cuh"

namespace fmpb {

// Size of the static scratch: 32 MiB on every device that loads the library,
// held until the process exits.  One product needs 2 F R B complex values.
constexpr size_t STATIC_SCRATCH_BYTES = (size_t)32 << 20;
static __device__ __align__(256) unsigned char g_static_scratch[STATIC_SCRATCH_BYTES];

namespace {
constexpr int MAX_DEVICES = 64;
std::mutex g_static_mu;
void* g_static_ptr[MAX_DEVICES] = {};
}  // namespace

// Device address of g_static_scratch on the current device.  The name of a
// __device__ array in host code is only a host-side stand-in, so the address
// is looked up once per device with that device current and then cached.
static fmpb_status static_scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_status(e, "cudaGetDevice");
  if (dev < 0 || dev >= MAX_DEVICES) {
    set_error("circulant_apply_static: device index %d beyond %d", dev, MAX_DEVICES);
    return FMPB_EINVAL;
  }
  std::lock_guard<std::mutex> lk(g_static_mu);
  if (!g_static_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return cuda_status(e, "cudaGetSymbolAddress(static scratch)");
    g_static_ptr[dev] = p;
  }
  *out = g_static_ptr[dev];
  return FMPB_OK;
}

}  // namespace fmpb

using namespace fmpb;

extern "C" fmpb_status fmpb_circulant_apply_static(const int32_t counts[3], int64_t B, const fmpb_c64* spec, int R,
                                                   const fmpb_c64* x, fmpb_c64* y, int accumulate, void* stream) {
  if (!counts || !spec || !x || !y || B < 1 || B > (1 << 20)) {
    set_error("circulant_apply_static: bad arguments (B must be 1..%d)", 1 << 20);
    return FMPB_EINVAL;
  }
  if (R < 1 || R > 4096) {
    set_error("circulant_apply_static: R out of range");
    return FMPB_EINVAL;
  }
  int M[3];
  for (int a = 0; a < 3; ++a) {
    if (counts[a] < 1 || counts[a] > 4096) {
      set_error("circulant_apply_static: count out of range");
      return FMPB_EINVAL;
    }
    M[a] = counts[a];
  }
  const CircShape sh = make_shape(M);
  // 2 F R B complex values, tested without forming a product that could
  // wrap: F R B <= limit  <=>  B <= limit / (F R)  (F < 2^40, R <= 4096)
  const size_t per_b = 2 * sizeof(cd) * (size_t)sh.F * (size_t)R;
  const size_t need = per_b * (size_t)B;
  if ((size_t)B > STATIC_SCRATCH_BYTES / per_b || need > STATIC_SCRATCH_BYTES) {
    set_error("circulant_apply_static: this product needs %zu bytes of scratch (2 F R B complex values, "
              "F = %lld, R = %d, B = %lld) but the static array holds %zu bytes",
              need, (long long)sh.F, R, (long long)B, STATIC_SCRATCH_BYTES);
    return FMPB_EINVAL;
  }
  void* scratch = nullptr;
  FMPB_TRY(static_scratch_address(&scratch));
  // Every scratch element the product reads is written earlier in the same
  // call, so nothing has to be cleared between calls.
  return circulant_apply(sh, B, (const cd*)spec, R, (const cd*)x, (cd*)y, accumulate != 0, (cd*)scratch,
                         (cudaStream_t)stream);
}
