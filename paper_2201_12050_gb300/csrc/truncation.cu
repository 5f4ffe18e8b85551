// Truncation number of the multipole expansion chosen from the cell itself.
//
// The paper asks for an n_t "sufficiently large" (Sec. 3.1) and shows in its
// accuracy study (Sec. 4) that the needed n_t grows with frequency.  The rule
// read from that: the smallest n_t in 4..MAX_NT for which the multipole form
// U_0 K(d) V_0 (Eq. (2dPeriodicFMM)) of the block of the nearest far cell
// reproduces the exact collocation block T_d (the same quadrature) on four
// probe vectors to a relative 1e-6:
//   ||(U_0 K(d) V_0 - T_d) X||_F <= 1e-6 ||T_d X||_F,
//   X_jp = exp(2 pi i frac((p + 1) j phi)), phi = (sqrt(5) - 1) / 2, p < 4.
// d is the far offset (max-norm >= 2) whose translation d . L is shortest
// (ties: the first in the order dz, dy, dx ascending); a grid without far
// cell pairs takes n_t = 4.  The tables of n_t are the leading
// (n_t + 1)^2 rows / columns of those of MAX_NT (every entry depends only on
// its own degrees and orders), so one build of T_d, V_0, U_0 and K(d) at
// MAX_NT serves every candidate.  T_d X runs on the device (FP64); the
// candidates' products, O(n B) each, on the host in FP64.
#include <cmath>
#include <vector>

#include "common.cuh"
#include "internal.cuh"
#include "multipole.cuh"
#include "profile.cuh"

namespace fmpb {

namespace {

constexpr int TRUNC_PROBES = 4;
constexpr double TRUNC_TOL = 1e-6;
constexpr int TRUNC_MIN = 4;

// TX[p][i] = sum_j T[i][j] X[p][j]: one warp per row i, fixed-order lane sums.
__global__ void k_probe_apply(const cd* __restrict__ T, const cd* __restrict__ X, cd* __restrict__ TX, int n) {
  const int lane = threadIdx.x & 31;
  const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (i >= n) return;   // uniform across the warp
  cd acc[TRUNC_PROBES];
  for (int p = 0; p < TRUNC_PROBES; ++p) acc[p] = mkc(0.0, 0.0);
  const cd* row = T + i * n;
  for (int j = lane; j < n; j += 32) {
    const cd t = row[j];
    for (int p = 0; p < TRUNC_PROBES; ++p) acc[p] = cfma(t, X[(int64_t)p * n + j], acc[p]);
  }
  for (int p = 0; p < TRUNC_PROBES; ++p) {
    for (int o = 16; o > 0; o >>= 1) {
      acc[p].x += __shfl_xor_sync(0xffffffffu, acc[p].x, o);
      acc[p].y += __shfl_xor_sync(0xffffffffu, acc[p].y, o);
    }
    if (lane == 0) TX[(int64_t)p * n + i] = acc[p];
  }
}

template <typename T>
fmpb_status talloc(T** p, size_t count) {
  if (cudaMalloc((void**)p, sizeof(T) * (count ? count : 1)) != cudaSuccess) {
    cudaGetLastError();
    set_error("truncation rule: cannot allocate %zu bytes on the device", sizeof(T) * count);
    return FMPB_ENOMEM;
  }
  return FMPB_OK;
}

}  // namespace

bool nearest_far_offset(const CellGrid& g, int32_t d[3]) {
  double best = INFINITY;
  bool found = false;
  for (int dz = 1 - g.M[2]; dz < g.M[2]; ++dz)
    for (int dy = 1 - g.M[1]; dy < g.M[1]; ++dy)
      for (int dx = 1 - g.M[0]; dx < g.M[0]; ++dx) {
        if (abs(dx) <= 1 && abs(dy) <= 1 && abs(dz) <= 1) continue;
        double d2 = 0.0;
        for (int c = 0; c < 3; ++c) {
          const double v = dx * g.L[0][c] + dy * g.L[1][c] + dz * g.L[2][c];
          d2 += v * v;
        }
        const double dist = sqrt(d2);
        if (dist < best) {
          best = dist;
          d[0] = dx;
          d[1] = dy;
          d[2] = dz;
          found = true;
        }
      }
  return found;
}

fmpb_status auto_truncation(const DeviceMesh& mesh, const CellGrid& g, double k, cd beta, int* nt_out, bool* met,
                            double* err_out, cudaStream_t st) {
  int32_t d[3] = {0, 0, 0};
  if (!nearest_far_offset(g, d)) {
    *nt_out = TRUNC_MIN;
    *met = true;
    if (err_out) *err_out = 0.0;
    return FMPB_OK;
  }
  const int n = mesh.n;
  const int Bmax = (MAX_NT + 1) * (MAX_NT + 1);
  // probe vectors X[p][j]
  std::vector<cd> X((size_t)TRUNC_PROBES * n);
  const double phi = (sqrt(5.0) - 1.0) / 2.0;
  for (int p = 0; p < TRUNC_PROBES; ++p)
    for (int j = 0; j < n; ++j) {
      const double t = fmod((double)(p + 1) * (double)j * phi, 1.0);
      X[(size_t)p * n + j] = mkc(cos(2.0 * PI * t), sin(2.0 * PI * t));
    }
  cd *T = nullptr, *Xd = nullptr, *TX = nullptr, *V = nullptr, *U = nullptr, *K = nullptr;
  fmpb_status s = talloc(&T, (size_t)n * n);
  if (s == FMPB_OK) s = talloc(&Xd, X.size());
  if (s == FMPB_OK) s = talloc(&TX, X.size());
  if (s == FMPB_OK) s = talloc(&V, (size_t)Bmax * n);
  if (s == FMPB_OK) s = talloc(&U, (size_t)Bmax * n);
  if (s == FMPB_OK) s = talloc(&K, (size_t)Bmax * Bmax);
  const int64_t dest0 = 0;
  double dvec[3];
  for (int c = 0; c < 3; ++c) dvec[c] = d[0] * g.L[0][c] + d[1] * g.L[1][c] + d[2] * g.L[2][c];
  if (s == FMPB_OK) s = build_blocks(mesh, g, k, beta, 1, d, &dest0, T, st);
  if (s == FMPB_OK) s = multipole_tables(mesh, k, beta, MAX_NT, V, U, st);
  if (s == FMPB_OK) s = m2l_blocks(MAX_NT, k, 1, dvec, &dest0, K, st);
  if (s == FMPB_OK && cudaMemcpyAsync(Xd, X.data(), sizeof(cd) * X.size(), cudaMemcpyHostToDevice, st) != cudaSuccess)
    s = cuda_status(cudaGetLastError(), "truncation probes");
  if (s == FMPB_OK) {
    FMPB_LAUNCH("probe_apply", st, k_probe_apply<<<grid_for((size_t)n * 32, 256), 256, 0, st>>>(T, Xd, TX, n));
    if (cudaGetLastError() != cudaSuccess) s = cuda_status(cudaGetLastError(), "probe_apply");
  }
  std::vector<cd> hTX(X.size()), hV((size_t)Bmax * n), hU((size_t)Bmax * n), hK((size_t)Bmax * Bmax);
  if (s == FMPB_OK &&
      (cudaMemcpyAsync(hTX.data(), TX, sizeof(cd) * hTX.size(), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
       cudaMemcpyAsync(hV.data(), V, sizeof(cd) * hV.size(), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
       cudaMemcpyAsync(hU.data(), U, sizeof(cd) * hU.size(), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
       cudaMemcpyAsync(hK.data(), K, sizeof(cd) * hK.size(), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
       cudaStreamSynchronize(st) != cudaSuccess))
    s = cuda_status(cudaGetLastError(), "truncation tables");
  cudaFree(T);
  cudaFree(Xd);
  cudaFree(TX);
  cudaFree(V);
  cudaFree(U);
  cudaFree(K);
  if (s != FMPB_OK) return s;
  // moments of the probes at MAX_NT: M[p][q] = sum_j V[q][j] X[p][j]
  std::vector<cd> Mo((size_t)TRUNC_PROBES * Bmax, mkc(0.0, 0.0));
  for (int p = 0; p < TRUNC_PROBES; ++p)
    for (int q = 0; q < Bmax; ++q) {
      cd a = mkc(0.0, 0.0);
      const cd* vq = &hV[(size_t)q * n];
      const cd* xp = &X[(size_t)p * n];
      for (int j = 0; j < n; ++j) a = cfma(vq[j], xp[j], a);
      Mo[(size_t)p * Bmax + q] = a;
    }
  double ref = 0.0;
  for (const cd& v : hTX) ref += v.x * v.x + v.y * v.y;
  ref = sqrt(ref);
  double err = INFINITY;
  std::vector<cd> Lc(Bmax);
  for (int nt = TRUNC_MIN; nt <= MAX_NT; ++nt) {
    const int B = (nt + 1) * (nt + 1);
    double e2 = 0.0;
    for (int p = 0; p < TRUNC_PROBES; ++p) {
      for (int q = 0; q < B; ++q) {
        cd a = mkc(0.0, 0.0);
        const cd* kq = &hK[(size_t)q * Bmax];
        const cd* mp = &Mo[(size_t)p * Bmax];
        for (int q2 = 0; q2 < B; ++q2) a = cfma(kq[q2], mp[q2], a);
        Lc[q] = a;
      }
      for (int i = 0; i < n; ++i) {
        cd y = mkc(0.0, 0.0);
        const cd* ui = &hU[(size_t)i * Bmax];
        for (int q = 0; q < B; ++q) y = cfma(ui[q], Lc[q], y);
        const cd r = csub(y, hTX[(size_t)p * n + i]);
        e2 += r.x * r.x + r.y * r.y;
      }
    }
    err = sqrt(e2) / ref;
    if (err <= TRUNC_TOL) {
      *nt_out = nt;
      *met = true;
      if (err_out) *err_out = err;
      return FMPB_OK;
    }
  }
  *nt_out = MAX_NT;
  *met = false;
  if (err_out) *err_out = err;
  return FMPB_OK;
}

}  // namespace fmpb
