// Collocation blocks T_delta (Sec. 2.2, Eq. (blockToeplizMatrix)) of the
// Burton-Miller operator (Sec. 2.1, Eq. (bm), Eq. (matrixBEM)) on nine-node
// quadrilaterals with discontinuous pressure of order 1 or 2: nb = 4 or 8
// dofs per element (dof e nb + a), collocated at the pressure nodes.  The
// element arithmetic is the host-and-device code of quad9p.cuh; here it is
// laid out for the device:
//   * one thread per (offset, collocation point, source element) evaluates
//     the far class (the 16-point table of quad9.cu) for all nb shapes at
//     once, and lists the near and very-near items;
//   * a warp per listed item shares its 64 (near) or 1,024 / 4,096 (very
//     near) points, formed from the element's monomials, and reduces the nb
//     columns in a fixed order;
//   * a warp per dof evaluates the self rule about its node (96 angular
//     nodes split between the lanes) for the nb columns of its element.
#include "common.cuh"
#include "internal.cuh"
#include "profile.cuh"
#include "quad9p.cuh"

namespace fmpb {

// Collocation data of every dof r = e nb + a: the node's point and normal,
// with the element's chord and area (corners 0, 2, 8 as v), in Elem for the
// kernels shared with the other elements (right-hand sides).
__global__ void k_q9p_colloc(const Q9Elem* __restrict__ q9, int ne, int order, Elem* __restrict__ el) {
  const Q9Basis B = q9p_basis(order);
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= ne * B.nb) return;
  const int e = r / B.nb, a = r - e * B.nb;
  double am[9][3];
  q9_monomials(q9[e].Y, am);
  double xi, eta;
  q9p_node(B, a, &xi, &eta);
  double y[3], yx[3], ye[3], J[3];
  q9_eval(am, xi, eta, y, yx, ye);
  q9_cross(yx, ye, J);
  const double dJ = sqrt(q9_dot(J, J));
  Elem E;
  const int corner[3] = {0, 2, 8};
  for (int c = 0; c < 3; ++c)
    for (int d = 0; d < 3; ++d) E.v[c][d] = q9[e].Y[corner[c]][d];
  for (int d = 0; d < 3; ++d) {
    E.c[d] = y[d];
    E.nrm[d] = J[d] / dJ;
  }
  E.area = q9[e].area;
  E.hmax = q9[e].hmax;
  el[r] = E;
}

// Entry of one column: dsign = -1 for the mirrored source cell of a
// half-space operator, whose nodes keep their order so that its computed
// normal is -R n (the terms linear in n_y, D and H, change sign).
template <bool SK>
__device__ __forceinline__ cd q9p_entry(cd D, cd H, cd S, cd K, double dsign, double k, cd beta) {
  D = cmulr(D, dsign);
  H = cmulr(H, dsign);
  return SK ? bm_entry_adm(D, H, S, K, k, beta) : bm_entry(D, H, k);
}

// One thread per item (o, r, f): offset o, collocation dof r (el), source
// element f (q9, far_tab: the cell itself, or the mirrored cell of a
// half-space operator); block o goes to out + dest[o] N N (N = ne nb dofs),
// stored by bw.  The items of a dof's own element in the zero offset are
// left to k_q9p_self.
template <bool SK>
__global__ void __launch_bounds__(128) k_q9p_blocks(const Elem* __restrict__ el, const Q9Elem* __restrict__ q9,
                                                    const double* __restrict__ far_tab, int ne, int order,
                                                    const double* __restrict__ shifts,
                                                    const int64_t* __restrict__ dest, int n_off, int zero_off,
                                                    cd* __restrict__ out, double k, cd beta, Q9Rules R,
                                                    double dsign, BlockWrite bw,
                                                    unsigned long long* __restrict__ near_list,
                                                    unsigned long long* __restrict__ near_count,
                                                    unsigned long long near_cap) {
  const Q9Basis B = q9p_basis(order);
  const int nb = B.nb;
  const size_t N = (size_t)ne * nb;
  const size_t per_off = N * ne;
  const size_t total = per_off * (size_t)n_off;
  const size_t sn = (size_t)ne;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int o = (int)(idx / per_off);
    const size_t rem = idx - (size_t)o * per_off;
    const int r = (int)(rem / sn);
    const int f = (int)(rem - (size_t)r * sn);
    if (o == zero_off && r / nb == f) continue;
    const Elem& T = el[r];
    const double x[3] = {T.c[0], T.c[1], T.c[2]};
    const double nx[3] = {T.nrm[0], T.nrm[1], T.nrm[2]};
    const double sh[3] = {shifts[3 * o], shifts[3 * o + 1], shifts[3 * o + 2]};
    const Q9Elem& F = q9[f];
    double dc[3];
    for (int d = 0; d < 3; ++d) dc[d] = x[d] - (F.c[d] + sh[d]);
    const double dist = sqrt(dc[0] * dc[0] + dc[1] * dc[1] + dc[2] * dc[2]);
    cd D[Q9P_MAXNB], H[Q9P_MAXNB], S[Q9P_MAXNB], K[Q9P_MAXNB];
    for (int c = 0; c < Q9P_MAXNB; ++c) D[c] = H[c] = S[c] = K[c] = mkc(0.0, 0.0);
    if (dist >= FAR_RATIO * F.hmax) {
#pragma unroll 1
      for (int p = 0; p < Q9_FAR; ++p) {
        const double* q = far_tab + (size_t)p * 7 * sn + f;
        const double dv[3] = {x[0] - (q[0] + sh[0]), x[1] - (q[sn] + sh[1]), x[2] - (q[2 * sn] + sh[2])};
        const double ny[3] = {q[3 * sn], q[4 * sn], q[5 * sn]};
        cd Dp = mkc(0.0, 0.0), Hp = mkc(0.0, 0.0), Sp = mkc(0.0, 0.0), Kp = mkc(0.0, 0.0);
        q9_kernels<SK>(dv, nx, ny, q[6 * sn], k, Dp, Hp, Sp, Kp);
        double xi, eta, w, Nv[Q9P_MAXNB];
        q9_rule_point(R, 0, p, &xi, &eta, &w);
        q9p_shape(B, xi, eta, Nv, nullptr);
        for (int c = 0; c < nb; ++c) {
          D[c] = cadd(D[c], cmulr(Dp, Nv[c]));
          H[c] = cadd(H[c], cmulr(Hp, Nv[c]));
          if (SK) {
            S[c] = cadd(S[c], cmulr(Sp, Nv[c]));
            K[c] = cadd(K[c], cmulr(Kp, Nv[c]));
          }
        }
      }
    } else {
      if (near_list) {
        const unsigned long long slot = atomicAdd(near_count, 1ull);
        if (slot < near_cap) {
          near_list[slot] = idx;
          continue;
        }
      }
      q9p_near_sum<SK>(F.Y, B, R, dist < NEAR_RATIO * F.hmax, x, nx, sh, k, 0, 1, D, H, S, K);
    }
    cd* row = out + (size_t)dest[o] * N * N + (size_t)r * N + (size_t)f * nb;
    for (int c = 0; c < nb; ++c) bw.put(row + c, q9p_entry<SK>(D[c], H[c], S[c], K[c], dsign, k, beta));
  }
}

// Fixed-order butterfly sum of nb complex accumulators over the warp.
__device__ __forceinline__ void q9p_warp_sum(cd* v, int nb) {
  for (int c = 0; c < nb; ++c)
    for (int off = 16; off > 0; off >>= 1) {
      v[c].x += __shfl_xor_sync(0xffffffffu, v[c].x, off);
      v[c].y += __shfl_xor_sync(0xffffffffu, v[c].y, off);
    }
}

// Near and very-near items listed by k_q9p_blocks, one warp per item; lane c
// stores column c after the reduction.
template <bool SK>
__global__ void __launch_bounds__(256) k_q9p_near(const Elem* __restrict__ el, const Q9Elem* __restrict__ q9, int ne,
                                                  int order, const double* __restrict__ shifts,
                                                  const int64_t* __restrict__ dest,
                                                  const unsigned long long* __restrict__ list,
                                                  const unsigned long long* __restrict__ count,
                                                  unsigned long long cap, cd* __restrict__ out, double k, cd beta,
                                                  Q9Rules R, double dsign, BlockWrite bw) {
  const Q9Basis B = q9p_basis(order);
  const int nb = B.nb;
  const size_t N = (size_t)ne * nb;
  const size_t per_off = N * ne;
  const size_t sn = (size_t)ne;
  const unsigned long long total = min(*count, cap);
  const int lane = threadIdx.x & 31;
  const unsigned long long nwarps = ((unsigned long long)gridDim.x * blockDim.x) >> 5;
  for (unsigned long long w = ((unsigned long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < total;
       w += nwarps) {
    const size_t idx = list[w];
    const int o = (int)(idx / per_off);
    const size_t rem = idx - (size_t)o * per_off;
    const int r = (int)(rem / sn);
    const int f = (int)(rem - (size_t)r * sn);
    const Elem& T = el[r];
    const double x[3] = {T.c[0], T.c[1], T.c[2]};
    const double nx[3] = {T.nrm[0], T.nrm[1], T.nrm[2]};
    const double sh[3] = {shifts[3 * o], shifts[3 * o + 1], shifts[3 * o + 2]};
    const Q9Elem& F = q9[f];
    double dc[3];
    for (int d = 0; d < 3; ++d) dc[d] = x[d] - (F.c[d] + sh[d]);
    const double dist = sqrt(dc[0] * dc[0] + dc[1] * dc[1] + dc[2] * dc[2]);
    cd D[Q9P_MAXNB], H[Q9P_MAXNB], S[Q9P_MAXNB], K[Q9P_MAXNB];
    for (int c = 0; c < Q9P_MAXNB; ++c) D[c] = H[c] = S[c] = K[c] = mkc(0.0, 0.0);
    q9p_near_sum<SK>(F.Y, B, R, dist < NEAR_RATIO * F.hmax, x, nx, sh, k, lane, 32, D, H, S, K);
    q9p_warp_sum(D, nb);
    q9p_warp_sum(H, nb);
    if (SK) {
      q9p_warp_sum(S, nb);
      q9p_warp_sum(K, nb);
    }
    cd* row = out + (size_t)dest[o] * N * N + (size_t)r * N + (size_t)f * nb;
    for (int c = 0; c < nb; ++c)
      if (lane == c) bw.put(row + c, q9p_entry<SK>(D[c], H[c], S[c], K[c], dsign, k, beta));
  }
}

// Self terms, one warp per dof r = e nb + a: row r, columns e nb + c of the
// zero-offset block, with the free term 1/2 (1 + beta) at c = a.
template <bool SK>
__global__ void __launch_bounds__(256) k_q9p_self(const Q9Elem* __restrict__ q9, int ne, int order,
                                                  cd* __restrict__ block0, double k, cd beta, Q9Rules R) {
  const Q9Basis B = q9p_basis(order);
  const int nb = B.nb;
  const size_t N = (size_t)ne * nb;
  const int lane = threadIdx.x & 31;
  const int r = (int)(((size_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  if (r >= (int)N) return;   // uniform across the warp
  const int e = r / nb, a = r - e * nb;
  Q9Node Nd;
  q9p_node_setup(q9[e].Y, B, a, Nd);
  cd D[Q9P_MAXNB], H[Q9P_MAXNB], S[Q9P_MAXNB], K[Q9P_MAXNB];
  for (int c = 0; c < Q9P_MAXNB; ++c) D[c] = H[c] = S[c] = K[c] = mkc(0.0, 0.0);
  for (int it = lane; it < Q9P_THETA; it += 32) q9p_self_theta<SK>(Nd, B, R.t24, R.w24, k, it, D, H, S, K);
  q9p_warp_sum(D, nb);
  q9p_warp_sum(H, nb);
  if (SK) {
    q9p_warp_sum(S, nb);
    q9p_warp_sum(K, nb);
  }
  cd* row = block0 + (size_t)r * N + (size_t)e * nb;
  for (int c = 0; c < nb; ++c)
    if (lane == c) {
      cd t = SK ? bm_entry_adm(D[c], H[c], S[c], K[c], k, beta) : bm_entry(D[c], H[c], k);
      if (c == a) t = cadd(t, mkc(0.5 + 0.5 * beta.x, 0.5 * beta.y));
      row[c] = t;
    }
}

// Scattered pressure at field points added to out[r][p] (which holds the
// incident field): one CTA per (rhs, point), the threads split the (cell,
// element) items, the partial sums are reduced in a fixed order.  With a
// plane, R_p times the same over the mirrored cell (refl: nodes R Y in their
// order), placed for cell c at its position with the axis component
// 2 offset - pos[axis].
template <bool SK>
__global__ void __launch_bounds__(256) k_field_q9(const Q9Elem* __restrict__ q9, const Q9Elem* __restrict__ refl,
                                                  PlaneDev pl, int ne, int order, CellGrid g,
                                                  double k, cd beta, int R, const cd* __restrict__ surf,
                                                  int64_t npts, const double* __restrict__ pts, cd* __restrict__ out,
                                                  Q9Rules Rq) {
  __shared__ double sre[256], sim[256];
  const int nb = order == 0 ? 1 : q9p_basis(order).nb;
  const size_t N = (size_t)ne * nb * g.ncells;
  const cd ikb = mkc(-k * beta.y, k * beta.x);
  const int64_t total = npts * R;
  const int64_t items = (int64_t)g.ncells * ne;
  for (int64_t idx = blockIdx.x; idx < total; idx += gridDim.x) {
    const int r = (int)(idx / npts);
    const int64_t p = idx - (int64_t)r * npts;
    const double x[3] = {pts[3 * p], pts[3 * p + 1], pts[3 * p + 2]};
    cd part = mkc(0.0, 0.0);
    for (int64_t it = threadIdx.x; it < items; it += blockDim.x) {
      const int c = (int)(it / ne), f = (int)(it - (int64_t)c * ne);
      double pos[3];
      g.cell_position(c, pos);
      const Q9Elem& F = q9[f];
      const cd* pd = surf + (size_t)r * N + ((size_t)c * ne + f) * nb;
      part = cadd(part, q9_field_element<SK>(F.Y, F.c, F.hmax, order, Rq, x, pos, k, ikb, 1.0, pd));
      if (pl.on) {
        const Q9Elem& Fm = refl[f];
        pos[pl.axis] = 2.0 * pl.offset - pos[pl.axis];
        part = cfma(pl.Rp, q9_field_element<SK>(Fm.Y, Fm.c, Fm.hmax, order, Rq, x, pos, k, ikb, -1.0, pd), part);
      }
    }
    sre[threadIdx.x] = part.x;
    sim[threadIdx.x] = part.y;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
      if ((int)threadIdx.x < s) {
        sre[threadIdx.x] += sre[threadIdx.x + s];
        sim[threadIdx.x] += sim[threadIdx.x + s];
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) out[idx] = cadd(out[idx], mkc(sre[0], sim[0]));
    __syncthreads();
  }
}

// ------------------------------------------------------------ host side --
fmpb_status field_scattered_q9(const DeviceMesh& m, const DeviceMesh* refl, const PlaneDev& pl, const CellGrid& g,
                               double k, cd beta, int R, const cd* surf, int64_t npts, const double* pts, cd* out,
                               cudaStream_t st) {
  if (m.nodes != 9 || !m.q9 || (pl.on && (!refl || !refl->q9 || refl->q9_ne != m.q9_ne))) {
    set_error("field: not a nine-node mesh, or a half-space operator without its mirrored cell");
    return FMPB_EINVAL;
  }
  const Q9Elem* rq = pl.on ? refl->q9 : m.q9;
  const int64_t total = npts * R;
  if (total <= 0) return FMPB_OK;
  const unsigned blocks = (unsigned)std::min<int64_t>(total, 152 * 16);
  if (beta.x == 0.0 && beta.y == 0.0)
    FMPB_LAUNCH("field_q9", st, k_field_q9<false><<<blocks, 256, 0, st>>>(m.q9, rq, pl, m.q9_ne, m.q9_order, g, k, beta, R, surf, npts, pts, out, m.q9r));
  else
    FMPB_LAUNCH("field_q9_adm", st, k_field_q9<true><<<blocks, 256, 0, st>>>(m.q9, rq, pl, m.q9_ne, m.q9_order, g, k, beta, R, surf, npts, pts, out, m.q9r));
  FMPB_CUDA(cudaGetLastError());
  return FMPB_OK;
}

fmpb_status upload_mesh_q9p(const double* nodes, int64_t nn, const int32_t* elems, int64_t n, int order,
                            DeviceMesh& m, cudaStream_t st) {
  if (order < 0 || order > 2) {
    set_error("mesh: pressure order must be 0, 1 or 2");
    return FMPB_EINVAL;
  }
  FMPB_TRY(upload_mesh_q9(nodes, nn, elems, n, m, st));
  m.q9_ne = (int)n;
  if (order == 0) return FMPB_OK;
  const Q9Basis B = q9p_basis(order);
  const int64_t N = n * B.nb;
  if (N > (1 << 20)) {
    set_error("mesh: %lld pressure dofs per cell exceed 2^20", (long long)N);
    return FMPB_EINVAL;
  }
  cudaFree(m.el);
  m.el = nullptr;
  FMPB_CUDA(cudaMalloc(&m.el, sizeof(Elem) * N));
  FMPB_LAUNCH("q9p_colloc", st, k_q9p_colloc<<<grid_for(N, 128), 128, 0, st>>>(m.q9, (int)n, order, m.el));
  FMPB_CUDA(cudaGetLastError());
  FMPB_CUDA(cudaStreamSynchronize(st));
  m.q9_order = order;
  m.n = (int)N;
  return FMPB_OK;
}

fmpb_status build_blocks_q9p(const DeviceMesh& m, const CellGrid& g, double k, cd beta, int n_off,
                             const int32_t* offsets, const int64_t* dest_host, cd* out, cudaStream_t st,
                             const ImageBlocks* img) {
  const int ne = m.q9_ne, order = m.q9_order;
  const DeviceMesh& src = img ? *img->source : m;
  if (m.nodes != 9 || !m.q9 || order < (img ? 0 : 1) || order > 2 || (int64_t)ne * q9p_basis(order).nb != m.n ||
      src.nodes != 9 || !src.q9 || src.q9_ne != ne || src.q9_order != order) {
    set_error("build_blocks_q9p: not a nine-node mesh with pressure of order 1 or 2 (0 too for image blocks), "
              "or a mirrored cell that differs from it");
    return FMPB_EINVAL;
  }
  const size_t N = (size_t)m.n;
  // shifts: -delta . lattice, or the image shifts given by the caller
  std::vector<double> shifts(3 * (size_t)n_off);
  int zero_off = -1;
  for (int o = 0; o < n_off; ++o) {
    const int32_t* dl = offsets + 3 * o;
    if (!img && dl[0] == 0 && dl[1] == 0 && dl[2] == 0) zero_off = o;
    for (int d = 0; d < 3; ++d)
      shifts[3 * o + d] = img ? img->shifts[3 * o + d]
                              : -(dl[0] * g.L[0][d] + dl[1] * g.L[1][d] + dl[2] * g.L[2][d]);
  }
  const BlockWrite bw = img ? BlockWrite{img->scale, 1, img->accumulate ? 1 : 0} : BlockWrite{mkc(1.0, 0.0), 0, 0};
  const double dsign = img ? -1.0 : 1.0;
  double* dshift = nullptr;
  int64_t* ddest = nullptr;
  FMPB_CUDA(cudaMalloc(&dshift, sizeof(double) * 3 * n_off));
  cudaError_t e = cudaMalloc(&ddest, sizeof(int64_t) * n_off);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(dshift, shifts.data(), sizeof(double) * 3 * n_off, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(ddest, dest_host, sizeof(int64_t) * n_off, cudaMemcpyHostToDevice, st);
  const size_t total = N * (size_t)ne * n_off;
  const unsigned long long near_cap = (unsigned long long)std::min<size_t>(total, (size_t)8 << 20);
  unsigned long long* near_list = nullptr;
  if (e == cudaSuccess) e = cudaMalloc(&near_list, sizeof(unsigned long long) * (near_cap + 1));
  unsigned long long* near_count = near_list ? near_list + near_cap : nullptr;
  if (e == cudaSuccess) e = cudaMemsetAsync(near_count, 0, sizeof(unsigned long long), st);
  if (e == cudaSuccess) {
    const unsigned blocks = (unsigned)std::min<size_t>(grid_for(total, 128), (size_t)152 * 64);
    const unsigned self_blocks = grid_for(N * 32, 256);
    const Q9Rules& R = m.q9r;
    cd* block0 = zero_off >= 0 ? out + (size_t)dest_host[zero_off] * N * N : nullptr;
    if (beta.x == 0.0 && beta.y == 0.0) {
      FMPB_LAUNCH("q9p_blocks", st, k_q9p_blocks<false><<<blocks, 128, 0, st>>>(m.el, src.q9, src.q9_far, ne, order, dshift, ddest, n_off, zero_off, out, k, beta, R, dsign, bw, near_list, near_count, near_cap));
      FMPB_LAUNCH("q9p_near", st, k_q9p_near<false><<<152 * 16, 256, 0, st>>>(m.el, src.q9, ne, order, dshift, ddest, near_list, near_count, near_cap, out, k, beta, R, dsign, bw));
      if (block0) FMPB_LAUNCH("q9p_self", st, k_q9p_self<false><<<self_blocks, 256, 0, st>>>(m.q9, ne, order, block0, k, beta, R));
    } else {
      FMPB_LAUNCH("q9p_blocks_adm", st, k_q9p_blocks<true><<<blocks, 128, 0, st>>>(m.el, src.q9, src.q9_far, ne, order, dshift, ddest, n_off, zero_off, out, k, beta, R, dsign, bw, near_list, near_count, near_cap));
      FMPB_LAUNCH("q9p_near_adm", st, k_q9p_near<true><<<152 * 16, 256, 0, st>>>(m.el, src.q9, ne, order, dshift, ddest, near_list, near_count, near_cap, out, k, beta, R, dsign, bw));
      if (block0) FMPB_LAUNCH("q9p_self_adm", st, k_q9p_self<true><<<self_blocks, 256, 0, st>>>(m.q9, ne, order, block0, k, beta, R));
    }
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(dshift);
  cudaFree(ddest);
  cudaFree(near_list);
  if (e != cudaSuccess) return cuda_status(e, "build_blocks_q9p");
  return FMPB_OK;
}

}  // namespace fmpb
