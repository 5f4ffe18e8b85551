// FMPBEM2 near field (Sec. 3.3): every unique near block S_delta of the
// FMPBEM is replaced by a multilevel FMM over an octree of the unit cell with
// its own truncation number n_t,near.  The product of all near blocks with a
// vector of every cell runs level by level over all cells at once:
//   P2M at the leaves, M2M up (Eq. (m2m)), M2L on the interaction lists of
//   every near offset (Eq. (m2l)), L2L down (Eq. (l2l)), L2P at the leaves,
//   plus the exact entries of the leaf pairs that are not well separated.
//
// Octree.  The root is the cube centred on the midpoint of the bounding box
// of the element centroids, with edge e_0 = its longest side x (1 + 1e-9);
// level l has boxes of edge e_0 / 2^l, and an element belongs to the box
// holding its centroid (indices clamped).  Boxes b (target cell) and b'
// (source cell shifted by s = -delta . L) of level l are well separated when
// |c_b - c_b' - s| >= 3 rho_l (1 - 1e-9), rho_l the largest distance from a
// level-l box centre to a vertex of its elements: Eq. (admissibility) with r
// = 1.5 rho_l, the two-centre expansion ratio at most 2/3 as for the cells.
//
// Translations.  With R(b) the regular translation, I_q(a + b) =
// sum_q' R_qq'(b) I_q'(a), from the coefficient table of Eq. (m2l) evaluated
// with I_l = j_l Y_l in place of O_l (K_reg):
//   R[q'][(n, -m)] = (-1)^m (2n+1)/(2n'+1) K_reg[(n, m)][q'],
//   M2M (child -> parent, b = c_child - c_parent):  T[q][q'] = conj(R[q][q'](b)),
//   L2L (parent -> child, same b):                  T[q'][q] = (2n+1)/(2n'+1) conj(R[q][q'](b)),
// consistent with moments of conj(I) and locals against conj(I) (Eq. (greenFMM)).
#include <algorithm>
#include <cmath>
#include <map>
#include <tuple>
#include <vector>

#include "ff.cuh"
#include "fmm2.cuh"
#include "multipole.cuh"
#include "profile.cuh"

namespace fmpb {

Near2::~Near2() {
  for (void* p : {(void*)parent, (void*)octant, (void*)child_start, (void*)child_idx, (void*)leaf_start,
                  (void*)leaf_elems, (void*)elem_leaf, (void*)V, (void*)U, (void*)Tm2m, (void*)Tl2l,
                  (void*)m2l_start, (void*)m2l_src, (void*)m2l_off, (void*)m2l_k, (void*)K, (void*)p2p_start,
                  (void*)p2p_j, (void*)p2p_off, (void*)p2p_val, (void*)offs})
    if (p) cudaFree(p);
}

// ---------------------------------------------------------------- kernels --
// M2M and L2L blocks from the regular table K_reg (in place of each L x 8
// block): see the header comment for the index map.
__global__ void k_regular_to_m2m_l2l(const cd* __restrict__ Kreg, int nt, int count, cd* __restrict__ Tm2m,
                                     cd* __restrict__ Tl2l) {
  const int B = (nt + 1) * (nt + 1);
  const int64_t total = (int64_t)count * B * B;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int t = (int)(e / ((int64_t)B * B));
    const int rem = (int)(e - (int64_t)t * B * B);
    const int a = rem / B, c = rem - a * B;   // R[a][c]
    int na, ma, nc, mc;
    q_to_nm(a, na, ma);
    q_to_nm(c, nc, mc);
    const int ct = nc * (nc + 1) - mc;        // (n_c, -m_c)
    const cd kv = Kreg[(int64_t)t * B * B + (int64_t)ct * B + a];
    const double sgn = (mc & 1) ? -1.0 : 1.0;
    const cd Rac = cmulr(kv, sgn * (2 * nc + 1) / (double)(2 * na + 1));
    Tm2m[(int64_t)t * B * B + (int64_t)a * B + c] = cconj(Rac);
    Tl2l[(int64_t)t * B * B + (int64_t)c * B + a] = cmulr(cconj(Rac), (2 * na + 1) / (double)(2 * nc + 1));
  }
}

// Mom[col][leaf][q] = sum_{j in leaf} V[q][j] x[col][j]
__global__ void k_near2_p2m(const cd* __restrict__ V, const int* __restrict__ leaf_start,
                            const int* __restrict__ leaf_elems, int nleaf, int leaf_base, int nbox, int n, int B,
                            int64_t columns, const cd* __restrict__ x, cd* __restrict__ Mom) {
  const int64_t total = columns * nleaf * B;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int q = (int)(e % B);
    const int64_t t = e / B;
    const int lf = (int)(t % nleaf);
    const int64_t col = t / nleaf;
    cd acc = mkc(0.0, 0.0);
    for (int p = leaf_start[lf]; p < leaf_start[lf + 1]; ++p) {
      const int j = leaf_elems[p];
      acc = cfma(V[(int64_t)q * n + j], x[col * n + j], acc);
    }
    Mom[(col * nbox + leaf_base + lf) * B + q] = acc;
  }
}

// parents of level l: Mom[col][b][q] = sum_children T_m2m[l][oct] Mom[col][child]
__global__ void k_near2_m2m(const cd* __restrict__ T, const int* __restrict__ child_start,
                            const int* __restrict__ child_idx, const int* __restrict__ octant, int b0, int nb,
                            int nbox, int B, int64_t columns, cd* __restrict__ Mom) {
  const int64_t total = columns * nb * B;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int q = (int)(e % B);
    const int64_t t = e / B;
    const int b = b0 + (int)(t % nb);
    const int64_t col = t / nb;
    cd acc = mkc(0.0, 0.0);
    for (int p = child_start[b]; p < child_start[b + 1]; ++p) {
      const int ch = child_idx[p];
      const cd* Tq = T + ((int64_t)octant[ch] * B + q) * B;
      const cd* mc = Mom + (col * nbox + ch) * B;
      for (int qp = 0; qp < B; ++qp) acc = cfma(Tq[qp], mc[qp], acc);
    }
    Mom[(col * nbox + b) * B + q] = acc;
  }
}

// Loc[col][b][q] = sum over the interaction list of b of K Mom[col - delta][b']
// with K and Mom as float-float pairs (the bulk of the near-field work runs
// on the FP32 pipe; GB300's FP64 rate is 1/58 of it)
__global__ void k_near2_m2l(const float4* __restrict__ K, const int* __restrict__ m2l_start,
                            const int* __restrict__ m2l_src, const int* __restrict__ m2l_off,
                            const int* __restrict__ m2l_k, const int* __restrict__ offs, int nbox, int B, int Mx,
                            int My, int Mz, int64_t columns, const float4* __restrict__ Mom, cd* __restrict__ Loc) {
  const int64_t Nc = (int64_t)Mx * My * Mz;
  const int64_t total = columns * nbox * B;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int q = (int)(e % B);
    const int64_t t = e / B;
    const int b = (int)(t % nbox);
    const int64_t col = t / nbox;
    const int64_t r = col / Nc;
    const int c = (int)(col - r * Nc);
    const int cx = c % Mx, cy = (c / Mx) % My, cz = c / (Mx * My);
    float rh = 0.f, rl = 0.f, ih = 0.f, il = 0.f;
    for (int p = m2l_start[b]; p < m2l_start[b + 1]; ++p) {
      const int* d = offs + 3 * m2l_off[p];
      const int sx = cx - d[0], sy = cy - d[1], sz = cz - d[2];
      if (sx < 0 || sx >= Mx || sy < 0 || sy >= My || sz < 0 || sz >= Mz) continue;
      const int64_t scol = r * Nc + ((int64_t)sz * My + sy) * Mx + sx;
      const float4* Kq = K + ((int64_t)m2l_k[p] * B + q) * B;
      const float4* ms = Mom + (scol * nbox + m2l_src[p]) * B;
      for (int qp = 0; qp < B; ++qp) ff_cmac(Kq[qp], ms[qp], rh, rl, ih, il);
    }
    Loc[(col * nbox + b) * B + q] = mkc((double)rh + (double)rl, (double)ih + (double)il);
  }
}

// children of level l + 1: Loc[col][ch][q'] += sum_q T_l2l[l][oct][q'][q] Loc[col][parent][q]
__global__ void k_near2_l2l(const cd* __restrict__ T, const int* __restrict__ parent, const int* __restrict__ octant,
                            int b0, int nb, int nbox, int B, int64_t columns, cd* __restrict__ Loc) {
  const int64_t total = columns * nb * B;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int q = (int)(e % B);
    const int64_t t = e / B;
    const int ch = b0 + (int)(t % nb);
    const int64_t col = t / nb;
    const cd* Tq = T + ((int64_t)octant[ch] * B + q) * B;
    const cd* lp = Loc + (col * nbox + parent[ch]) * B;
    cd acc = Loc[(col * nbox + ch) * B + q];
    for (int qp = 0; qp < B; ++qp) acc = cfma(Tq[qp], lp[qp], acc);
    Loc[(col * nbox + ch) * B + q] = acc;
  }
}

// y[col][i] = sum_q U[i][q] Loc[col][leaf(i)][q] + sum of the exact entries of
// row i; the exact entries and x as float-float pairs (FP32 pipe)
__global__ void k_near2_l2p_p2p(const cd* __restrict__ U, const int* __restrict__ elem_leaf,
                                const int64_t* __restrict__ p2p_start, const int* __restrict__ p2p_j,
                                const int* __restrict__ p2p_off, const float4* __restrict__ p2p_val,
                                const int* __restrict__ offs, int n, int nbox, int B, int Mx, int My, int Mz,
                                int64_t columns, const cd* __restrict__ Loc, const float4* __restrict__ xff,
                                cd* __restrict__ y) {
  const int64_t Nc = (int64_t)Mx * My * Mz;
  const int64_t total = columns * n;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % n);
    const int64_t col = e / n;
    const cd* Ui = U + (int64_t)i * B;
    const cd* li = Loc + (col * nbox + elem_leaf[i]) * B;
    cd acc = mkc(0.0, 0.0);
    for (int q = 0; q < B; ++q) acc = cfma(Ui[q], li[q], acc);
    const int64_t r = col / Nc;
    const int c = (int)(col - r * Nc);
    const int cx = c % Mx, cy = (c / Mx) % My, cz = c / (Mx * My);
    float rh = 0.f, rl = 0.f, ih = 0.f, il = 0.f;
    for (int64_t p = p2p_start[i]; p < p2p_start[i + 1]; ++p) {
      const int* d = offs + 3 * p2p_off[p];
      const int sx = cx - d[0], sy = cy - d[1], sz = cz - d[2];
      if (sx < 0 || sx >= Mx || sy < 0 || sy >= My || sz < 0 || sz >= Mz) continue;
      const int64_t scol = r * Nc + ((int64_t)sz * My + sy) * Mx + sx;
      ff_cmac(p2p_val[p], xff[scol * n + p2p_j[p]], rh, rl, ih, il);
    }
    y[e] = cadd(acc, mkc((double)rh + (double)rl, (double)ih + (double)il));
  }
}

static unsigned grid_of(int64_t total) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, 152 * 32));
}

size_t near2_scratch_elems(const Near2& t, int64_t columns) { return 2 * (size_t)columns * t.nbox * t.B; }

fmpb_status near2_apply(const Near2& t, const int M[3], int R, const cd* x, const float4* xff, cd* y, cd* scratch,
                        cudaStream_t st) {
  const int64_t columns = (int64_t)R * M[0] * M[1] * M[2];
  const int B = t.B;
  cd* Mom = scratch;
  cd* Loc = scratch + (size_t)columns * t.nbox * B;
  const int L = t.L;
  const int nleaf = t.base[L + 1] - t.base[L];
  FMPB_LAUNCH("near2_p2m", st, k_near2_p2m<<<grid_of(columns * nleaf * B), 256, 0, st>>>(t.V, t.leaf_start, t.leaf_elems, nleaf, t.base[L], t.nbox, t.n, B, columns, x, Mom));
  for (int l = L - 1; l >= 0; --l) {
    const int nb = t.base[l + 1] - t.base[l];
    FMPB_LAUNCH("near2_m2m", st, k_near2_m2m<<<grid_of(columns * nb * B), 256, 0, st>>>(t.Tm2m + (size_t)l * 8 * B * B, t.child_start, t.child_idx, t.octant, t.base[l], nb, t.nbox, B, columns, Mom));
  }
  // the moments as float-float pairs for the M2L products (in place)
  FMPB_TRY(spectrum_to_ff(Mom, (size_t)columns * t.nbox * B, st));
  FMPB_LAUNCH("near2_m2l", st, k_near2_m2l<<<grid_of(columns * t.nbox * B), 256, 0, st>>>(reinterpret_cast<const float4*>(t.K), t.m2l_start, t.m2l_src, t.m2l_off, t.m2l_k, t.offs, t.nbox, B, M[0], M[1], M[2], columns, reinterpret_cast<const float4*>(Mom), Loc));
  for (int l = 0; l < L; ++l) {
    const int nb = t.base[l + 2] - t.base[l + 1];
    FMPB_LAUNCH("near2_l2l", st, k_near2_l2l<<<grid_of(columns * nb * B), 256, 0, st>>>(t.Tl2l + (size_t)l * 8 * B * B, t.parent, t.octant, t.base[l + 1], nb, t.nbox, B, columns, Loc));
  }
  FMPB_LAUNCH("near2_l2p_p2p", st, k_near2_l2p_p2p<<<grid_of(columns * t.n), 256, 0, st>>>(t.U, t.elem_leaf, t.p2p_start, t.p2p_j, t.p2p_off, reinterpret_cast<const float4*>(t.p2p_val), t.offs, t.n, t.nbox, B, M[0], M[1], M[2], columns, Loc, xff, y));
  FMPB_CUDA(cudaGetLastError());
  return FMPB_OK;
}

// ---------------------------------------------------------------- builder --
template <typename T>
static fmpb_status upload(T** dst, const std::vector<T>& h, size_t& bytes, cudaStream_t st) {
  const size_t cnt = std::max<size_t>(h.size(), 1);
  FMPB_CUDA(cudaMalloc((void**)dst, sizeof(T) * cnt));
  bytes += sizeof(T) * cnt;
  if (!h.empty()) FMPB_CUDA(cudaMemcpyAsync(*dst, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice, st));
  return FMPB_OK;
}

fmpb_status near2_plan(const double* verts, const int32_t* tris, int n, const CellGrid& g, int levels, int nt_near,
                       const std::vector<int32_t>& near_off, Near2& t, Near2Host& h, int npe) {
  if (nt_near < 1 || nt_near > MAX_NT) {
    set_error("FMPBEM2: n_t,near must be 1..%d", MAX_NT);
    return FMPB_EINVAL;
  }
  std::vector<double> cen(3 * (size_t)n);
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  for (int j = 0; j < n; ++j)
    for (int d = 0; d < 3; ++d) {
      const double c = npe == 9 ? verts[3 * (int64_t)tris[9 * j + 4] + d]
                                : (verts[3 * tris[3 * j] + d] + verts[3 * tris[3 * j + 1] + d] +
                                   verts[3 * tris[3 * j + 2] + d]) / 3.0;
      cen[3 * j + d] = c;
      lo[d] = std::min(lo[d], c);
      hi[d] = std::max(hi[d], c);
    }
  double c0[3], corner[3], e0 = 0.0;
  for (int d = 0; d < 3; ++d) {
    c0[d] = 0.5 * (lo[d] + hi[d]);
    e0 = std::max(e0, hi[d] - lo[d]);
  }
  e0 *= 1.0 + 1e-9;
  if (!(e0 > 0.0)) e0 = 1.0;   // all centroids at one point: a single box at every level
  for (int d = 0; d < 3; ++d) corner[d] = c0[d] - 0.5 * e0;
  using Key = std::tuple<int, int, int>;
  auto key_of = [&](int l, int j) {
    const double e = e0 / std::ldexp(1.0, l);
    int id[3];
    for (int d = 0; d < 3; ++d) {
      int v = (int)std::floor((cen[3 * j + d] - corner[d]) / e);
      id[d] = std::min(std::max(v, 0), (1 << l) - 1);
    }
    return Key(id[0], id[1], id[2]);
  };
  if (levels <= 0) {   // the shallowest tree with at most 32 elements per leaf on average (depth <= 8)
    levels = 8;
    for (int l = 1; l <= 8; ++l) {
      std::map<Key, int> occ;
      for (int j = 0; j < n; ++j) occ[key_of(l, j)] = 1;
      if ((double)n / occ.size() <= 32.0) {
        levels = l;
        break;
      }
    }
  }
  if (levels > 10) {
    set_error("FMPBEM2: octree depth must be 0..10");
    return FMPB_EINVAL;
  }
  const int L = levels;
  t.L = L;
  t.nt = nt_near;
  t.B = (nt_near + 1) * (nt_near + 1);
  t.n = n;
  t.n_off = (int)(near_off.size() / 3);
  // boxes of every level, ordered by (z, y, x); radius rho_l
  std::vector<std::map<Key, int>> index(L + 1);
  std::vector<std::vector<Key>> keys(L + 1);
  std::vector<double> rho(L + 1, 0.0);
  t.base.assign(L + 2, 0);
  auto centre = [&](int l, const Key& kk, double c[3]) {
    const double e = e0 / std::ldexp(1.0, l);
    const int id[3] = {std::get<0>(kk), std::get<1>(kk), std::get<2>(kk)};
    for (int d = 0; d < 3; ++d) c[d] = corner[d] + (id[d] + 0.5) * e;
  };
  for (int l = 0; l <= L; ++l) {
    std::vector<Key> ks;
    for (int j = 0; j < n; ++j) ks.push_back(key_of(l, j));
    std::vector<Key> u = ks;
    std::sort(u.begin(), u.end(), [](const Key& a, const Key& b) {
      return std::make_tuple(std::get<2>(a), std::get<1>(a), std::get<0>(a)) <
             std::make_tuple(std::get<2>(b), std::get<1>(b), std::get<0>(b));
    });
    u.erase(std::unique(u.begin(), u.end()), u.end());
    keys[l] = u;
    for (size_t b = 0; b < u.size(); ++b) index[l][u[b]] = (int)b;
    for (int j = 0; j < n; ++j) {
      double c[3];
      centre(l, ks[j], c);
      for (int a = 0; a < npe; ++a) {
        const double* v = verts + 3 * (int64_t)tris[(int64_t)npe * j + a];
        const double dx = v[0] - c[0], dy = v[1] - c[1], dz = v[2] - c[2];
        rho[l] = std::max(rho[l], std::sqrt(dx * dx + dy * dy + dz * dz));
      }
    }
    t.base[l + 1] = t.base[l] + (int)u.size();
  }
  t.nbox = t.base[L + 1];
  // parents, octants, children
  std::vector<int> parent(t.nbox, -1), octant(t.nbox, 0), cstart(t.nbox + 1, 0), cidx;
  std::vector<std::vector<int>> ch(t.nbox);
  for (int l = 1; l <= L; ++l)
    for (size_t b = 0; b < keys[l].size(); ++b) {
      const Key& kk = keys[l][b];
      const Key pk(std::get<0>(kk) / 2, std::get<1>(kk) / 2, std::get<2>(kk) / 2);
      const int gid = t.base[l] + (int)b, pg = t.base[l - 1] + index[l - 1][pk];
      parent[gid] = pg;
      octant[gid] = (std::get<0>(kk) & 1) + 2 * (std::get<1>(kk) & 1) + 4 * (std::get<2>(kk) & 1);
      ch[pg].push_back(gid);
    }
  for (int b = 0; b < t.nbox; ++b) {
    cstart[b + 1] = cstart[b] + (int)ch[b].size();
    cidx.insert(cidx.end(), ch[b].begin(), ch[b].end());
  }
  // leaves: elements and leaf centres
  const int nleaf = t.base[L + 1] - t.base[L];
  std::vector<std::vector<int>> lel(nleaf);
  std::vector<int> elem_leaf(n);
  std::vector<double> lcen(3 * (size_t)n);
  for (int j = 0; j < n; ++j) {
    const Key kk = key_of(L, j);
    const int lf = index[L][kk];
    lel[lf].push_back(j);
    elem_leaf[j] = t.base[L] + lf;
    centre(L, kk, &lcen[3 * j]);
  }
  std::vector<int> lstart(nleaf + 1, 0), lelems;
  for (int lf = 0; lf < nleaf; ++lf) {
    lstart[lf + 1] = lstart[lf] + (int)lel[lf].size();
    lelems.insert(lelems.end(), lel[lf].begin(), lel[lf].end());
  }
  // interaction lists of every near offset (pairs reached from the roots)
  struct M2LEntry {
    int tgt, src, off, kid;
  };
  std::vector<M2LEntry> m2l;
  std::map<std::tuple<int, int, int, int, int>, int> kid_of;   // (level, dkey x3, offset)
  std::vector<double> dvecs;
  std::vector<std::vector<std::pair<int, int>>> prow(n);        // per target element: (off, j)
  for (int o = 0; o < t.n_off; ++o) {
    const int32_t* dl = &near_off[3 * o];
    double s[3];
    for (int d = 0; d < 3; ++d) s[d] = -(dl[0] * g.L[0][d] + dl[1] * g.L[1][d] + dl[2] * g.L[2][d]);
    std::vector<std::tuple<int, int, int>> stack{{0, 0, 0}};   // (level, local a, local b)
    while (!stack.empty()) {
      const auto [l, a, b] = stack.back();
      stack.pop_back();
      double ca[3], cb[3], dv[3];
      centre(l, keys[l][a], ca);
      centre(l, keys[l][b], cb);
      for (int d = 0; d < 3; ++d) dv[d] = ca[d] - (cb[d] + s[d]);
      const double dist = std::sqrt(dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2]);
      if (dist >= 3.0 * rho[l] * (1.0 - 1e-9)) {
        const Key& ka = keys[l][a];
        const Key& kb = keys[l][b];
        const auto kk = std::make_tuple(l, std::get<0>(ka) - std::get<0>(kb), std::get<1>(ka) - std::get<1>(kb),
                                        std::get<2>(ka) - std::get<2>(kb), o);
        auto it = kid_of.find(kk);
        int kid;
        if (it == kid_of.end()) {
          kid = (int)kid_of.size();
          kid_of[kk] = kid;
          for (int d = 0; d < 3; ++d) dvecs.push_back(ca[d] - cb[d] - s[d]);
        } else {
          kid = it->second;
        }
        m2l.push_back({t.base[l] + a, t.base[l] + b, o, kid});
      } else if (l == L) {
        for (int i : lel[a])
          for (int j : lel[b]) prow[i].push_back({o, j});
      } else {
        for (int ca_ : ch[t.base[l] + a])
          for (int cb_ : ch[t.base[l] + b]) stack.emplace_back(l + 1, ca_ - t.base[l + 1], cb_ - t.base[l + 1]);
      }
    }
  }
  // M2L lists by target box
  std::stable_sort(m2l.begin(), m2l.end(), [](const M2LEntry& a, const M2LEntry& b) { return a.tgt < b.tgt; });
  std::vector<int> mstart(t.nbox + 1, 0), msrc, moff, mk;
  for (const auto& e : m2l) {
    ++mstart[e.tgt + 1];
    msrc.push_back(e.src);
    moff.push_back(e.off);
    mk.push_back(e.kid);
  }
  for (int b = 0; b < t.nbox; ++b) mstart[b + 1] += mstart[b];
  t.n_m2l = (int64_t)m2l.size();
  t.n_k = (int64_t)kid_of.size();
  // exact entries by target element; the slot of each (i, i) of the zero offset
  std::vector<int64_t> pstart(n + 1, 0), plist, self_slot(n, -1);
  std::vector<int> pj, poff;
  int zero_off = -1;
  for (int o = 0; o < t.n_off; ++o)
    if (near_off[3 * o] == 0 && near_off[3 * o + 1] == 0 && near_off[3 * o + 2] == 0) zero_off = o;
  for (int i = 0; i < n; ++i) {
    for (const auto& [o, j] : prow[i]) {
      if (o == zero_off && j == i) self_slot[i] = (int64_t)plist.size();
      plist.push_back(((int64_t)o * n + i) * n + j);
      pj.push_back(j);
      poff.push_back(o);
    }
    pstart[i + 1] = (int64_t)plist.size();
  }
  t.n_p2p = (int64_t)plist.size();
  h.parent = std::move(parent);
  h.octant = std::move(octant);
  h.cstart = std::move(cstart);
  h.cidx = std::move(cidx);
  h.lstart = std::move(lstart);
  h.lelems = std::move(lelems);
  h.elem_leaf = std::move(elem_leaf);
  h.lcen = std::move(lcen);
  h.mstart = std::move(mstart);
  h.msrc = std::move(msrc);
  h.moff = std::move(moff);
  h.mk = std::move(mk);
  h.dvecs = std::move(dvecs);
  h.pstart = std::move(pstart);
  h.plist = std::move(plist);
  h.pj = std::move(pj);
  h.poff = std::move(poff);
  h.self_slot = std::move(self_slot);
  h.e0 = e0;
  return FMPB_OK;
}

fmpb_status near2_build(const DeviceMesh& m, const CellGrid& g, const double* verts, const int32_t* tris, double k,
                        cd beta, int levels, int nt_near, const std::vector<int32_t>& near_off, Near2& t,
                        cudaStream_t st) {
  const int n = m.n;
  Near2Host h;
  FMPB_TRY(near2_plan(verts, tris, n, g, levels, nt_near, near_off, t, h, m.nodes));
  const int L = t.L, B = t.B;
  const double e0 = h.e0;
  const auto &parent = h.parent, &octant = h.octant, &cstart = h.cstart, &cidx = h.cidx, &lstart = h.lstart,
             &lelems = h.lelems, &elem_leaf = h.elem_leaf, &mstart = h.mstart, &msrc = h.msrc, &moff = h.moff,
             &mk = h.mk, &pj = h.pj, &poff = h.poff;
  const auto& lcen = h.lcen;
  const auto& dvecs = h.dvecs;
  const auto &pstart = h.pstart, &plist = h.plist, &self_slot = h.self_slot;
  // device structure
  size_t& by = t.bytes;
  FMPB_TRY(upload(&t.parent, parent, by, st));
  FMPB_TRY(upload(&t.octant, octant, by, st));
  FMPB_TRY(upload(&t.child_start, cstart, by, st));
  FMPB_TRY(upload(&t.child_idx, cidx, by, st));
  FMPB_TRY(upload(&t.leaf_start, lstart, by, st));
  FMPB_TRY(upload(&t.leaf_elems, lelems, by, st));
  FMPB_TRY(upload(&t.elem_leaf, elem_leaf, by, st));
  FMPB_TRY(upload(&t.m2l_start, mstart, by, st));
  FMPB_TRY(upload(&t.m2l_src, msrc, by, st));
  FMPB_TRY(upload(&t.m2l_off, moff, by, st));
  FMPB_TRY(upload(&t.m2l_k, mk, by, st));
  FMPB_TRY(upload(&t.p2p_start, pstart, by, st));
  FMPB_TRY(upload(&t.p2p_j, pj, by, st));
  FMPB_TRY(upload(&t.p2p_off, poff, by, st));
  FMPB_TRY(upload(&t.offs, std::vector<int>(near_off.begin(), near_off.end()), by, st));
  // tables: P2M / L2P about the leaf centres
  double* dcen = nullptr;
  FMPB_CUDA(cudaMallocAsync(&dcen, sizeof(double) * 3 * n, st));
  FMPB_CUDA(cudaMemcpyAsync(dcen, lcen.data(), sizeof(double) * 3 * n, cudaMemcpyHostToDevice, st));
  FMPB_CUDA(cudaMalloc(&t.V, sizeof(cd) * (size_t)B * n));
  FMPB_CUDA(cudaMalloc(&t.U, sizeof(cd) * (size_t)B * n));
  by += 2 * sizeof(cd) * (size_t)B * n;
  FMPB_TRY(multipole_tables(m, k, beta, nt_near, t.V, t.U, st, dcen));
  // M2M / L2L of every level and octant from the regular table
  const int ntr = std::max(1, 8 * L);
  FMPB_CUDA(cudaMalloc(&t.Tm2m, sizeof(cd) * (size_t)ntr * B * B));
  FMPB_CUDA(cudaMalloc(&t.Tl2l, sizeof(cd) * (size_t)ntr * B * B));
  by += 2 * sizeof(cd) * (size_t)ntr * B * B;
  if (L > 0) {
    std::vector<double> bv;
    std::vector<int64_t> dest;
    for (int l = 0; l < L; ++l) {
      const double e = e0 / std::ldexp(1.0, l + 1);
      for (int oc = 0; oc < 8; ++oc) {
        bv.push_back(((oc & 1) - 0.5) * e);
        bv.push_back((((oc >> 1) & 1) - 0.5) * e);
        bv.push_back((((oc >> 2) & 1) - 0.5) * e);
        dest.push_back((int64_t)dest.size());
      }
    }
    cd* Kreg = nullptr;
    FMPB_CUDA(cudaMallocAsync(&Kreg, sizeof(cd) * (size_t)ntr * B * B, st));
    FMPB_TRY(m2l_blocks(nt_near, k, ntr, bv.data(), dest.data(), Kreg, st, true));
    FMPB_LAUNCH("near2_translations", st, k_regular_to_m2m_l2l<<<grid_of((int64_t)ntr * B * B), 256, 0, st>>>(Kreg, nt_near, ntr, t.Tm2m, t.Tl2l));
    FMPB_CUDA(cudaFreeAsync(Kreg, st));
  }
  // M2L blocks of the unique translations
  FMPB_CUDA(cudaMalloc(&t.K, sizeof(cd) * (size_t)std::max<int64_t>(t.n_k, 1) * B * B));
  by += sizeof(cd) * (size_t)std::max<int64_t>(t.n_k, 1) * B * B;
  if (t.n_k > 0) {
    std::vector<int64_t> dest(t.n_k);
    for (int64_t i = 0; i < t.n_k; ++i) dest[i] = i;
    FMPB_TRY(m2l_blocks(nt_near, k, (int)t.n_k, dvecs.data(), dest.data(), t.K, st));
    FMPB_TRY(spectrum_to_ff(t.K, (size_t)t.n_k * B * B, st));   // read as float-float pairs
  }
  // exact entries of the leaf pairs that are not well separated
  FMPB_CUDA(cudaMalloc(&t.p2p_val, sizeof(cd) * (size_t)std::max<int64_t>(t.n_p2p, 1)));
  by += sizeof(cd) * (size_t)std::max<int64_t>(t.n_p2p, 1);
  if (t.n_p2p > 0) {
    int64_t* dlist = nullptr;
    int64_t* dslot = nullptr;
    FMPB_CUDA(cudaMallocAsync(&dlist, sizeof(int64_t) * t.n_p2p, st));
    FMPB_CUDA(cudaMallocAsync(&dslot, sizeof(int64_t) * n, st));
    FMPB_CUDA(cudaMemcpyAsync(dlist, plist.data(), sizeof(int64_t) * t.n_p2p, cudaMemcpyHostToDevice, st));
    FMPB_CUDA(cudaMemcpyAsync(dslot, self_slot.data(), sizeof(int64_t) * n, cudaMemcpyHostToDevice, st));
    FMPB_TRY(build_entries(m, g, k, beta, t.n_off, near_off.data(), dlist, t.n_p2p, dslot, t.p2p_val, st));
    FMPB_TRY(spectrum_to_ff(t.p2p_val, (size_t)t.n_p2p, st));   // read as float-float pairs
    FMPB_CUDA(cudaFreeAsync(dlist, st));
    FMPB_CUDA(cudaFreeAsync(dslot, st));
  }
  FMPB_CUDA(cudaFreeAsync(dcen, st));
  FMPB_CUDA(cudaStreamSynchronize(st));
  return FMPB_OK;
}

}  // namespace fmpb
