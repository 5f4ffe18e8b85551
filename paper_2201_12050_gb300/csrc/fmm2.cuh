// FMPBEM2 near field (fmm2.cu): the unique near blocks S_delta of the FMPBEM
// approximated by a multilevel FMM over an octree of the unit cell (Sec. 3.3).
#pragma once
#include <vector>

#include "common.cuh"
#include "internal.cuh"

namespace fmpb {

// Device tables of the multilevel near field; boxes of all levels are
// numbered together (level l holds global ids base[l] .. base[l+1]-1).
struct Near2 {
  int L = 0, nt = 0, B = 0, n = 0, n_off = 0;
  int nbox = 0;                       // boxes of all levels
  std::vector<int> base;              // L + 2 entries
  int* parent = nullptr;              // [nbox] global id of the parent (-1 at the root)
  int* octant = nullptr;              // [nbox] child octant within the parent
  int* child_start = nullptr;         // [nbox + 1] CSR of the children
  int* child_idx = nullptr;
  int* leaf_start = nullptr;          // [nleaf + 1] CSR of the elements of each leaf
  int* leaf_elems = nullptr;
  int* elem_leaf = nullptr;           // [n] global id of each element's leaf
  cd* V = nullptr;                    // B x n, P2M about each element's leaf centre
  cd* U = nullptr;                    // n x B, L2P about each element's leaf centre
  cd* Tm2m = nullptr;                 // L x 8 x B x B: child (level l+1) -> parent (level l)
  cd* Tl2l = nullptr;                 // L x 8 x B x B: parent (level l) -> child (level l+1)
  int* m2l_start = nullptr;           // [nbox + 1] CSR by target box
  int* m2l_src = nullptr;             // source box (global id)
  int* m2l_off = nullptr;             // near offset index
  int* m2l_k = nullptr;               // translation block index
  cd* K = nullptr;                    // n_k x B x B M2L blocks (float-float pairs)
  int64_t n_m2l = 0, n_k = 0;
  int64_t* p2p_start = nullptr;       // [n + 1] CSR by target element
  int* p2p_j = nullptr;               // source element
  int* p2p_off = nullptr;             // near offset index
  cd* p2p_val = nullptr;              // exact entries (float-float pairs)
  int64_t n_p2p = 0;
  int* offs = nullptr;                // n_off x 3 near offsets
  size_t bytes = 0;
  ~Near2();
};

// Host half of the build: the octree, the interaction lists and the exact
// entries' indices (no CUDA call).  Fills the scalar fields and `base` of t.
struct Near2Host {
  std::vector<int> parent, octant, cstart, cidx, lstart, lelems, elem_leaf, mstart, msrc, moff, mk, pj, poff;
  std::vector<double> lcen, dvecs;
  std::vector<int64_t> pstart, plist, self_slot;
  double e0 = 0.0;
};
// npe: nodes per element (3: triangles, centroid; 9: nine-node
// quadrilaterals, the centre node 4); box radii run over all of them.
fmpb_status near2_plan(const double* verts, const int32_t* tris, int n, const CellGrid& g, int levels, int nt_near,
                       const std::vector<int32_t>& near_off, Near2& t, Near2Host& h, int npe = 3);

// Builds the tree, the interaction lists of every near offset and the device
// tables (Sec. 3.3, Eqs. (m2m), (m2l), (l2l)).  verts/tris: the host mesh;
// levels: octree depth L >= 0 (0 picks the depth giving about 32 elements
// per leaf); nt_near: truncation of the expansions.
fmpb_status near2_build(const DeviceMesh& m, const CellGrid& g, const double* verts, const int32_t* tris, double k,
                        cd beta, int levels, int nt_near, const std::vector<int32_t>& near_off, Near2& out,
                        cudaStream_t st);

// y (=) sum_delta S~_delta x_{c - delta} for R right-hand sides (complex
// double, cell-major; xff: the same vector as float-float pairs); scratch:
// near2_scratch_elems complex values.
size_t near2_scratch_elems(const Near2& t, int64_t columns);
fmpb_status near2_apply(const Near2& t, const int M[3], int R, const cd* x, const float4* xff, cd* y, cd* scratch,
                        cudaStream_t st);

}  // namespace fmpb
