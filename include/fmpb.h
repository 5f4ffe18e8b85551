/*
 * fmpb.h -- C ABI of the GB300 finite-periodic fast multipole BEM library.
 *
 * Method: Jelich, Zhao, Chen, Marburg, "Fast multipole boundary element
 * method for the acoustic analysis of finite periodic structures"
 * (arXiv 2201.12050).  A unit-cell boundary mesh is repeated on a lattice of
 * M_x x M_y x M_z cells (Sec. 2.2).  The Burton-Miller collocation operator
 * of a rigid boundary (Sec. 2.1, Eq. (bm) with dp/dn = 0) is applied either
 *   - in the FMPBEM form S + U K V (Sec. 3.2, Eq. (2dPeriodicFMM)): the
 *     near-field blocks S_delta (|delta|_inf <= 1), the P2M/L2P tables V_0,
 *     U_0 shared by all cells and the multilevel block Toeplitz M2L matrix K,
 *     or
 *   - in the PBEM form T (Sec. 2.2, Eq. (toeplitzBEM)): one dense n x n block
 *     per cell offset,
 * and every block Toeplitz product is evaluated as a zero-padded block
 * circulant convolution by FFT over the cell grid (Sec. 2.4, Eqs.
 * (diagonalized), (modifiedFourierTransform1/2); Sec. 3.5, Eq.
 * (FMPBEMsystem)).
 *
 * Conventions shared by every call
 *   - Complex numbers are interleaved doubles (fmpb_c64), the layout of
 *     torch.complex128 and std::complex<double>.
 *   - A cell is c = (iz*M_y + iy)*M_x + ix; dof i of cell c has global
 *     index c*n + i (n = triangles of the unit cell).  Vectors with R
 *     right-hand sides are RHS-major: element (r, c*n + i) at r*N + c*n + i.
 *   - Pointer arguments documented "device" must point to memory of the
 *     current CUDA device; "host" pointers are read before the call returns.
 *     The caller owns every buffer it passes; the library never frees them.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Work is
 *     enqueued on it; calls returning device results do not synchronise
 *     unless documented.  Calls on one operator share its scratch memory
 *     and must be ordered on one stream.
 *   - Every call returns a status.  No call aborts, traps or prints.  On
 *     error the outputs are undefined (except FMPB_ENOCONV, see
 *     fmpb_solve) and fmpb_last_error() describes the failure.
 */
#ifndef FMPB_H
#define FMPB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FMPB_VERSION_MAJOR 0
#define FMPB_VERSION_MINOR 1

typedef struct { double re, im; } fmpb_c64;

typedef enum {
  FMPB_OK = 0,
  FMPB_EINVAL = -1,    /* invalid argument (null pointer, size, option) */
  FMPB_ENOMEM = -2,    /* device or host allocation failed */
  FMPB_EMESH = -3,     /* bad mesh: index out of range, degenerate triangle */
  FMPB_EADMISS = -4,   /* FMM form forced on a cell the expansion cannot separate */
  FMPB_ENOCONV = -5,   /* GMRES reached maxit before the tolerance */
  FMPB_ETIMEOUT = -6,  /* a bounded wait expired */
  FMPB_ENAN = -7,      /* NaN or Inf in an input vector */
  FMPB_ECUDA = -8      /* a CUDA runtime call failed */
} fmpb_status;

/* FMPB_FORM_FMM2: the FMM form with every unique near block approximated by
 * a multilevel FMM over an octree of the unit cell (FMPBEM2, Sec. 3.3). */
typedef enum { FMPB_FORM_AUTO = -1, FMPB_FORM_FMM = 0, FMPB_FORM_PBEM = 1, FMPB_FORM_FMM2 = 2 } fmpb_form;
/* FP64: spectrum and tables as float-float pairs (FP64-class accuracy).
 * FP32: spectrum in complex FP32 (half the bytes per product).
 * BF16: FMM form only.  Near-field blocks and P2M/L2P tables rounded to
 *       BF16 (FP64 -> FP32 -> BF16, nearest even each time) and applied on
 *       the tensor cores with FP32 accumulation (see fmpb_offset_gemm_bf16);
 *       the input vector is rounded the same way per product.  M2L spectrum
 *       in complex FP32.  Relative error of a product about 1e-3.
 * MIXED: both spectra; fmpb_matvec uses the accurate one and fmpb_solve
 *        runs GMRES-IR (inner solves on the FP32 spectrum, accurate outer
 *        residuals).  In the FMM form the inner products also run the near
 *        field, P2M and L2P on the tensor cores as BF16 does, and the operator
 *        keeps both the float-float and the BF16 tables. */
typedef enum { FMPB_FP64 = 0, FMPB_FP32 = 1, FMPB_BF16 = 2, FMPB_MIXED = 3 } fmpb_precision;

/* Incident fields: a plane wave amp e^{i k d.x} (Eq. (planewave); vec = unit
 * direction d) or a monopole amp e^{i k r}/r, r = |x - x_s| (vec = source
 * position x_s; amp is the pressure amplitude at 1 m; the source must not
 * lie on the surface). */
/* Boundary elements (Sec. 2.1): flat three-node triangles, or the paper's
 * nine-node quadratic quadrilaterals.  Both carry one constant pressure per
 * element, collocated at the centroid (triangle) or at the parameter centre
 * y(0, 0) (quadrilateral). */
typedef enum { FMPB_ELEM_TRI3 = 0, FMPB_ELEM_QUAD9 = 1 } fmpb_element;

typedef enum { FMPB_INC_PLANE = 0, FMPB_INC_MONOPOLE = 1 } fmpb_incident_kind;
typedef struct {
  int32_t kind;      /* fmpb_incident_kind */
  double vec[3];
  fmpb_c64 amp;
} fmpb_incident;

/* Finite lattice (Sec. 2.2, Fig. PeriodicArray2d): counts[a] cells along
 * lattice vector vectors[a] (metres).  counts[a] = 1 for an unused axis. */
typedef struct {
  int32_t counts[3];
  double vectors[3][3];
} fmpb_lattice;

/* Human-readable description of the last error on the calling thread; valid
 * until the next library call on that thread.  Never NULL. */
const char *fmpb_last_error(void);
/* Library version as (major << 16) | minor. */
int fmpb_version(void);

/* ------------------------------------------------------------------------
 * Operator: everything the matrix-vector product needs for one
 * (unit-cell mesh, lattice, wavenumber), resident on the current device.
 * ---------------------------------------------------------------------- */
typedef struct fmpb_operator fmpb_operator;

typedef struct {
  int form;        /* fmpb_form; AUTO picks FMM when the nearest far cell
                      (|delta|_inf >= 2) lies at least 3 cell radii away, so that
                      the two-centre expansion of Eq. (greenFMM) converges with
                      ratio 2 rho / |d| <= 2/3; else PBEM.  FMM forced with
                      |d| <= 2 rho is refused (EADMISS). */
  int n_t;         /* truncation number of the FMM form (Eq. (greenFMM)), 1..20;
                      0 = the truncation rule: the smallest n_t in 4..20 whose
                      U_0 K(d) V_0 reproduces the exact collocation block of
                      the nearest far cell d (max-norm offset >= 2, shortest
                      translation) on four fixed probe vectors
                      x_j = exp(2 pi i frac((p+1) j phi)), phi = (sqrt 5 - 1)/2,
                      p < 4, to a relative 1e-6 (Frobenius norm over the
                      probes).  If none does, AUTO falls back to the PBEM
                      form and a forced FMM form takes n_t = 20.  A grid
                      without far cells takes 4.  fmpb_operator_info reports
                      the n_t chosen. */
  int precision;   /* fmpb_precision: FMPB_FP64 (default), FMPB_FP32, FMPB_BF16
                      (FMM form only) or FMPB_MIXED */
  /* Uniform normalised surface admittance beta = beta_re + i beta_im
   * (Eq. (admittance): dp/dn = i k beta p with n out of the fluid, i.e.
   * dp/dn_m = -i k beta p with the mesh normal); 0 + 0i (the value of a
   * zero-initialised struct) is the rigid surface.  The matrix gains
   * (beta/2) delta_ij - i k beta (S_ij + (i/k) K_ij) with S = int G and
   * K = int dG/dn_x (Eq. (bm), Eq. (matrixBEM)); the FMM form adds
   * i k beta int conj(I) dA to the P2M table. */
  double beta_re;
  double beta_im;
  /* Half-space (Sec. 2.3, Eq. (green3dHalf)): halfspace = 1 replaces G by
   * G_h(x, y) = G(x, y) + R_p G(x, y^), y^ the mirror image of y in the plane
   * {x : x[plane_axis] = plane_offset}; 0 (zero-initialised) is full space.
   * Every lattice axis with more than one cell must be parallel to the plane
   * or perpendicular to it (at most one); a perpendicular axis makes the image
   * part a block Hankel matrix (Eq. (blockToeplizMatrixSymmetry)), applied as
   * the block Toeplitz product of the cell-reversed vector (Sec. 2.4).  The
   * mesh of every cell must lie on one side of the plane (touching allowed).
   * The image part is stored beside the full-space one (PBEM form with a
   * perpendicular axis: a second spectrum; FMM form: image near blocks, a
   * P2M table of the mirrored cell and a second M2L spectrum, Eq.
   * (2dPeriodicFMM_halfspace)); PBEM with the lattice parallel to the plane
   * adds the image blocks to the one block Toeplitz pattern.  Precisions
   * FP64, FP32, and MIXED in the PBEM form. */
  int32_t halfspace;
  int32_t plane_axis;   /* 0, 1, 2 */
  double plane_offset;
  double Rp_re;         /* reflection coefficient R_p (1: rigid plane, -1: soft) */
  double Rp_im;
  /* FMPBEM2 form (FMPB_FORM_FMM2, FP64, full space): truncation number
   * n_t,near of the multilevel near field (0: 6) and the depth of the cell's
   * octree (0: the shallowest with at most 32 elements per leaf on average).
   * The root is the cube on the centroids' bounding box; boxes of a level are
   * well separated at centre distance >= 3 x their largest centre-to-vertex
   * distance (Eq. (admissibility)); pairs that never are keep their exact
   * entries (P2P). */
  int32_t n_t_near;
  int32_t near_levels;
  /* fmpb_element of the mesh (0, zero-initialised: flat triangles).  With
   * FMPB_ELEM_QUAD9 `tris` holds ntri x 9 node indices per element (node
   * (i, j) of its 3 x 3 grid at 3 j + i, i along xi, parameter values -1, 0,
   * 1; y_xi x y_eta into the fluid).  Such operators run in the PBEM form
   * (FP64, FP32 or MIXED; AUTO picks it) or the FMM form (FP64 or FP32; its
   * P2M table integrates each element with the 4 x 4 far-class rule and each
   * point's normal), in full or half space.  Field points and the
   * insertion loss take every pressure order, in full and half space. */
  int32_t element;
  /* Order of the discontinuous pressure on FMPB_ELEM_QUAD9 elements (0,
   * zero-initialised: one constant per element at its centre; 1: 2 x 2 nodes
   * at +-1/sqrt(3), bilinear; 2: the eight-node serendipity element on
   * [-sqrt(3/5), sqrt(3/5)]^2), collocated at the nodes with dof e nb + a.
   * Every order runs the PBEM and FMM forms of FMPB_ELEM_QUAD9 (the P2M table
   * weights the far rule by each shape N_b). */
  int32_t pressure_order;
} fmpb_operator_opts;

typedef struct {
  int64_t n;             /* triangles (dofs) per cell */
  int64_t n_cells;       /* M_x M_y M_z */
  int64_t N;             /* n * n_cells */
  int32_t dim;           /* lattice axes with more than one cell */
  int32_t form;          /* fmpb_form actually built */
  int32_t n_t;           /* truncation number (FMM form), 0 for PBEM */
  int64_t B;             /* circulant block size: (n_t+1)^2 (FMM) or n (PBEM) */
  int32_t P[3];          /* padded circulant length per axis, >= 2 M_a - 1 */
  int64_t F;             /* P[0] P[1] P[2] */
  int32_t n_near;        /* near offsets stored (3^dim) in the FMM form, else 0 */
  size_t bytes_device;   /* device memory held by the operator (tables only) */
  int32_t precision;     /* fmpb_precision of the stored spectrum(s) */
  double beta_re;        /* surface admittance the operator was built with */
  double beta_im;
  int32_t halfspace;     /* 1 for a half-space operator */
  int32_t hankel_axis;   /* lattice axis perpendicular to the plane, -1 if none */
  int32_t n_near_image;  /* image offsets evaluated exactly (FMM form), else 0 */
  int32_t image_separate;/* 1 if the image part has its own tables and products */
  int32_t near_levels;   /* FMPBEM2: octree depth, else 0 */
  int64_t n_m2l_near;    /* FMPBEM2: M2L pairs over all near offsets */
  int64_t n_p2p_near;    /* FMPBEM2: exact entries kept */
  int32_t element;       /* fmpb_element of the mesh */
  int32_t pressure_order;/* pressure order of FMPB_ELEM_QUAD9 elements (n = elements x nodes) */
  double n_t_rule_err;   /* the truncation rule's relative probe error at the n_t
                            chosen (n_t = 0 requested), else -1 */
} fmpb_operator_info;

/*
 * Builds the operator on the current device.
 *   verts  host, nv x 3 doubles: unit-cell vertex coordinates (metres).  The
 *          mesh origin is the cell's expansion centre.
 *   tris   host, ntri x 3 int32: vertex indices of each flat triangle, wound
 *          so that (v1-v0) x (v2-v0) points from the body into the fluid
 *          (ntri x 9 node indices with opts->element = FMPB_ELEM_QUAD9).
 *   k      wavenumber omega/c > 0 (Eq. (helmholtz)).
 *   opts   may be NULL (AUTO form, the truncation rule for n_t, FP64).
 * Builds, all on the device: element geometry and quadrature rules; the
 * offset blocks (all (2M-1)^d offsets in the PBEM form, the 3^d near offsets
 * in the FMM form) by the collocation quadrature of Eq. (bm); in the FMM
 * form the P2M/L2P tables (Eqs. (p2m), (l2p)) and the M2L blocks of every
 * far offset (Eqs. (m2l), (wigner)); finally the FFT of the circulant first
 * block column over the padded cell grid (Eq. (blockDiagonal)).  The input
 * arrays are copied; the stream is synchronised before return.
 * Errors: EINVAL (sizes, k <= 0, options), EMESH (index out of range or
 * zero-area triangle), EADMISS (FMM forced but not admissible), ENOMEM,
 * ECUDA.  *out is set only on success and is freed by
 * fmpb_operator_destroy.
 */
fmpb_status fmpb_operator_create(const double *verts, int64_t nv, const int32_t *tris, int64_t ntri,
                                 const fmpb_lattice *lattice, double k,
                                 const fmpb_operator_opts *opts, void *stream,
                                 fmpb_operator **out);
fmpb_status fmpb_operator_get_info(const fmpb_operator *op, fmpb_operator_info *info);
/* Frees the operator's device memory (synchronises the device first).  NULL is a no-op. */
void fmpb_operator_destroy(fmpb_operator *op);

/*
 * Right-hand side of Eq. (bm) for R incident plane waves
 * p_inc = amp_r exp(i k d_r . x) (Eq. (planewave)):
 * b_r(x_i) = p_inc(x_i) + (i/k) dp_inc/dn(x_i) at every collocation point.
 *   dirs  host, R x 3 unit vectors; amps host, R values (NULL = all 1).
 *   b     device, R x N.
 */
fmpb_status fmpb_rhs_plane_wave(const fmpb_operator *op, int R, const double *dirs,
                                const fmpb_c64 *amps, fmpb_c64 *b, void *stream);
/*
 * Right-hand sides of R incident fields of any kind (fmpb_incident, host
 * array of R), with their images R_p p_inc(M x) for a half-space operator:
 * b_r(x_i) = p_inc(x_i) + (i/k) dp_inc/dn(x_i).  fmpb_rhs_plane_wave is the
 * plane-wave case.   b device, R x N.
 */
fmpb_status fmpb_rhs_incident(const fmpb_operator *op, int R, const fmpb_incident *inc, fmpb_c64 *b,
                              void *stream);

/*
 * y = A x for R vectors at once, A the collocation operator of the chosen
 * form (Eq. (FMPBEMsystem) or the PBEM product of Sec. 2.4).
 *   x, y  device, R x N each, must not overlap.
 */
fmpb_status fmpb_matvec(const fmpb_operator *op, int R, const fmpb_c64 *x, fmpb_c64 *y,
                        void *stream);

typedef struct {
  double tol;        /* relative residual ||b - A p|| / ||b||; <= 0 selects 1e-8 */
  int restart;       /* GMRES restart length m, 1..1000; 0 selects 30 */
  int maxit;         /* total iteration cap per RHS; 0 selects 1000 */
  int timeout_ms;    /* wall-clock cap for the whole call; 0 = none */
  double inner_tol;  /* MIXED operators: relative tolerance of each inner FP32
                        GMRES solve; <= 0 selects 1e-4 */
} fmpb_solve_opts;

typedef struct {
  int iters;            /* Arnoldi iterations used (summed over inner solves) */
  int converged;        /* 1 if the residual met tol */
  double relres_est;    /* residual estimate (Givens recursion; outer residual for MIXED) */
  double relres_true;   /* ||b - A p|| / ||b|| recomputed with the accurate operator */
  int refinements;      /* outer refinement steps (MIXED operators), else 0 */
} fmpb_solve_info;

/*
 * Solves A p_r = b_r for R right-hand sides by restarted GMRES (Sec. 4)
 * with x0 = 0 and no preconditioner.  Arnoldi: classical Gram-Schmidt with
 * reorthogonalisation (the delayed form DCGS2 for operators with a
 * float-float product, else CGS2 with a second pass when the first removes
 * more than half of ||w||^2), on a Krylov basis stored as float-float pairs
 * (48-bit significands, FP32 pipe); Givens rotations, Hessenberg data, the
 * new rotation, the residual estimate, the solution update and the true
 * residual in FP64.  All vectors live on the device; the host sequences
 * launches and reads the per-RHS convergence flags once every few
 * iterations (4 at first, more while the residual falls slowly); in between,
 * the Arnoldi kernels of converged right-hand sides return at once on their
 * device-side flag.  MIXED operators run GMRES-IR:
 * FP32-spectrum inner solves to inner_tol, outer residuals with the accurate
 * operator, until tol.
 *   b, p   device, R x N; p is overwritten.
 *   opts   may be NULL (defaults); info host, R entries, may be NULL.
 * Returns FMPB_ENOCONV if some RHS missed the tolerance within maxit (p
 * then holds the last iterate and info is filled), FMPB_ETIMEOUT if
 * timeout_ms expired (same guarantees), FMPB_ENAN if b holds NaN/Inf.
 * Synchronises the stream.
 */
fmpb_status fmpb_solve(const fmpb_operator *op, int R, const fmpb_c64 *b, fmpb_c64 *p,
                       const fmpb_solve_opts *opts, fmpb_solve_info *info, void *stream);

/*
 * Solves the systems of n_ops operators at once (Sec. 4's GMRES, as in
 * fmpb_solve), e.g. one lattice at several frequencies, R right-hand sides
 * each: A_o p_{o,r} = b_{o,r}.  The Arnoldi steps of all n_ops R systems run
 * together, one product sequence per iteration.  When the operators share
 * one shape and apply their FMM form on the tensor cores (BF16 operators,
 * and the inner products of MIXED ones: same mesh size, lattice and n_t,
 * full space), every step of that product (near field, P2M, DFT passes,
 * per-frequency M2L products, L2P) is one launch over all operators (Sec.
 * 3.5, Eq. (FMPBEMsystem) applied to the stacked moments); otherwise each
 * operator applies its own product within the shared iteration.  Every
 * system keeps its own Krylov basis, residual and convergence test, so each
 * result matches its own fmpb_solve up to rounding.
 *   ops    host array of n_ops (1..16) operators with one N; MIXED operators
 *          only with MIXED ones.
 *   b, p   device, n_ops x R x N: system (o, r) at ((o R) + r) N; p is
 *          overwritten.  R n_ops <= 4096.
 *   info   host, n_ops x R entries (same order), may be NULL.
 * Allocates the batched product's scratch per call; returns as fmpb_solve
 * (FMPB_ECUDA also if a tensor-core wait of any operator gave up).
 * Synchronises the stream.
 */
fmpb_status fmpb_solve_batch(const fmpb_operator *const *ops, int n_ops, int R, const fmpb_c64 *b, fmpb_c64 *p,
                             const fmpb_solve_opts *opts, fmpb_solve_info *info, void *stream);

/*
 * Synchronises the stream and reports whether any tensor-core product of
 * this operator (BF16 precision) gave up waiting for its MMAs since the
 * operator was built: every such wait is bounded (about one second), and a
 * kernel that gives up skips its output, frees its tensor memory and raises
 * a flag instead of hanging.  Returns FMPB_OK, or FMPB_ECUDA when the flag
 * is set (every product since then is invalid).  fmpb_solve runs this check
 * itself before returning.
 */
fmpb_status fmpb_operator_check(const fmpb_operator *op, void *stream);

/*
 * Total pressure at field points in the fluid (Eq. (cbie) with c(x) = 1):
 * p(x) = p_inc(x) + sum_j int_{E_j} dG/dn_y(x, y) dA_y p_j over every
 * element of every cell (direct sum); an operator built with an admittance
 * beta adds i k beta int_{E_j} G(x, y) dA_y p_j (dp/dn_m = -i k beta p).
 *   p     device, R x N surface pressure.   dirs, amps as in fmpb_rhs_plane_wave.
 *   pts   device, npts x 3 points (must not lie on an element).
 *   out   device, R x npts.
 */
fmpb_status fmpb_field(const fmpb_operator *op, int R, const fmpb_c64 *p, const double *dirs,
                       const fmpb_c64 *amps, int64_t npts, const double *pts, fmpb_c64 *out,
                       void *stream);
/* fmpb_field for incident fields of any kind (host array of R); for a
 * half-space operator the sums include R_p times the mirrored elements and
 * the incident fields their images. */
fmpb_status fmpb_field_incident(const fmpb_operator *op, int R, const fmpb_c64 *p, const fmpb_incident *inc,
                                int64_t npts, const double *pts, fmpb_c64 *out, void *stream);

/*
 * Insertion loss of Eq. (insertionloss) at npts observation points:
 * IL = 20 log10(sum_i |p_inc(x_i)| / sum_i |p(x_i)|), the R incident fields
 * (host array) and their solutions p (device, R x N) acting together; p_inc
 * and p include the images of a half-space operator.   pts device, npts x 3;
 * *il host, in dB.  Errors: EINVAL (sizes, or a total field that vanishes).
 */
fmpb_status fmpb_insertion_loss(const fmpb_operator *op, int R, const fmpb_c64 *p, const fmpb_incident *inc,
                                int64_t npts, const double *pts, double *il, void *stream);

/* ------------------------------------------------------------------------
 * Building blocks (the same kernels the operator uses), for callers that
 * assemble their own products and for table-level checks.
 * ---------------------------------------------------------------------- */

/*
 * Host-side plan of a half-space operator (no device work): the lattice axis
 * perpendicular to the plane {x : x[plane_axis] = plane_offset} (-1 if
 * none), the image offsets whose mirrored cell is within 2 r of the target
 * cell (evaluated exactly in the FMM form, Eq. (admissibilityMirror)) and
 * the smallest distance to a farther mirrored cell (1e300 if none).
 * Errors: EINVAL (bad plane or a lattice axis neither parallel nor
 * perpendicular to the plane), EMESH (cells on both sides of the plane).
 */
fmpb_status fmpb_halfspace_plan(const double *verts, int64_t nv, const int32_t *tris, int64_t ntri,
                                const fmpb_lattice *lattice, int plane_axis, double plane_offset,
                                int32_t *hankel_axis, int32_t *n_near_image, double *dmin_far_image);
/* The same plan on nine-node quadrilaterals (elems: n x 9 node indices; the
 * one-side check reads the element centres, node 4, and all nodes). */
fmpb_status fmpb_halfspace_plan_q9(const double *nodes, int64_t nn, const int32_t *elems, int64_t n,
                                   const fmpb_lattice *lattice, int plane_axis, double plane_offset,
                                   int32_t *hankel_axis, int32_t *n_near_image, double *dmin_far_image);

/*
 * Host-side plan of the FMPBEM2 near field (FMPB_FORM_FMM2, Sec. 3.3), with
 * no device work: the octree depth used (near_levels 0 = automatic), the M2L
 * pairs over all near offsets of the lattice, the exact entries kept for
 * the leaf pairs that are never well separated, and the distinct M2L
 * translations.  n_t_near only validates (0 = 6).  Errors: EINVAL.
 */
fmpb_status fmpb_near2_plan_counts(const double *verts, int64_t nv, const int32_t *tris, int64_t ntri,
                                   const fmpb_lattice *lattice, int near_levels, int n_t_near,
                                   int32_t *levels_out, int64_t *n_m2l, int64_t *n_p2p,
                                   int64_t *n_translations);
/* The same plan on nine-node quadrilaterals (elems: n x 9 node indices; the
 * octree of the element centres, node 4, with box radii over all nine nodes). */
fmpb_status fmpb_near2_plan_counts_q9(const double *nodes, int64_t nn, const int32_t *elems, int64_t n,
                                      const fmpb_lattice *lattice, int near_levels, int n_t_near,
                                      int32_t *levels_out, int64_t *n_m2l, int64_t *n_p2p,
                                      int64_t *n_translations);

/*
 * Collocation blocks T_delta of Eq. (blockToeplizMatrix) (Sec. 2.2): entry
 * (i, j) couples collocation point i of the cell at the origin with
 * triangle j of the cell displaced by -delta . lattice vectors:
 *   T_delta[i][j] = 1/2 [delta = 0, i = j] - int_{E_j} (dG/dn_y + (i/k) d2G/dn_x dn_y).
 *   offsets host, n_off x 3 int32 (delta_x, delta_y, delta_z).
 *   out     device, n_off x ntri x ntri, row-major per block.
 */
fmpb_status fmpb_build_blocks(const double *verts, int64_t nv, const int32_t *tris, int64_t ntri,
                              const fmpb_lattice *lattice, double k, int n_off,
                              const int32_t *offsets, fmpb_c64 *out, void *stream);
/*
 * The same blocks for a surface of uniform normalised admittance beta
 * (Eq. (admittance) in Eq. (bm)); fmpb_build_blocks is beta = 0:
 *   T_delta[i][j] += [delta = 0, i = j] beta/2 - i k beta int_{E_j} (G + (i/k) dG/dn_x).
 * The self term's int G is the closed form of int 1/r plus the polar rule on
 * (e^{ikr} - 1)/r; its int dG/dn_x vanishes on the flat element.
 * Errors: as fmpb_build_blocks, and EINVAL for a non-finite beta.
 */
fmpb_status fmpb_build_blocks_admittance(const double *verts, int64_t nv, const int32_t *tris, int64_t ntri,
                                         const fmpb_lattice *lattice, double k, double beta_re,
                                         double beta_im, int n_off, const int32_t *offsets,
                                         fmpb_c64 *out, void *stream);

/*
 * The blocks T_delta of fmpb_build_blocks_admittance on nine-node quadratic
 * quadrilaterals (Sec. 2.1, Eq. (matrixBEM)) with one constant pressure per
 * element collocated at its centre y(0, 0):
 *   nodes   host, nn x 3 doubles.
 *   elems   host, n x 9 int32 node indices (node (i, j) of the element's 3 x 3
 *           grid at 3 j + i, i along xi, parameter values -1, 0, 1;
 *           y_xi x y_eta points into the fluid).
 *   out     device, n_off x n x n, row-major per block.
 * Regular entries by class of d = |x_i - y_j(0, 0)| against the longest
 * chord h_j between adjacent corners: d >= 4 h: 4 x 4 Gauss-Legendre;
 * 1.5 h <= d < 4 h: 8 x 8; closer: 8 x 8 on each parameter quarter.  Self
 * entries: polar coordinates about the centre (four triangles, 16 x 16
 * Gauss-Legendre each); D, S, K directly and H as the Hadamard finite part
 * from the Laurent expansion of the integrand in the polar radius.
 * Errors: EINVAL (sizes, k <= 0, non-finite beta), EMESH (node index out of
 * range, non-finite node, vanishing Jacobian), ENOMEM, ECUDA.
 */
fmpb_status fmpb_build_blocks_q9(const double *nodes, int64_t nn, const int32_t *elems, int64_t n,
                                 const fmpb_lattice *lattice, double k, double beta_re, double beta_im,
                                 int n_off, const int32_t *offsets, fmpb_c64 *out, void *stream);

/*
 * fmpb_build_blocks_q9 with discontinuous pressure of order 1 or 2 (see
 * fmpb_operator_opts.pressure_order): N = n nb dofs per cell (nb = 4 or 8),
 * dof e nb + a collocated at node a of element e, column f nb + b weighted
 * by shape N_b.
 *   out     device, n_off x N x N, row-major per block.
 * Rules: regular classes as fmpb_build_blocks_q9 but the very-near one on
 * 4 x 4 (order 1) or 8 x 8 (order 2) parameter sub-squares of 8 x 8 points;
 * the element's own entries of a node by a 24 x 24 polar rule about the node
 * with the finite part of N_b H (the shape function's gradient enters the
 * 1/rho coefficient).
 * Errors: as fmpb_build_blocks_q9, and EINVAL for another order.
 */
fmpb_status fmpb_build_blocks_q9p(const double *nodes, int64_t nn, const int32_t *elems, int64_t n, int order,
                                  const fmpb_lattice *lattice, double k, double beta_re, double beta_im,
                                  int n_off, const int32_t *offsets, fmpb_c64 *out, void *stream);

/*
 * P2M table V_0 (B x n, Eq. (p2m)) and L2P table U_0 (n x B, Eq. (l2p) and
 * its normal derivative, scaled by -(ik/4pi)(2n'+1)), B = (n_t+1)^2,
 * coefficient (n', m) at q = n'(n'+1) + m.  Either output may be NULL.
 */
fmpb_status fmpb_multipole_tables(const double *verts, int64_t nv, const int32_t *tris,
                                  int64_t ntri, double k, int n_t, fmpb_c64 *V0, fmpb_c64 *U0,
                                  void *stream);
/* The same tables for a surface of uniform normalised admittance beta:
 * V_0[q][j] += i k beta int_{E_j} conj(I_q) dA (the single layer that the
 * admittance adds to Eq. (p2m)); U_0 is unchanged.  beta = 0 is
 * fmpb_multipole_tables. */
fmpb_status fmpb_multipole_tables_admittance(const double *verts, int64_t nv, const int32_t *tris,
                                             int64_t ntri, double k, double beta_re, double beta_im,
                                             int n_t, fmpb_c64 *V0, fmpb_c64 *U0, void *stream);

/*
 * M2L blocks K(d) (B x B each, Eqs. (m2l), (wigner)) for n_d translation
 * vectors d = x_c - y_c.   dvecs host, n_d x 3;  out device, n_d x B x B.
 */
fmpb_status fmpb_m2l_blocks(double k, int n_t, int n_d, const double *dvecs, fmpb_c64 *out,
                            void *stream);

/*
 * Offset-indexed complex block products on the tensor cores, the form shared
 * by the near field (Sec. 3.2: y_c = sum_delta S_delta p_{c - delta}) and by
 * P2M / L2P (Sec. 3.5, one offset delta = 0):
 *   y[r][c] (+)= sum_o T_o x[r][c - delta_o]
 * for every right-hand side r < R and cell c of the counts[0] x counts[1] x
 * counts[2] grid (cell index (c_z counts[1] + c_y) counts[0] + c_x); terms
 * whose source cell c - delta_o lies outside the grid are skipped.
 *   offsets  host, n_off x 3 int32 (delta_x, delta_y, delta_z), 1 <= n_off <= 27.
 *   T        device, n_off x m x k complex blocks, row-major.
 *   x        device, R x n_cells x k;   y device, R x n_cells x m.
 *   accumulate  0: y = result;  1: y += result.
 * Arithmetic: T and x are rounded to BF16 (FP64 -> FP32 -> BF16, nearest
 * even at each step); the products run on the tensor cores (tcgen05, complex
 * numbers as 2 x 2 real blocks) with FP32 accumulation; y is complex double.
 * So the result equals the exact product of the rounded inputs up to FP32
 * accumulation error.  Allocates its BF16 copies of T and x per call and
 * synchronises the stream.  FMPB_EINVAL, before any device call, for m or k
 * outside 1..2^20, R outside 1..4096, counts outside 1..4096, more than 2^30
 * cells or more than 65,535 x 128 columns (cells x R); FMPB_ECUDA if a
 * bounded wait in the kernel gave up (see fmpb_operator_check).
 */
fmpb_status fmpb_offset_gemm_bf16(const int32_t counts[3], int n_off, const int32_t *offsets,
                                  int64_t m, int64_t k, const fmpb_c64 *T, int R, const fmpb_c64 *x,
                                  fmpb_c64 *y, int accumulate, void *stream);

/*
 * The same with a second product in the same FP32 accumulation, the form of
 * the FMM product's near field plus its L2P term (Sec. 3.5:
 * y_c = sum_delta S_delta p_{c - delta} + U_0 L_c):
 *   y[r][c] (+)= sum_o T_o x[r][c - delta_o] + T2 x2[r][c]
 *   T2  device, m x k2 complex;   x2  device, R x n_cells x k2;  1 <= k2 <= 2^20.
 * Same rounding, allocation and error behaviour as fmpb_offset_gemm_bf16.
 */
fmpb_status fmpb_offset_gemm2_bf16(const int32_t counts[3], int n_off, const int32_t *offsets,
                                   int64_t m, int64_t k, const fmpb_c64 *T, int R, const fmpb_c64 *x,
                                   int64_t k2, const fmpb_c64 *T2, const fmpb_c64 *x2, fmpb_c64 *y,
                                   int accumulate, void *stream);

/*
 * Padded circulant lengths P_a (smallest 2,3,5,7-smooth integer >= 2 M_a - 1,
 * 1 for M_a = 1) and F = P_0 P_1 P_2 for a cell grid.
 */
fmpb_status fmpb_circulant_shape(const int32_t counts[3], int32_t P[3], int64_t *F);

/*
 * Spectrum of a multilevel block Toeplitz matrix (Eq. (blockDiagonal)):
 * Lambda_f = sum_delta T_delta exp(-2 pi i f . (delta mod P) / P).
 *   blocks  device, (2M_x-1)(2M_y-1)(2M_z-1) x B x B, offsets ordered with
 *           delta_x fastest, each from 1-M_a to M_a-1.
 *   spec    device, F x B x B (frequency-major).
 * FMPB_EINVAL, before any device call, for B outside 1..2^20, counts outside
 * 1..4096, more than 2^24 cells, or F B^2 values beyond 2^59.
 */
fmpb_status fmpb_circulant_spectrum(const int32_t counts[3], int64_t B, const fmpb_c64 *blocks,
                                    fmpb_c64 *spec, void *stream);

/*
 * y (+)= T x for the block Toeplitz T whose spectrum is `spec`, through the
 * pruned FFT, the per-frequency B x B products and the pruned inverse FFT
 * (Sec. 2.4).   x, y device, R x (n_cells B), cell-major as above.
 *   accumulate  0: y = T x;  1: y += T x.
 * Allocates its scratch (about 2 F R B complex values) per call.  B must be
 * 1..2^20 and F R B below 2^59 (FMPB_EINVAL otherwise).
 */
fmpb_status fmpb_circulant_apply(const int32_t counts[3], int64_t B, const fmpb_c64 *spec, int R,
                                 const fmpb_c64 *x, fmpb_c64 *y, int accumulate, void *stream);

/*
 * The product of fmpb_circulant_apply in complex FP32 (Sec. 2.4): the
 * spectrum rounded to complex FP32, the pruned forward and inverse DFT
 * passes, their intermediate values and the per-frequency products in FP32
 * (8 bytes per value).  This is how FP32 operators and the inner solves of
 * MIXED operators apply their block Toeplitz parts; relative accuracy about
 * 1e-6.  Same arguments and layouts as fmpb_circulant_apply; every padded
 * length must split into two factors of at most 16 (all lengths up to 256
 * except a few, e.g. 245), else FMPB_EINVAL.  Allocates its FP32 copy of the
 * spectrum and its scratch per call and synchronises the stream.
 */
fmpb_status fmpb_circulant_apply_f32(const int32_t counts[3], int64_t B, const fmpb_c64 *spec, int R,
                                     const fmpb_c64 *x, fmpb_c64 *y, int accumulate, void *stream);

/*
 * The product of fmpb_circulant_apply with the per-frequency products
 * Y_f = Lambda_f X_f on the tensor cores (tcgen05, BF16 inputs, FP32
 * accumulation): Lambda_f and X_f are rounded to BF16 (Lambda: FP64 -> FP32 ->
 * BF16; X_f: its float-float DFT value -> FP32 -> BF16, nearest even at each
 * step); the pruned forward and inverse DFTs run in float-float as in
 * fmpb_circulant_apply.  The result equals the exact circulant product with
 * the rounded Lambda_f and X_f up to FP32 accumulation.  This is how BF16
 * operators (and the inner solves of MIXED operators in the FMM form) apply
 * their M2L translations.  Same arguments and layouts as
 * fmpb_circulant_apply; F must not exceed 65,535.  Allocates its BF16 copy of
 * the spectrum and its scratch per call, synchronises the stream; FMPB_ECUDA
 * if a bounded wait of the tensor-core kernel gave up.
 */
fmpb_status fmpb_circulant_apply_bf16(const int32_t counts[3], int64_t B, const fmpb_c64 *spec, int R,
                                      const fmpb_c64 *x, fmpb_c64 *y, int accumulate, void *stream);

/*
 * Same product as fmpb_circulant_apply, for callers that cannot allocate
 * device memory during the call (for example a program whose device memory
 * belongs to another runtime's pool, or a latency-bound loop that cannot
 * accept the synchronisation an allocation may cause).  This entry point has
 * no counterpart in the paper; it only changes where the temporaries live.
 *   - Allocates nothing: no cudaMalloc, cudaFree or allocating library call.
 *     The scratch (2 F R B complex values) comes from one static device
 *     array of 32 MiB, which every device that loads the library holds until
 *     the process exits.  Products needing more than 32 MiB of scratch return
 *     FMPB_EINVAL with the required size in fmpb_last_error().
 *   - The first call on a device looks up that array's device address (with
 *     the device current) and caches it for the life of the process; make
 *     that first call before any stream capture.  A device reset
 *     (cudaDeviceReset) or a release of the primary context reloads the
 *     library's device code, so the cached address is then stale: do not
 *     call this entry point after either.
 *   - B must be 1..2^20; counts, R and the 32 MiB limit are checked on the
 *     host, before any CUDA call, without an overflowing size product.
 *   - Every call on a device shares the same array.  The array keeps the
 *     last call's contents, but nothing in it needs clearing: each call
 *     writes every element it reads.  Calls that may overlap on the GPU
 *     (different streams, or different host threads) race on the array and
 *     must be serialised by the caller.
 * Arguments, layouts and results are those of fmpb_circulant_apply.
 */
fmpb_status fmpb_circulant_apply_static(const int32_t counts[3], int64_t B, const fmpb_c64 *spec, int R,
                                        const fmpb_c64 *x, fmpb_c64 *y, int accumulate, void *stream);

/* ------------------------------------------------------------------------
 * Serving: a request loop over many (mesh, lattice, k) problems.
 *
 * Requests (a unit-cell mesh, a lattice, a wavenumber and R incident plane
 * waves) are queued and served by two worker threads, each with its own
 * CUDA stream, so that batches overlap on the device.  Operators are kept
 * resident per (mesh, lattice, k, form, precision) in a cache with LRU
 * eviction.  A request is admitted when its operator and solve workspace fit
 * in the HBM budget (after evicting idle operators).  Queued requests that
 * share an operator are merged into one multi-RHS solve (continuous
 * batching: new arrivals join the next batch while others run).  Each RHS
 * runs its own Krylov iteration, so a result does not depend on what else
 * was batched with it.  The paper has no serving layer; this is the systems
 * pattern around its solver.
 * ---------------------------------------------------------------------- */
typedef struct fmpb_server fmpb_server;

typedef struct {
  size_t hbm_budget_bytes;   /* 0 = 80% of the device memory free at creation */
  int max_batch_rhs;         /* right-hand sides merged into one solve; 0 = 64 */
  int cache_entries;         /* resident operators kept; 0 = 8 */
  int precision;             /* fmpb_precision of the operators the server builds */
  double tol;                /* GMRES relative tolerance; <= 0 selects 1e-8 */
  int restart;               /* GMRES restart; 0 = 200 */
  int maxit;                 /* iteration cap; 0 = 3000 */
} fmpb_server_opts;

typedef struct {
  const double *verts;       /* host, nv x 3, copied at submit */
  int64_t nv;
  const int32_t *tris;       /* host, ntri x 3, copied at submit */
  int64_t ntri;
  fmpb_lattice lattice;
  double k;
  int form;                  /* fmpb_form */
  int n_t;                   /* FMM truncation number; 0 = the truncation rule */
  int R;                     /* plane waves, 1..64 */
  const double *dirs;        /* host, R x 3 unit vectors, copied at submit */
  const fmpb_c64 *amps;      /* host, R amplitudes or NULL (all 1), copied at submit */
} fmpb_request;

typedef struct {
  fmpb_status status;        /* of this request only */
  int R;
  int iters_max;             /* largest GMRES iteration count among its RHS */
  double relres_true_max;    /* largest true relative residual among its RHS */
  int cache_hit;             /* 1 if its operator was resident when it started */
  int batched_with;          /* requests in the same solve, itself included */
  double queue_ms, build_ms, solve_ms, latency_ms;   /* submit -> completion */
} fmpb_result;

typedef struct {
  int64_t submitted, completed, failed, cache_hits, batches;
  double p50_ms, p99_ms, mean_ms;         /* latency over completed requests */
  double solves_per_s;                    /* completed requests / (last completion - first submit) */
  size_t hbm_in_use, hbm_high_water;      /* resident operators + running workspaces */
} fmpb_server_stats;

/* Creates the server on the current device.  opts may be NULL. */
fmpb_status fmpb_server_create(const fmpb_server_opts *opts, fmpb_server **out);
/*
 * Queues a request.  p_out (host, R x N complex, N = ntri * cells) receives
 * the surface pressure; it must stay valid until fmpb_server_wait returns for
 * this ticket.  Returns at once; EINVAL on malformed requests.
 */
fmpb_status fmpb_server_submit(fmpb_server *srv, const fmpb_request *req, fmpb_c64 *p_out, uint64_t *ticket);
/* Waits (bounded by timeout_ms; <= 0 waits without limit) for a ticket and
 * fills *res.  ETIMEOUT if still running.  A ticket can be waited once. */
fmpb_status fmpb_server_wait(fmpb_server *srv, uint64_t ticket, int timeout_ms, fmpb_result *res);
fmpb_status fmpb_server_get_stats(fmpb_server *srv, fmpb_server_stats *stats);
/* Finishes queued work, stops the workers, frees every cached operator. */
void fmpb_server_destroy(fmpb_server *srv);

/* ------------------------------------------------------------------------
 * Telemetry (no counterpart in the paper; it reports wall-clock times of
 * assembly and products only, Sec. 4).
 * ---------------------------------------------------------------------- */

/* Number of CUDA kernels this library has launched in the process. */
uint64_t fmpb_kernel_launches(void);
/* Enables (1) or disables (0) per-kernel timing: a CUDA event pair recorded
 * on the launching stream around every kernel launch from then on. */
void fmpb_profile_enable(int on);
/* Drops the recorded timings (events are recycled). */
fmpb_status fmpb_profile_reset(void);
/* Waits for the recorded events and writes a JSON object
 * {"kernel": [launches, total_ms], ...} into buf (len bytes, NUL-terminated).
 * EINVAL if buf is too small. */
fmpb_status fmpb_profile_summary(char *buf, size_t len);

/* Writes a JSON list of the tile shapes the tensor-core autotuner chose:
 * the first product of each shape (device, rows m, depth k, columns,
 * offsets; single products and operator batches apart, "batched", one
 * choice for every operator count of a batch) times the tile variants (128
 * or 256 output rows and 128 or 256 output columns per CTA) on the caller's
 * stream and keeps the fastest;
 * every entry lists the chosen tile and the time of each variant (ms, in
 * the order 128x256, 256x256, 256x128, 128x128); "kernel": "tc_gemm".
 * It also lists the plans the DFT-pass autotuner chose ("kernel": "dft"):
 * the first out-of-place, non-accumulating pass of each shape (device,
 * arithmetic and storage formats, padded length P, inputs Pin, outputs Pout;
 * its inner extent and line count are reported, but later passes of the
 * shape take its plan whatever theirs, so that operators batched together
 * round as they do alone) times the direct form, the radix-2 form (FP32 passes of length 8,
 * 16 or 32) and every split P = P1 P2 into factors of at most 16 and keeps
 * the fastest; "chosen" and "ms" name them ("direct<P>", "fft2_<P>",
 * "split<P1>").  EINVAL if buf is too small. */
fmpb_status fmpb_tuning_summary(char *buf, size_t len);

/* Forces one tile variant of the tensor-core offset GEMM for all later
 * products in this process (0: 128x256, 1: 256x256, 2: 256x128,
 * 3: 128x128 output rows x columns per CTA), or restores autotuning (-1).
 * For tests and tuning studies; the variants give the same results up to
 * FP32 accumulation order.  EINVAL outside -1..3. */
fmpb_status fmpb_set_tile_variant(int variant);

/* Forces one plan kind for every later DFT pass of the circulant products in
 * this process, where the pass has it: 0 the direct form (inputs in
 * registers), 1 the two-factor form with the split of fewest multiply-adds,
 * 2 the radix-2 form (FP32 passes of length 8, 16 or 32); a pass without the
 * requested kind takes the model's plan.  -1 restores the autotuner.  For
 * tests and tuning studies: the plans give the same results up to rounding.
 * EINVAL outside -1..2. */
fmpb_status fmpb_set_dft_plan(int kind);

#ifdef __cplusplus
}
#endif

#endif /* FMPB_H */
