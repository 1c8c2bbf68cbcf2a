/*
 * femamg.h -- C ABI of the GB300 solver for the P1 finite element system
 *
 *     (rho K + M) u = f,   K_ij = int grad phi_j . grad phi_i,  M_ij = int phi_j phi_i,
 *                          f_i  = int ubar phi_i
 *
 * of the reduced optimality system -rho Lap(u) + u = ubar in the unit cube, u = 0 on
 * its boundary (Langer, Steinbach, Yang, "Robust discretization and solvers for elliptic
 * optimal control problems with energy regularization", arXiv 2102.03515: Sec. 1 eq.
 * (sigular), Sec. 2 eq. (linsys)).  The system is solved by conjugate gradients
 * preconditioned by one algebraic-multigrid V-cycle with one pre- and one post-smoothing
 * step (Sec. 3.1 eq. (amgpre); Sec. 4), stopped on a relative residual (Sec. 4).
 *
 * Conventions for every entry point:
 *  - Every call returns a fem_status and never aborts the process.  On failure,
 *    fem_last_error() returns a message for the calling thread.
 *  - "stream" is a cudaStream_t (pass the caller's current stream, or NULL for the
 *    legacy default stream).  Work is stream-ordered; a call returns once the results
 *    it reports on the host are available.
 *  - Pointers named *_dev are device pointers owned by the caller, contiguous, FP64,
 *    in unknown order; pointers named *_host are host pointers borrowed for the duration
 *    of the call.  Handles (fem_system, amg_hier, pcg_batch) are owned by the library
 *    and released by the matching *_destroy call.
 *  - Unknowns: the interior vertices (i,j,k), 1 <= i,j,k <= n-1, of the (n+1)^3 vertex
 *    grid, numbered (i-1) + (n-1)*((j-1) + (n-1)*(k-1)); boundary vertices carry the
 *    homogeneous Dirichlet value and are not unknowns (V_h = S_h^1 cap H_0^1, Sec. 2).
 *  - Matrices are kept in "CSR4": CSR whose rows are padded to a multiple of 4 entries
 *    with (column -1, value 0) so that every row starts on a 16-byte boundary.
 */
#ifndef FEMAMG_H
#define FEMAMG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  FEM_OK = 0,
  FEM_EINVAL = 1,        /* invalid argument (null handle, bad size, bad option)        */
  FEM_ENOMEM = 2,        /* device or host allocation failed, or over the memory budget */
  FEM_ECUDA = 3,         /* a CUDA runtime call failed                                  */
  FEM_ENOCONV = 4,       /* max_iter reached; the best iterate is still written          */
  FEM_EBREAKDOWN = 5,    /* <p, A p> <= 0 or a NaN appeared in a CG scalar             */
  FEM_ECANCELLED = 6,    /* the caller's cancel flag was raised                         */
  FEM_EDEVCHECK = 7,     /* a device-side consistency check failed (see message)        */
  FEM_EUNSUPPORTED = 8   /* input outside what this build handles (see message)         */
} fem_status;

/* ------------------------------------------------------------------ mesh + target */

/* Kuhn mesh of the unit cube: n^3 cubes, each split into the 6 tetrahedra along the
 * monotone lattice paths from its corner (i,j,k) to (i+1,j+1,k+1) (the paper's
 * admissible simplicial decomposition, Sec. 2; the Kuhn type is this library's choice).
 * xyz_host, if not NULL, gives all (n+1)^3 vertex coordinates (x,y,z interleaved,
 * vertex (i,j,k) at index i + (n+1)*(j + (n+1)*k)), e.g. a jittered grid; NULL means the
 * uniform grid h*(i,j,k), h = 1/n.  Requires 2 <= n <= 1290. */
typedef struct {
  int32_t n;
  const double* xyz_host;
} fem_kuhn_desc;

/* Targets of Sec. 4: FEM_TARGET_SINE (4.1), FEM_TARGET_BOX = 1 on (lo,hi)^3 (4.2),
 * FEM_TARGET_SINE_PLUS_ONE (4.3), and FEM_TARGET_BUMPS: sum_b a_b exp(-|x-c_b|^2/(2 w_b^2))
 * (synthetic batched/serving targets).  Arrays are host pointers of length nb (3*nb for
 * centres); nb <= 64.
 * FEM_TARGET_QUADVALS: any ubar in L2 (Sec. 2), given by its values at the quadrature points
 * of the load vector: quadvals_dev (device, read during the call) holds 4 doubles per tet,
 * [tet][q], the value at the point with barycentric weight (5 + 3 sqrt 5)/20 on the tet's
 * local vertex q and (5 - sqrt 5)/20 on the other three.  Tets are numbered as the mesh
 * gives them (fem_assemble_mesh, fem_mesh), and 6 c + p on the Kuhn mesh: cube
 * c = i + n (j + n k), path p over the axis orders (x,y,z), (x,z,y), (y,x,z), (y,z,x),
 * (z,x,y), (z,y,x), with local vertices corner, +e_a, +e_a+e_b, +(1,1,1).  Only the load
 * vector uses it (fem_assemble*, fem_assemble_rhs); calls that evaluate ubar elsewhere
 * (fem_errors, fem_recover, fem_error_indicator, fem_assemble_rhs_noalloc) return
 * FEM_EINVAL for it. */
typedef enum {
  FEM_TARGET_SINE = 0,
  FEM_TARGET_BOX = 1,
  FEM_TARGET_BUMPS = 2,
  FEM_TARGET_SINE_PLUS_ONE = 3,
  FEM_TARGET_QUADVALS = 4
} fem_target_kind;

typedef struct {
  int32_t kind;
  int32_t nb;
  const double* centers_host;
  const double* widths_host;
  const double* amps_host;
  double lo, hi;
  const double* quadvals_dev;   /* FEM_TARGET_QUADVALS only (else ignored) */
} fem_target;

/* Operator storage for the finest level. */
typedef enum {
  FEM_FMT_AUTO = 0,     /* 15-point stencil on the uniform grid, CSR4 otherwise */
  FEM_FMT_STENCIL = 1,  /* matrix-free stencil (uniform grid only)              */
  FEM_FMT_CSR = 2       /* CSR4 always                                           */
} fem_format;

typedef struct {
  int32_t format;       /* fem_format                                            */
  int32_t keep_pencil;  /* 1: keep K and M separately (needed by batched solves) */
} fem_assemble_opts;

typedef struct fem_system_s* fem_system;

/* A general conforming tetrahedral mesh (host arrays, read during the call only): nv
 * vertices with coordinates xyz[3*nv]; nt tets given by 4 vertex indices each in tet[4*nt]
 * (either orientation); dirichlet[nv] != 0 marks the vertices on which u = 0 (the boundary
 * of Omega, Sec. 2: V_h = S_h^1 cap H_0^1).  The unknowns are the other vertices, numbered
 * in increasing vertex order. */
typedef struct {
  int64_t nv;
  int64_t nt;
  const double* xyz;
  const int32_t* tet;
  const uint8_t* dirichlet;
} fem_mesh_desc;

/* Assemble K, M and f = (int ubar phi_i)_i (Sec. 2, entries below eq. (linsys)) on the
 * interior unknowns and form A = rho K + M (eq. (linsys)).  K and M come from the P1
 * element matrices |tau| grad(lambda_a).grad(lambda_b) and |tau|(1+delta_ab)/20; f uses
 * the 4-point degree-2 rule of Hammer and Stroud on each tetrahedron.  rho > 0.
 * opts may be NULL (defaults: AUTO format, no pencil).  On success *out owns all
 * device storage of the system. */
fem_status fem_assemble(const fem_kuhn_desc* mesh, double rho, const fem_target* target,
                        const fem_assemble_opts* opts, void* stream, fem_system* out);

typedef struct {
  int64_t n;          /* cells per side                                 */
  int64_t N;          /* unknowns (n-1)^3                               */
  int64_t nnz;        /* stored entries of the CSR4 form (with padding) */
  double h, rho;
  int32_t is_stencil; /* finest level applied matrix-free               */
  int32_t has_pencil;
} fem_system_info;

fem_status fem_system_get_info(fem_system sys, fem_system_info* info);

/* Load vector of another target on the same mesh: f_dev[i] = int ubar phi_i (the rule of
 * fem_assemble), length N.  Used to feed many targets to one batch. */
fem_status fem_assemble_rhs(fem_system sys, const fem_target* target, double* f_dev,
                            void* stream);

/* fem_assemble_rhs without any device allocation (the paper has no counterpart: this is
 * an interface for callers that cannot allocate).  Callers that cannot call cudaMalloc --
 * code running while another allocator holds nearly all of the GPU's memory, callers with
 * a fixed pre-reserved budget, latency-critical loops that must not pay for an allocation
 * and its implicit synchronisation -- get the same f_dev as fem_assemble_rhs, computed in a
 * fixed 17 MB scratch array that the library holds on every GPU it is loaded on until the
 * process exits.  Limits: Kuhn meshes with n <= 64 cells per side, at most 64 bumps, and
 * targets given by formula (FEM_TARGET_QUADVALS is not taken); other inputs return
 * FEM_EINVAL with a message naming the limit.  The first call on each device looks up the
 * array's device address.  Every call synchronises its stream before it returns (the bump
 * parameters are copied from the caller's host arrays), so no call may be made during a
 * stream capture.  All calls share the array: calls that overlap on the GPU (different
 * streams without ordering) race and must not be issued. */
fem_status fem_assemble_rhs_noalloc(fem_system sys, const fem_target* target, double* f_dev,
                                    void* stream);

/* fem_assemble on a general tetrahedral mesh: the same K, M (P1 element matrices) and f
 * (4-point Hammer-Stroud rule per tet), rows built vertex by vertex over the incident tets in
 * increasing tet order; CSR4 operator (no stencil).  Limits: at most 64 tets per vertex and
 * 128 distinct neighbours per row (FEM_EUNSUPPORTED beyond), nt < 2^31.  A degenerate tet
 * (zero volume) or a vertex index out of range gives FEM_EINVAL.  fem_errors, fem_recover,
 * fem_assemble_rhs, the AMG variants and PCG accept the resulting system; batched sessions
 * need keep_pencil as usual. */
fem_status fem_assemble_mesh(const fem_mesh_desc* mesh, double rho, const fem_target* target,
                             const fem_assemble_opts* opts, void* stream, fem_system* out);

/* Copy the assembled load vector f (length N) into f_dev. */
fem_status fem_system_get_rhs(fem_system sys, double* f_dev, void* stream);

/* The vertex of every unknown (the dof -> vertex map), vert_dev: device int64[N].  Kuhn mesh:
 * vertex i + (n+1) (j + (n+1) k) of the interior point (i, j, k); general mesh: the index in
 * the mesh's vertex array (unknowns follow increasing vertex order).  Lets a caller evaluate
 * its own functions at the unknowns' vertices. */
fem_status fem_system_dof_vertices(fem_system sys, int64_t* vert_dev, void* stream);

/* Export A = rho K + M (which = 0), K (1) or M (2) in CSR4: rowptr_dev int32[N+1],
 * col_dev int32[nnz], val_dev double[nnz] with nnz from fem_system_get_info. */
fem_status fem_system_export(fem_system sys, int32_t which, int32_t* rowptr_dev,
                             int32_t* col_dev, double* val_dev, void* stream);

/* y = A x for the system's operator (the operator of eq. (linsys)) in FP64.  x_dev, y_dev:
 * device FP64 [N], distinct.  Synchronises the stream. */
fem_status fem_spmv(fem_system sys, const double* x_dev, double* y_dev, void* stream);

/* y = A x as CG's iterations apply it, reps times after one untimed application; ms_out
 * receives the mean device time of one operator launch (CUDA events on `stream`).  CSR4
 * systems (jittered and general meshes): the FP64 product of fem_spmv.  The matrix-free
 * operator of the uniform grid: double-float arithmetic on the FP32 pipe -- x rounded to 48
 * significant bits and split into two FP32 numbers (once, before the timed launches), the
 * four stencil coefficients held exactly as three FP32 numbers each, the sums of each
 * coefficient class and the products carried by error-free transformations -- so that each
 * y_i is within 2^-44 sum_j |a_ij x_j| of the exact product (FP64: a few 2^-53); when some
 * x_i != 0 lies outside 2^-74 <= |x_i| < 2^101 the product is FP64 instead.  pcg_solve
 * recomputes the residual with the FP64 operator at the end and continues from its iterate
 * when that residual is above the tolerance.  Errors: FEM_EINVAL (null argument, reps < 1). */
fem_status fem_spmv_timed(fem_system sys, const double* x_dev, double* y_dev, int32_t reps,
                          void* stream, double* ms_out);

void fem_system_destroy(fem_system sys);

/* ------------------------------------------------------------------ post-processing */

/* Errors of a discrete solution against w = scale * target (Sec. 4.1, Tables 1-3: with
 * target = FEM_TARGET_SINE and scale = 1 / (3 rho pi^2 + 1), w is the exact u_rho of the
 * reduced problem; with scale = 1, w is the target ubar itself):
 *   l2sq = ||w - u_h||^2_{L2},  h1sq = ||grad (w - u_h)||^2_{L2},
 * u_h the P1 function with the nodal values u_dev (length N, interior unknowns) and zero
 * on the boundary.  Integrals run over every tet of the mesh with the 4-point
 * Hammer-Stroud rule applied on each child of qlevel (0..2) rounds of Bey's red
 * refinement (4 * 8^qlevel points per tet), in FP64 with a fixed-order reduction.  h1sq is
 * NaN for targets without a gradient here (box, bumps).  Errors: FEM_EINVAL (null
 * argument, qlevel out of range, bad target). */
typedef struct {
  double l2sq;
  double h1sq;
} fem_errors_result;
fem_status fem_errors(fem_system sys, const double* u_dev, const fem_target* target,
                      double scale, int32_t qlevel, void* stream, fem_errors_result* out);

/* Control and adjoint of the optimal control problem recovered from the state u_h
 * (Sec. 2: z = (ubar - u) / rho from the gradient equation, p = -rho u): at every
 * unknown's vertex x_i, z_i = (ubar(x_i) - u_i) / rho and p_i = -rho u_i, rho the
 * system's.  u_dev, z_dev, p_dev: device arrays of length N (z_dev or p_dev may be
 * null).  Errors: FEM_EINVAL (null sys / u_dev / target, bad target). */
fem_status fem_recover(fem_system sys, const double* u_dev, const fem_target* target,
                       double* z_dev, double* p_dev, void* stream);

/* ------------------------------------------------------------------ adaptive meshes */

/* The adaptive runs of Sec. 4.2-4.3 refine the mesh where a residual error indicator is
 * large.  These calls keep a general tetrahedral mesh on the device, compute the indicator
 * of a solution on it, mark the tets with the largest indicators and refine them locally,
 * so that solve -> estimate -> mark -> refine -> assemble runs without host copies of the
 * mesh. */

/* Residual error indicator of the reduced problem -rho Lap u + u = ubar (eq. (linsys) in
 * strong form) for the P1 solution u_dev (length N, zero on Dirichlet vertices) on a system
 * from fem_assemble_mesh / fem_assemble_on_mesh: per tet T, after Verfurth's robust
 * estimator for reaction-diffusion problems,
 *   eta_T^2 = a_T^2 ||ubar - u_h||^2_{L2(T)}
 *           + 1/2 sum_{interior faces F of T} rho^{-1/2} a_F |F| (rho [grad u_h . n_F])^2,
 *   a_S = min(h_S / sqrt(rho), 1),  h_S the longest edge of S,
 * rho the system's.  The volume integral uses the rule of fem_errors of the given qlevel
 * (0..2).  eta2_dev: device array of nt doubles (nt of the mesh, tets in the mesh's order);
 * *total (may be null) receives sum_T eta_T^2 (fixed-order reduction).  Errors: FEM_EINVAL
 * (null argument, Kuhn-mesh system, qlevel out of range, bad target, a face shared by more
 * than two tets). */
fem_status fem_error_indicator(fem_system sys, const double* u_dev, const fem_target* target,
                               int32_t qlevel, double* eta2_dev, void* stream, double* total);

/* Bulk marking: with S(t) = sum of the eta2_dev[i] >= t and t* the largest double with
 * S(t*) >= theta * S(0), mark_dev[i] = (eta2_dev[i] >= t*) (ties at t* all marked; nothing is
 * marked when every value is 0).  t* is found by bisection on the bits of non-negative
 * doubles, each S by a fixed-order reduction.  eta2_dev: n finite values >= 0 (device);
 * mark_dev: n bytes (device).  *threshold and *nmarked may be null.  Errors: FEM_EINVAL
 * (n < 1, theta outside (0, 1], a negative or non-finite value). */
fem_status fem_mark_bulk(const double* eta2_dev, int64_t n, double theta, uint8_t* mark_dev,
                         void* stream, double* threshold, int64_t* nmarked);

typedef struct fem_mesh_s* fem_mesh;

/* Copy a conforming mesh (fem_mesh_desc, host arrays) to the device.  The mesh must be a
 * manifold partition: every face in one or two tets (FEM_EINVAL otherwise, and for a zero
 * volume or a vertex index out of range).  The Dirichlet flags must mark the vertices on the
 * boundary: refinement flags its new boundary vertices the same way. */
fem_status fem_mesh_create(const fem_mesh_desc* mesh, void* stream, fem_mesh* out);

typedef struct {
  int64_t nv;
  int64_t nt;
} fem_mesh_info;
fem_status fem_mesh_get_info(fem_mesh m, fem_mesh_info* info);

/* Copy the mesh to host arrays of nv * 3 doubles, nt * 4 int32 and nv bytes (any may be
 * null). */
fem_status fem_mesh_download(fem_mesh m, double* xyz, int32_t* tet, uint8_t* dirichlet,
                             void* stream);

/* Local refinement by longest-edge bisection (Rivara) with conforming closure: every tet
 * with mark_dev[t] != 0 (device, nt bytes of the current mesh) is bisected on its longest
 * edge, and every tet that then holds a bisected edge is bisected on its own longest edge,
 * in passes, until the mesh is conforming again.  Deterministic:
 *   - edge order: squared length (dx*dx + dy*dy) + dz*dz without fused multiply-add, ties
 *     to the smaller vertex pair (min, max);
 *   - a tet (v0..v3) with longest edge at local positions i < j and midpoint
 *     m = 0.5 * (x_a + x_b) becomes, at its index, the tet with v_j replaced by m, and the
 *     tet with v_i replaced by m is appended; appended tets follow their parents' order;
 *   - the new vertices of a pass follow the order of the first tet that bisects their edge;
 *   - a new vertex is a Dirichlet vertex when it lies on a boundary face.
 * stats (may be null): passes, new vertices and new tets.  Errors: FEM_EINVAL (null
 * argument), FEM_EUNSUPPORTED (2^31 tets or vertices). */
typedef struct {
  int32_t passes;
  int64_t new_vertices;
  int64_t new_tets;
} fem_refine_stats;
fem_status fem_mesh_refine(fem_mesh m, const uint8_t* mark_dev, void* stream,
                           fem_refine_stats* stats);

/* fem_assemble_mesh on a device mesh (the mesh is copied: it may be refined or destroyed
 * afterwards). */
fem_status fem_assemble_on_mesh(fem_mesh m, double rho, const fem_target* target,
                                const fem_assemble_opts* opts, void* stream, fem_system* out);

void fem_mesh_destroy(fem_mesh m);

/* ------------------------------------------------------------------ AMG */

/* Smoothers: Chebyshev of degree `degree` on D^{-1}A, one l1-Jacobi step, or symmetric
 * Gauss-Seidel as in Sec. 3.1 (one forward sweep on the way down, one backward sweep on
 * the way up), run class by class over a greedy colouring of the matrix graph (nodes
 * visited by decreasing hash priority, each taking the smallest colour unused by its
 * already coloured neighbours). */
typedef enum {
  AMG_SMOOTHER_CHEBYSHEV = 0,
  AMG_SMOOTHER_L1_JACOBI = 1,
  AMG_SMOOTHER_SGS = 2
} amg_smoother;
/* Coarsening: smoothed aggregation (default), or the paper's red-black colouring with
 * averaging interpolation (Sec. 3.1 after KF1998: visit the unknowns in a fixed order; an
 * unmarked one becomes coarse and its unmarked matrix-graph neighbours fine; a fine unknown
 * is interpolated by the average of its coarse neighbours).  The visiting order of the
 * red-black split: decreasing hash priority (default), or the unknowns' index order
 * (AMG_ORDER_NATURAL: on the Kuhn grid the lexicographic order coarsens to every other grid
 * point, and the iteration counts follow the paper's Table 4; the parallel rounds that find
 * the greedy set then take about 3 (n - 1) rounds). */
typedef enum { AMG_COARSEN_SA = 0, AMG_COARSEN_RED_BLACK = 1 } amg_coarsening;
typedef enum { AMG_ORDER_HASH = 0, AMG_ORDER_NATURAL = 1 } amg_order;
typedef enum { AMG_PREC_FP64 = 0, AMG_PREC_FP32 = 1, AMG_PREC_BF16 = 2 } amg_precision;

/* Smoothed-aggregation set-up on the device; Sec. 3.1 coarsens by red-black colouring
 * and averaging interpolation, this library by smoothed aggregation (rules below); both
 * build A_c = P^T A P by Galerkin's method (Sec. 3.1).
 *   strength: |a_ij| >= theta sqrt(a_ii a_jj); MIS-2 roots by hashed priorities (seed);
 *   P = (I - omega D^{-1} A_F) P_tent, omega = 4/(3 lambda_F) (Gershgorin bound);
 *   coarsest level (<= coarse_max unknowns): dense FP64 inverse.
 * precision selects the V-cycle arithmetic: FP64, FP32, or BF16-stored matrix values
 * with FP32 vectors/accumulation; the coarsest solve is FP64 in every case. */
typedef struct {
  double theta;          /* strength threshold, default 0.05                   */
  int32_t smoother;      /* amg_smoother, default Chebyshev                     */
  int32_t degree;        /* Chebyshev degree per smoothing step, default 2      */
  double cheb_ratio;     /* interval [lambda/ratio, lambda], default 6          */
  int32_t coarse_max;    /* default 256                                         */
  int32_t max_levels;    /* default 16                                          */
  int32_t precision;     /* amg_precision, default FP64                         */
  uint32_t seed;         /* priority seed, default 0                            */
  double rho_setup;      /* > 0: build the hierarchy from rho_setup K + M (needs the
                            pencil; the finest operator of solves is unchanged);
                            default 0 = the system's rho                        */
  int32_t coarsening;    /* amg_coarsening, default smoothed aggregation         */
  int32_t max_row;       /* a level whose restriction R, product A P or coarse
                            operator R A P would have a row with more than max_row
                            entries becomes the coarsest level (dense inverse if it
                            has <= coarse_max unknowns, else the smoother alone);
                            1..8192, default (and 0) 8192, the products' limit      */
  int32_t order;         /* amg_order of the red-black split, default hash        */
} amg_opts;

typedef struct amg_hier_s* amg_hier;

/* opts may be NULL for defaults.  The hierarchy refers to sys's storage: destroy it
 * before the system. */
fem_status amg_setup(fem_system sys, const amg_opts* opts, void* stream, amg_hier* out);

/* Fill opts with the defaults. */
void amg_default_opts(amg_opts* opts);

typedef struct {
  int32_t levels;
  int64_t rows[32];      /* unknowns per level        */
  int64_t nnz[32];       /* stored CSR4 entries       */
  double lmax[32];       /* Gershgorin bound of D^-1 A per level */
  double setup_ms;
  int64_t pnnz[32];      /* stored CSR4 entries of P_l (0 on the coarsest level) */
  int64_t rnnz[32];      /* stored CSR4 entries of R_l                            */
  int32_t finest_stencil;/* 1: the finest level is applied matrix-free           */
  int32_t colours[32];   /* Gauss-Seidel colours per level (SGS smoother; else 0) */
} amg_hier_info;

fem_status amg_hier_get_info(amg_hier h, amg_hier_info* info);

/* Export level l (0 = finest): which = 0 A_l, 1 P_l, 2 R_l = P_l^T (CSR4, FP64 values;
 * sizes from amg_hier_get_info / the row counts of consecutive levels), which = 3 the
 * aggregate of each node of level l (int32 in col_dev, -1 = isolated; with red-black
 * coarsening the coarse index of coarse nodes and -1 for fine ones; rowptr/val unused),
 * which = 4 the Gauss-Seidel colour of each node (int32 in col_dev; SGS smoother only). */
fem_status amg_hier_export(amg_hier h, int32_t level, int32_t which, int32_t* rowptr_dev,
                           int32_t* col_dev, double* val_dev, int64_t* nnz_out, void* stream);

/* z = V(r): one V-cycle with zero initial guess (eq. (amgpre) applied recursively). */
fem_status amg_vcycle(amg_hier h, const double* r_dev, double* z_dev, void* stream);

/* The same V-cycle applied `reps` times (reps >= 1) from one CUDA graph of a single
 * application, for callers that apply the preconditioner many times (their own Krylov
 * method, a timing of the V-cycle alone): z = V(r) after the call; *ms_out (may be null)
 * receives the mean device time of one application, measured with CUDA events around the
 * graph replays on `stream`.  Errors: FEM_EINVAL (null argument, reps < 1). */
fem_status amg_vcycle_graph(amg_hier h, const double* r_dev, double* z_dev, int32_t reps,
                            void* stream, double* ms_out);

/* The Galerkin product A_{l+1} = R_l (A_l P_l) of level `level` (Sec. 3.1: the coarse
 * operator P^T A P), computed again from the hierarchy's A_l, P_l, R_l reps times after one
 * untimed product, into scratch storage (the hierarchy is not changed).  ms_out receives the
 * mean device time of one product (CUDA events on `stream`: both SpGEMM launches and the
 * compaction), ap_entries_out the entries of A_l P_l.  Errors: FEM_EINVAL (null hierarchy,
 * reps < 1, a level without a coarse operator, or a finest level kept without its FP64
 * matrix). */
fem_status amg_galerkin_timed(amg_hier h, int32_t level, int32_t reps, void* stream,
                              double* ms_out, int64_t* ap_entries_out);

void amg_hier_destroy(amg_hier h);

/* ------------------------------------------------------------------ PCG */

typedef enum { PCG_STOP_RESIDUAL = 0, PCG_STOP_PRECONDITIONED = 1 } pcg_stop;

typedef struct {
  double tol;               /* default 1e-8                                           */
  int32_t max_iter;         /* default 1000                                           */
  int32_t stop;             /* PCG_STOP_RESIDUAL: ||r||/||f|| <= tol (default);
                               PCG_STOP_PRECONDITIONED: sqrt(<r,z>/<r0,z0>) <= tol;
                               r is CG's updated residual: the true residual (relres
                               below) can differ from it by about cond(A) x 1e-16, so
                               near that level relres may end slightly above tol      */
  int32_t flexible;         /* -1 auto (on for FP32/BF16 V-cycles), 0 off, 1 on        */
  int32_t use_x0;           /* 1: u_dev holds the initial guess, 0: start from zero    */
  int32_t use_graph;        /* 1: replay iterations as a CUDA graph (default 1)       */
  const volatile int32_t* cancel_host; /* optional host flag; nonzero cancels: read
                               on the host after every chunk of two iterations,
                               while the next chunk is already queued; the solve
                               then returns FEM_ECANCELLED with its iterate so far,
                               unless it converged or stopped by the end of the
                               chunks it ran (then its own status is returned)      */
} pcg_opts;

typedef struct {
  int32_t iterations;
  int32_t status;           /* fem_status of the solve                                 */
  double relres;            /* ||f - A u|| / ||f||, recomputed at the end: in FP64, or
                               for tol >= 1e-10 on the uniform grid with the
                               double-float operator (rows within 2^-44 sum|a_ij u_j|) */
  double prec_relres;       /* sqrt(<r,z>/<r0,z0>) at the last iteration               */
  double solve_ms;          /* device time of the iterations (CUDA events)             */
} pcg_result;

void pcg_default_opts(pcg_opts* opts);

/* Solve (rho K + M) u = f by CG preconditioned with the V-cycle of hier (Sec. 4), or
 * with the diagonal when hier is NULL.  f_dev NULL means the assembled load vector.
 * nrhs = 1: u_dev is length N.  nrhs > 1: f_dev/u_dev are [N][nrhs] row-major and
 * rho_k_host gives one rho per column (the system must keep its pencil, the hierarchy
 * must come from amg_setup on it); each column is an independent solve.  res points to
 * nrhs results.  Returns FEM_OK when every column converged.  On the uniform grid the
 * columns' CG operator (nrhs > 1 and batch sessions) runs in double-float arithmetic --
 * search directions rounded to 48 bits, each row within 2^-44 sum_j |a_ij p_j| as for
 * fem_spmv_timed -- when tol >= 1e-12, and in FP64 for smaller tolerances; a column whose
 * direction leaves the pairs' range takes FP64 for that iteration. */
fem_status pcg_solve(fem_system sys, amg_hier hier, const double* f_dev, double* u_dev,
                     int32_t nrhs, const double* rho_k_host, const pcg_opts* opts,
                     void* stream, pcg_result* res);

/* ------------------------------------------------------------------ BDDC (Sec. 3.2)
 *
 * CG on the interface Schur complement S_C u_C = g preconditioned by the two-level BDDC
 * preconditioner P^-1 = R_D^T (T_sub + T_0) R_D of Sec. 3.2, on the uniform Kuhn mesh split
 * into `slabs` slabs of whole cube layers along z (slab s: layers [floor(s n / slabs),
 * floor((s+1) n / slabs))).  Interface: the slabs - 1 vertex planes between slabs; primal
 * constraints: the average over each plane; scaling D = 1/2 (every interface unknown lies in
 * two slabs).  Each slab assembles its own Neumann and internal systems from its tets (the
 * P1 element matrices of the global system) and solves them with FP64 AMG-PCG to inner_tol.
 * A process may set up a range of the slabs [slab_begin, slab_end): the sums over slabs then
 * go through `reduce` (every rank passes the same sequence of calls; interface and coarse
 * vectors are replicated); with all slabs in one process, reduce may be null.  The stopping
 * test of bddc_solve is ||r_C|| <= tol ||g|| on the interface system; res->relres is the
 * global ||f - A u|| / ||f|| in FP64, res->iterations the CG iterations. */
typedef struct bddc_s* bddc_solver;
typedef void (*fem_allreduce_fn)(double* buf, int64_t count, int32_t on_device, void* ctx);
typedef struct {
  int32_t slabs;        /* 2 <= slabs <= n/2                                         */
  int32_t slab_begin;   /* slabs owned by this process: [slab_begin, slab_end)        */
  int32_t slab_end;     /* 0: up to slabs                                             */
  double inner_tol;     /* relative residual of the subdomain AMG-PCG solves, < 1e-6 */
} bddc_opts;

/* The slab layers (host only, no GPU needed): layer_begin[0..slabs] (nullable) and the
 * interface unknowns (slabs - 1) (n - 1)^2.  FEM_EINVAL for n < 4 or slabs out of range. */
fem_status fem_bddc_partition(int32_t n, int32_t slabs, int32_t* layer_begin,
                              int64_t* interface_unknowns);

/* Set up the owned slabs' systems, hierarchies, constraint solves and the coarse matrix of
 * a Kuhn-mesh system (uniform grid).  Errors: FEM_EINVAL (null argument, a general or
 * jittered mesh, slabs out of range, inner_tol outside (0, 1e-6)), FEM_ENOCONV (a
 * constraint solve did not converge), FEM_ENOMEM. */
fem_status bddc_setup(fem_system sys, const bddc_opts* opts, fem_allreduce_fn reduce, void* ctx,
                      void* stream, bddc_solver* out);

/* Solve A u = f (f_dev: device [N], null for the assembled load vector) into u_dev (device
 * [N]; on every rank the whole solution after the final all-reduce).  Statuses as
 * pcg_solve (FEM_ENOCONV after opts->max_iter interface iterations). */
fem_status bddc_solve(bddc_solver b, const double* f_dev, double* u_dev, const pcg_opts* opts,
                      fem_allreduce_fn reduce, void* ctx, void* stream, pcg_result* res);

/* Wall time of bddc_setup in ms. */
double bddc_get_setup_ms(bddc_solver b);

void bddc_destroy(bddc_solver b);

/* Discrete H^-1 error of a solution (Tables 3, 6 and 8 report ||ubar - u_h||^2 in H^-1
 * without stating its discrete form): with w = scale * target,
 *   hm1sq = r^T K^-1 r,   r_i = (w - u_h, phi_i)_{L2} = scale * f_i(target) - (M u)_i,
 * the square of sup_v (w - u_h, v) / ||grad v|| over the P1 functions v with zero boundary
 * values.  f(target) is the load vector fem_assemble builds for that target (the same
 * quadrature), M and K the system's mass and stiffness matrices, u_h the P1 function with
 * the nodal values u_dev (length N, interior unknowns).  K^-1 r comes from CG preconditioned
 * by an FP64 smoothed-aggregation V-cycle built on K (default amg_opts), started from zero,
 * to ||r_k|| <= tol ||r||; hm1sq is then accurate to about tol^2 cond(K) relative (CG's
 * iterate y_k has r^T y_k = y_k^T K y_k, short of r^T K^-1 r by the squared energy norm of
 * its error).  A uniform Kuhn mesh rebuilds K and M from its stencils; any other system needs
 * keep_pencil at assembly.  The call allocates the stiffness system and its hierarchy and
 * frees them before it returns; it synchronises the stream.  *hm1sq_out receives the value
 * (0 when r = 0), *res (may be null) the stiffness solve's result.  Errors: FEM_EINVAL (null
 * sys / u_dev / target / hm1sq_out, tol outside (0, 1), bad target, a non-uniform system
 * without its pencil), or the stiffness solve's status (FEM_ENOCONV, ...), with the value of
 * the last iterate still written. */
fem_status fem_error_hm1(fem_system sys, const double* u_dev, const fem_target* target,
                         double scale, double tol, void* stream, double* hm1sq_out,
                         pcg_result* res);

/* ------------------------------------------------------------------ batched sessions */

/* A batch session holds up to `slots` independent solves on one system/hierarchy, each
 * with its own rho and right-hand side, advanced together one CG iteration per step
 * (multi-vector SpMM-PCG, no counterpart in the paper).  Slots are admitted and retired
 * between steps, so new solves join while others are in flight (continuous batching).
 * Results of a slot do not depend on the other slots. */
typedef struct pcg_batch_s* pcg_batch;

fem_status pcg_batch_create(fem_system sys, amg_hier hier, int32_t slots, const pcg_opts* opts,
                            void* stream, pcg_batch* out);
/* Load f_dev (length N) and rho into a free slot; *slot_out receives its index. */
fem_status pcg_batch_admit(pcg_batch b, const double* f_dev, double rho, int32_t* slot_out,
                           void* stream);
/* Run `iters` CG iterations for every active slot (one CUDA-graph replay per iteration). */
fem_status pcg_batch_step(pcg_batch b, int32_t iters, void* stream);
/* Host snapshot per slot: status (-1 free, 0 running, 1 converged, 2 failed), iterations,
 * recurrence residual ||r||/||f||.  Arrays of length slots. */
fem_status pcg_batch_poll(pcg_batch b, int32_t* state_host, int32_t* iters_host,
                          double* relres_host, void* stream);
/* Copy the slot's iterate into u_dev (length N), free the slot. */
fem_status pcg_batch_retire(pcg_batch b, int32_t slot, double* u_dev, void* stream);
/* Bytes of device memory a session with these sizes allocates (admission control). */
int64_t pcg_batch_footprint(fem_system sys, amg_hier hier, int32_t slots);
void pcg_batch_destroy(pcg_batch b);

/* ------------------------------------------------------------------ misc */

/* Message of the last failure on this thread ("" if none). */
const char* fem_last_error(void);

/* Launch-shape autotuner (no counterpart in the paper).  Kernels with several launch
 * shapes -- lanes per row of the CSR SpMV, tile rows and planes per block of the stencil,
 * block shape of the multivector kernels -- are timed once per operator shape with CUDA
 * events, inside amg_setup (single-vector kernels) and pcg_batch_create / batched
 * pcg_solve (multivector kernels), never while a stream is being captured.  The fastest
 * variant is cached for the process under (kernel, rows, stored entries, slots) and used
 * by every later launch of that shape; untuned shapes take a fixed default.  A choice
 * changes only the order of floating-point sums.  Environment: FEM_AUTOTUNE=0 disables
 * timing (defaults everywhere); FEM_AUTOTUNE_CACHE=<file> reads choices from and appends
 * new ones to a text file ("kernel rows entries slots variant" per line).
 *
 * fem_autotune_report: the cache as JSON text, {"enabled": bool, "entries": [{"kernel",
 * "a", "b", "c", "source": "timed"|"file", "pick", "pick_name", "variants": [{"name",
 * "us"}]}]}.  The string is owned by the library (thread-local) and valid until the
 * thread's next call.
 * fem_autotune_clear: forgets every choice and pin (later launches take defaults until
 * tuned again); does not touch the cache file.
 * fem_autotune_pin: forces variant `variant` of kernel family `kernel` for every shape
 * ("stencil_f32", "stencil_f64": 0 shared-memory planes, 1..5 column marching;
 * "csr_f64", "csr_f32", "csr_bf16": lanes per row 1 << variant; "mv_stencil_f32",
 * "mv_stencil_f64", "mv_csr_f32", "mv_csr_f64": see fem_autotune_report's variant names);
 * variant < 0 removes the pin.  A pin outside a family's range is ignored.  Returns
 * FEM_EINVAL for a null kernel name. */
const char* fem_autotune_report(void);
void fem_autotune_clear(void);
fem_status fem_autotune_pin(const char* kernel, int32_t variant);

/* Measured FP64 fused multiply-add throughput of the current GPU in TFLOP/s (2 flops per
 * FMA): `reps` timed launches (CUDA events on the stream, after one untimed launch) of a
 * kernel with 8 independent FMA chains per thread and 8 blocks of 256 threads per SM.  The
 * ceiling of the FP64 kernels, which this GPU's FP64 rate makes ALU-bound rather than
 * HBM-bound.  Synchronises the stream.  Errors: FEM_EINVAL (null tflops_out, reps < 1). */
fem_status fem_measure_fp64_rate(int32_t reps, void* stream, double* tflops_out);

/* Library version string. */
const char* fem_version(void);

/* Number of this library's kernels launched so far in the process (CUDA-graph replays
 * count every kernel they run). */
int64_t fem_kernel_launches(void);

#ifdef __cplusplus
}
#endif

#endif /* FEMAMG_H */
