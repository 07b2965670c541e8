/*
 * dgell.h -- C ABI of the GB300 (sm_103a) matrix-free hp-DG elliptic solver.
 *
 * Method: symmetric interior penalty DG (SIPG) discretisation of
 *     -Lap u + f u = g  in Omega,   u = g_D on the Dirichlet boundary,
 * on h- and p-non-conforming hexahedral meshes (Vincent, Pfeiffer & Fischer,
 * arXiv:1907.01572, Sec. II.A-II.D), with a Chebyshev/CG-eigenvalue smoothed
 * multigrid V-cycle (Sec. II.E, Algs. 3-5) preconditioning flexible CG
 * (Alg. 2), and Newton-Raphson (Alg. 1) for the puncture equation (Sec. III.D).
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Every call returns an int status: DG_OK (0) or one of DG_ERR_*.
 *    dg_last_error() returns a thread-local message for the last failure.
 *  - Vectors are element-blocked: element e of a level owns the contiguous
 *    block [dof_off[e], dof_off[e] + (p_e+1)^3); inside the block the LGL node
 *    (a, b, c) (a along x fastest) is at a + n b + n^2 c, n = p_e + 1.
 *    Element order on the finest level is the order of the mesh description;
 *    on coarser levels it is the order of each coarse element's first
 *    appearance while scanning the finer level (dg_level_leaves reports it).
 *  - Levels follow the paper: 0 is the coarsest, L = n_levels - 1 the finest
 *    (the input mesh).  level = -1 means the finest.
 *  - "device" pointers are CUDA global-memory pointers on the context's
 *    device; they are owned by the caller unless stated otherwise and must
 *    stay valid until the work queued on the context's stream has finished.
 *    All device work is queued on the stream given at context creation.
 *  - Precision codes: DG_FP64 (double vectors, double arithmetic),
 *    DG_FP32 (float vectors, float arithmetic), DG_BF16 (dg_apply only:
 *    bfloat16 input vector, FP32 arithmetic, float output vector).
 */
#ifndef DGELL_H
#define DGELL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DGELL_VERSION 125

enum {
    DG_OK = 0,
    DG_ERR_INVALID = 1,        /* bad argument, malformed mesh (not 2:1, p out of range, ...) */
    DG_ERR_OOM = 2,            /* device allocation failed */
    DG_ERR_CUDA = 3,           /* a CUDA runtime call failed */
    DG_ERR_NOT_CONVERGED = 4,  /* iteration cap reached; statistics are filled */
    DG_ERR_BREAKDOWN = 5,      /* non-finite or non-positive Krylov scalar */
    DG_ERR_UNSUPPORTED = 6     /* valid request this library version does not implement */
};

typedef enum { DG_FP64 = 0, DG_FP32 = 1, DG_BF16 = 2 } dg_prec;

typedef enum {
    DG_MAP_AFFINE = 0,      /* block map = identity on the box [lo, hi]^3 */
    DG_MAP_SINE_WARP = 1    /* x_i += a sin(2 pi k_i x_i) sin(2 pi k_{i+1} x_{i+1}), cyclic i */
} dg_map_kind;

/* Boundary condition of a block face on the domain boundary (Sec. II.A.2,
 * eqs. DirichletBC, NeumannBC, RobinBC).  This version implements Dirichlet
 * data only: a mesh with a Neumann or Robin tag on a boundary face is
 * rejected by dg_mesh_create with DG_ERR_UNSUPPORTED. */
typedef enum { DG_BC_DIRICHLET = 0, DG_BC_NEUMANN = 1, DG_BC_ROBIN = 2 } dg_bc_kind;

typedef enum {
    DG_BLOCK_HEX8 = 0,      /* trilinear map through 8 corners (a box or any parallelepiped) */
    DG_BLOCK_WEDGE = 1,     /* cubed-sphere block between the cube of half-width a and the sphere r */
    DG_BLOCK_SHELL = 2      /* cubed-sphere block of the shell r1 < r < r2, 1/r linear in xi_2 */
} dg_block_kind;

/* One macro-element of a multi-block mesh (Sec. II.A.1; the cubed-sphere
 * domains of Sec. III).  Its map takes the reference cube [-1, 1]^3 to:
 *  HEX8:  sum over corners c = i + 2 j + 4 k of corners[c] times the
 *         trilinear weight of (i, j, k) in {0, 1}^3;
 *  WEDGE: (1 - t) P + t r P / |P|, P = a (s e_d + xi_0 e_t1 + xi_1 e_t2),
 *         t = (xi_2 + 1) / 2, for cube face `face` = 2 d + (s > 0);
 *  SHELL: R(t) P / |P| with 1 / R(t) = (1 - t) / r1 + t / r2.
 * Wedge and shell frames: (t1, t2) = (d+1, d+2) mod 3 for s = +1 and
 * (d+2, d+1) mod 3 for s = -1, so xi_2 points outward and the frame is
 * right-handed.  Blocks meet face to face in any relative orientation; the
 * library finds the block connectivity by matching block face corners. */
typedef struct {
    int kind;              /* dg_block_kind */
    int face;              /* WEDGE, SHELL: cube face 2 d + (s > 0) */
    double corners[8][3];  /* HEX8 */
    double a, r;           /* WEDGE: cube half-width, sphere radius */
    double r1, r2;         /* SHELL: inner and outer radius */
} dg_block;

/* Mesh description (Sec. II.A.1).  With n_blocks = 0: one macro-element, the
 * box [lo, hi]^3 (map_kind, warp_*), refined as an octree.  With n_blocks > 0:
 * the blocks above, element e in block elem_block[e] (lo, hi and map_kind are
 * ignored).  All arrays are HOST memory; dg_ctx_create copies them.  leaves:
 * n_elems x 4 ints (level, ix, iy, iz) in the element's block frame (level
 * <= 15), a level-l leaf covers 1 / 2^l of its block along each axis; leaves
 * must tile every block with at most 2:1 level difference across faces,
 * block interfaces included.  p: n_elems degrees in 1..8.  Geometry is
 * isoparametric: the block map is sampled at each element's own LGL nodes. */
typedef struct {
    double lo[3];
    double hi[3];
    int map_kind;          /* dg_map_kind */
    double warp_amp;       /* a of DG_MAP_SINE_WARP */
    int warp_k[3];         /* k_i of DG_MAP_SINE_WARP */
    int n_elems;
    const int* leaves;     /* host, n_elems * 4 */
    const int* p;          /* host, n_elems */
    int n_blocks;          /* 0: single box */
    const dg_block* blocks;    /* host, n_blocks */
    const int* elem_block;     /* host, n_elems */
    const int* bc;             /* host, 6 per block (6 for the single box), face 2 d + (s > 0):
                                  the dg_bc_kind of that block face where it lies on the domain
                                  boundary (ignored on faces glued to another block); NULL: all
                                  Dirichlet */
} dg_mesh_desc;

/* A validated mesh: the description's copy with its multigrid hierarchy
 * (Sec. II.E.3) and block connectivity, built on the host.  Contexts and
 * footprint queries take it; it may be destroyed once they are made. */
typedef struct dg_mesh dg_mesh;

/* Discretisation options.  penalty_c is C of eq. (penaltyparameter),
 * sigma = C p_m^2 / h_m; <= 0 selects the default 10. */
typedef struct {
    double penalty_c;
    int reserved[4];
} dg_disc_opts;

typedef struct dg_ctx dg_ctx;

typedef struct {
    int n_levels;
    int n_elems;           /* of the requested level */
    int64_t n_dofs;        /* of the requested level */
    int64_t n_vol_qp;      /* volume GL points of the level (sum of (p+1)^3) */
    int64_t n_bnd_qp;      /* Dirichlet-boundary mortar GL points of the level */
    int n_mortars;
    int max_p;
    size_t device_bytes;   /* device memory held by the whole context */
    double apply_flops;    /* floating-point operations of one dg_apply on the level
                              (sum factorisation: 24 n^4 + 18 n^3 per element volume,
                              per mortar side 4 n^3 + 12 q n^2 + 16 q^2 n + 20 q^2) */
} dg_level_info;

int dg_version(void);
const char* dg_last_error(void);

/* Validates a mesh description (Sec. II.A.1: octree leaves tiling every
 * block, 2:1 across faces and block interfaces, degrees 1..8, block maps;
 * boundary tags) and builds, on the host, its block connectivity and its
 * multigrid hierarchy (Sec. II.E.3: surrogate coarsening + 2:1 rebalancing,
 * coarse degree = min over children).  The library copies every array of
 * desc.  Errors: DG_ERR_INVALID (malformed description), DG_ERR_UNSUPPORTED
 * (a Neumann or Robin tag on a boundary face).  No device work. */
int dg_mesh_create(const dg_mesh_desc* desc, dg_mesh** out);
void dg_mesh_destroy(dg_mesh* mesh);

/* Uploads a mesh: mortar tables, the 1-D operator tables and all geometry
 * (eqs. Jacobian, Surface-Jacobian, the normal, eq. penaltyparameter) on the
 * device, for every level of the mesh's hierarchy.  The context keeps its own
 * copy of what it needs from mesh.  stream: a cudaStream_t (NULL = legacy
 * default stream).  Synchronises the stream before return. */
int dg_ctx_create(const dg_mesh* mesh, const dg_disc_opts* opts, void* stream, dg_ctx** out);
void dg_ctx_destroy(dg_ctx* ctx);

/* Device bytes dg_ctx_create would hold for this mesh (admission control);
 * host-only, no device work. */
int dg_ctx_footprint(const dg_mesh* mesh, const dg_disc_opts* opts, size_t* bytes);

int dg_level_info_get(dg_ctx* ctx, int level, dg_level_info* info);

/* Host copies of a level's leaves (n_elems x 4), degrees (n_elems) and
 * element DOF offsets (n_elems + 1).  Any pointer may be NULL. */
int dg_level_leaves(dg_ctx* ctx, int level, int* leaves, int* p, int64_t* dof_off);

/* Host copy of a level's element block indices (n_elems; all 0 for a
 * single-box mesh). */
int dg_level_blocks(dg_ctx* ctx, int level, int* elem_block);

/* Physical coordinates (device, double, 3 x n) of the level's volume GL
 * points (SoA: x[0..n), y[n..2n), z[2n..3n)), element by element, point
 * (i, j, k) of element e at vol_qp_off[e] + i + q j + q^2 k, q = p_e + 1.
 * Same for the Dirichlet-boundary mortar points (bnd).  Either may be NULL. */
int dg_quadrature_points(dg_ctx* ctx, int level, double* vol_xyz, double* bnd_xyz);

/* y = L x: the SIPG operator of eq. (lh2) (stiffness + consistency +
 * symmetry + penalty on interior and Dirichlet mortars, plus the zeroth-order
 * term int f u v when one was set with dg_set_zeroth_order), applied
 * matrix-free on level `level` (Sec. II.A.5, eq. harald-stiff; mortar
 * integrals with hp mortar projection, mortar figure).  x, y: device
 * vectors of the level's n_dofs in precision prec (double for DG_FP64,
 * float for DG_FP32; DG_BF16: x bfloat16, y float); x and y must not
 * overlap.  Asynchronous. */
int dg_apply(dg_ctx* ctx, int level, int prec, const void* x, void* y);

/* dg_apply on nvec vectors held in HOST memory: y_r = L x_r, r < nvec (the
 * operator of eq. (lh2) as for dg_apply).  hx: HOST, nvec input vectors of the
 * level's n_dofs values each, back to back; hy: HOST, nvec outputs in the same
 * layout; double for DG_FP64, float for DG_FP32 (DG_BF16: DG_ERR_UNSUPPORTED).
 * The copy of vector r+1 to the device and of vector r-1 back run on two copy
 * streams of the context while vector r is applied on its stream, through two
 * device staging slots per direction that the context allocates on first use
 * (4 n_dofs values of the precision, kept until dg_ctx_destroy; not counted by
 * dg_ctx_footprint).  The host buffers should be page-locked (cudaHostAlloc or
 * cudaHostRegister) for the copies to overlap the applies; pageable memory
 * gives the same results.  Asynchronous: the context's stream waits for the
 * last copy, so hy is complete once that stream is synchronised; hx and hy
 * must stay untouched until then.  nvec = 0 does nothing.  Not for use
 * inside stream capture (the first call allocates). */
int dg_apply_host(dg_ctx* ctx, int level, int prec, int nvec, const void* hx, void* hy);

/* Right-hand side F_h of eq. (equationFh2) on the finest level:
 * F = int g v - int_{Gamma_D} g_D n.grad v + int_{Gamma_D} sigma g_D v.
 * g_qp: device double values of g at the finest level's volume GL points
 * (dg_quadrature_points order) or NULL for g = 0; gD_qp: device double values
 * of g_D at the boundary mortar points or NULL for g_D = 0.  F: device
 * double, n_dofs.  Asynchronous. */
int dg_rhs(dg_ctx* ctx, const double* g_qp, const double* gD_qp, double* F);

/* Chebyshev smoother (Alg. 4) with CG spectral bound (Alg. 5).  Smooths
 * J x = b on `level` in place: n_eigs CG steps (which also update x) give
 * lambda_max by Gershgorin on the Lanczos tridiagonal; then n_cheb Chebyshev
 * steps on [lambda_max / Lambda, lambda_max].  b, x: device vectors of the
 * level in precision prec.  lambda_max_out: host pointer or NULL (forces a
 * stream synchronisation when given). */
typedef struct {
    int n_eigs;        /* N_iter,eigs; <= 0 -> 15 */
    int n_cheb;        /* N_iter,Cheb; <= 0 -> 15 */
    double Lambda;     /* lambda_max / lambda_min; <= 0 -> 20 */
    double lam_scale;  /* the Chebyshev interval uses lam_scale x the CG estimate of lambda_max
                          (a safety factor against an underestimate on strongly stretched
                          meshes); <= 0 -> 1, the paper's Alg. 4 */
    double lam_fixed;  /* > 0: no CG steps; the Chebyshev steps use lambda_max = lam_fixed on
                          every level (a linear smoother, Alg. 4 with a given bound instead of
                          Alg. 5's estimate); <= 0 -> the CG estimate (the paper) */
} dg_cheb_opts;

int dg_smooth(dg_ctx* ctx, int level, int prec, const void* b, void* x,
              const dg_cheb_opts* opts, double* lambda_max_out);

/* dg_smooth without any device allocation.  The paper has no counterpart:
 * this entry point exists for callers that cannot call cudaMalloc when they
 * smooth (all free device memory already handed to a caching allocator or
 * admitted to other work, or loops that cannot take cudaMalloc's implicit
 * device synchronisation).  Same arguments, algorithm and results as
 * dg_smooth (on levels of at most 1024 DOFs dg_smooth applies the assembled
 * operator and this call the matrix-free one, so there FP32 results agree up
 * to rounding, which the CG steps amplify), but its work vectors and
 * reduction scratch live in one
 * fixed-size array compiled into the library (about 6 MB, reserved on every
 * GPU that loads the library until the process exits), so the level must have
 * at most 262,144 DOFs (larger levels: DG_ERR_INVALID).  The first call on a
 * device looks up the array's device address (cudaGetSymbolAddress, that
 * device current): make it before any stream capture.  All calls share the
 * array and it keeps the previous call's contents (the call clears what must
 * start at zero); calls whose GPU work overlaps -- other streams, other
 * threads -- race on it. */
int dg_smooth_static(dg_ctx* ctx, int level, int prec, const void* b, void* x,
                     const dg_cheb_opts* opts, double* lambda_max_out);

/* Multigrid V-cycle (Alg. 3) as a preconditioner: v = VCYCLE(f) on the
 * finest level, starting from v = 0 on every level, pre- and post-smoothing
 * with dg_smooth's smoother, restriction = transpose of the prolongation
 * (eq. temp-G), coarse level: smoother (coarse = 0) or exact Cholesky
 * solve (coarse = 1).  f, v: device vectors of the finest level in prec. */
typedef struct {
    dg_cheb_opts cheb;
    int coarse;        /* 0: smoother on level 0 (paper), 1: dense Cholesky */
    int smoother;      /* 0: Chebyshev with CG eigenvalue bound (Alg. 4, 5);
                          1: Schwarz smoother (Alg. 6) with element subdomains and no overlap:
                          n_schwarz cycles of r = b - J x, element-local CG on the element
                          diagonal blocks J_ee dx_e = r_e (all elements at once, to local_tol
                          or local_iters steps), x += schwarz_omega dx;
                          2: Schwarz smoother (Alg. 6) with overlapping subdomains, one per
                          element: its nodes and the touching elements' nodes that coincide
                          with its boundary nodes (one overlap layer), weights w_h of
                          eq. (schwarz_weight) at zero overlap width (1, 1/2, 1/4, 1/8 inside,
                          on faces, edges, corners), exact local solves with inverses of
                          R_s J R_s^T built on first use (and after a change of the
                          operator's coefficients); n_schwarz cycles of r = b - J x,
                          x += sum_s R_s^T W_s (R_s J R_s^T)^-1 R_s r.  Levels with one degree
                          and conforming faces only (else DG_ERR_UNSUPPORTED) */
    int n_schwarz;     /* <= 0 -> 3 (the paper's typical N_s) */
    int local_iters;   /* <= 0 -> 20 */
    double local_tol;  /* relative; <= 0 -> 1e-3 (the paper's local tolerance) */
    double schwarz_omega;  /* damping; <= 0 -> 0.7 (without overlap the paper's weights are 1) */
} dg_mg_opts;

int dg_vcycle(dg_ctx* ctx, int prec, const void* f, void* v, const dg_mg_opts* opts);

/* Flexible CG (Alg. 2) on the finest level, FP64 vectors, preconditioned by
 * the V-cycle in precision opts->mg_prec (DG_FP64: the plain FP64 form;
 * DG_FP32: FP32 V-cycle inside the FP64 Krylov loop, i.e. mixed precision).
 * b, x: device double, n_dofs; x holds the initial guess on entry.  Stops
 * when ||b - J x||_2 <= tol ||b||_2 (recursive residual, confirmed with a
 * true FP64 residual: while the true one is still above tol, FCG restarts
 * from x with r = b - J x, at most 3 times) or after max_iter iterations in
 * all. */
typedef struct {
    double tol;        /* relative residual target; <= 0 -> 1e-10 */
    int max_iter;      /* N_iter,FCG; <= 0 -> 100 */
    int mg_prec;       /* precision of the V-cycle: DG_FP64 or DG_FP32 */
    int use_mg;        /* 0: no preconditioner (plain CG iterates) */
    dg_mg_opts mg;
    int graph_mode;    /* 0: after one eager V-cycle, capture it once as a CUDA graph and
                          replay it (needs a non-default stream); 1: always launch eagerly */
} dg_solver_opts;

typedef struct {
    int iterations;
    double rel_residual;       /* true ||b - J x|| / ||b|| at exit */
    double rel_residual_rec;   /* recursive residual at exit */
    double seconds;            /* host wall time of the call */
    int status;
} dg_solve_stats;

int dg_solve(dg_ctx* ctx, const double* b, double* x, const dg_solver_opts* opts, dg_solve_stats* stats);

/* Zeroth-order term int f u v of eq. (lh2) on the finest level:
 * coef_qp: device double values of f at the finest level's volume GL
 * points (NULL clears the term).  Coarse levels get the Galerkin form
 * O^H = I^T O^h I of eq. (operator_oh) as dense per-element blocks. */
int dg_set_zeroth_order(dg_ctx* ctx, const double* coef_qp);

/* Puncture initial data (Sec. III.D, eqs. Two_Punctures_PDE, Two_Punctures_Aij):
 * R(u) = -Lap u - beta (1 + alpha (1 + u))^-7, u = 0 on the box boundary,
 * 1/alpha = sum m_I / (2 r_I), beta = alpha^7 A_ij A^ij / 8,
 * A_ij = sum_I 3 / (2 r_I^2) [P_i n_j + P_j n_i - (delta_ij - n_i n_j) P.n]
 *      + 3 / r_I^3 [n_i (S x n)_j + n_j (S x n)_i]
 * (the printed spin term read with t_(ij) = (t_ij + t_ji) / 2). */
typedef struct {
    int n;                 /* number of punctures, <= 16 */
    double m[16];
    double c[16][3];       /* positions */
    double P[16][3];       /* linear momenta */
    double S[16][3];       /* spins (zero for non-spinning punctures) */
} dg_puncture_params;

/* Evaluates alpha, beta at the finest level's volume GL points and keeps
 * them in the context for dg_newton_*. */
int dg_puncture_setup(dg_ctx* ctx, const dg_puncture_params* params);

/* Weak residual R(u) (device double, n_dofs) of the puncture equation
 * (DG_ERR_INVALID unless the puncture problem is the one set up last). */
int dg_puncture_residual(dg_ctx* ctx, const double* u, double* R);

/* Power-law source (the constant-density star of Sec. III.C,
 * Lap psi + 2 pi rho psi^5 = 0, in the coercive form):
 * R(u) = L u - F - int c u^power v, Jacobian zeroth-order term
 * -power c u^(power-1),
 * with the nonlinearity evaluated at the volume GL points (as the paper
 * does for that problem).  coef_qp: device double, c at the finest level's
 * volume GL points (dg_quadrature_points order), copied; power: 1..9; F:
 * device double n_dofs forcing vector (e.g. dg_rhs with g = 0 for the
 * Dirichlet data), copied, or NULL.  Makes this the problem of dg_newton_*. */
int dg_power_source_setup(dg_ctx* ctx, const double* coef_qp, int power, const double* F);

/* Weak residual R(u) of the nonlinear problem set up last (puncture or
 * power-law source). */
int dg_nonlinear_residual(dg_ctx* ctx, const double* u, double* R);

/* One Newton step (Alg. 1) on the nonlinear problem set up last: sets the
 * Jacobian's zeroth-order term (puncture: 7 alpha beta (1 + alpha (1 + u))^-8),
 * solves J du = -R(u) with dg_solve and updates u += du.  u: device double,
 * n_dofs.  residual_norm_out: host, ||R(u)||_2 before the step (may be NULL). */
int dg_newton_step(dg_ctx* ctx, double* u, const dg_solver_opts* opts, dg_solve_stats* stats,
                   double* residual_norm_out);

/* Newton-Raphson: at most max_newton steps until ||R(u)||_2 < tol_newton. */
int dg_newton_solve(dg_ctx* ctx, double* u, double tol_newton, int max_newton,
                    const dg_solver_opts* opts, int* steps_out, double* residual_norm_out);

/* Inter-level transfer between level `coarse_level` (H) and coarse_level + 1
 * (h) (Sec. II.E.6): direction 0 = prolongation, out_h += I_h^H in_H
 * (eq. psi-interpolation); direction 1 = restriction of a weak residual,
 * out_H = (I_h^H)^T in_h (eq. temp-G).  Device vectors in prec. */
int dg_transfer(dg_ctx* ctx, int coarse_level, int prec, int direction, const void* in, void* out);

/* A-posteriori error estimator eta^2(e) of eq. (Eta2_Local) (Sec. II.D) on
 * the finest level, for -Lap u + f u = g with Dirichlet data g_D:
 *   eta^2(e) = h_e^2 p_e^2 ||f u - g - Lap u||^2_e
 *            + sum over e's interior mortars of
 *                h_m / p_m ||[[grad u]] . n||^2_m + sigma p_m^2 / h_m ||[[u]]||^2_m
 *            + sum over e's Dirichlet mortars of sigma p_m^2 / h_m ||u - g_D||^2_m
 * (eqs. Eta2_Ingredients, Eta2_Integrals, weights as printed there), with
 * h_e the largest distance between two vertices of e, p_m, h_m and sigma
 * those of the operator's penalty (eq. penaltyparameter), Lap u the exact
 * Laplacian of the mapped polynomial on the isoparametric element, and
 * every norm by the operator's own GL quadrature.  Each interior mortar's
 * terms count in full for both of its elements.  Geometry: the isoparametric
 * interpolant on single-box meshes, the exact block maps (with their second
 * derivatives in Lap u) on multi-block meshes, as in the operator.
 * u: device double, n_dofs; g_qp, f_qp: device double values at the finest
 * level's volume GL points (dg_quadrature_points order), NULL for 0 (pass
 * the coefficient given to dg_set_zeroth_order as f_qp); gD_qp: device
 * double values at the Dirichlet mortar points, NULL for 0.  eta2: device
 * double, n_elems (output).  Queues one FP64 apply of u (overwriting the
 * level's trace buffer), on single boxes a node-coordinate kernel, and the
 * estimator kernel; takes n_dofs doubles (single box: 4 n_dofs) of
 * stream-ordered scratch (cudaMallocAsync) for the duration of the call.
 * Asynchronous. */
int dg_estimate(dg_ctx* ctx, const double* u, const double* g_qp, const double* f_qp, const double* gD_qp,
                double* eta2);

/* dg_estimate with a fiducial grid (Sec. II.D, the fiducial-grid paragraph;
 * Problem C's compactified grid): on a multi-block mesh, `fiducial` (HOST,
 * n_fiducial = the mesh's block count) gives other maps for the same blocks
 * (same kinds and cube faces, other corners or radii; e.g. the shell pulled
 * in from r2 = 1e9 to a moderate radius).  The integrands R_e and J_{m,.}
 * stay those of the physical grid; the weights of every norm (w det J,
 * w S^m), h_e, h_m and sigma are the fiducial grid's.  fiducial = NULL is
 * dg_estimate.  The geometry of the mortars on the fiducial grid is computed
 * into stream-ordered scratch (7 doubles per mortar point) for the call.
 * DG_ERR_INVALID: single-box mesh with a fiducial grid, block count, kinds or
 * faces that differ, or a fiducial grid that folds a face. */
int dg_estimate_fiducial(dg_ctx* ctx, const dg_block* fiducial, int n_fiducial, const double* u,
                         const double* g_qp, const double* f_qp, const double* gD_qp, double* eta2);

/* hp-AMR driving strategy (Sec. II.D, Algorithm 4, smooth-pred).  Host code,
 * no context and no GPU needed. */
typedef enum { DG_AMR_NONE = 0, DG_AMR_P_REFINE = 1, DG_AMR_H_REFINE = 2 } dg_amr_action;
typedef enum {
    DG_MARK_FRACTION = 0,   /* refine the ceil(theta n) elements with the largest eta^2 (ties: lower index) */
    DG_MARK_MEAN = 1        /* refine where eta^2 > theta * mean(eta^2) (sum in element order) */
} dg_mark_kind;

typedef struct {
    int criterion;          /* dg_mark_kind */
    double theta;           /* FRACTION: share of elements in (0, 1]; MEAN: factor >= 0 on the mean
                               (DG_ERR_INVALID outside these ranges) */
    double gamma_h;         /* Algorithm 4's gamma_h; <= 0 selects 0.25 */
    double gamma_p;         /* Algorithm 4's gamma_p; <= 0 selects 0.1 */
    int p_max;              /* largest degree; <= 0 selects 8 (the library's limit) */
    int level_max;          /* deepest octree level; <= 0 selects 15 (the library's limit) */
} dg_amr_opts;

/* Marks elements (opts->criterion) and applies Algorithm 4 to each marked
 * one: h-refine when eta2[e] > pred[e], else p-refine; a p-refinement at
 * p_max becomes an h-refinement, an h-refinement at level_max a
 * p-refinement (nothing when p = p_max too).  pred_next[e] is what the
 * element carries on: gamma_p eta2[e] (p-refined), the prediction of each
 * child gamma_h 2^-3 2^(-2 p_e) eta2[e] (h-refined), pred[e] (unchanged).
 * Start with pred = +inf for the p-first start the text of Sec. II.D
 * describes, 0 for Algorithm 4 taken literally.  All arrays HOST, n_elems
 * long: eta2, pred, p, level (in), action (dg_amr_action), pred_next (out). */
int dg_hp_mark(int n_elems, const double* eta2, const double* pred, const int* p, const int* level,
               const dg_amr_opts* opts, int* action, double* pred_next);

/* Applies the actions to a single-box leaf set (dg_mesh_desc leaves and p)
 * and then refines further until every pair of face neighbours differs by
 * at most one level (2:1).  h-refined elements become their 8 children
 * (child c = i + 2 j + 4 k at (2 ix + i, 2 iy + j, 2 iz + k), in place of
 * the parent) with the parent's degree and prediction pred_next[e];
 * p-refined ones get p + 1; children of balance-only refinements keep the
 * degree and get pred_init.  parent_out[k]: the input element new leaf k
 * lies in.  HOST arrays.  *n_out receives the new element count; the
 * outputs (leaves_out 4 per element, p_out, pred_out, parent_out; any may
 * be NULL) are written when n_out <= max_out, else DG_ERR_INVALID is
 * returned with *n_out set (call again with enough room).  DG_ERR_INVALID
 * also for an h-refinement past level 15, a degree past 8, or leaves
 * outside their level's index range. */
int dg_hp_refine(int n_elems, const int* leaves, const int* p, const int* action, const double* pred_next,
                 double pred_init, int max_out, int* n_out, int* leaves_out, int* p_out, double* pred_out,
                 int* parent_out);

/* dg_hp_refine for any mesh description (dg_ctx_create's): with blocks,
 * leaves are refined and 2:1-balanced inside their blocks and across block
 * interfaces (the block connectivity found as for dg_ctx_create); children
 * stay in their parent's block (block_out, may be NULL).  mesh->leaves,
 * mesh->p and mesh->elem_block are the input elements; action and pred_next
 * are n_elems long.  Same outputs, ordering and errors as dg_hp_refine, plus
 * DG_ERR_INVALID for a bad block description. */
int dg_hp_refine_mesh(const dg_mesh_desc* mesh, const int* action, const double* pred_next, double pred_init,
                      int max_out, int* n_out, int* leaves_out, int* p_out, int* block_out, double* pred_out,
                      int* parent_out);

/* Vector helpers used by the binding's tests and the bench (device memory,
 * on the context stream): precision conversion double <-> float. */
int dg_convert(dg_ctx* ctx, int64_t n, int src_prec, const void* src, int dst_prec, void* dst);

/* Kernel launches issued by the library since context creation (counter of
 * this library's own kernels). */
int64_t dg_launch_count(dg_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* DGELL_H */
