/*
 * enp_dg.h -- C ABI of the GB300 (sm_103a) discontinuous Galerkin operator for
 * the electroneutral Nernst-Planck equations in charge-conservation form (CNP).
 *
 * The operator is the DG scheme of Sec. 3.3 (Eq. NPDG for the species
 * c_1..c_{m-1}, Eq. chargeDG for the potential Phi; c_m is eliminated by
 * Eq. substitution), on structured tensor-product quadrilateral (2D) and
 * hexahedral (3D) meshes with a nodal Gauss-Lobatto basis of degree p and
 * Gauss-Legendre quadrature with q = p + 2 points per direction (Sec. 4:
 * "higher-order quadrature rules compared to the polynomial degree").
 *
 * Vector layout (every double/float vector argument): device memory, caller
 * owned, contiguous, indexed [b][f][e][i]:
 *   b  operating point, 0 <= b < batch (enp_disc_desc.batch);
 *   f  field: 0 = Phi (charge-conservation rows), k = c_k for k = 1..m-1;
 *   e  element, lexicographic with x fastest;
 *   i  node, lexicographic with x fastest, (p+1)^dim per element.
 * This is the block ordering [R_Phi; R_c1; ...; R_c(m-1)] of Sec. 4 (Eq. blockmatrix).
 *
 * Calls are asynchronous on the handle's CUDA stream unless stated. They return
 * an enp_status; on failure enp_last_error() gives a message. No call throws,
 * aborts or traps. Device pointers must be 8-byte aligned (4 for float).
 * A handle is not thread-safe: one host thread at a time.
 */
#ifndef ENP_DG_H
#define ENP_DG_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct enp_dg* enp_handle;

typedef enum {
  ENP_OK = 0,
  ENP_ERR_INVALID_ARG = 1,   /* a null pointer, an out-of-range size or parameter */
  ENP_ERR_CUDA = 2,          /* a CUDA runtime error (message in enp_last_error) */
  ENP_ERR_OOM = 3,           /* device allocation failed */
  ENP_ERR_NONFINITE = 4,     /* a NaN/Inf was found where the call checks for one */
  ENP_ERR_NOT_CONVERGED = 5, /* an iterative solve stopped at its iteration limit */
  ENP_ERR_TIMEOUT = 6,       /* reserved: no call of this build returns it (no device-side
                                waits; host-driven loops end at their iteration limits) */
  ENP_ERR_UNSUPPORTED = 7    /* a valid configuration this build does not implement */
} enp_status;

/* Boundary face tags (one byte per boundary face). The boundary classification of
 * Sec. 2.1 (inlet, outlet, wall, electrode), plus DIRICHLET for manufactured
 * solutions (Sec. 5.1: "all boundary conditions ... prescribed using the exact
 * solutions"), imposed weakly in Nitsche form. */
enum {
  ENP_FACE_WALL = 1,       /* Eq. wall: no term */
  ENP_FACE_INLET = 2,      /* Eq. inlet: + int (u.n) c_k^in v */
  ENP_FACE_OUTLET = 3,     /* Eq. NPDG outlet term: + int (q_k.n) c_k v */
  ENP_FACE_DIRICHLET = 4,  /* exterior state from enp_set_sources */
  ENP_FACE_ELECTRODE0 = 5  /* electrode j = tag - 5 (j < 4), Butler-Volmer Eq. bv */
};

enum { ENP_VEL_CONSTANT = 0, ENP_VEL_PLATE = 1 };
#define ENP_MAX_SPECIES 4

/* Structured box mesh. Host arrays, read during enp_dg_create only.
 * coords[a]: n_el[a]+1 strictly increasing vertex coordinates along axis a.
 * face_tag[s]: boundary side s = 2a + (0 low, 1 high), one tag per face, faces
 * numbered lexicographically over the remaining axes (lowest axis fastest). */
typedef struct {
  int dim;                          /* 2 or 3 */
  int n_el[3];                      /* elements per axis (n_el[2] ignored in 2D) */
  const double* coords[3];
  const unsigned char* face_tag[6];
} enp_mesh_desc;

/* Physical parameters (Sec. 2). mu_k = D_k / RT (Eq. NE). F = RT = 1 gives the
 * nondimensional form of Sec. 2.3 when concentrations are scaled by c^in.
 * velocity_kind CONSTANT: u = (vel_params[0..2]).
 * velocity_kind PLATE (Sec. 5.2): flow axis A = vel_params[0], normal axis
 *   N = vel_params[1], wall at y0 = vel_params[2], height H = vel_params[3],
 *   mean speed vel_params[4]: u_A = 6 u_avg s (H - s) / H^2, s = x_N - y0.
 * Butler-Volmer (Eq. bv), with the reductant the solid electrode (ratio 1):
 *   J_n = J_0 [exp(alpha1 n F/RT (phi_app_j - Phi)) - (c_o/c_ref)^gamma exp(-alpha2 n F/RT (phi_app_j - Phi))],
 *   g_ox = J_n / (n F) (species row of the oxidant, if not c_m), g = z_ox J_n / n
 *   (charge row). J_0 is constant, or with bv_J0_axis >= 0 the profile
 *   3/5 J_0 [2 - ((t - w/2)/(w/2))^2], t = x_axis - lo, w = hi - lo (Sec. 5.2). */
typedef struct {
  int m;                            /* species, 2 <= m <= ENP_MAX_SPECIES; z[m-1] != 0 */
  double z[ENP_MAX_SPECIES];
  double D[ENP_MAX_SPECIES];
  double c_in[ENP_MAX_SPECIES];
  double F, RT;
  int velocity_kind;
  double vel_params[8];
  int bv_oxidant;                   /* species index of the oxidant (0-based), -1: no reaction */
  double bv_J0, bv_alpha1, bv_alpha2, bv_n, bv_gamma, bv_c_ref;
  double bv_phi_app[4];             /* applied potential of electrodes 0..3 */
  int bv_J0_axis;
  double bv_J0_lo, bv_J0_hi;
} enp_physics_desc;

/* Discretisation: delta_p = C_IP p^2 / h (Eq. deltap) with h the element
 * diagonal (mean of both elements on an interior face); the paper uses C_IP = 10. */
typedef struct {
  int p;          /* 1..4 in 3D, 1..3 in 2D */
  int q;          /* Gauss points per direction; must be p + 2 */
  double C_IP;
  int batch;      /* operating points carried by every vector, >= 1 */
} enp_disc_desc;

/* Create an operator handle. Uploads the mesh, tags and basis tables, using
 * stream (a cudaStream_t, may be 0) for every later call. Synchronises once.
 * On hexahedral meshes the handle also owns the face buffer through which the
 * face kernel hands each face's terms to the element kernel: faces x 4 x m x
 * (p+1)^2 x batch doubles (about 3 E of the faces; 154 MB per operating point
 * for 64x32x16 elements at p = 3, m = 3). Calls on one handle share it and the
 * solver workspace, so they must not overlap on the GPU (use one handle per
 * concurrent stream). Errors: INVALID_ARG (bad descriptor), UNSUPPORTED (p, q,
 * m or dim outside the compiled set), OOM, CUDA. *out is NULL on failure. */
enp_status enp_dg_create(enp_handle* out, const enp_mesh_desc* mesh,
                         const enp_physics_desc* phys, const enp_disc_desc* disc,
                         void* stream);
enp_status enp_dg_destroy(enp_handle h);

/* Sizes: DOFs per operating point (m * E * (p+1)^dim), fields, nodes and
 * quadrature points per element, boundary faces. Any pointer may be NULL. */
enp_status enp_dg_sizes(enp_handle h, long long* n_dof, int* n_fields, int* n_nodes,
                        int* n_qpoints, int* n_bfaces);

/* Replace the stream later calls run on (a cudaStream_t). */
enp_status enp_set_stream(enp_handle h, void* stream);

/* Optional problem data, copied into handle-owned device memory (NULL clears):
 *   src [m][E][q^dim]: volume sources at the Gauss points (field 0: f of
 *       Eq. chargeDG; field k: R_k of Eq. NPDG), subtracted as -int src v;
 *   dir [m][NBF][q^(dim-1)]: exterior states (Phi, c_1..c_{m-1}) at the Gauss
 *       points of every boundary face (side-major, face order as face_tag,
 *       points lexicographic, lower axis fastest); read on DIRICHLET faces.
 * Both are device pointers, read before the call returns. */
enp_status enp_set_sources(enp_handle h, const double* src, const double* dir);

/* Applied electrode potentials per operating point, host array [batch][4]
 * (NULL: every operating point uses bv_phi_app). Copied. */
enp_status enp_set_phi_app(enp_handle h, const double* phi_app);

/* Physical coordinates of the volume Gauss points [E][q^dim][3] and of the
 * boundary-face Gauss points [NBF][q^(dim-1)][3] (device pointers, either NULL). */
enp_status enp_quadrature_points(enp_handle h, double* xq, double* xbq);

/* Arithmetic of the FP64 operator on hexahedral meshes: enp_residual,
 * enp_jvp, enp_vjp, enp_block_diagonal (and the FP64 block-Jacobi setup), and
 * the FP64 residual and J v inside the Newton and FGMRES solvers; vectors stay
 * FP64 in and out either way. dR/dtheta and the sweep's face terms always use
 * the FP64 kernels.
 *   ENP_ARITH_F64  (default): native FP64 arithmetic. GB300 issues 2 FP64
 *                  fused multiply-adds per clock per SM, so this path is bound
 *                  by the FP64 pipe.
 *   ENP_ARITH_DF32: double-float arithmetic on the FP32 pipe (each value the
 *                  unevaluated sum of two binary32 numbers, about 48 significant
 *                  bits; error-free TwoSum/TwoProd building blocks). Agrees with
 *                  the FP64 evaluation to about 1e-14 relative; magnitudes below
 *                  2^-126 are flushed to zero and above 2^127 overflow.
 * The paper computes in FP64 (Sec. 4.3); this is an implementation choice of
 * the same operator. On 2D meshes the call is accepted and the operator stays
 * FP64. Takes effect at the next call. Errors: INVALID_ARG. */
#define ENP_ARITH_F64 0
#define ENP_ARITH_DF32 1
enp_status enp_set_arithmetic(enp_handle h, int arith);
enp_status enp_get_arithmetic(enp_handle h, int* arith);

/* r = R(u): the left-hand sides of Eq. NPDG (rows f = 1..m-1) and Eq. chargeDG
 * (rows f = 0), tested with every basis function. u, r: [batch][m][E][Np]. */
enp_status enp_residual(enp_handle h, const double* u, double* r);

/* jv = J(u) v, the Gateaux derivative of R at u in direction v (Eq. blockmatrix),
 * matrix-free (Sec. 4.3). d|x|/dx is taken as 0 at x = 0. */
enp_status enp_jvp(enp_handle h, const double* u, const double* v, double* jv);

/* The same in single precision (inner Krylov operator of the mixed-precision
 * solve): u, v, jv are float vectors in the same layout. */
enp_status enp_jvp_f32(enp_handle h, const float* u, const float* v, float* jv);

/* jtw = J(u)^T w, the adjoint of enp_jvp, by element-local recomputation (no
 * stored quadrature-point state). The paper has no adjoint; this is the
 * transpose of Eq. blockmatrix. */
enp_status enp_vjp(enp_handle h, const double* u, const double* w, double* jtw);

/* c_m = -(1/z_m) sum_{k<m} z_k c_k at every node (Eq. substitution): the
 * eliminated concentration. u: [batch][m][E][Np]; cm: [batch][E][Np]. */
enp_status enp_recover_cm(enp_handle h, const double* u, double* cm);

/* out[b] = <x_b, y_b> for every operating point b (host array of batch
 * doubles). Reduced on the device in a fixed order (warp shuffles, one partial
 * per thread block, then one block), so the result does not depend on timing.
 * Synchronises the stream. */
enp_status enp_inner_product(enp_handle h, const double* x, const double* y, double* out);

/* The element-diagonal blocks of J(u): for every element K, the derivative of
 * K's rows with respect to K's own unknowns (volume terms and K's side of every
 * face term, all fields coupled). The "element-wise Jacobi" of Sec. 4.2, which
 * ignores inter-element couplings. blocks: device [batch][E][nb][nb] row-major,
 * nb = m * Np, row/column index f * Np + i. */
enp_status enp_block_diagonal(enp_handle h, const double* u, double* blocks);

/* Assemble and invert the element-diagonal blocks of J(u) (Gauss-Jordan with
 * partial pivoting) and keep the inverses in handle-owned memory, stored as
 * 0 = FP64, 1 = FP32, 2 = BF16. Storage 0 assembles and inverts in FP64; 1 and 2
 * assemble (with the FP32 operator) and invert in FP32: the preconditioner of
 * a flexible Krylov method need not be exact. Synchronises.
 * Errors: NONFINITE if a block is singular or not finite. */
enp_status enp_block_jacobi_setup(enp_handle h, const double* u, int storage);

/* y = M^{-1} x with M the preconditioner of the last setup: the inverse block
 * diagonal (or, with enp_set_sweep on, the downwind block Gauss-Seidel sweep),
 * plus the coarse correction when the two-level preconditioner is on.
 * x, y: device [batch][m][E][Np], not overlapping. Runs on the handle's stream.
 * Errors: INVALID_ARG before a setup. */
enp_status enp_block_jacobi_apply(enp_handle h, const double* x, double* y);

/* The same with FP32 vectors, as the FP32 Krylov solve of the mixed-precision
 * Newton method applies it (the sweep's upstream face terms in FP32). */
enp_status enp_block_jacobi_apply_f32(enp_handle h, const float* x, float* y);

/* Memory strategy of the block inverses for large batches: point = -1 (the
 * default) stores one set of element-block inverses per operating point;
 * point >= 0 stores only the inverses of operating point `point` and applies
 * them to every operating point of the batch (a lagged, shared
 * preconditioner: FGMRES is flexible and needs no exact one). The blocks are
 * assembled and inverted one operating point at a time either way, so the
 * setup's FP32 staging holds one point's blocks. For the plate reactor at
 * p = 4 (147,456 elements, blocks of 250 x 250) one set is 36.9 GB in FP32 and
 * 18.4 GB in BF16: eight sets would not fit next to the Krylov basis in
 * 288 GB, one does. The two-level coarse correction stays per point.
 * Takes effect at the next setup. Errors: INVALID_ARG. */
enp_status enp_set_shared_blocks(enp_handle h, int point);

/* Choose the preconditioner that the next enp_block_jacobi_setup builds (and
 * that FGMRES and Newton then use). two_level = 0: block-Jacobi alone (the
 * element-wise Jacobi of Sec. 4.2, the default). two_level = 1 (hexahedral
 * meshes): block-Jacobi plus an additive coarse correction on the element-mean
 * potential, P V(P^T r), with P the constant on the potential nodes of each
 * element; A0 = P^T J_PhiPhi(u) P, a 7-point stencil on the element grid, is
 * assembled exactly from 7 coloured J v products at setup, and V is one
 * multigrid V-cycle on it (2 x 2 x 2 Galerkin aggregation, red-black
 * Gauss-Seidel, 2 + 2 sweeps per level, prolongation over-corrected by 1.8; the coarsest grid, of at most 128
 * cells, solved with its dense inverse, or by 100 sweeps if it is singular to
 * working accuracy; the levels of at most 8192 cells run in one launch). A0 is
 * assembled with the FP64 operator when the block inverses are stored in FP64,
 * else with the FP32 one; the V-cycle runs in FP32 (it only preconditions). The Schur-complement-like stiffness of the potential
 * equation (Sec. 3.3) is what block-Jacobi alone cannot reduce.
 * Takes effect at the next setup. Errors: INVALID_ARG (two_level not 0 or 1),
 * UNSUPPORTED (two_level = 1 on a 2D mesh). */
enp_status enp_set_preconditioner(enp_handle h, int two_level);

/* Options of the coarse solve of the two-level preconditioner (defaults 1, 2,
 * 1.8): `cycles` V-cycles per application (1..8; each further cycle solves
 * for the correction of the level-0 residual), `smooth` red-black Gauss-Seidel
 * sweeps before and after each coarse step (1..8), and `omega` (0 < omega <= 3)
 * multiplying every prolongated coarse correction. Piecewise-constant
 * aggregation makes each Galerkin level about twice as stiff as the
 * operator it approximates, so the plain correction comes out too small:
 * omega near 2 compensates (on the plate reactor, 1.8 cut the FGMRES
 * iterations by a quarter at 147k elements). Errors: INVALID_ARG. */
enp_status enp_set_coarse_options(enp_handle h, int cycles, int smooth, double omega);

/* Replace the block-Jacobi part of the preconditioner by one downwind block
 * Gauss-Seidel sweep (on = 1; 0 keeps block-Jacobi; 2, the default, chooses:
 * the sweep on hexahedral meshes with a non-zero velocity and at least 128
 * elements along the flow axis, block-Jacobi otherwise), hexahedral meshes:
 * z = (D + L)^-1 r, D the element-diagonal blocks of the last setup and L the
 * coupling of every element to its upstream neighbour along the flow axis (the
 * plate-flow axis in the sign of its mean speed, or the largest component of a
 * constant velocity, in its direction). The element planes across that axis
 * are solved in flow order, one launch per plane: each element evaluates the
 * face term of J(u) z between it and its upstream neighbour (the face kernel's
 * arithmetic, at the u of the last setup, z of the plane solved before) and
 * applies its block inverse. With upwind advection dominating, this carries
 * information along the whole channel in one application, where block-Jacobi
 * moves it one element per Krylov iteration (Pe = 1e4 in the plate reactor of
 * Sec. 5.2); it costs about 9 us per plane, so it pays on long channels (on the
 * plate reactor: 1.5x faster linear solves at 192 elements along the flow,
 * slower at 96 and below, hence the automatic threshold). Combines with the
 * two-level correction (added after the sweep). Takes effect at the next
 * enp_block_jacobi_setup, which then also keeps a copy of u.
 * Errors: INVALID_ARG, UNSUPPORTED (on = 1 on a 2D mesh). */
enp_status enp_set_sweep(enp_handle h, int on);

/* a0: device [batch][E][7] = the level-0 coarse operator of the last setup,
 * entries (self, -x, +x, -y, +y, -z, +z) of each element's row of
 * P^T J_PhiPhi P (zero where the neighbour does not exist).
 * Errors: INVALID_ARG if the two-level preconditioner has not been set up. */
enp_status enp_coarse_operator(enp_handle h, double* a0);

typedef struct {
  int restart;   /* Krylov vectors per cycle (FGMRES(restart)), at most 255 */
  int max_it;    /* total iterations */
  double rtol;   /* stop when ||b - A x|| <= max(rtol ||b||, atol) */
  double atol;
  int graph;     /* 1: capture one restart cycle in a CUDA graph and replay it (one
                    launch and one host read per cycle; the graph always runs whole
                    cycles, a converged point stays frozen) */
} enp_krylov_opts;

typedef struct {
  int iterations;
  int converged;
  double initial_norm;       /* largest ||b - A x0|| over operating points */
  double residual_norm;      /* largest final ||b - A x|| */
  double relative_residual;  /* largest final ||b - A x|| / ||b|| */
} enp_krylov_stats;

/* Solve J(u_lin) x = b by flexible GMRES (the outer solver of Sec. 4.3, which
 * tolerates a preconditioner that varies between iterations), right-
 * preconditioned with the preconditioner of the last enp_block_jacobi_setup
 * (block-Jacobi, plus the coarse potential correction when the two-level
 * preconditioner is on; identity if none), classical Gram-Schmidt applied twice. x holds the initial guess on
 * entry. Every operating point of the batch is solved independently. stats is
 * a host pointer (may be NULL); the call synchronises.
 * Errors: NOT_CONVERGED (x holds the last iterate), NONFINITE, OOM, CUDA. */
enp_status enp_fgmres_solve(enp_handle h, const double* u_lin, const double* b, double* x,
                            const enp_krylov_opts* opts, enp_krylov_stats* stats);

/* The same with the single-precision operator and Krylov vectors (float
 * u_lin, b, x): the inner solve of the mixed-precision Newton method. */
enp_status enp_fgmres_solve_f32(enp_handle h, const float* u_lin, const float* b, float* x,
                                const enp_krylov_opts* opts, enp_krylov_stats* stats);

typedef struct {
  int max_it;            /* Newton iterations */
  double rtol, atol;     /* stop when ||R(u)|| <= max(rtol ||R(u0)||, atol) */
  double armijo_c;       /* sufficient decrease: ||R(u + lam du)|| <= (1 - c lam) ||R(u)|| */
  int max_backtracks;    /* halvings of lam per iteration */
  int bj_storage;        /* block-Jacobi storage: 0 FP64, 1 FP32, 2 BF16 */
  int mixed;             /* 1: inner FGMRES with the FP32 operator and vectors */
  enp_krylov_opts krylov;
  int pc_lag;            /* rebuild the preconditioner every pc_lag Newton iterations
                            (<= 1: every iteration), and after an inner solve that did
                            not converge; between rebuilds the preconditioner of an
                            earlier iterate is kept (FGMRES needs no exact one) */
  int device_loop;       /* 1: the Newton iterations between preconditioner setups run
                            as one CUDA graph launch whose conditional WHILE nodes loop
                            over the FGMRES restart cycles, the line-search trial steps
                            and the Newton steps, with device-side iteration counts and
                            stopping tests (the host acts once per setup; the graph is
                            captured on the first call and reused while the
                            preconditioner, the sizes and the options stay the same).
                            Same iterates as 0 (the eager loop), up to the rounding of
                            whole restart cycles: converged points are frozen. */
} enp_newton_opts;

typedef struct {
  int iterations;
  int krylov_iterations;
  int converged;
  double initial_norm;
  double residual_norm;
  double history[64];    /* ||R|| after each iteration (largest over operating points) */
  int setups;            /* preconditioner setups */
  double setup_seconds;  /* wall time in preconditioner setups */
  double krylov_seconds; /* wall time in the inner FGMRES solves */
} enp_newton_stats;

/* Newton's method with backtracking line search (Sec. 4) on R(u) = 0, in
 * place on u (device, [batch][m][E][Np]). An iteration rebuilds the
 * preconditioner at u (every iteration, or every opts->pc_lag iterations) and
 * solves J du = -R with FGMRES to opts->krylov.rtol. Synchronises.
 * Errors: NOT_CONVERGED, NONFINITE, OOM, CUDA. */
enp_status enp_newton_solve(enp_handle h, double* u, const enp_newton_opts* opts,
                            enp_newton_stats* stats);

/* The initial guess of Sec. 4.3 ("Implementation"), in place on u: every
 * concentration at its inlet value c_k^in (every node, every operating point),
 * and the potential from the charge-conservation equation (Eq. chargeDG) at
 * these constant concentrations, starting from the potential in u. With
 * Butler-Volmer electrodes that equation is nonlinear in Phi, so it is solved
 * by the Newton method of enp_newton_solve on the potential rows alone: the
 * species rows of the system are replaced by c_k - c_k^in, with unit rows in
 * J and in the element blocks, so the concentrations stay at c^in and the
 * preconditioner (block-Jacobi, plus the coarse potential correction when the
 * two-level preconditioner is on) acts on the potential block. The paper
 * solves each linear system of this step with its potential-block solver to a
 * relative tolerance of 1e-2: opts->krylov.rtol = 1e-2 follows it. The
 * downwind sweep is not used here. The preconditioner of the last setup is
 * replaced (set up again before a separate enp_block_jacobi_apply).
 * Synchronises. Errors as enp_newton_solve. */
enp_status enp_initial_guess(enp_handle h, double* u, const enp_newton_opts* opts,
                             enp_newton_stats* stats);

/* Continuation in the applied potential for operating points that Newton
 * cannot reach from a plain initial guess (strongly driven Butler-Volmer
 * electrodes, Eq. bv, Sec. 5.2): solves R(u; lambda Phi_app) = 0 for a rising
 * sequence of lambda ending at 1, each stage by enp_newton_solve from the
 * previous stage's solution. The increment starts at step0, is multiplied by
 * grow after a converged stage (up to step_max), and is halved after a failed
 * one, whose iterate is discarded. Stages with lambda < 1 stop at stage_rtol
 * within stage_max_it iterations; the last stage uses opts as given. */
typedef struct {
  double step0, step_max, step_min;  /* increments of lambda, 0 < step_min <= step0 <= step_max <= 1 */
  double grow;                       /* >= 1 */
  double stage_rtol;                 /* Newton tolerance of the stages with lambda < 1 */
  int stage_max_it;                  /* Newton iterations of those stages */
} enp_continuation_opts;

typedef struct {
  int stages;             /* Newton solves run, converged or not */
  int failed_stages;
  int newton_iterations;  /* over all stages */
  int krylov_iterations;
  double lambda;          /* the last converged lambda (1 on success) */
  enp_newton_stats last;  /* the last stage run */
} enp_continuation_stats;

/* u: device [batch][m][E][Np], on entry the initial guess for the first stage
 * (lambda = step0), on return the solution at the last converged lambda.
 * phi_app: host [batch][4], the target potentials; on return the handle's
 * applied potentials are the target ones. stats: host pointer (may be NULL).
 * With the environment variable ENP_CONTINUATION_LOG set, two progress lines
 * per stage (lambda, status, Newton and FGMRES iterations, elapsed time; the
 * stage's ||R|| / ||R_0|| after each Newton iteration) go to stderr. Synchronises. Errors: NOT_CONVERGED (the increment fell below
 * step_min), INVALID_ARG, NONFINITE, OOM, CUDA. */
enp_status enp_newton_continuation(enp_handle h, double* u, const double* phi_app,
                                   const enp_continuation_opts* copts,
                                   const enp_newton_opts* opts, enp_continuation_stats* stats);

/* Choose the tile shapes of the hexahedral operator for this handle's degree
 * and field count: for each of R, J v, J^T w (FP64-accurate, in the handle's
 * arithmetic), J v (FP32) and R (FP32), first every feasible number of faces
 * per thread block of the face kernel, then every feasible number of elements
 * per thread block of the element kernel, is timed on this mesh (three
 * launches of the whole operator, CUDA events), and the fastest is kept for the
 * process (per degree, field count, mode and arithmetic). chosen (host, 5 ints,
 * may be NULL) receives the elements per block in that order. Allocates and
 * frees three work vectors; synchronises. No-op in 2D. */
enp_status enp_autotune(enp_handle h, int* chosen);

/* The tile shapes in use for this handle (host arrays of 5 ints, either NULL):
 * elements per block and faces per block of R, J v, J^T w (in the handle's
 * arithmetic), J v (FP32), R (FP32); 0 = the built-in default. */
enp_status enp_launch_shapes(enp_handle h, int* eb, int* fpb);

/* Number of parameters theta of enp_param_jacobian / enp_param_vjp: 2m + 3,
 * ordered (D_1..D_m, c_in_1..c_in_{m-1}, phi_app of electrodes 0..3). */
enp_status enp_param_count(enp_handle h, int* n_theta);

/* dR/dtheta_j for every parameter j, exactly (the residual evaluated with
 * forward-tangent coefficients): D_k enters through D_k, z_k mu_k F, a_km and
 * kappa (Eq. NE, Eq. charge2), c_in through the inlet term and phi_app through
 * Butler-Volmer (Eq. bv). The paper has no derivative with respect to its
 * parameters; this is the parameter Jacobian of Eq. NPDG / Eq. chargeDG.
 * dRdtheta: device [n_theta][batch][m][E][Np]. Hexahedra only (UNSUPPORTED in 2D). */
enp_status enp_param_jacobian(enp_handle h, const double* u, double* dRdtheta);

/* dtheta[b][j] = <w_b, dR_b/dtheta_j>: the parameter part of the adjoint.
 * w: device [batch][m][E][Np]; dtheta: host [batch][n_theta]. Synchronises. */
enp_status enp_param_vjp(enp_handle h, const double* u, const double* w, double* dtheta);

/* dtheta[j] = sum_b <w_b, dR_b/dtheta_j>: the same, summed over the operating
 * points on the device (in batch order), for one parameter vector shared by the
 * whole batch. dtheta: host [n_theta]. Synchronises. */
enp_status enp_param_vjp_total(enp_handle h, const double* u, const double* w, double* dtheta);

/* enp_inner_product without any device allocation. The paper has no
 * counterpart: this entry point exists for callers that cannot call cudaMalloc,
 * such as a host application that owns all device memory through its own pool,
 * or a latency-critical loop that cannot afford cudaMalloc's cost and implicit
 * device synchronisation. It needs no handle.
 *   out[b] = <x_b, y_b> for b < batch, x and y device arrays [batch][n],
 *   out a device array of batch doubles; asynchronous on `stream` (a
 *   cudaStream_t, may be 0). The same kernels, grid and summation order as
 *   enp_inner_product on a handle with n DOFs and `batch` operating points,
 *   so the two give the same bits.
 * The partial sums live in one fixed array of ENP_NOALLOC_MAX_BATCH x 608
 * doubles in the library's static device memory, held by every GPU that loads
 * the library until the process exits. batch > ENP_NOALLOC_MAX_BATCH returns
 * ENP_ERR_INVALID_ARG without launching anything.
 * The first call on a device looks up the array's device address (with that
 * device current); make that first call before any stream capture.
 * All calls share the array, and it keeps the last call's contents (each call
 * writes every entry it reads, so nothing needs clearing): calls that overlap
 * on the GPU (on different streams, or from different threads) race. */
#define ENP_NOALLOC_MAX_BATCH 32
enp_status enp_inner_product_noalloc(const double* x, const double* y, long long n, int batch,
                                     double* out, void* stream);

/* Message of the last failed call on this handle ("" if none). The pointer is
 * owned by the handle and valid until the next call on it. */
const char* enp_last_error(enp_handle h);

#ifdef __cplusplus
}
#endif
#endif /* ENP_DG_H */
