/* imga.h -- C ABI of the GB300 (sm_103a) immersogeometric VMS residual / Jacobian-vector library.
 *
 * The library evaluates, on one GPU, the hot path of the immersogeometric octree LES method of
 * Saurabh et al., "Industrial scale large eddy simulations with adaptive octree meshes using
 * immersogeometric analysis" (arXiv:2009.00706):
 *
 *   imga_build_mesh   octree refined by region predicates, 2:1 balanced, Morton ordered, meshed
 *                     with hanging nodes (Sec. "Octree based Mesh Generation", Algorithm 3);
 *                     triangles distributed to the elements they overlap (Algorithm 1), element
 *                     markers In/Out/Intercepted (Algorithm 5), adaptive sub-cell quadrature of the
 *                     Intercepted elements (Sec. "Adaptive Quadrature", Fig. GP) and the surface
 *                     quadrature of the Nitsche terms (Eq. weakbc).
 *   imga_classify     normal-based in/out test with ray-tracing fallback (Algorithm 6).
 *   imga_residual     VMS residual, Eqs. (ALE-VMS-form), (vms), (uprime), (pprime), plus the
 *                     Nitsche weak Dirichlet terms, Eq. (weakbc), scattered to the nodes through
 *                     the hanging-node operator M_e^T (Algorithm 2).
 *   imga_jvp          the exact directional derivative J(u) v of imga_residual: the matrix of
 *                     Algorithms 2 and 4 applied without being formed.
 *   imga_newton_step  Newton iterations with right-preconditioned GMRES(m) (appendix "Details of
 *                     solver selection": Newton line search + Krylov solver).
 *
 * Conventions
 *   - Node vectors are DEVICE pointers to float64 [n_nodes][4] = (u, v, w, p), node-major, owned
 *     by the caller; the mesh handle owns every other device array.  Nodes are the independent
 *     (non-hanging) octree nodes in Morton order of their integer coordinates.
 *   - Streams are passed as void* (a cudaStream_t, NULL = the legacy default stream).  Compute
 *     calls are asynchronous on that stream; imga_build_mesh and imga_newton_step synchronise.
 *   - Inputs are never written.  Every call returns a status; nothing aborts or traps.  The
 *     message of the last failure on the calling thread is imga_last_error().
 *   - One mesh handle belongs to the device it was built on; calls using it must run with that
 *     device current or pass pointers of that device.  A mesh owns one per-call node workspace,
 *     so residual / J v calls on the same mesh must not overlap on the GPU (issue them on one
 *     stream, or order the streams), and must come from one host thread at a time (the mesh's
 *     side streams, fork / join events and cached graphs are shared by its calls).
 */
#ifndef IMGA_H
#define IMGA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    IMGA_OK = 0,
    IMGA_ERR_INVALID_ARG = 1,   /* bad pointer, size or parameter                         */
    IMGA_ERR_CUDA = 2,          /* a CUDA runtime call failed                             */
    IMGA_ERR_OOM = 3,           /* device or host allocation failed                       */
    IMGA_ERR_SURFACE = 4,       /* degenerate triangle (zero area) in the surface         */
    IMGA_ERR_TIMEOUT = 5,       /* a device-side wait ran out of its iteration budget      */
    IMGA_ERR_NOT_CONVERGED = 6, /* Newton / GMRES stopped before the tolerance            */
    IMGA_ERR_NUMERIC = 7        /* NaN or Inf in a residual norm                          */
} imga_status;

typedef struct imga_mesh_s* imga_mesh;

/* Refinement region: octants meeting the region are refined to `level` (the user predicate of
 * Sec. "Octree based Mesh Generation").  kind 0: spherical band |‖x-c‖-r| <= w, par = (cx, cy,
 * cz, r, w); kind 1: closed box, par = (x0, y0, z0, x1, y1, z1); kind 2: cone along +x, par =
 * (apex x, y, z, length, radius at the apex, tan(half angle)), tested at the octant centre
 * inflated by half its diagonal. */
typedef struct {
    int kind;
    int level;          /* 0 .. 14 */
    double par[8];
} imga_region;

typedef struct {
    double lo[3], hi[3];    /* box; the root cube has the largest edge, origin lo; every edge must
                               be a whole number of base-level cells                         */
    int base_level;         /* level everywhere, 0 .. 14                                       */
    int n_regions;
    const imga_region* regions;
    int quad_max_split;     /* L_max of the adaptive sub-cell quadrature, 0 .. 4               */
} imga_mesh_params;

typedef struct {
    double rho, mu, dt;
    int time_scheme;        /* 0 backward Euler, 1 Crank-Nicolson, 2 BDF2                       */
    double C_b;             /* Nitsche penalty constant: tau_B = C_b mu / h_b                   */
    double C_I;             /* inverse-estimate constant in tau_M                               */
    double g_body[3];       /* velocity prescribed on the immersed surface (weakly)             */
    double u_inf[3];        /* velocity prescribed on the box faces (strongly, not the outlet)  */
    int drop_visc_strong;   /* 1: drop mu grad(div u) from the strong momentum residual         */
    /* g of Eq. (weakbc) per surface point, overriding g_body there: DEVICE float64
     * [n_surface_points][3] in the order of imga_export_surface_points (a rotating or deforming
     * body, or an exact solution prescribed on the surface), or NULL for g_body everywhere.  Read
     * by the residual, J v and element-Jacobian calls; nodes touched by no active element keep
     * U = (g_body, 0). */
    const double* g_points;
} imga_physics;

typedef struct {
    int64_t n_elem, n_nodes, n_hanging;
    int64_t n_out, n_in, n_cut;          /* element markers                                       */
    int64_t n_cut_points;                /* sub-cell quadrature points of the Intercepted elements */
    int64_t n_surface_points;            /* Nitsche quadrature points kept                        */
    int64_t n_tri, n_bt;                 /* triangles, (element, triangle) background pairs       */
    int64_t n_rays;                      /* ray-parity casts made while building                  */
    int64_t hi_int[3];                   /* box extent in integer units (2^20 per root edge)      */
    double scale;                        /* physical length of one integer unit                   */
    double setup_ms[4];                  /* octree+mesh, background triangles, markers+quadrature, upload */
} imga_mesh_info;

/* Build the mesh and every geometric table on `device` (synchronous).  tri_xyz_host: host
 * float64 [n_tri][3][3], counter-clockwise seen from outside each closed body (n_tri may be 0:
 * no immersed body).  On success *out owns the mesh; free it with imga_destroy_mesh.
 * device < 0 builds the host tables only (octree, nodes, background triangles) for inspection:
 * no GPU is touched, and the compute calls reject such a mesh with IMGA_ERR_INVALID_ARG. */
imga_status imga_build_mesh(const double* tri_xyz_host, int64_t n_tri, const imga_mesh_params* params, int device,
                            imga_mesh* out);
/* Free the mesh and every device array it owns (cached graphs, solver workspace, profiling events).
 * NULL is a no-op.  The caller's work on the mesh must be finished or queued before the call: the
 * device frees synchronise the device.  The handle is invalid afterwards. */
void imga_destroy_mesh(imga_mesh mesh);

/* Several independent problems in one mesh, so that one launch of each residual / J v / Jacobian
 * kernel covers all of them.  Problem p has its own surface, octree parameters and viscosity mu
 * (the mu of the imga_physics passed to later calls is ignored; rho, dt, the time scheme, C_b, C_I,
 * g_body and u_inf are shared).  Every problem must use the same box origin and root size.  Its
 * nodes and elements come in problem order: imga_mesh_problems gives the offsets.  Node vectors
 * of the batched mesh are the concatenation of the problems' vectors.  imga_classify is refused
 * (classify against a problem's own mesh). */
typedef struct {
    const double* tri_xyz_host;
    int64_t n_tri;
    imga_mesh_params params;
    double mu;
} imga_problem;
imga_status imga_build_mesh_batch(const imga_problem* problems, int n_problems, int device, imga_mesh* out);
/* number of problems (1 for an ordinary mesh) and elem_off / node_off [n_problems + 1] (host) */
imga_status imga_mesh_problems(imga_mesh mesh, int* n_problems, int64_t* elem_off, int64_t* node_off);
/* Sizes and set-up timings of the mesh (host struct filled by the call).  Errors: IMGA_ERR_INVALID_ARG
 * for a null mesh or info. */
imga_status imga_mesh_get_info(imga_mesh mesh, imga_mesh_info* info);

/* Coordinates of the independent nodes, float64 [n_nodes][3] = lo + node_ijk * scale, in the node
 * order of every node vector (Sec. "Octree based Mesh Generation": nodes of the octree mesh).  For
 * a mesh built on a device, xyz is a device pointer of that device, written by a copy on `stream`
 * that the call waits for; for a mesh built host-only (device < 0), xyz is a host pointer and
 * stream is ignored.  Errors: IMGA_ERR_INVALID_ARG (null mesh or xyz), IMGA_ERR_OOM, IMGA_ERR_CUDA. */
imga_status imga_node_coords(imga_mesh mesh, double* xyz, void* stream);

/* Host copies of the mesh tables (every pointer may be NULL to skip it).  anchors [n_elem][3]
 * integer anchors; levels [n_elem]; conn [n_elem][8] corner -> node index, or n_nodes + h for
 * hanging node h (corner c has bits (c&1, c>>1&1, c>>2&1) along x, y, z); node_ijk [n_nodes][3];
 * hang_parents [n_hanging][4] (-1 padded); hang_np [n_hanging] (2 edge, 4 face). */
imga_status imga_mesh_export(imga_mesh mesh, uint32_t* anchors, uint8_t* levels, int32_t* conn, uint32_t* node_ijk,
                             int32_t* hang_parents, int8_t* hang_np);
/* Host copies of marker [n_elem] (0 Out, 1 In, 2 Intercepted) and corner flags [n_elem] (bit c
 * set: corner c is In), Algorithm 5. */
imga_status imga_export_markers(imga_mesh mesh, int8_t* marker, uint8_t* corner_flags);
/* Host copies of the sub-cell quadrature: offsets [n_elem + 1] into points [n_cut_points][4] =
 * (xi_x, xi_y, xi_z, reference weight) on the element's reference cube [-1, 1]^3. */
imga_status imga_export_cut_points(imga_mesh mesh, int64_t* offsets, double* points);
/* Host copy of the background triangles B_T (Algorithm 1): offsets [n_elem + 1] into tri_ids
 * [n_bt], each element's triangles in increasing order. */
imga_status imga_export_background(imga_mesh mesh, int32_t* offsets, int32_t* tri_ids);
/* Host copy of the surface quadrature [n_surface_points][10] = (x, y, z, n_x, n_y, n_z, weight,
 * h_b, element, triangle); n is the fluid-outward normal. */
imga_status imga_export_surface_points(imga_mesh mesh, double* out);

/* In/out flags of n points (Algorithm 6): pts_dev float64 [n][3] device, flags_dev uint8 [n]
 * device, 1 = In, 0 = Out (points outside the box are Out).  A point in an element whose box meets
 * no triangle takes that element's stored marker (Algorithm 5): no triangle crosses the element,
 * and the paper stores the markers so that such tests are not repeated.  A point in an element
 * with background triangles gets the normal test over them, and ray parity when the test is
 * undecided (Algorithm 6).  With IMGA_OPT_CLASSIFY_RAYS every point in the box goes to ray parity
 * instead: the conventional test of the paper's in/out comparison (Table in-out).  Both modes give
 * the same flags. */
imga_status imga_classify(imga_mesh mesh, const double* pts_dev, int64_t n, uint8_t* flags_dev, void* stream);
/* How imga_classify settled its points, summed over the calls on this mesh since it was built or
 * last reset (host int64 counts[4]): [0] points in elements without background triangles, given
 * the stored marker; [1] points given the normal test; [2] the points among them that the test
 * decided; [3] points sent to ray parity.  Points outside the box are not counted.  The paper's
 * success fraction of the normal test is P_s = counts[2] / counts[1], and P_f = 1 - P_s.
 * Synchronises the mesh's device; reset = 1 zeroes the counts after reading them.  Errors:
 * IMGA_ERR_INVALID_ARG (null argument, host-only or batched mesh), IMGA_ERR_CUDA. */
imga_status imga_classify_counts(imga_mesh mesh, int64_t* counts, int reset);

/* Residual R(u) [n_nodes][4] (device).  u_prev2 is read by BDF2 only (may be NULL otherwise);
 * f is a nodal body force [n_nodes][4] (components 0..2 used) or NULL.  precision 0: FP64
 * throughout; 1: element arithmetic in FP32 with FP64 nodal gathers and FP64 accumulation; the
 * velocity jump u - g at every surface point and the Nitsche penalty tau_B w.(u - g) with its
 * accumulation stay in FP64 (tau_B = C_b mu / h_b reaches 100 C_b mu / h on sliver cut cells).  Rows of strong Dirichlet nodes hold U - g; rows of nodes touched by no
 * active element (In-only nodes, Algorithm 1) hold U - (g_body, 0). */
imga_status imga_residual(imga_mesh mesh, const double* u, const double* u_prev, const double* u_prev2,
                          const double* f, const imga_physics* phys, int precision, double* R, void* stream);

/* Jacobian-vector product J(u) v [n_nodes][4] (device), the derivative of imga_residual in the
 * direction v (the inflow indicator of the Nitsche advective term is held fixed). */
imga_status imga_jvp(imga_mesh mesh, const double* u, const double* u_prev, const double* u_prev2, const double* f,
                     const imga_physics* phys, int precision, const double* v, double* Jv, void* stream);

/* imga_jvp that allocates nothing.  No counterpart in the paper: this entry point exists for
 * callers that cannot allocate device memory when they apply the operator -- processes whose
 * device memory is capped or handed out once at start-up (a GPU shared through a memory-limited
 * partition, an application that reserves all of its memory up front and treats any later
 * cudaMalloc as a failure).  It computes exactly what imga_jvp computes, on the caller's
 * inputs and into the caller's output, but its per-call node workspace is a fixed device array
 * of 32 MiB compiled into the library, which every GPU that loads the library holds until the
 * process exits, instead of the workspace of the mesh handle.
 *   Limit: (16 + 4 if f != NULL) x (n_nodes + n_hanging) x (4 bytes for precision 1, 8 bytes
 *   for precision 0) must not exceed 32 MiB; larger meshes are rejected with
 *   IMGA_ERR_INVALID_ARG and a message giving the bytes needed.
 *   The first call on a device looks the array up on that device (cudaGetSymbolAddress, with
 *   that device current); make that first call before any stream capture.
 *   Every call on every mesh shares the one array, and each call overwrites all of the part it
 *   uses before reading it, so nothing has to be cleared between calls; calls that overlap on
 *   the GPU race on the array: issue them on one stream or order their streams.
 *   The mesh's device must be current.  Calls no cudaMalloc, cudaFree or other allocating
 *   routine, and records no profiling events (imga_profile does not see these calls). */
imga_status imga_jvp_noalloc(imga_mesh mesh, const double* u, const double* u_prev, const double* u_prev2,
                             const double* f, const imga_physics* phys, int precision, const double* v, double* Jv,
                             void* stream);

/* Replace the default strong Dirichlet rows (u = u_inf on every box face but the outlet x = hi,
 * p = 0 on the outlet) by mask_dev uint8 [n_nodes] (bit k: component k prescribed) and values
 * val_dev float64 [n_nodes][4].  Both device pointers; copied.  Pass NULL, NULL to restore. */
imga_status imga_set_dirichlet(imga_mesh mesh, const uint8_t* mask_dev, const double* val_dev, void* stream);

/* Block pattern of the Jacobian assembled in 4 x 4 blocks, K = sum_e M_e^T k_e M_e (Algorithms 2
 * and 4): block (i, j) is present when nodes i and j both enter one element through M_e, as corners
 * or as parents of a hanging corner (Algorithm 3).  Every element counts, In elements too, so the
 * pattern depends on the octree alone; every diagonal block is present.  Host arrays: indptr
 * [n_nodes + 1] (int64) and indices [*n_blocks] (int32, increasing within each block row); pass
 * NULL for both to read *n_blocks first.  Built on the host at the first call and kept by the mesh;
 * works on host-only and batched meshes (block-diagonal over the problems).  Errors:
 * IMGA_ERR_INVALID_ARG (null mesh or n_blocks), IMGA_ERR_OOM. */
imga_status imga_bsr_pattern(imga_mesh mesh, int64_t* n_blocks, int64_t* indptr, int32_t* indices);

/* The Jacobian assembled in 4 x 4 blocks on the block pattern of imga_bsr_pattern (Algorithms 2 and 4:
 * K = sum_e M_e^T k_e M_e, the matrix that imga_jvp applies without forming it, in the element
 * precision `precision`, accumulated in float64), rows of prescribed components replaced by identity
 * rows as in imga_residual.  vals: DEVICE float64 [n_blocks][4][4] (row component, column component),
 * written on `stream`.  The first call on a mesh copies the block pattern to the device (kept by the
 * mesh).  The scatter adds with float64 atomics: entries may differ in the last bits between runs.
 * Errors: IMGA_ERR_INVALID_ARG, IMGA_ERR_OOM, IMGA_ERR_CUDA. */
imga_status imga_bsr_assemble(imga_mesh mesh, const double* u, const double* u_prev, const double* u_prev2,
                              const double* f, const imga_physics* phys, int precision, double* vals, void* stream);
/* y = K x with an assembled matrix vals of this mesh's block pattern; x, y DEVICE float64 [n_nodes][4].
 * Needs the pattern on the device (any earlier imga_bsr_assemble or imga_multilevel_setup). */
imga_status imga_bsr_spmv(imga_mesh mesh, const double* vals, const double* x, double* y, void* stream);

/* Multilevel preconditioner by block coarsening of the assembled Jacobian (no counterpart in the
 * paper, whose solver uses additive Schwarz; its conclusion asks for preconditioners suited to the
 * method).  Level 0 is imga_bsr_assemble's matrix; level l + 1 sums `agg` consecutive block rows and
 * columns of level l (ranges of the Morton node order) over their free unknowns (not identity or empty
 * rows of level 0, not dead rows of coarser levels), A_{l+1} = P^T A_l P with P one 1 per free row; a
 * coarse unknown no free row reaches gets an identity row; the level with at most `coarse_max` block
 * rows (<= 24) is inverted densely.  imga_multilevel_apply runs one V-cycle z = B r: `sweeps` block-
 * Jacobi sweeps damped by `omega` on each level, restriction, the coarse correction, prolongation and
 * `sweeps` sweeps more.  precision 0: assembly, hierarchy and V-cycle in float64; 1: element
 * arithmetic and the whole hierarchy in float32 (the assembly accumulates in float64); r, z stay
 * float64 DEVICE [n_nodes][4].  Setup assembles at the given state (asynchronous on `stream`; the
 * patterns of the levels are built on the host on the first call for an (agg, coarse_max) pair and
 * kept by the mesh).  Errors: IMGA_ERR_INVALID_ARG, IMGA_ERR_OOM, IMGA_ERR_CUDA. */
imga_status imga_multilevel_setup(imga_mesh mesh, const double* u, const double* u_prev, const double* u_prev2,
                                  const double* f, const imga_physics* phys, int precision, int agg, int coarse_max,
                                  int sweeps, double omega, void* stream);
imga_status imga_multilevel_apply(imga_mesh mesh, const double* r, double* z, void* stream);
/* number of levels (0 before any setup), block rows per level (host int64 [24], may be NULL) and
 * whether the dense inverse of the last level met a singular pivot (synchronises; may be NULL) */
imga_status imga_multilevel_info(imga_mesh mesh, int* n_levels, int64_t* rows, int* singular);

/* Force of the fluid on the immersed body, F DEVICE float64 [3], at the state u (spatial terms at
 * theta u + (1 - theta) u_prev as in imga_residual).  The paper reports drag coefficients (Sec.
 * "Validation: flow past a sphere") without printing the formula; this is the weak-boundary reading:
 * the surface terms of Eq. (weakbc) tested with w = e_i, summed over all nodes (partition of unity),
 *     F_i = sum_q w_q [ -(sigma(u_s, p) n)_i - [u.n < 0] rho (u.n) (u - g)_i + tau_B (u - g)_i ],
 * n the fluid-outward normal, g per point as in imga_physics.g_points; the force that keeps the
 * discrete momentum balance.  Float64 throughout; partial sums in a fixed order (same bits on every
 * call).  C_d = 2 F_x / (rho U^2 A).  The first call allocates 6 KiB kept by the mesh. */
imga_status imga_surface_force(imga_mesh mesh, const double* u, const double* u_prev, const imga_physics* phys,
                               double* F, void* stream);

/* Element Jacobians k_e = d r_e / d u_e for a list of elements (Algorithm 4's element matrix, before
 * the hanging correction M_e^T k_e M_e of Algorithm 2): elems_dev int32 [n] device, distinct
 * element indices; K_dev float64 [n][32][32] device, row a*4+i (corner a, component i), column
 * b*4+k, with respect to the element's own corner values (volume + Nitsche terms; In elements give
 * zeros).  precision as in imga_residual. */
imga_status imga_element_jacobians(imga_mesh mesh, const double* u, const double* u_prev, const double* u_prev2,
                                   const double* f, const imga_physics* phys, int precision, const int32_t* elems_dev,
                                   int64_t n, double* K_dev, void* stream);

typedef struct {
    int gmres_m;            /* restart length of GMRES (1 .. 63), e.g. 50                          */
    int max_newton;         /* Newton iterations at most (<= 32)                                   */
    int max_krylov;         /* GMRES iterations per Newton iteration at most                      */
    double rtol, atol;      /* stop when ||R(u)|| <= max(rtol ||R(u_0)||, atol)                     */
    double krylov_rtol;     /* inner tolerance: ||J du + R|| <= krylov_rtol ||R||                 */
    int precision;          /* J v and preconditioner precision: 0 FP64, 1 mixed (FP32 elements)  */
    int precond;            /* 0 none, 1 block-Jacobi (nodal 4x4 diagonal blocks of J), 2 block-Jacobi
                               plus the learned element-block correction of `learned`, 3 block-
                               Jacobi plus the exact element-block correction the network is
                               trained to reproduce, 4 one V-cycle of the multilevel preconditioner
                               (rebuilt from the assembled Jacobian at every Newton iterate, in the
                               precision of `precision`).  With 2 or 3, a linear solve that does not
                               reach krylov_rtol is redone with block-Jacobi alone (counted in
                               imga_solver_stats.fallbacks)                                     */
    int line_search;        /* 1: backtracking (Armijo, c = 1e-4, halving, <= 12 trials)          */
    const void* learned;    /* imga_mlp for precond 2 (n_in 1027, n_out 1024), else NULL         */
    double learned_omega;   /* weight of the learned correction, e.g. 0.5                          */
    /* linear solver of the Newton steps: 0 GMRES(m) on the matrix-free J v; 1 BiCGStab (the solver
     * of the paper's appendix) on the Jacobian assembled in 4 x 4 blocks (imga_bsr_assemble), the
     * assembled matrix also judging the linear tolerance */
    int linear_solver;
    /* precond 4, the multilevel preconditioner of imga_multilevel_setup: block rows per aggregate
     * (0: 6), block rows of the dense last level at most (0: 16, at most 24), damped block-Jacobi
     * sweeps before and after the coarse correction (0: 1) and their weight (0: 0.5) */
    int ml_agg, ml_coarse_max, ml_sweeps;
    double ml_omega;
} imga_solver_opts;

typedef struct {
    int newton_its, krylov_its;
    int krylov_per_newton[32];
    double res_norm[33];    /* float64 ||R|| before the first and after every Newton iteration   */
    double time_ms;
    int converged;
    int fallbacks;          /* linear solves redone with block-Jacobi (precond 2, 3)              */
    double krylov_rel[32];  /* ||b - J du|| / ||b|| reached by each Newton iteration's linear solve  */
} imga_solver_stats;

/* Newton iterations on R(u) = 0 from u_inout (device [n_nodes][4], updated in place), each linear
 * step solved by right-preconditioned GMRES(m) with classical Gram-Schmidt applied twice, every
 * vector and reduction in float64; convergence is judged on the float64 residual.  Synchronous.
 * The mesh keeps the Krylov workspace ((m + 1) + 8 vectors + 2 x 16 n_nodes doubles) for later
 * calls.  On a batched mesh one solve covers every problem (the system is block diagonal over
 * them); the Krylov space, the norms and the stopping test are global, so the hardest problem sets
 * the iteration count.  With IMGA_OPT_GRAPHS the whole solve replays as one CUDA graph.
 * Returns IMGA_ERR_NOT_CONVERGED (stats filled) when the tolerance is not reached. */
imga_status imga_newton_step(imga_mesh mesh, double* u_inout, const double* u_prev, const double* u_prev2,
                             const double* f, const imga_physics* phys, const imga_solver_opts* opts,
                             imga_solver_stats* stats, void* stream);

/* n_steps time steps of the scheme of phys (Sec. "Validation: flow past a sphere": the sphere is run in
 * time and its drag recorded): every step solves R(u^{n+1}; u^n, u^{n-1}) = 0 by imga_newton_step with
 * `opts`, starting from u^n, then shifts the levels; BDF2 takes backward Euler for its first step.
 * u (in: u^n, out: the last level) and u_prev (in: u^{n-1}, ignored by the first step; out: the level
 * before the last) are DEVICE [n_nodes][4].  force_hist (host [n_steps][3], may be NULL) receives
 * imga_surface_force after every step, newton_hist / krylov_hist (host [n_steps], may be NULL) the
 * iterations.  Synchronous; allocates two node vectors for the call.  Returns IMGA_ERR_NOT_CONVERGED
 * after the first step whose Newton solve misses its tolerance (histories filled up to it). */
imga_status imga_time_steps(imga_mesh mesh, double* u, double* u_prev, const double* f, const imga_physics* phys,
                            const imga_solver_opts* opts, int n_steps, double* force_hist, int* newton_hist,
                            int* krylov_hist, void* stream);

/* ---- weighted partition into k parts with halo exchange -------------------------------------------
 * Sec. "Partitioning": the Morton order of the elements is cut into k contiguous ranges of equal total
 * weight under Eq. (Wpart), W(e) = n_Vgp(e)/8 + (T_s/T_v) n_Sgp(e)/8 (volume points evaluated: 8 for
 * Out, the kept sub-cell points for Intercepted, 0 for In; n_Sgp its surface points), ts_over_tv the
 * measured cost ratio T_s/T_v.  Part p owns the nodes it is the lowest part to touch through M_e and
 * keeps the other nodes its elements touch as ghosts (the ghost layer of Sec. "Octree based Mesh
 * Generation").  imga_partition_residual / imga_partition_jvp compute imga_residual / imga_jvp as k
 * parts on this GPU with the data flow of a multi-GPU step: owned rows in, halo gather of the ghost
 * rows through explicit send / receive buffers, the element kernels of each part on its own sub-mesh,
 * halo reduce-add of the ghost rows into their owners (in part order, prescribed components skipped),
 * owned rows out.  Vectors are the global DEVICE [n_nodes][4] ones.  On a mesh built host-only the
 * partition holds the split and the halo lists only (unit weights; the compute calls refuse it).
 * Refused: batched meshes, meshes with imga_set_dirichlet rows, physics with g_points.  The partition
 * reads the mesh, which must outlive it. */
typedef struct imga_partition_s* imga_partition;
imga_status imga_partition_build(imga_mesh mesh, int k, double ts_over_tv, imga_partition* out);
void imga_partition_destroy(imga_partition part);
/* *k parts; host arrays (each may be NULL): elem_off [k + 1] element ranges, weight [k] their Eq.
 * (Wpart) weight, n_owned [k], n_ghost [k] */
imga_status imga_partition_info(imga_partition part, int* k, int64_t* elem_off, double* weight, int64_t* n_owned,
                                int64_t* n_ghost);
/* part p's nodes (host int64 [n_owned + n_ghost], global indices, owned first) and the owning part of
 * each ghost (host int32 [n_ghost]); either may be NULL */
imga_status imga_partition_nodes(imga_partition part, int p, int64_t* nodes, int32_t* ghost_owner);
imga_status imga_partition_residual(imga_partition part, const double* u, const double* u_prev, const double* u_prev2,
                                    const double* f, const imga_physics* phys, int precision, double* R, void* stream);
imga_status imga_partition_jvp(imga_partition part, const double* u, const double* u_prev, const double* u_prev2,
                               const double* f, const imga_physics* phys, int precision, const double* v, double* Jv,
                               void* stream);

/* ---- learned block preconditioner -------------------------------------------------------------
 * A 3-layer MLP (ReLU, widths n_in -> width -> width -> n_out) with BF16 weights and activations on
 * the tensor cores, FP32 accumulation and FP32 master weights, trained by Adam on the mean squared
 * error sum (y - t)^2 / (2 n).  As a preconditioner (imga_solver_opts.precond = 2) it maps each active
 * element's Jacobian block, scaled by its mean |diagonal| s_e, plus (log h, Intercepted flag,
 * log10(1 + local Re)) to a 32 x 32 correction C_e, and GMRES uses
 *     P^-1 v = D^-1 v + omega sum_e M_e^T (C_e / s_e) M_e v      (free rows only),
 * D the nodal block-Jacobi diagonal.  The paper has no learned component: its conclusion asks for
 * preconditioners tailored to the method for matrix-free solvers.  Device pointers unless named host. */
typedef struct imga_mlp_s* imga_mlp;
imga_status imga_mlp_create(int n_in, int width, int n_out, uint64_t seed, int device, imga_mlp* out);
/* frees the network's weights and optimiser state; NULL is a no-op */
void imga_mlp_destroy(imga_mlp mlp);
/* number of parameters and the padded input width the layout uses (W1 is width x n_in_pad) */
imga_status imga_mlp_shape(imga_mlp mlp, int64_t* n_params, int* n_in_pad);
/* FP32 master weights in the order W1 [width][n_in_pad], b1, W2 [width][width], b2, W3 [n_out][width],
 * b3 (host array of n_params floats); set = 1 writes them (and resets Adam), set = 0 reads. */
imga_status imga_mlp_params(imga_mlp mlp, float* host, int set);
/* Y [n][n_out] = MLP(X [n][ldx], first n_in columns), float32 device arrays */
imga_status imga_mlp_forward(imga_mlp mlp, const float* X, int64_t ldx, int64_t n, float* Y, void* stream);
/* loss and gradient (host, n_params floats, same order as the weights) over all n samples */
imga_status imga_mlp_gradient(imga_mlp mlp, const float* X, int64_t ldx, const float* T, int64_t n, double* loss,
                              float* grad_host, void* stream);
/* `epochs` passes of Adam (lr, beta 0.9 / 0.999) over mini-batches of `batch` rows in order;
 * loss_hist (host, may be NULL) receives the mean training loss of each epoch. */
imga_status imga_mlp_train(imga_mlp mlp, const float* X, int64_t ldx, const float* T, int64_t n, int epochs, int batch,
                           float lr, double* loss_hist, void* stream);
/* Network inputs X [n][ldx] (ldx >= 1027) and, when T != NULL, targets T [n][1024] =
 * (K_e/s_e + 0.1 I)^-1 - blockdiag4(K_e/s_e + 0.1 I)^-1 of the listed elements, plus their scales
 * s_e [n]; float32 device arrays.  Allocates a temporary float64 [n][32][32] buffer.  (The shift of
 * the target is 0.1, not 1e-3: an element's constant-pressure mode is nearly singular.) */
imga_status imga_precond_dataset(imga_mesh mesh, const double* u, const double* u_prev, const double* u_prev2,
                                 const double* f, const imga_physics* phys, int precision, const int32_t* elems_dev,
                                 int64_t n, int ldx, float* X, float* T, float* scale, void* stream);
/* C [M][N] = A [M][K] B[N][K]^T with A, B rounded to BF16, FP32 accumulation (the GEMM of the network) */
imga_status imga_gemm_bf16(int M, int N, int K, const float* A, const float* B, float* C, void* stream);

/* Options of a mesh.  IMGA_OPT_GRAPHS (value 1 on, 0 off, default off): imga_residual and imga_jvp
 * run as CUDA graphs -- the first call with a given set of pointers, precision and physics
 * captures (on a private stream) node preparation, the Out-element, Intercepted-element and surface kernels (the last
 * three on parallel branches) and the strong rows; later identical calls replay that graph (up to
 * 32 graphs are kept per mesh), ordered after the work already queued on the caller's stream and
 * before anything queued on it later.  The first call for a key must not itself run inside a stream
 * capture.  imga_set_dirichlet drops the cached graphs.  Profiling (imga_profile) bypasses them. */
/* IMGA_OPT_AUTOTUNE (value 1): the next imga_residual / imga_jvp call of each precision and kind
 * (residual or J v) first times the Intercepted-element kernel in every tile shape -- 2, 4 or 8
 * warps per block (8 in mixed precision only), elements in Morton order or longest first -- and the
 * persistent Out-element kernel with 1 to 5 resident blocks per SM, on the call's own inputs, and
 * keeps the fastest of each for that mesh.  This follows the cost model of
 * Eq. (Wpart): the bucket of elements with uneven quadrature counts (8 to 4096 points).  Tuning
 * synchronises the stream, allocates (once per mesh) a 4-byte-per-element index of the Intercepted
 * list, and is skipped inside a stream capture and by imga_jvp_noalloc.  Value 0 restores the default
 * shape (4 warps, Morton order).  Both values drop the cached graphs. */
/* IMGA_OPT_CLASSIFY_RAYS (value 1 on, 0 off, default off): imga_classify sends every point to ray
 * parity, skipping the stored markers and the normal test; for the comparison of Table in-out. */
/* IMGA_OPT_DETERMINISTIC (value 1 on, the default; 0 off): how imga_residual / imga_jvp (and
 * imga_jvp_noalloc) sum the element vectors into the nodes (o2n of Algorithm 2).  On, every element
 * kernel writes its 8 x 4 contributions to a slot owned by the mesh (a volume slot per Out or
 * Intercepted element in the element precision, a float64 surface slot per element of the dense
 * surface bucket and per point of the sparse one), and one pass over the nodes sums each node's slot
 * rows in the fixed order of a node -> (slot, corner, hanging weight) list built with the mesh, in
 * float64 (mixed precision: a float-float sum of the float32 rows, then float64), and applies the
 * strong rows: two calls with the same inputs give the same bits.  Off, the element kernels add into
 * the output with float64 atomics, whose order, and so the last bits, vary from run to run.  Both
 * values drop the cached graphs. */
/* IMGA_OPT_FUSED (value 1 on, 0 off, default off): imga_residual and imga_jvp (and the solvers built
 * on them) evaluate the Out and Intercepted buckets in ONE persistent launch.  Its warps drain a
 * device work queue: first the Intercepted elements, one per claim, by decreasing point count (a
 * warp's rounds of 32 points: Eq. (Wpart)'s volume cost); then the Out elements, 4 per warp item
 * and 8 items per claim.  The surface (Nitsche) kernels and the float64 penalty run beside it on a
 * side stream (IMGA_OPT_CONCURRENT) or after it.  Results equal the bucketed launches' up to the
 * order of the float64 atomic additions, and bit for bit with IMGA_OPT_DETERMINISTIC.  The first
 * switch-on builds the queue (a synchronous upload).  Fails with IMGA_ERR_CUDA if that fails. */
/* IMGA_OPT_FUSED_SPLIT (value 1 .. 4, default 4): how many of the fused kernel's 4 warps per block
 * start on the Intercepted elements; the others start on the Out elements and take what is left of
 * the Intercepted ones at the end, so latency-bound work can share the SMs with the
 * arithmetic-bound Out elements. */
/* IMGA_OPT_CONCURRENT (value 1 on, the default; 0 off): the bucketed imga_residual / imga_jvp launch
 * the Intercepted-element and surface kernels on two side streams of the mesh, forked after the node
 * preparation and joined before the node sums, so they run beside the Out-element kernel (direct
 * calls and captured graphs alike).  Off: every kernel on the caller's stream, one after the other
 * (each kernel then runs alone, e.g. to time it).  The results are the same bit for bit with
 * IMGA_OPT_DETERMINISTIC. */
enum { IMGA_OPT_GRAPHS = 1, IMGA_OPT_AUTOTUNE = 2, IMGA_OPT_CLASSIFY_RAYS = 3, IMGA_OPT_DETERMINISTIC = 4, IMGA_OPT_FUSED = 5,
       IMGA_OPT_FUSED_SPLIT = 6, IMGA_OPT_CONCURRENT = 7 };
imga_status imga_set_option(imga_mesh mesh, int option, int64_t value);

/* The tile shapes in use.  shape[8] = {warps per block, longest-first order} for
 * [float64, mixed] x [residual, J v].  If ms is non-null, ms[24] receives the per-launch milliseconds
 * of the last tuning for the same 4 cases x 6 candidates (warps 2, 4, 8) x (Morton, longest first);
 * an entry is 0 where not measured. */
imga_status imga_tuning(imga_mesh mesh, int32_t* shape, float* ms);
/* The Out-element bucket's tuning (IMGA_OPT_AUTOTUNE also times the persistent interior kernel with 1,
 * 2, 3 and 4 resident blocks per SM, and in mixed precision 5 with a register allocation made for 5,
 * and keeps the fastest): bps[4] for [float64, mixed] x [residual, J v] (0: not tuned, the occupancy
 * limit is used); if ms is non-null, ms[20] the per-launch milliseconds of the candidates 1 .. 5
 * (0 where not measured). */
imga_status imga_tuning_interior(imga_mesh mesh, int32_t* bps, float* ms);
/* The fused launch (IMGA_OPT_FUSED): counts[6] = {1 if on, Intercepted elements in its queue, elements
 * of the warp-per-element surface kernel, points of the thread-per-point surface kernel (those two
 * run beside it), Out elements, IMGA_OPT_FUSED_SPLIT}. */
imga_status imga_fused_info(imga_mesh mesh, int64_t* counts);

/* Per-kernel timing with CUDA events recorded on the caller's stream around every kernel that
 * imga_residual / imga_jvp launch.  enable = 1 starts (and zeroes) the counters, 0 stops.
 * imga_profile_read synchronises the device and returns, per kernel class (0 Out elements,
 * 1 Intercepted elements, 2 Nitsche surface points, 3 strong rows or node sums, 4 node preparation,
 * 5 the fused launch of IMGA_OPT_FUSED), the summed milliseconds ms[6] and the kernel launch
 * counts launches[6] since profiling was enabled
 * (node preparation is one timed span of up to two kernels; the surface class counts its
 * thread-per-point and warp-per-element kernels separately). */
imga_status imga_profile(imga_mesh mesh, int enable);
imga_status imga_profile_read(imga_mesh mesh, double* ms, int64_t* launches);

/* Self-check of the float64 <-> float32 conversions that the mixed-precision kernels do on the
 * integer pipes (no counterpart in the paper: it is an implementation device of this library).
 * Runs n cases on `device` -- random bit patterns, round-to-nearest-even ties, the edges of the
 * float32 normal range, zeros, subnormals, infinities and NaNs -- derived from `seed`, and stores in
 * *mismatches the number whose result differs in any bit from the hardware conversion (NaN: from
 * being NaN).  Synchronous.  Errors: IMGA_ERR_INVALID_ARG (n < 0, null output), IMGA_ERR_CUDA. */
imga_status imga_selftest_conversions(int device, int64_t n, uint64_t seed, int64_t* mismatches);

/* Measured throughput of an arithmetic pipe of `device`, for roofline denominators (no counterpart in
 * the paper): 8 independent chains of fused multiply-adds per thread, 8 blocks of 256 threads per SM,
 * best of 3 timed launches (synchronous).  kind 0: FP32 FMA; 1: packed FP32x2 FMA (two per
 * instruction); 2: FP64 FMA.  *tflops = 2 x FMAs / second / 1e12.  Errors: IMGA_ERR_INVALID_ARG,
 * IMGA_ERR_CUDA. */
imga_status imga_peak_flops(int device, int kind, double* tflops);

/* Message of the last failing call on the calling thread ("" if none has failed).  The string
 * is owned by the library and stays valid until the next failing call on the same thread. */
const char* imga_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* IMGA_H */
