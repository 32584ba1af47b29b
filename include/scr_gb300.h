/*
 * scr_gb300.h - C ABI of the GB300 (sm_103a) SCR-FGMRES + AMG block solver.
 *
 * The library solves, on one GPU, the two linear systems of every Newton
 * step of the segregated predictor multi-corrector of Liu et al. (arXiv
 * 2206.06996):
 *
 *   1. the velocity-pressure block system  calA x = b,
 *        calA = [[A, B], [C, D]]   (Sec. 5.2.1; blocks defined in Sec. 3.5,
 *        eqs. ABCD_block_matrices_fluid / _solid),
 *      by FGMRES (Sec. 5.2.1, "outer level") preconditioned with the Schur
 *      complement reduction P_SCR (App. B, Algorithm 1), whose Schur
 *      complement S = D - C A^{-1} B is applied matrix-free (App. B,
 *      Algorithm 2), with AMG preconditioners P_A = P_I = AMG(A) and
 *      P_S = AMG(Shat), Shat = D - C diag(A)^{-1} B (Sec. 5.2.1);
 *   2. the mesh-motion system (harmonic extension, Sec. 2.2 and 5.2.2) by
 *      CG preconditioned with AMG.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Status: every function returns an int: SCR_OK (0) or an error code
 *   below.  No C++ exception crosses the boundary.  scr_last_error() returns
 *   a message for the last failure on the calling thread.
 * - Matrices are block CSR (scr_bsr): nb_rows x nb_cols blocks of br x bc
 *   scalars, 0-based int32 row_ptr[nb_rows+1] and col_idx[nnzb] with column
 *   indices sorted within each row, values block after block, each block
 *   row-major.  Blocks: A 3x3 over velocity nodes, B 3x1, C 1x3, D 1x1 over
 *   pressure indices (nodes first, then the duplicated interface pressures
 *   of Sec. 3.3).  Dirichlet degrees of freedom arrive as identity rows with
 *   zeroed columns.
 * - Vectors: velocity nodes interleaved (x, y, z) for all n_v nodes, then all
 *   n_p pressures: length 3 n_v + n_p.  The mesh system uses n_m nodes with
 *   three interleaved displacement components (length 3 n_m).
 * - Sign: the paper solves calA dx = -R; the caller passes b = -R.
 * - Ownership: the caller owns every pointer it passes; set-up functions
 *   deep-copy their inputs (converting precision and layout) and keep
 *   nothing the caller gave.  Output vectors are caller-allocated.
 * - ptr_is_device: 0 = host pointers (copied in and out on the handle's
 *   stream), 1 = device pointers of the current device.
 * - Streams: all work is ordered on the stream given to scr_create; calls
 *   return after the stream work they need has finished, except where noted.
 */
#ifndef SCR_GB300_H
#define SCR_GB300_H

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define SCR_OK 0
#define SCR_INVALID_ARG 1
#define SCR_CUDA_ERROR 2
#define SCR_NOT_CONVERGED 3 /* x holds the best iterate; iters/residual valid */
#define SCR_DEVICE_TIMEOUT 4 /* reserved: no kernel of this library waits on another */
#define SCR_SINGULAR 5

/* arithmetic of the preconditioner (the outer FGMRES, the Gram-Schmidt
   steps, the operator calA and the final residual are always FP64) */
#define SCR_FP64 0
#define SCR_MIXED 1 /* A, Shat and the AMG hierarchies in FP32 */

/* preconditioners of the outer FGMRES (Sec. 5.2.1) */
#define SCR_PC_SCR 0    /* Schur complement reduction, App. B Algorithm 1 (S applied by Algorithm 2) */
#define SCR_PC_SIMPLE 1 /* SIMPLE: Shat for S and diag(A) in the upper factor, no inner level */
#define SCR_PC_SIMPLEC 2 /* SIMPLEC (Sec. 5.2.1): SIMPLE with diag(A) replaced, in Shat and in the upper
                            factor, by the diagonal lumped from |A|: d_i = sum_j |a_ij| */

/* hierarchies for scr_amg_apply / scr_export */
#define SCR_HIER_A 0
#define SCR_HIER_SHAT 1
#define SCR_HIER_MESH 2

/* what scr_export returns */
#define SCR_EXPORT_OPERATOR 0    /* level operator A_l (level 0 of SCR_HIER_SHAT is Shat) */
#define SCR_EXPORT_PROLONGATOR 1 /* smoothed prolongator P_l */
#define SCR_EXPORT_AGGREGATES 2  /* aggregate id per block row of level l (-1: none), into col_idx */
#define SCR_EXPORT_ROOTS 3       /* root block row of each aggregate of level l (the distance-2
                                    independent node that seeded it), n_agg entries into col_idx */
#define SCR_EXPORT_BLOCK_B 4     /* the set-up B, C, D blocks of the block system (level 0; which is */
#define SCR_EXPORT_BLOCK_C 5     /* ignored); with SCR_EXPORT_OPERATOR of SCR_HIER_A level 0 (A) they */
#define SCR_EXPORT_BLOCK_D 6     /* give back the whole Jacobian the solver holds */

typedef struct scr_ctx* scr_handle;

/* Solver settings (Sec. 6, table of solver settings; outer tolerance
   tightened to 1e-8).  Defaults from scr_default_opts. */
typedef struct {
  double rtol;        /* outer FGMRES relative residual ||b - calA x|| / ||b||, 1e-8 */
  int max_it;         /* outer iteration cap n^max, 200 */
  int restart;        /* outer FGMRES restart length, 30 */
  double rtol_A;      /* intermediate GMRES on A (Alg. 1 steps 1, 5), delta_A = 1e-3 */
  double rtol_S;      /* intermediate GMRES on S (Alg. 1 step 3), delta_S = 1e-3 */
  double rtol_I;      /* inner GMRES on A inside Alg. 2, delta_I = 1e-3 */
  int max_A, max_S, max_I; /* 200 each */
  int restart_inner;  /* restart of the intermediate/inner GMRES, 30 */
  int precision;      /* SCR_FP64 or SCR_MIXED */
  int precond;        /* SCR_PC_SCR (Algorithm 1, default), SCR_PC_SIMPLE or SCR_PC_SIMPLEC */
  double amg_theta;   /* strength threshold, 0.08 */
  int amg_max_levels; /* 10 */
  int amg_coarse_size;/* block rows at which coarsening stops, 64 */
  int amg_nu;         /* l1-Jacobi sweeps before and after the coarse correction, 1 */
  double amg_trunc;   /* prolongator truncation factor (AMG settings table: 0.3) */
  int amg_pmax;       /* at most this many blocks per prolongator row (AMG settings table: 5; 0 = no cap) */
  int autotune;       /* 1: time the SpMV lane-group widths at set-up and keep the fastest */
  int amg_smoother;   /* 0: l1-Jacobi (amg_nu sweeps); 1: Chebyshev on D^{-1}A (default) */
  int amg_degree;     /* Chebyshev degree, 3 */
  int spmv_group;     /* 0: autotune/heuristic; 1..16: lanes per block row; 101..116: 100 + lanes per
                         scalar row; 301..316: 300 + lanes per block row of the 16-byte kernels on
                         the padded copy (matrices without one use the scalar-row kernel with
                         that many lanes) (forces the product kernel of every matrix) */
  int sell;           /* 0: slab products; W > 0: products with A, Shat and L use a sliced block-ELL
                         copy with rows sorted by length inside windows of W block rows
                         (W a multiple of 32, at most 1024); default 0 */
  int vec;            /* 1 (default): A and Shat (and their FP32 copies) also keep a padded copy in
                         which every block row's column indices and scalar rows start on 16-byte
                         boundaries (zero padding), and the autotuner also times the kernels that
                         read it with 16-byte vector loads; 0: slab products only */
  int inner_vcycles;  /* 0 (default): Algorithm 2's inner A solve is GMRES + P_I to rtol_I (the paper);
                         k in 1..64: k steps of Richardson's iteration preconditioned by one V-cycle
                         (x_1 = M b, x_{i+1} = x_i + M (b - A x_i)): a fixed linear operator with no
                         host synchronisation (the outer FGMRES is flexible) */
  int inter_vcycles;  /* the same for the intermediate A solves of Algorithm 1 (steps 1 and 5) and of
                         SIMPLE / SIMPLEC; 0 (default): GMRES + P_A to rtol_A */
  int newton;         /* scr_corrector / scr_corrector_ale: 0 (default) hold the tangent of the last
                         scr_setup fixed (modified Newton); 1 re-assemble it on the GPU at every
                         iteration's state (scr_assemble_tangent) before that iteration's solve, as
                         the paper's multi-corrector does */
  int pdl;            /* 1 (default): the product kernels are launched with programmatic stream
                         serialization: a product's CTAs start while the previous kernel drains,
                         prefetch their own rows of the stored matrix into L2 and wait
                         (griddepcontrol.wait) before reading any vector; 0: ordinary launches.
                         Results are the same either way (measured: FP64 step 1084 -> 1069 ms,
                         mixed 626 -> 615 ms on the 616k-node tube).
                         Like spmv_group and l2_prefetch it is process-wide: the last scr_create sets it */
  int tangent_resetup;/* how scr_assemble_tangent (and the Newton corrector) set the solve up on the
                         new tangent: 1 (default) scr_update_values (the aggregates, truncation
                         positions and product patterns of the first set-up kept); 0 a full
                         scr_setup */
  int mapped_scalars; /* how the Krylov residual estimates reach the host after each iteration:
                         1 (default) kernels write mapped pinned host memory; 0 a device buffer
                         and one 16-byte copy to pinned memory before the stream synchronisation
                         (measured 0.4 % slower) */
  int l2_prefetch;    /* scalar-row products: each CTA prefetches into L2 the values and indices of
                         the CTA this many indices ahead (bulk L2 prefetch); 0 off; default 192 */
  int amg_coarse_bf16;/* mixed form only: 1 (default) stores the values of the coarse AMG levels
                         (operators and transfers of levels >= 1) in BF16, rounded to nearest even
                         from the FP32 copy; products still use FP32 vectors and FP32 sums;
                         0 keeps them in FP32 */
  int cuda_graphs;    /* 1 (default): each AMG hierarchy records one V-cycle as a CUDA graph at its
                         first use after set-up and replays it (between copies to and from two
                         staging vectors) for every later V-cycle; 0: every V-cycle launched
                         kernel by kernel.  V-cycles run kernel by kernel while scr_profile_begin
                         is active.  Results are the same either way. */
  int graph_krylov;   /* device loops: each preconditioner application (Algorithm 1, SIMPLE or SIMPLEC)
                         is recorded once per set-up as one CUDA graph and replayed; in it every
                         intermediate and inner GMRES runs as a device-side loop (conditional WHILE
                         and IF graph nodes: restart cycles, Arnoldi steps, restart), its convergence
                         test evaluated on the GPU, so the host waits once per outer FGMRES iteration
                         instead of once per inner iteration.  1: always; 0: host-driven inner loops;
                         2 (default): device loops for block systems of at most 1,000,000 unknowns
                         (times nrhs), where they were measured faster (small systems: 7-16 %),
                         host-driven above (2.5M unknowns: 0.5-1.3 % slower with device loops).
                         Direct launches while scr_profile_begin is active.  Results are the same
                         either way. */
  int nrhs;           /* right-hand sides of the block solve: 1 (default, scr_solve) or 8
                         (scr_solve_multi: the block products act on 8 interleaved vectors at once) */
  double mm_rtol;     /* mesh CG relative residual, 1e-8 */
  int mm_max_it;      /* mesh CG iteration cap, 500 */
  int verbose;        /* 0 quiet */
} scr_opts;

typedef struct {
  int nb_rows, nb_cols, br, bc, nnzb;
  const int* row_ptr;
  const int* col_idx;
  const double* val;
} scr_bsr;

#define SCR_SMOOTH_L1 0
#define SCR_SMOOTH_CHEB 1

/* destination of scr_export (host pointers; pass NULL arrays to query sizes) */
typedef struct {
  int nb_rows, nb_cols, br, bc, nnzb;
  int* row_ptr;
  int* col_idx;
  double* val;
} scr_bsr_out;

/* counters and timings of the last set-up and solves on a handle */
typedef struct {
  int outer_iters;      /* FGMRES iterations of the last scr_solve */
  int a_solves;         /* intermediate A solves (Alg. 1 steps 1 and 5) */
  int a_iters;          /* GMRES iterations inside them */
  int s_iters;          /* GMRES iterations on S (Alg. 1 step 3) */
  int i_iters;          /* inner GMRES iterations (Alg. 2) */
  int vcycles_A, vcycles_S, vcycles_M;
  int mm_iters;         /* mesh CG iterations of the last mm_solve */
  double rel_res;       /* final FP64 ||b - calA x|| / ||b|| of the last scr_solve */
  double mm_rel_res;
  double setup_ms, solve_ms, mm_setup_ms, mm_solve_ms; /* host wall clock */
  long long kernel_launches;  /* library launches issued in this process so far */
  long long spmv_bytes;       /* modelled HBM bytes of the SpMV-type launches (process total) */
  int levels_A, levels_S, levels_M;
  int syncs;                  /* host waits on device scalars */
  int kernel_A, kernel_Shat;  /* product kernel codes chosen for A and Shat in the solver
                                 precision (see scr_opts.spmv_group; 0 = heuristic) */
  int pc_graph_runs;          /* preconditioner applications of the last solve replayed from
                                 the recorded graph (scr_opts.graph_krylov) */
} scr_stats;

/* Fill o with the defaults listed above.  Never fails for non-NULL o. */
int scr_default_opts(scr_opts* o);

/* Create a solver context on the current CUDA device.  cuda_stream is a
   cudaStream_t (NULL: the legacy default stream).  o may be NULL
   (defaults).  The handle owns all device memory it allocates. */
int scr_create(scr_handle* h, const scr_opts* o, void* cuda_stream);

/* Free every resource of h (NULL is accepted). */
int scr_destroy(scr_handle h);

/* Set-up of the block system (Sec. 5.2.1): copies A, B, C, D, forms
   Shat = D - C diag(A)^{-1} B on the GPU (sparse product), builds the AMG
   hierarchies of A and Shat.  Shapes: A n_v x n_v (3x3), B n_v x n_p (3x1),
   C n_p x n_v (1x3), D n_p x n_p (1x1).  SCR_INVALID_ARG on a shape or
   block-size mismatch, a missing diagonal block of A or a zero diagonal
   entry of A; SCR_CUDA_ERROR on device failure. */
int scr_setup(scr_handle h, const scr_bsr* A, const scr_bsr* B, const scr_bsr* C,
              const scr_bsr* D, int ptr_is_device);

/* New values for the block system of the last scr_setup, with the same
   sizes and the same sparsity patterns (row_ptr and col_idx equal to the
   set-up's; checked on the device, SCR_INVALID_ARG when they differ): the
   numeric re-set-up of a Newton step whose Jacobian keeps its pattern.  The
   values are copied in, Shat = D - C diag(A)^{-1} B is recomputed on its
   stored pattern (Sec. 5.2.1), and both AMG hierarchies are recomputed on
   their stored patterns: the aggregates of the first set-up are kept, the
   smoothed prolongators are recomputed from the new operators and
   truncated to the positions the first set-up kept (rescaled to the new
   row sums), and the Galerkin operators, smoother data (Chebyshev interval,
   guard), coarsest inverse and lower-precision copies follow.  Ownership,
   pointers and errors as scr_setup; not for batched handles. */
int scr_update_values(scr_handle h, const scr_bsr* A, const scr_bsr* B, const scr_bsr* C, const scr_bsr* D,
                      int ptr_is_device);

/* Solve calA x = b to the outer tolerance (FGMRES + P_SCR, x_0 = 0).
   b, x: length 3 n_v + n_p.  Returns SCR_NOT_CONVERGED if the outer cap is
   reached (x = last iterate).  The final relative residual is recomputed in
   FP64 with calA (scr_residual). */
int scr_solve(scr_handle h, const double* b, double* x, int ptr_is_device);

/* ---------------- batched form: many independent systems at once --------
   nb independent block systems (each as in scr_setup, arrays A[i] ...
   D[i]) are set up and solved together as one block-diagonal system, so
   every kernel launch of the solve covers all members; the AMG aggregates
   never cross members (they have no connections), so each level of the
   hierarchies stays block-diagonal.  The outer tolerance is tightened to
   rtol * min_i ||b_i|| / ||b||, which guarantees ||b_i - calA_i x_i|| <=
   rtol ||b_i|| for every member; the per-member FP64 relative residuals
   are available from scr_batch_residuals.  Member i's vectors have length
   3 n_v(i) + n_p(i) in the usual order.  Errors as in scr_setup /
   scr_solve; SCR_NOT_CONVERGED if a member with b_i != 0 misses rtol. */
int scr_setup_batch(scr_handle h, int nb, const scr_bsr* A, const scr_bsr* B, const scr_bsr* C,
                    const scr_bsr* D, int ptr_is_device);
int scr_solve_batch(scr_handle h, const double* const* b, double* const* x, int ptr_is_device);
int scr_batch_residuals(scr_handle h, double* rel_res /* nb entries */);

/* Iteration counts of the last scr_solve: outer FGMRES and the sum of all
   intermediate and inner GMRES iterations. */
int scr_iters(scr_handle h, int* outer, int* inner_total);

/* FP64 ||b - calA x||_2 / ||b||_2 of the last scr_solve. */
int scr_residual(scr_handle h, double* rel_res);

/* Several right-hand sides with one set-up (the block product form of the
   multi-right-hand-side solve): for a handle created with nrhs = 8, solves
   calA x_c = b_c for c = 0..7.  b and x are arrays of 8 pointers to vectors
   laid out as for scr_solve (host pointers when dev == 0, device pointers
   otherwise; the caller owns them).  Inside, the right-hand sides are
   interleaved (entry i of b_c at i * 8 + c), so every product with A, B, C,
   D, Shat and the AMG levels reads the stored blocks once for all eight
   columns; one FGMRES runs on the interleaved system with the tolerance
   rtol * min_c ||b_c|| / ||b||, which bounds every column's relative
   residual by rtol.  rel_res (8 doubles, may be NULL) receives each
   column's FP64 ||b_c - calA x_c|| / ||b_c||.  Returns SCR_NOT_CONVERGED if
   a column misses rtol; SCR_INVALID_ARG before scr_setup or for NULL
   pointers.  With nrhs = 1 it solves one right-hand side like scr_solve.
   scr_solve, scr_setup_batch, scr_apply_* and scr_amg_apply on the block
   hierarchies take nrhs = 1 handles only.  Not in the paper: the
   multi-right-hand-side form is an addition of this library. */
int scr_solve_multi(scr_handle h, const double* const* b, double* const* x, int dev, double* rel_res);

/* Resistance outlets (Sec. 3.5, outlet coupling matrix): the momentum block
   of calA becomes A + sum_j c_j a_j a_j^T, with a_j[3 A + i] = the integral
   of N_A n_i over outlet j and c_j = alpha_f gamma dt m_j (m_j = dP/dQ of the
   outlet model).  a: n_out vectors of len = 3 n_v doubles one after
   another, c: n_out doubles (host memory, copied).  Takes effect at the
   next scr_setup: every product with A on the Krylov path and calA add the
   rank-1 terms (one dot and one update per outlet), diag(A) in Shat and in
   SIMPLE's update includes sum_j c_j a_j^2; the AMG hierarchies are built
   from the sparse A.  n_out = 0 removes the outlets.  SCR_INVALID_ARG for
   NULL arrays, a non-finite coefficient, or (at scr_setup) len != 3 n_v,
   nrhs != 1 or SCR_PC_SIMPLEC. */
int scr_set_outlets(scr_handle h, int n_out, int len, const double* a, const double* c);

/* Residual assembly on the GPU (Sec. 3.2 fluid and Sec. 3.5 solid element
   residuals of the unified-continuum VMS formulation on linear tets, 4-point
   Gauss rule; the element loop of the segregated multi-corrector step).
   scr_assembly_setup copies the mesh (host arrays): node coordinates xyz
   (3 n_nodes), velocity connectivity ien and pressure-index connectivity
   pien (4 n_elem each, 0-based; pressure indices < n_p), element type (0
   fluid, 1 solid) and the velocity Dirichlet flag per node (dir_v, may be
   NULL).  scr_assemble_residual writes R = [R_m (3 n_nodes) | R_p (n_p)], the raw
   residual before any Dirichlet rows, at the state v (3 n_nodes, at
   t_{n+alpha_f}), p (n_p), vhat (mesh velocity), vdot (at t_{n+alpha_m})
   and u (solid displacement); vhat, vdot and u may be NULL (zero).  Host
   pointers when dev == 0, device pointers otherwise.  Every run adds the
   same terms in the same order (per-element values, then a fixed-order sum
   per row).  SCR_INVALID_ARG for NULL arrays, sizes < 0 or out-of-range
   connectivity. */
typedef struct {
  int n_nodes, n_elem, n_p;
  const double* xyz;
  const int* ien;
  const int* pien;
  const unsigned char* etype;
  const unsigned char* dir_v;
} scr_mesh;
typedef struct {
  double rho_f, mu_f;        /* fluid density and dynamic viscosity */
  double rho_s, E_s, nu_s;   /* solid density, Young's modulus, Poisson ratio */
  double dt, rho_inf;        /* time step, generalized-alpha spectral radius */
  double c_m_solid, c_c_solid; /* solid stabilisation constants */
} scr_physics;
int scr_assembly_setup(scr_handle h, const scr_mesh* m, const scr_physics* ph);
int scr_assemble_residual(scr_handle h, const double* v, const double* vhat, const double* p,
                          const double* vdot, const double* u, double* R, int dev);

/* Tangent assembly on the GPU (Sec. 3.5: the consistent tangent K =
   alpha_m dR/d(ydot) + alpha_f gamma dt dR/dy of the element residuals of
   scr_assemble_residual, with tau_M and tau_C evaluated at the state and held
   fixed; generalized-alpha weights from scr_physics.rho_inf and dt).  At the
   state v, p (at t_{n+alpha_f}), vhat (mesh velocity; may be NULL: zero) and
   vdot (at t_{n+alpha_m}; may be NULL: zero), host pointers when dev == 0,
   device pointers otherwise, it writes the blocks A, B, C, D into the
   sparsity pattern of the matrices of the last scr_setup, with the velocity
   Dirichlet nodes of scr_assembly_setup as identity rows of A (the input
   convention: the pattern holds no other block in a Dirichlet row or column
   of A, B, C), and then runs the set-up of the block solve on them (Shat,
   AMG hierarchies, lower-precision copies), so the next scr_solve solves
   with this Jacobian.  The element tangents are formed one thread per
   (element, column vertex) and summed per stored block in increasing
   element order, so every run gives the same values.  The pattern is
   captured at the first call after a caller's scr_setup; the solid
   displacement does not enter (the solid is linearised at the reference
   state).  SCR_INVALID_ARG without scr_setup (not batched) and
   scr_assembly_setup on the same mesh, or for NULL v, p. */
int scr_assemble_tangent(scr_handle h, const double* v, const double* vhat, const double* p, const double* vdot,
                         int dev);

/* Segregated multi-corrector iterations (Sec. 3.5) on the GPU: with the
   tangent of the last scr_setup held fixed (modified Newton; with the option
   newton = 1 the tangent is re-assembled at every iteration's state by
   scr_assemble_tangent before that iteration's solve) and the mesh
   of scr_assembly_setup held fixed (no mesh-motion update inside the loop),
   n_iter times: R = scr_assemble_residual at the state (plus the outlet
   tractions m_j (a_j^T v) a_j of scr_set_outlets, with m_j = c_j / (alpha_f
   gamma dt)), b = -R with the velocity Dirichlet rows zeroed, solve calA x = b (SCR-FGMRES + AMG, the
   handle's options), then vdot += alpha_m x_v, v += alpha_f gamma dt x_v,
   p += alpha_f gamma dt x_p, u += (alpha_f gamma dt)^2 / alpha_m x_v
   (generalized-alpha weights from scr_physics.rho_inf and dt).  v, vdot, u
   (3 n_nodes) and p (n_p) are updated in place (host pointers when dev ==
   0, device pointers otherwise); res_norms (host, n_iter + 1 doubles)
   receives ||b|| before each solve and after the last update.  Returns
   SCR_NOT_CONVERGED if an inner solve missed rtol (the iterations still
   run); SCR_INVALID_ARG without both set-ups on the same mesh or with
   nrhs != 1. */
int scr_corrector(scr_handle h, double* v, double* p, double* vdot, double* u, int n_iter, double* res_norms,
                  int dev);

/* Mesh motion for scr_corrector_ale (Sec. 3.5, steps 3-4; Sec. 5.2.2).
   After scr_assembly_setup.  n_fluid fluid nodes; fluid_id (n_nodes of the
   assembly mesh) maps a node to its fluid ordinal or -1, every ordinal used
   exactly once; dir_m (n_fluid) flags the Dirichlet mesh nodes; follow
   (n_fluid) flags those that take the solid displacement of their node (the
   fluid-solid interface; the other Dirichlet nodes are held at zero), and
   follow without dir_m is an error; L_raw (n_fluid x n_fluid, 1x1 blocks)
   is the mesh Laplacian WITHOUT boundary conditions, used to lift the
   Dirichlet data into the right-hand side of the eliminated system that
   mm_setup received.  All arrays are host memory, copied (the caller keeps
   ownership).  A later scr_assembly_setup drops the coupling.  SCR_INVALID_ARG
   on NULL, sizes or maps that do not fit. */
int scr_mesh_coupling(scr_handle h, int n_fluid, const int* fluid_id, const unsigned char* dir_m,
                      const unsigned char* follow, const scr_bsr* L_raw);

/* scr_corrector with the mesh moving inside the loop (Sec. 3.5, steps 3-4).
   The state enters at the same-Y predictor, so u at entry is u_n.  Before
   every residual evaluation: u_{n+1} = u_n + (u - u_n) / alpha_f; the
   Dirichlet data g (u_{n+1} on follow nodes, zero on the other Dirichlet
   mesh nodes); uhat_{n+1} from CG + AMG (mm_setup's hierarchy, mm_rtol) on
   the eliminated mesh system with right-hand side g on Dirichlet rows and
   -(L_raw g) on the free rows; vhat_{n+1} = (uhat_{n+1} - uhat_n) / (gamma
   dt) + (gamma - 1) / gamma vhat_n and vhat_{n+alpha_f} = vhat_n + alpha_f
   (vhat_{n+1} - vhat_n) at the fluid nodes (zero elsewhere), passed to the
   residual as the mesh velocity.  The element geometry stays that of
   scr_assembly_setup.  uhat_n, vhat_n (may be NULL: zero) and uhat (out:
   uhat_{n+1} after the last update) have 3 n_fluid interleaved entries, host
   or device like the state (dev).  Returns SCR_NOT_CONVERGED if an inner
   block solve or a mesh solve missed its tolerance (the iterations still
   run); SCR_INVALID_ARG without scr_mesh_coupling and mm_setup on the same
   n_fluid, or as scr_corrector. */
int scr_corrector_ale(scr_handle h, double* v, double* p, double* vdot, double* u, const double* uhat_n,
                      const double* vhat_n, double* uhat, int n_iter, double* res_norms, int dev);

/* Counters and timings (see scr_stats). */
int scr_get_stats(scr_handle h, scr_stats* s);

/* Mesh-motion set-up (Sec. 5.2.2): L is n_m x n_m with 1x1 blocks,
   symmetric positive definite after the Dirichlet rows were made identity;
   builds the AMG hierarchy of L (applied to the three displacement
   components). */
int mm_setup(scr_handle h, const scr_bsr* L, int ptr_is_device);

/* CG + AMG on (L kron I_3) u = g; g, u: length 3 n_m interleaved. */
int mm_solve(scr_handle h, const double* g, double* u, int ptr_is_device);

/* Iterations and FP64 relative residual of the last mm_solve. */
int mm_iters(scr_handle h, int* iters, double* rel_res);

/* Message of the last error on this thread ("" if none). */
const char* scr_last_error(void);

/* ---------------- single steps of the path (device pointers) ----------
   These run exactly the kernels the solver uses, for parity checks. */

/* y = calA x, the fused block product (Sec. 5.2.1). */
int scr_apply_op(scr_handle h, const double* x, double* y);

/* y = P^{-1} r for the handle's preconditioner: Algorithm 1 of App. B
   (SCR_PC_SCR) or P_SIMPLE^{-1} (SCR_PC_SIMPLE, Sec. 5.2.1; SCR_PC_SIMPLEC: P_SIMPLEC^{-1}). */
int scr_apply_pc(scr_handle h, const double* r, double* y);

/* y_p = S x_p = D x_p - C A^{-1} B x_p, Algorithm 2 of App. B. */
int scr_apply_schur(scr_handle h, const double* xp, double* yp);

/* x = one V-cycle of hierarchy `which` applied to b (x_0 = 0).  For
   SCR_HIER_MESH, b and x hold three interleaved components. */
int scr_amg_apply(scr_handle h, int which, const double* b, double* x);

/* Number of levels of hierarchy `which` (0 if not set up). */
int scr_amg_levels(scr_handle h, int which, int* n_levels);

/* ---------------- kernel timing (CUDA events on the handle's stream) ----
   Between scr_profile_begin and scr_profile_end every launch of the chosen
   kernel class is bracketed by a pair of CUDA events recorded on the
   launching stream; scr_profile_end waits for the stream and returns the
   launch count, the summed event time and the algorithmic bytes and
   flops of those launches (bytes: stored values and column indices once,
   the source vector once, the destination written once plus the vectors
   the epilogue reads; flops: 2 per stored scalar and right-hand side). */
#define SCR_PROF_SPMV_A 0   /* products with A (level 0, solver precision) */
#define SCR_PROF_BLOCK_OP 1 /* the fused calA product */
typedef struct {
  long long launches;  /* launches of the class in the region */
  long long timed;     /* launches with an event pair (capacity-limited) */
  double ms;           /* summed event time of the timed launches */
  double bytes;        /* algorithmic bytes of the timed launches */
  double flops;        /* flops of the timed launches */
} scr_kprof;
int scr_profile_begin(scr_handle h, int kernel_class, int capacity);
int scr_profile_end(scr_handle h, scr_kprof* out);

/* The autotuner's kernel choices (scr_opts.autotune) live in a process-wide
   cache keyed by block shape, block rows and columns, stored blocks, value
   precision (plus whether the matrix has the padded 16-byte copy of the
   vec option) and right-hand sides.  scr_tune_save writes every cached
   decision to a text file, one per line; scr_tune_load adds the decisions of
   such a file to the cache for the current device, so later set-ups of
   matrices with those keys skip the timing and use the stored kernels.  Use:
   reproduce one run's choices in another, e.g. under a profiler, whose
   instrumentation distorts the timings the autotuner relies on.  The paper
   has no counterpart.  Errors: SCR_INVALID_ARG for a NULL path, a file that
   cannot be opened or a malformed line (nothing is added then). */
int scr_tune_save(const char* path);
int scr_tune_load(const char* path);

/* Copy a level operator, prolongator or the aggregates of a hierarchy to
   host arrays in the block CSR layout above.  Call once with NULL arrays to
   receive the sizes, then again with arrays of those sizes. */
int scr_export(scr_handle h, int which, int level, int kind, scr_bsr_out* out);

/* y = M x for a block matrix given in device memory (any br, bc in {1,3}),
   on stream cuda_stream, with the same block-row kernel the solver uses.
   x has nb_cols*bc entries, y nb_rows*br. */
int scr_bsr_spmv(const scr_bsr* M, const double* x, double* y, void* cuda_stream);

/* y = M x like scr_bsr_spmv, but without allocating any device memory.
   The paper has no counterpart: this entry point exists for callers that
   cannot let a library call cudaMalloc/cudaFree: hosts whose device memory
   is owned by another allocator or fixed at start-up (a library's own
   allocation can fail there or starve the owner), and code that must not
   call cudaFree, which waits for the whole device.  Its scratch (the matrix
   values in the kernel's row layout and a validation flag) is one static
   device array that every GPU loading the library keeps until the process
   exits; matrices with more than 2,097,152 stored scalars (nnzb * br * bc,
   16 MiB) are rejected with SCR_INVALID_ARG.  The first call on each device
   looks up the array's device address (cudaGetSymbolAddress) with that
   device current and keeps it for the life of the process, so do not call
   it on a device after cudaDeviceReset.  Every call validates the indices
   on the device, copies the result flag back to the host and synchronises
   the stream twice (before the product and after it).  All calls share the
   array: calls whose work overlaps on the GPU (different streams, or
   different host threads) race and give wrong results; serialise them.
   Arguments, layout and errors are those of scr_bsr_spmv. */
int scr_bsr_spmv_noalloc(const scr_bsr* M, const double* x, double* y, void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* SCR_GB300_H */
