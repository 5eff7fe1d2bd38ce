/*
 * feti.h -- C ABI of the GB300 (sm_103a) classical / all-floating FETI solver.
 *
 * The library solves the linear(ized) elasticity systems of Sec. 3.2 of
 * Augustin, Holzapfel & Steinbach, "Classical and all-floating FETI methods
 * for the simulation of arterial tissues" by the dual method of Sec. 4:
 * tearing into subdomains (Sec. 4.1), all-floating treatment of Dirichlet
 * conditions (Sec. 4.2, Eq. jumpoperatorAF), generalized local inverses and
 * projected preconditioned CG on the multipliers (Sec. 4.3, Eqs.
 * classicalFetiF, projection, dualProblem) with the lumped, Dirichlet or
 * identity preconditioner (Sec. 4.4, Eqs. LumpedVK, DirichletVK).
 *
 * Conventions for every call:
 *  - Host arrays passed to feti_create are read during the call and copied;
 *    the caller keeps ownership.  The library owns all device memory it
 *    allocates and frees it in feti_destroy.
 *  - DOF numbering: dof = 3 * node + component (component 0, 1, 2 = x, y, z).
 *  - Every call returns a feti_status.  On failure the context keeps a
 *    message readable with feti_last_error.  No call exits, aborts or traps.
 *  - Calls on one context are not thread-safe; different contexts are
 *    independent.  All device work of a context runs on its stream.
 *  - There is no CPU fallback: without a usable CUDA device feti_create
 *    returns FETI_ERR_CUDA.
 */
#ifndef FETI_H
#define FETI_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  FETI_OK = 0,
  FETI_ERR_INVALID_ARG = 1,      /* null pointer, size out of range, bad option */
  FETI_ERR_PARTITION = 2,        /* empty subdomain or unsupported kernel dimension */
  FETI_ERR_ELEMENT_INVERTED = 3, /* a tetrahedron with non-positive volume or det F <= 0 */
  FETI_ERR_LOCAL_SINGULAR = 4,   /* non-positive pivot in a local Cholesky factorization */
  FETI_ERR_KERNEL_DETECT = 5,    /* rigid-body kernel detection failed */
  FETI_ERR_BREAKDOWN = 6,        /* PCG breakdown: (p, F p) <= 0 or not finite */
  FETI_ERR_NOT_CONVERGED = 7,    /* PCG reached maxit above tolerance */
  FETI_ERR_NEWTON_DIVERGED = 8,  /* Newton did not reach its tolerance */
  FETI_ERR_TIMEOUT = 9,          /* a bounded device wait gave up */
  FETI_ERR_OOM = 10,             /* device allocation failed */
  FETI_ERR_CUDA = 11,            /* any other CUDA runtime error */
  FETI_ERR_STATE = 12,           /* call made in the wrong order */
  FETI_ERR_IO = 13               /* checkpoint file not writable, unreadable or corrupt */
} feti_status;

/* feti_material.kind: FETI_LINEAR_ISO -- Hooke's law (E, nu); FETI_HGO_TWO_FIBRE
 * -- the two-fibre hyperelastic energy (P1 only); FETI_LINEAR_ISO_P0 -- Hooke's
 * law with the volumetric part carried by a piecewise-constant pressure that
 * is condensed out element by element (Sec. 3.2, static condensation): the
 * P2-P0 element on 10-node meshes; on 4-node meshes identical to
 * FETI_LINEAR_ISO (the element mean of div u is div u itself). */
enum { FETI_LINEAR_ISO = 0, FETI_HGO_TWO_FIBRE = 1, FETI_LINEAR_ISO_P0 = 2 };
enum { FETI_CLASSICAL = 0, FETI_ALL_FLOATING = 1 };             /* feti_options.method */
enum { FETI_PREC_IDENTITY = 0, FETI_PREC_LUMPED = 1, FETI_PREC_DIRICHLET = 2 };
/* feti_options.precision: FETI_FP64 -- every operator in FP64; FETI_MIXED --
 * FP32 copies of the dense local operators F_i and S_i inside the PCG,
 * FP64 vectors, dot products, projection, coarse solve and an FP64 outer
 * residual (iterative refinement on the dual problem);
 * FETI_MIXED_F32FACTOR -- as FETI_MIXED, but the local factorizations
 * themselves run in FP32 (F_i and S_i come out of the FP32 elimination), and
 * every FP64-accurate use of K_i^+ (dual right-hand side, outer residual,
 * recovery) is an FP32 triangular solve refined against the FP64 element
 * matrices (mixed-precision iterative refinement); linear solves only. */
enum { FETI_FP64 = 0, FETI_MIXED = 1, FETI_MIXED_F32FACTOR = 2 };

/* Mesh T_N of Sec. 3.2 and its non-overlapping decomposition (Sec. 4, Eq.
 * decomposition).  coords: [n_nodes*3] reference coordinates; tets:
 * [n_tets*nodes_per_tet] node ids, positive orientation; part: [n_tets]
 * subdomain id in [0, n_parts).  Every subdomain must own at least one
 * tetrahedron.  nodes_per_tet: 4 (P1; 0 is read as 4) or 10 (P2, straight
 * edges: the four vertices, then the midpoints of the edges (0,1), (0,2),
 * (0,3), (1,2), (1,3), (2,3); linear materials only; Sec. 5.1, Table 3). */
typedef struct {
  int32_t n_nodes;
  const double* coords;
  int32_t n_tets;
  const int32_t* tets;
  const int32_t* part;
  int32_t n_parts;
  int32_t nodes_per_tet;
} feti_mesh;

/* Material of Sec. 3.1.  LINEAR_ISO: Hooke with (E, nu).  HGO_TWO_FIBRE:
 * Psi = kappa/2 (J-1)^2 + c/2 (I1bar-3) + sum_f k1/(2 k2) (exp(k2 (I4bar_f-1)^2)-1)
 * (Eqs. isoaniso, iso, aniso_1, aniso_2), a fibre family contributing only
 * while I4bar_f - 1 > 1e-12; fibres: [n_tets*6] = a1, a2 per element (unit
 * vectors, reference configuration), required for HGO_TWO_FIBRE. */
typedef struct {
  int32_t kind;
  double E, nu;
  double c, k1, k2, kappa;
  const double* fibres;
} feti_material;

/* Boundary data (Sec. 3, Eqs. Dirichlet and Neumann).
 * dir_dof: [n_dir] strictly increasing DOFs with prescribed values dir_val.
 * press_tri: [n_press*3] triangles oriented so that (x1-x0) x (x2-x0) points
 * into the solid, press_owner: [n_press] the tetrahedron owning each face;
 * a pressure p pushes along that area vector (P1-consistent: a third of the
 * force to each vertex).  trac_tri/trac_owner likewise, with the constant
 * traction vector traction[3] per unit reference area.  On 10-node meshes the
 * faces have 6 nodes (v0, v1, v2, then the midpoints of (v0,v1), (v1,v2),
 * (v2,v0)) and the consistent load of a flat face goes a third to each edge
 * midpoint (the vertex shape functions integrate to zero); a pressure there
 * does not follow the deformation. */
typedef struct {
  int32_t n_dir;
  const int32_t* dir_dof;
  const double* dir_val;
  int32_t n_press;
  const int32_t* press_tri;
  const int32_t* press_owner;
  double pressure;
  int32_t n_trac;
  const int32_t* trac_tri;
  const int32_t* trac_owner;
  double traction[3];
} feti_bc;

typedef struct {
  int32_t method;      /* FETI_CLASSICAL or FETI_ALL_FLOATING */
  int32_t precond;     /* FETI_PREC_* */
  int32_t precision;   /* FETI_FP64, FETI_MIXED or FETI_MIXED_F32FACTOR */
  double tol;          /* stop when ||P r_k||_2 <= tol ||P r_0||_2 */
  int32_t maxit;       /* PCG iteration limit */
  int32_t chunk;       /* PCG iterations per CUDA-graph launch (0: default 16) */
  int32_t follower;    /* nonzero: pressure follows the deformed surface (Newton) */
  int32_t n_load_steps;
  double newton_tol;
  int32_t newton_maxit;
  double inner_tol;    /* FETI_MIXED: relative tolerance of each inner solve (0: 1e-4) */
  int32_t max_outer;   /* FETI_MIXED: limit on refinement passes (0: 20) */
  int32_t no_tensor_cores; /* FP32 block GEMM: 0 = autotuner picks tensor cores if faster,
                              1 = CUDA cores only, 2 = tensor cores whenever they run cleanly
                              (fastest staging variant), 3 / 4 / 5 / 6 / 7 = only the
                              register-staged / bulk-copy staged / tensor-map (TMA) fed /
                              warp-specialised TMA-fed 3-stage / 2-stage tensor-core kernel,
                              8 / 9 / 10 = only the persistent kernel (over all tiles,
                              double-buffered accumulators) with 3 / 3 / 2 raw A copies
                              and 2 / 3 / 2 tail slots in flight, two / two / three CTAs
                              per SM */
  int32_t per_subdomain;   /* nonzero: the dense local applies of F_i and S_i are launched once per
                              subdomain (p launches per apply, the plain non-batched form) instead
                              of one batched launch over all subdomains; same results, for
                              measuring what batching buys */
  int32_t symmetric;       /* FP32 single-vector local applies: 0 = the autotuner picks the
                              symmetric kernel (reads only the lower block-triangle of F_i / S_i)
                              when it is faster, 1 = full rows only, 2 = symmetric always
                              (fastest variant), 3 = symmetric, streamed through shared memory,
                              4 = symmetric, one CTA per subdomain (transposed partial sums
                              reduced in shared memory, no second pass) */
  uint64_t spin_timeout_ns; /* budget of each main-loop mbarrier wait of the streamed symmetric
                               apply and the warp-specialised tensor-core block GEMM, in ns,
                               counted as SM clock cycles at the device's maximum clock
                               (0: 0.1 s).  A wait that runs out stops the
                               kernel's pipeline, waits for its copies and tensor-core products in
                               flight (those drain waits keep a fixed budget of 2e8 clock cycles),
                               releases tensor memory and flags the call, which then returns
                               FETI_ERR_TIMEOUT; the context stays usable.  The same budget bounds
                               each dependency wait of the sparse coarse solve. */
  int32_t coarse_form;      /* the coarse problem (G^T G)^-1 of the projection (Sec. 4.3):
                               0 = automatic (sparse from 1536 coarse columns on), 1 = dense
                               explicit inverse (block elimination; each projection a dense
                               matvec), 2 = sparse: supernodal Cholesky over a nested-dissection
                               order of the subdomain graph (fronts eliminated level by level),
                               each projection a forward and a backward sweep over the supernodes
                               run as one task-graph kernel whose waits are bounded as above */
  int32_t local_form;       /* the local apply y_i = K_i^+ v_i of F inside the PCG (Sec. 4.3):
                               0 = automatic (explicit), 1 = explicit F_i = (S_i[b',b'])^-1 applied
                               as a dense matvec, 2 = implicit: forward and backward triangular
                               sweeps over the local Cholesky factor on the placed boundary
                               vector every iteration, the paper's sparse-direct form (FETI_FP64
                               only; the block form, the allocation-free apply and the
                               preconditioner stay explicit) */
  int32_t workspace_mb;     /* device memory of the dense elimination workspace (Sec. 4.4: the
                               local factorizations and the Schur complements S_i, F_i): the
                               subdomains are eliminated in consecutive groups whose (n + n_b')^2
                               matrices fit this many MiB (at least one subdomain per group), one
                               workspace reused by every group, and after each group the
                               interior columns of its factor (L_II, L_bI) are copied into a
                               compact array that the K^+ solves use (the boundary block of K^+
                               through the explicit F_i).  0 = automatic (12288 MiB), -1 = one
                               group holding every subdomain.  The implicit local form keeps the
                               whole factor (one group). */
} feti_options;

typedef struct {
  int32_t iterations;      /* PCG iterations (F applications after lambda_0; mixed: inner total) */
  int32_t converged;
  double rel_residual;     /* ||P r_k|| / ||P r_0|| at exit */
  double cond_est;         /* Lanczos estimate from the CG coefficients */
  double t_setup_ms;       /* element matrices + local assembly + factorizations */
  double t_pcg_ms;         /* lambda_0 -> stop, device time */
  double t_total_ms;
  int64_t n_lambda;        /* number of multipliers */
  int64_t coarse_dim;      /* columns of G */
  int32_t newton_iters;    /* total Newton iterations (feti_newton) */
  double newton_rel_res;   /* final relative residual (feti_newton) */
  int32_t outer_iterations; /* FETI_MIXED: refinement passes (FP64 residuals) */
} feti_report;

typedef struct feti_ctx feti_ctx;

/* Builds the decomposition on the host (local numbering, multipliers, kernels,
 * fixing DOFs) and uploads the problem to the current CUDA device.  stream: a
 * cudaStream_t to run on, or NULL for a library-owned stream.  No numerical
 * work on the device yet. */
feti_status feti_create(feti_ctx** out, const feti_mesh* mesh, const feti_material* mat,
                        const feti_bc* bc, const feti_options* opt, void* stream);

/* The same argument checks and host decomposition as feti_create (Sec. 4.1
 * tearing and the multiplier rows, Sec. 4.3 kernels R_i and the coarse space,
 * Sec. 5.2 fixing DOFs, the sparse coarse ordering, the workspace groups)
 * without any CUDA device or device memory: a host plan for checking and
 * sizing a decomposition.  Only the host getters accept the context
 * (feti_get_sizes, feti_get_coarse_info, feti_get_factor_info,
 * feti_get_index_maps, feti_get_fixing, feti_last_error); every call that
 * needs the device returns FETI_ERR_STATE.  Free with feti_destroy. */
feti_status feti_create_plan(feti_ctx** out, const feti_mesh* mesh, const feti_material* mat,
                             const feti_bc* bc, const feti_options* opt);

/* Linear problem: element matrices, local assembly, local factorizations,
 * dense local operators, coarse problem, then projected PCG and recovery.
 * Writes the displacement [n_nodes*3] to u_out (host or device pointer;
 * u_on_device says which).  report may be NULL. */
feti_status feti_solve(feti_ctx* ctx, double* u_out, int32_t u_on_device, feti_report* report);

/* Block form: nrhs (1..16) load cases at once, f_k = load_scale[k] * f (the
 * pressure and traction loads scaled; Dirichlet data must be homogeneous).
 * The nrhs projected CG recurrences share every operator apply: each dense
 * local operator entry read from memory feeds nrhs products (a batched GEMM
 * instead of a matvec).  A converged right-hand side is frozen while the
 * others continue.  u_out: [nrhs][n_nodes*3], host or device.  report:
 * iterations = shared iteration count (until the last right-hand side
 * converged), summed over refinement passes for FETI_MIXED. */
feti_status feti_solve_multi(feti_ctx* ctx, const double* load_scale, int32_t nrhs, double* u_out,
                             int32_t u_on_device, feti_report* report);

/* Nonlinear problem (Sec. 3.2, Eq. loadStepping): tau = s / n_load_steps,
 * Newton with one FETI solve per step until ||R|| <= newton_tol ||tau f_ext||.
 * Requires FETI_HGO_TWO_FIBRE.  Writes U [n_nodes*3] like feti_solve. */
feti_status feti_newton(feti_ctx* ctx, double* u_out, int32_t u_on_device, feti_report* report);

/* Load steps first_step .. last_step (1 <= first_step <= last_step <=
 * n_load_steps) of the load-stepped Newton method of feti_newton, starting
 * from U_start [n_nodes*3] -- the displacement after load step first_step - 1
 * (NULL: zero, the unloaded state; first_step = 1 with NULL is feti_newton).
 * U_start and u_out are host or device pointers as u_on_device says.  The
 * continuation of a long run from a checkpoint (Sec. 5.3 runs hundreds of
 * load steps).  pcg_per_step / newton_per_step (host arrays of
 * last_step - first_step + 1 entries, may be NULL) receive the PCG iterations
 * (summed over the FETI solves of the step) and the Newton iterations each
 * load step took. */
feti_status feti_newton_steps(feti_ctx* ctx, const double* U_start, int32_t first_step, int32_t last_step,
                              double* u_out, int32_t u_on_device, int32_t* pcg_per_step, int32_t* newton_per_step,
                              feti_report* report);

/* Checkpoint of a load-stepped run: the state after load step `step` of
 * n_load_steps, tau = step / n_load_steps (Eq. loadStepping), and U [n_dofs]
 * (host array).  Binary file: magic "FETICKP1", n_dofs (int64), step,
 * n_load_steps (int32), tau (double), U (n_dofs doubles), FNV-1a 64-bit hash
 * of all preceding bytes; native byte order.  Written to "<path>.tmp" and
 * renamed over path.  Host-only (no CUDA call, no context); FETI_ERR_IO when the
 * file cannot be written. */
typedef struct {
  int64_t n_dofs;
  int32_t step;
  int32_t n_load_steps;
  double tau;
} feti_checkpoint_info;
feti_status feti_checkpoint_write(const char* path, const double* U, int64_t n_dofs, int32_t step,
                                  int32_t n_load_steps, double tau);
/* Reads a checkpoint: header into *info (may be NULL) and, with U != NULL,
 * the displacement into U (capacity doubles; too small: FETI_ERR_INVALID_ARG).
 * U == NULL reads the header only.  FETI_ERR_IO for a missing, truncated or
 * corrupt file (bad magic, sizes or hash); U is written only after the hash
 * matched. */
feti_status feti_checkpoint_read(const char* path, double* U, int64_t capacity, feti_checkpoint_info* info);

/* Element level of Sec. 3.2 (Eq. Tangent and the residual K(U)): for every
 * tetrahedron the 12x12 tangent K_e (30x30 on 10-node meshes; row-major,
 * local DOF 3 * node + component, nodes in tets order) into Ke_out
 * [n_tets*144] ([n_tets*900]), and for the
 * hyperelastic material the internal force f_e = V (F S grad N_a) into
 * fe_out [n_tets*12] (may be NULL; unused for the linear materials), at the
 * displacement U [n_nodes*3] (NULL = zero).  U and the outputs are host or
 * device pointers as u_on_device / out_on_device say.  Fails with
 * FETI_ERR_ELEMENT_INVERTED if det F <= 0 anywhere. */
feti_status feti_elements(feti_ctx* ctx, const double* U, int32_t u_on_device, double* Ke_out, double* fe_out,
                          int32_t out_on_device);

/* Sizes of the decomposition: out[0] n_lambda, out[1] coarse_dim, out[2]
 * sum of local DOFs, out[3] sum of boundary DOFs, out[4] n_parts. */
feti_status feti_get_sizes(const feti_ctx* ctx, int64_t out[5]);

/* Form of the coarse problem (G^T G)^-1 (Sec. 4.3) chosen at feti_create:
 * out[0] 0 no coarse space, 1 dense explicit inverse, 2 sparse supernodal
 * Cholesky; for the sparse form out[1] supernodes, out[2] height of the
 * assembly tree, out[3] entries of the factor (lower triangle of each
 * diagonal block plus its panel), out[4] tasks of one forward + backward
 * sweep, out[5] doubles of the factorization workspace (held only during
 * set-up); for the dense form out[3] = coarse_dim^2. */
feti_status feti_get_coarse_info(const feti_ctx* ctx, int64_t out[6]);

/* Storage of the local factorizations (Sec. 4.4) chosen at feti_create:
 * out[0] groups of subdomains eliminated one after another in the reused
 * workspace, out[1] elements of that workspace, out[2] elements the whole
 * dense workspace would take (every subdomain at once), out[3] elements of the
 * compact interior factor kept for the K^+ solves (0 when the whole factor is
 * kept), out[4] bytes per element (8 FP64, 4 FP32 factorizations). */
feti_status feti_get_factor_info(const feti_ctx* ctx, int64_t out[5]);

/* Multiplier rows in canonical order (Sec. 4.1, Fig. 3a, fully redundant):
 * interface rows by (global node, component, subdomain pair i<j) with +1 on
 * i and -1 on j, then (all-floating) Dirichlet rows by (node, component,
 * subdomain) with +1.  Host arrays of n_lambda*2 entries: row_sub (-1 pad),
 * row_ldof (local DOF = 3 * local node + component, local nodes = the
 * subdomain's global node ids in increasing order), row_sign; weight and b
 * have n_lambda entries.  Any pointer may be NULL. */
feti_status feti_get_index_maps(const feti_ctx* ctx, int32_t* row_sub, int32_t* row_ldof,
                                int8_t* row_sign, double* weight, double* b);

/* Fixing DOFs of the generalized inverses (Sec. 5.2, regularization by
 * fixing nodes): fix_ptr [n_parts+1] and fix_ldof [fix_ptr[n_parts]], local
 * DOFs per subdomain in selection order.  Either pointer may be NULL. */
feti_status feti_get_fixing(const feti_ctx* ctx, int32_t* fix_ptr, int32_t* fix_ldof);

/* Hot-path benchmark hook: after feti_solve (or feti_prepare), applies the
 * dual operator and the preconditioner n_apply times back to back to device
 * vectors: q = F v, then z = M^-1 q (Sec. 4.3, Eq. classicalFetiF, and Sec.
 * 4.4, Eq. feti_preconditioner), without projection; v, q, z are device
 * arrays of n_lambda doubles.  The applies run as one CUDA graph (captured on
 * the first call for a given (v, q, z, n_apply) and replayed afterwards) on
 * the context's stream; *ms_per_apply (may be NULL) receives the average
 * device time per apply of this launch.  Returns after the launch completed. */
feti_status feti_dual_apply(feti_ctx* ctx, const double* v, double* q, double* z,
                            int32_t n_apply, double* ms_per_apply);

/* Block benchmark hook: like feti_dual_apply on blocks v, q, z of
 * [n_lambda][nrhs] doubles (row-major, nrhs contiguous per multiplier). */
feti_status feti_dual_apply_multi(feti_ctx* ctx, const double* v, double* q, double* z, int32_t nrhs,
                                  int32_t n_apply, double* ms_per_apply);

/* Allocation-free variant of feti_dual_apply (one apply: q = F v, then
 * z = M^-1 q; v, q, z: device arrays of n_lambda doubles).  The paper has no
 * counterpart: this call exists for callers that must not allocate device
 * memory after setup -- a fixed memory budget reserved at start-up, a
 * latency-critical loop that cannot take cudaMalloc's implicit device
 * synchronisation, or work issued while another component holds the
 * allocator.  It allocates nothing and creates no graph or event: its local
 * scratch vectors live in one static device array of 2^20 doubles (8 MiB)
 * that every GPU loading the library keeps until process exit.
 *  - Limit: a decomposition needs about 2.5 x (sum of boundary DOFs) doubles;
 *    larger ones are rejected with FETI_ERR_INVALID_ARG and a message.
 *  - Set-up happens in feti_create, with the context's device current: it
 *    looks up the array's device address (cudaGetSymbolAddress), which also
 *    makes the runtime load the module holding the array there, so no call of
 *    this function loads code or reserves memory.  Call it with the same
 *    device current (another device: FETI_ERR_INVALID_ARG).  An error left
 *    pending by earlier CUDA work is reported (FETI_ERR_CUDA), not cleared.
 *  - The work is enqueued on the context's stream and the call returns
 *    without waiting.  All calls share the array: calls whose work overlaps
 *    on the GPU (other streams, other contexts) race on it.  Every scratch
 *    entry is written before it is read, so nothing needs clearing.
 *  - Requires feti_prepare (or feti_solve) on this context first. */
feti_status feti_dual_apply_noalloc(feti_ctx* ctx, const double* v, double* q, double* z);

/* Runs the setup part of feti_solve (element matrices through coarse
 * factorization) without PCG. */
feti_status feti_prepare(feti_ctx* ctx);

/* Dominant per-iteration kernel (dense local F_i apply with fused gather):
 * its device time averaged over the launches inside the last feti_dual_apply
 * (timed by event nodes around each launch in that graph), the algorithmic
 * bytes one launch must move (each of the n(n+1)/2 distinct entries of the
 * symmetric F_i once, gathered multipliers,
 * local outputs) and its floating-point operations (2 per F_i entry). */
feti_status feti_kernel_stats(const feti_ctx* ctx, double* gemv_ms, double* gemv_bytes,
                              double* gemv_flops);

/* Element kernel of the last feti_elements call (the P1 tangent and
 * internal-force kernel of Sec. 3, hyperelastic or linear): its device time
 * (CUDA events on the context's stream around the one launch), the
 * algorithmic bytes it must move (connectivity 16 B, fibres 48 B, the
 * symmetric tangent 78 x 8 B and the force 12 x 8 B per element, coordinates
 * and displacement 48 B per node, each read once) and the element count.
 * Zeros before the first feti_elements call. */
feti_status feti_element_stats(const feti_ctx* ctx, double* elem_ms, double* elem_bytes,
                               double* n_elements);

/* Launch schedules of the dense local applies chosen by the setup-time
 * autotuner (timed on the real operators, fastest kept): out[0..1] rows per
 * warp step and rows per CTA of the FP64 F_i apply, out[2..3] of the FP64
 * preconditioner apply, out[4..7] the same for the FP32 copies (rows per warp
 * step -G, rows 32 = symmetric kernel on 32-row panels, load groups of
 * G % 100 rows with an L2 prefetch G / 100 tiles ahead; G = 64: panels
 * streamed through shared memory; G = 300 + g: one CTA per subdomain, load
 * groups of g rows), out[8..11]
 * the FP32 block-form GEMMs (rows per warp step 0 / -1 / -2 / -3 / -4 =
 * tensor-core kernel with register-staged / bulk-copy staged / tensor-map fed
 * operands / warp-specialised 3-stage / 2-stage; both entries -1 = block form
 * not tuned yet). */
feti_status feti_get_schedule(const feti_ctx* ctx, int32_t out[12]);

/* FETI_MIXED_F32FACTOR: the number of FP64 refinement corrections each
 * application of K_i^+ takes (chosen at setup: corrections are added while
 * the largest relative residual ||g - K_rr x|| / ||g|| over the subdomains,
 * on a fixed pseudo-random g, still halves and exceeds 1e-14; at most 12) and
 * that residual.  Zeros for the other forms or before setup. */
feti_status feti_get_refinement(const feti_ctx* ctx, int32_t* steps, double* residual);

/* Sets the main-loop wait budget of feti_options.spin_timeout_ns for the
 * later calls on this context, in ns taken literally (100000000 = the default
 * 0.1 s); a budget below one clock cycle, e.g. 0, makes every main-loop wait
 * give up at its first check (the pipelines then always stop, drain and
 * report FETI_ERR_TIMEOUT: a way to exercise that path).  Captured graphs
 * read the budget at every launch.  Host blocking: waits for the context's
 * stream. */
feti_status feti_set_spin_timeout(feti_ctx* ctx, uint64_t spin_timeout_ns);

const char* feti_last_error(const feti_ctx* ctx);
void feti_destroy(feti_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* FETI_H */
