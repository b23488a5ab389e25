/*
 * afd.h -- C ABI of the assembly-free deflated finite element hot path of the
 * augmented topological level-set method (Deng & Suresh, arXiv 2203.15115).
 *
 * The library solves K u = f (Eq. 1.1, Sec. 3.5) on a voxel mesh of nx*ny*nz
 * trilinear hexahedra (Sec. 3.8 step 1) with one Young's modulus per element,
 * without assembling K, by Jacobi-preconditioned conjugate gradients deflated
 * with the rigid-body modes of agglomerated node groups (Sec. 3.5).  It then
 * evaluates the compliance J = f^T u (Eqs. 1.3-1.4), per-element sensitivity
 * fields (Eqs. 3.2, 3.3, 3.5 and the element-sensitivity fallback of Sec. 3.1),
 * and extracts the next topology from the combined level-set (Eqs. 3.6, 3.17).
 *
 * Conventions (the paper is silent on them):
 *   element (i,j,k), 0<=i<nx:  e = i + nx*(j + ny*k)
 *   node    (i,j,k), 0<=i<=nx: n = i + (nx+1)*(j + (ny+1)*k)
 *   DOF = 3*n + c, c in {0:x, 1:y, 2:z};  element edge h (option, default 1)
 *   multi-RHS arrays are RHS-major: value (r, d) at r*ndof + d.
 *
 * Ownership: the library allocates and owns all device memory it uses; the
 * caller owns every pointer it passes.  Host pointers are read/written only
 * during the call.  Device pointers (flag *_on_device = 1) must point to
 * memory of the mesh's device and stay valid until the call returns; the call
 * is ordered on the mesh's CUDA stream and returns after that stream has
 * finished the work unless stated otherwise.
 *
 * Errors: every int-returning call returns AFD_OK (0) or a negative AFD_ERR_*
 * code; afd_last_error() returns a thread-local message for the last failure.
 * No call aborts the process; device loops are iteration-capped and report a
 * status word, so an unconverged or singular system is an error code, not a
 * hang.
 */
#ifndef AFD_H_
#define AFD_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  AFD_OK = 0,
  AFD_ERR_INVALID_ARG = -1,     /* bad size, null pointer, NaN/negative modulus ... */
  AFD_ERR_OOM = -2,             /* device allocation failed, or a budget was exceeded */
  AFD_ERR_NOT_CONVERGED = -3,   /* iteration cap reached; u still holds the best iterate */
  AFD_ERR_COARSE_SINGULAR = -4, /* the coarse matrix W^T K W is singular: its inversion (blocked Gauss-Jordan
                                   sweeps of the SPD matrix) met a pivot <= 0 (e.g. no supports) */
  AFD_ERR_NAN = -5,             /* a residual norm became NaN or Inf */
  AFD_ERR_CUDA = -6,            /* a CUDA runtime call failed */
  AFD_ERR_STATE = -7            /* call out of order (e.g. solve before set_loads_bcs) */
};

enum { AFD_FP64 = 0, AFD_MIXED = 1 };        /* solver precision */
/* arithmetic type of a stencil call: FP32 on float data, FP64 on double data, or double-float on double data
 * (each value an unevaluated sum of two floats, about 44 significant bits, on the FP32 pipes) */
enum { AFD_F32 = 0, AFD_F64 = 1, AFD_F64_DF = 2 };
enum {
  AFD_SENS_STRAIN_ENERGY = 0,  /* s_e = u_e^T (E_e K0) u_e; sums to J (Sec. 3.1 fallback) */
  AFD_SENS_TJ = 1,             /* Eq. 3.2 at the element centroid, as printed */
  AFD_SENS_VON_MISES = 2       /* von Mises stress at the element centroid (Eq. 3.3's measure) */
};

typedef struct afd_mesh afd_mesh;

typedef struct {
  int precision;      /* AFD_MIXED (FP32 inner DPCG in FP64 iterative refinement) or AFD_FP64 */
  int group;          /* deflation agglomeration: elements per group edge (g); 0 = automatic */
  double nu;          /* Poisson ratio (default 0.3, Sec. 4) */
  double h;           /* element edge length (default 1) */
  double e_void;      /* modulus given to removed elements by the level-set update (default 1e-3) */
  int max_iter;       /* cap on inner DPCG iterations per solve (default 20000) */
  int max_refine;     /* cap on FP64 refinement steps in AFD_MIXED (default 12) */
  double inner_tol;   /* floor of the inner relative tolerance in AFD_MIXED (default 2e-5) */
  int check_every;    /* DPCG iterations per captured CUDA graph between host checks (default 16) */
  int autotune;       /* 1 (default): at the first solve, time the stencil's z depth per CTA and keep the fastest */
  int persistent;     /* AFD_MIXED inner solves: 0 (default) CUDA-graph chunks of check_every iterations,
                         one kernel per phase; 1 one cooperatively launched persistent kernel per inner
                         solve with grid-wide barriers between its phases (afd_solver_phase_times) */
  int stencil_warps;  /* FP32 stencil CTA: 8 or 16 warps; 0 (default) = chosen by the autotuner/heuristic */
  int stencil_planes; /* FP32 stencil: node planes per CTA (>= 1); 0 (default) = autotuner/heuristic.
                         When both are set the autotuner does not run. */
  int pdl;            /* 1: the kernels of a captured DPCG iteration chunk use programmatic dependent launch
                         (each may be scheduled while its predecessor finishes its reductions); 0 (default):
                         plain stream order, measured faster on the 128x64x64 workload */
  double inner_aim;   /* AFD_MIXED: each inner solve aims at inner_aim * rel_tol in the true relative residual
                         (not below inner_tol); default 0.7, in (0, 1) */
  int coarse_fp64;    /* AFD_MIXED: 1 builds W^T K W from FP64 element products and inverts it in FP64 (its
                         FP32 rounding is applied in the FP32 inner iterations); 0 (default) builds it from
                         FP32 element products summed in FP64 and inverts it in FP32 (same inner iteration
                         counts on the measured workloads at a lower set-up cost).  AFD_FP64 is always FP64. */
  int residual_fp64;  /* AFD_MIXED: 0 (default) evaluates the refinement residual f - K u from the FP64 u and f
                         in double-float arithmetic (AFD_F64_DF) when rel_tol >= 1e-10 and every nonzero
                         ||f|| lies in [1e-20, 1e20], else in FP64 (and again in FP64 if its norm is not
                         finite); 1 always in FP64.  The double-float residual's rounding is a few 2^-44 of
                         the element forces, far below the tolerances it serves, at a fraction of FP64's
                         cost on GB300. */
} afd_options;

typedef struct {
  int iters;            /* inner DPCG iterations (summed over refinement steps) */
  int refine_steps;     /* FP64 residual evaluations after the first (AFD_MIXED) */
  double rel_residual;  /* final ||f - K u||_2 / ||f||_2 over free DOFs, FP64 */
  double ms;            /* wall time of the solve call */
  int status;           /* AFD_OK or AFD_ERR_NOT_CONVERGED / AFD_ERR_NAN for this RHS */
} afd_stats;

/* Fill *opt with the defaults listed above. */
void afd_default_options(afd_options* opt);

/* Create a mesh of nx*ny*nz hexahedra (Sec. 3.8 step 1).  cuda_stream is a
 * cudaStream_t of the current device (NULL = the legacy default stream); every
 * later call on the mesh is ordered on it.  opt may be NULL (defaults); it is
 * copied.  nx, ny, nz >= 1 and the DOF count must fit in int32 indices. */
int afd_create_mesh(int nx, int ny, int nz, const afd_options* opt, void* cuda_stream, afd_mesh** out);

/* Per-element Young's modulus E_e (length nx*ny*nz, element order above),
 * FP64, each finite and > 0.  Invalidates the coarse factor (rebuilt lazily
 * by the next solve: E = W^T K W and its Cholesky factor, FP64). */
int afd_set_element_moduli(afd_mesh* m, const double* E, int E_on_device);

/* Loads and supports: n_rhs load cases f (n_rhs*ndof, FP64, RHS-major) and a
 * fixed-DOF mask (ndof bytes, nonzero = displacement fixed to 0; shared by all
 * load cases).  Loads on fixed DOFs are ignored.  Resets the warm start. */
int afd_set_loads_bcs(afd_mesh* m, int n_rhs, const double* f, int f_on_device,
                      const uint8_t* fixed_dof_mask, int mask_on_device);

/* Solve K u = f for every load case to ||f - K u||_2 <= rel_tol ||f||_2 over
 * the free DOFs (Eq. 1.1).  warm_start = 1 starts from the previous solution
 * kept in the mesh (the level-set iterations of Sec. 3.2), 0 from u = 0.
 * per_rhs (nullable) receives n_rhs stats; u_out (nullable) receives
 * n_rhs*ndof FP64 displacements.  Returns AFD_ERR_NOT_CONVERGED if any load
 * case missed the tolerance (u_out still written). */
int afd_solve(afd_mesh* m, double rel_tol, int warm_start, afd_stats* per_rhs,
              double* u_out, int u_on_device);

/* J_r = f_r^T u_r for every load case (Eqs. 1.3-1.4), FP64, host output. */
int afd_compliance(afd_mesh* m, double* J_out);

/* Per-element field of the given kind for every load case from the current
 * solution: out has n_rhs*nelem floats, RHS-major. */
int afd_sensitivity(afd_mesh* m, int kind, float* out, int out_on_device);

/* p-norm of the element von Mises stresses, (sum_e sigma_vm,e^p)^(1/p), per
 * load case (the stress measure of Eq. 3.3), FP64, host output. */
int afd_pnorm_stress(afd_mesh* m, double p, double* out);

/* Adjoint topological sensitivity of the p-norm stress (Eq. 3.3, read with
 * the adjoint state): sigma_PN = (sum_e s_e^p)^(1/p) of the centroid von Mises
 * stresses of the current solution (afd_pnorm_stress), the adjoint lambda
 * solving K lambda = -d sigma_PN / d u on the free DOFs (the same solver,
 * precision, coarse space and rel_tol as afd_solve; adj_stats per load case,
 * nullable), and per element at the centroid
 *   T_sigma = 4/(1+nu) sigma(u):eps(lambda) - (1-3 nu)/(1-nu^2) tr sigma(u) tr eps(lambda).
 * out: n_rhs*nelem floats, RHS-major; lambda_out (nullable): n_rhs*ndof.
 * The solution u is left unchanged.  AFD_ERR_NOT_CONVERGED if an adjoint
 * solve stopped above rel_tol (out is still written). */
int afd_stress_sensitivity(afd_mesh* m, double p, double rel_tol, float* out, int out_on_device, afd_stats* adj_stats,
                           double* lambda_out, int lambda_on_device);

/* Modal analysis for the eigenvalue constraint of Sec. 3.8 (Eq. 3.4 needs the
 * modes): the n_modes smallest eigenpairs of K_ff phi = lambda M_ff phi
 * (lambda = omega^2) on the mesh's moduli and supports.  The paper gives no
 * mass matrix; M is lumped, every node of element e receiving
 * rho_e h^3 / 8 per direction with rho_e = rho * E_e (density follows the
 * modulus).  Block LOBPCG on a block of n_modes + 2 vectors, preconditioned
 * by K^-1 from the mesh's solver (its precision and options, relative
 * tolerance 3e-2): each step forms the residuals K phi - lambda M phi, solves
 * for the new directions W of the vectors not yet converged (soft locking)
 * and takes the Rayleigh-Ritz pairs of span[X, W, P]
 * (FP64 Gram matrices; a small generalised eigenproblem on the device,
 * directions scaled and truncated against dependence).  Stops when every
 * requested pair has ||K phi - lambda M phi|| <= tol lambda ||M phi|| (free
 * DOFs), else after max_iter steps with AFD_ERR_NOT_CONVERGED (outputs still
 * written).  AFD_ERR_NAN if an eigenvalue is not positive (supports that
 * leave a rigid-body mode).
 * n_modes in [1, 10]; rho > 0.
 * lam_out: n_modes doubles (host), ascending.  modes_out (nullable):
 * n_modes*ndof, M-orthonormal, zero on fixed DOFs, sign arbitrary.
 * iters_out / solve_iters_out (nullable): LOBPCG steps; inner DPCG
 * iterations summed over the steps (the largest per step).
 * The load cases are kept; the static solution is discarded (afd_solve
 * again before afd_compliance or afd_sensitivity).  The modes stay in the
 * mesh for afd_eigen_sensitivity. */
int afd_modal(afd_mesh* m, int n_modes, double rho, double tol, int max_iter, double* lam_out, double* modes_out,
              int modes_on_device, int* iters_out, int* solve_iters_out);

/* Topological sensitivity of the eigenvalues (Eq. 3.4) for the modes of the
 * last afd_modal, per element at the centroid:
 *   T_lambda = sigma(phi):eps(phi) - lambda rho_e |phi(centroid)|^2,
 * phi(centroid) the mean of the element's eight nodal vectors.
 * out: n_modes*nelem floats, mode-major.  AFD_ERR_STATE without modes. */
int afd_eigen_sensitivity(afd_mesh* m, float* out, int out_on_device);

/* Linear buckling for the buckling constraint of Sec. 3.8 (Eq. 3.5 needs the
 * modes): the n_modes smallest positive load factors lambda of
 * (K + lambda K_G) phi = 0 on the free DOFs, lambda the factor on load case 0
 * at which the structure buckles.  The pre-buckling state is the mesh's
 * current static solution of load case 0 (afd_solve first): its stress at each
 * element centroid, held constant over the element, gives the geometric
 * stiffness K_G^e[(a,i),(b,j)] = delta_ij int grad N_a . S_e grad N_b (exact
 * cube integrals).  Block LOBPCG for the smallest eigenvalues theta of
 * K_G phi = theta K phi (lambda = -1/theta), block n_modes + 2, with
 * K^-1 by the mesh's solver (relative tolerance 3e-2) as the preconditioner,
 * soft locking of converged vectors
 * and Rayleigh-Ritz on [X, W, P] (FP64 Gram matrices, directions scaled and
 * truncated against dependence on the device).  It targets the smallest
 * positive factors even when the reversed load buckles first.
 * Stops when every requested pair has ||K_G phi - theta K phi|| <= tol |theta| ||K phi||,
 * else after max_iter steps with AFD_ERR_NOT_CONVERGED (outputs written).
 * AFD_ERR_NAN if the load gives fewer than n_modes positive factors.
 * lam_out: n_modes doubles ascending; modes_out (nullable): n_modes*ndof,
 * K-orthonormal, zero on fixed DOFs, sign arbitrary.  n_modes in [1, 10].
 * The load cases are kept; the static solution is discarded.  The modes
 * stay in the mesh for afd_buckling_sensitivity (a later afd_modal replaces
 * them, and the other way round). */
int afd_buckling(afd_mesh* m, int n_modes, double tol, int max_iter, double* lam_out, double* modes_out,
                 int modes_on_device, int* iters_out, int* solve_iters_out);

/* Sensitivity of the buckling load factors (Eq. 3.5) for the modes of the last
 * afd_buckling, per element: phi_e^T (E_e K0 - lambda K_sigma^e) phi_e with
 * the paper's K_sigma read as -K_G (its buckling equation (K - lambda
 * K_sigma) phi = 0), so that the element terms of a mode sum to zero.
 * out: n_modes*nelem floats, mode-major.  AFD_ERR_STATE without modes. */
int afd_buckling_sensitivity(afd_mesh* m, float* out, int out_on_device);

/* Level-set update (Eqs. 3.6, 3.17-3.18): for every load case r compute the
 * field of `kind`, divide it by its largest magnitude, add the fields with
 * weights[r] (float32, fixed order), keep the k = round(v * nelem) elements
 * with the largest value (ties keep the lower element index), set their
 * modulus to 1 and the others to opt.e_void.  tau_out (nullable) receives the
 * cut value, kept_out (nullable, host, nelem bytes) the kept mask.  When the
 * call on this mesh just before was afd_sensitivity of the same kind, its
 * fields are reused (nothing in between can have changed u or the moduli). */
int afd_levelset_update(afd_mesh* m, int kind, const double* weights, double volume_fraction,
                        double* tau_out, uint8_t* kept_out);

/* afd_levelset_update with the casting constraint of Sec. 3.7 applied to the
 * combined field before the cut (see afd_casting_scan): axis 0/1/2 = x/y/z,
 * parting in [0, n_axis] elements (0 or n_axis: a one-piece draw).  The kept
 * set then covers, on every line along the axis and on each side of the
 * parting plane, a run of elements starting at the plane (no undercut). */
int afd_levelset_update_cast(afd_mesh* m, int kind, const double* weights, double volume_fraction, int axis,
                             int parting, double* tau_out, uint8_t* kept_out);

/* Level-set update from caller-given fields (Eqs. 3.6, 3.17-3.18), e.g. the
 * compliance and stress sensitivities of the Sec. 3.8 algorithm: nfields
 * per-element float32 fields (field-major, nfields*nelem, host or device),
 * each divided by its largest magnitude, multiplied by weights[i] and added
 * (float32, fixed order), then the casting scan when axis >= 0 (parting as in
 * afd_levelset_update_cast; axis < 0: none), the cut keeping round(v nelem)
 * elements, and the new moduli (kept 1, others opt.e_void). */
int afd_levelset_update_fields(afd_mesh* m, const float* fields, int fields_on_device, int nfields,
                               const double* weights, double volume_fraction, int axis, int parting, double* tau_out,
                               uint8_t* kept_out);

/* Casting constraint (Sec. 3.7) on a per-element float field, in place on the
 * device (keys: nx*ny*nz floats, element order e = i + nx (j + ny k)): along
 * every line parallel to `axis`, each half of the part (element index >=
 * parting, or below it) is replaced, from its far face toward the parting
 * plane, by key'(c) = max(key(c), nextafter(key'(previous), +inf)), a running
 * maximum raised by one float32 step per element.  The paper states the
 * constraint (the level set must not decrease along the casting direction)
 * without a formula; this is the reading.  Stream-ordered on cuda_stream;
 * returns after it has finished.  AFD_ERR_INVALID_ARG for a bad axis or
 * parting index. */
int afd_casting_scan(float* keys, int nx, int ny, int nz, int axis, int parting, void* cuda_stream);

/* ---- lower-level entry points (the pieces of the path, used by the tests) ---- */

/* y = K u on the free DOFs (rows and columns of fixed DOFs act as zero), in
 * FP32 (arith = AFD_F32: u, y float), FP64 (AFD_F64: double) or double-float
 * arithmetic on double data (AFD_F64_DF: u, y double); n_rhs vectors of ndof
 * values, RHS-major.  Device pointers only. */
int afd_apply_stiffness(afd_mesh* m, int arith, int n_rhs, const void* u, void* y);

/* One search-direction step of the inner FP32 deflated PCG iteration (Sec.
 * 3.5), as the solver runs it: for each of n_rhs load cases
 *   p = z + W mu + beta p_old   on the free DOFs (0 on fixed DOFs),
 *   q = K p                     (rows of fixed DOFs 0),
 * formed by the solver's fused FP32 stencil in the mesh's current CTA shape
 * (afd_set_stencil_shape pins it), and *pq_out = p.q per case (host, nullable).
 * z, p_old, p_out, q_out: device float, RHS-major with stride ndof; mu: device
 * double, n_rhs x n_c coarse coefficients (6 rigid modes per group, the order
 * of afd_deflation_w); beta: host, n_rhs values.  Needs moduli and loads
 * (the supports); builds the coarse problem if it is stale.  Used by the tests
 * to check every stencil variant element by element. */
int afd_apply_search_direction(afd_mesh* m, int n_rhs, const float* z, const float* p_old, const double* mu,
                               const double* beta, float* p_out, float* q_out, double* pq_out);

/* Deflation operators (Sec. 3.5): out = W^T v (n_rhs*6*N_g) and
 * out = W y (n_rhs*ndof), FP64, device pointers.  Group G's 6 values are
 * (T_x, T_y, T_z, R_x, R_y, R_z): force sums and moments about the group's
 * node centroid. */
int afd_deflation_wt(afd_mesh* m, int n_rhs, const double* v, double* out);
int afd_deflation_w(afd_mesh* m, int n_rhs, const double* y, double* out);

/* The inverse of W^T K W (n_c x n_c, row-major, host doubles) as the solver
 * forms it: FP32 on AFD_MIXED meshes (FP64 with opt.coarse_fp64 and on
 * AFD_FP64 meshes), from the unit-diagonal scaled matrix by blocked
 * Gauss-Jordan sweeps without pivoting (E is SPD).  Rebuilds the coarse
 * matrix from the current moduli and supports and leaves the solver's coarse
 * data stale.  AFD_ERR_COARSE_SINGULAR when a pivot of the scaled matrix is
 * <= 1e-6 (FP32) / 1e-12 (FP64) or not finite.  Used by the tests. */
int afd_coarse_inverse(afd_mesh* m, double* out_host);

/* Number of coarse unknowns 6*N_g, and the dense coarse matrix W^T K W
 * (n_c*n_c FP64, host) built from the current moduli and supports. */
int afd_coarse_size(afd_mesh* m);
int afd_coarse_matrix(afd_mesh* m, double* out_host);

/* Keep the k largest of n float keys (device), ties toward the lower index:
 * kept (device, n bytes) = 1/0, *tau_out = the k-th largest key (host).
 * Runs on cuda_stream and returns after it finishes. */
int afd_select_topk(const float* keys, int64_t n, int64_t k, uint8_t* kept, float* tau_out,
                    void* cuda_stream);

/* The same selection as afd_select_topk without allocating device memory.
 * The paper has no counterpart: this is for callers that cannot call
 * cudaMalloc -- code whose device memory belongs to another allocator (a
 * framework's caching allocator that already holds the memory) and
 * latency-sensitive loops where cudaMalloc/cudaFree would synchronise the
 * device.  The scratch (about 17 KB: the selection state and one counter per
 * 4096 keys) is a file-scope device array that every device loading this
 * library keeps until the process exits.  Limit: n <= 16,777,216 keys; larger
 * n returns AFD_ERR_INVALID_ARG without touching the device.  The first call
 * on a device looks up the array's device address (once, with that device
 * current); make that first call before any stream capture.  Every call
 * shares the one array and re-initialises it; calls that overlap on the GPU
 * (e.g. on two streams at once) race and give undefined results.  Returns
 * after cuda_stream has finished, like afd_select_topk.  keys and kept must be
 * device memory of one device; the call runs with that device current and
 * uses that device's array.  The looked-up address is cached for the life of
 * the process: do not keep using the library across a cudaDeviceReset. */
int afd_select_topk_noalloc(const float* keys, int64_t n, int64_t k, uint8_t* kept, float* tau_out,
                            void* cuda_stream);

/* Time `launches` back-to-back stiffness applies y = K u (the solver's
 * kernel and launch geometry, arith AFD_F32, AFD_F64 or AFD_F64_DF, n_rhs vectors, device
 * pointers, one launch per vector) on the mesh's stream with CUDA events
 * recorded on that stream; *ms_out = mean device time per round of n_rhs
 * launches.  Measurement aid (Sec. 3.5 names
 * memory access as the bottleneck of the assembly-free solve). */
int afd_time_stiffness(afd_mesh* m, int arith, int n_rhs, const void* u, void* y, int launches, double* ms_out);

/* Number of CUDA kernels this mesh has launched so far (a CUDA-graph replay
 * counts its kernel nodes). */
int64_t afd_kernel_launches(const afd_mesh* m);

/* Node planes per CTA of the FP32 stiffness kernel (chosen by the autotuner at
 * the first mixed solve when opt.autotune is set, else by a size heuristic). */
int afd_stencil_depth(const afd_mesh* m);

/* Warps per CTA of the FP32 stiffness kernel (8 or 16); chosen with the depth. */
int afd_stencil_warps(const afd_mesh* m);

/* Pin the FP32 stencil's variant and CTA shape (8 or 16 warps, planes >= 1,
 * clipped to the mesh) on an existing mesh; the autotuner then leaves this mesh
 * alone.  Variant (async_staging): 0 two node rows per thread, the next plane
 * prefetched into registers; 1 the same with a cp.async ring two planes ahead
 * in shared memory; 2 two row bands per CTA packed into the lanes of every
 * float2, cp.async ring; 3 variant 2 with two load cases in the lanes instead
 * of two bands, for solves of two or more load cases (one load case runs
 * variant 2). */
int afd_set_stencil_shape(afd_mesh* m, int warps, int planes, int async_staging);

/* The FP32 stencil variant in use (the async_staging values above). */
int afd_stencil_async(const afd_mesh* m);

/* Measurement aid for the CUDA-graph inner solver: continues the last FP32
 * inner DPCG iteration of a completed AFD_MIXED solve for `iters` iterations
 * (no stopping test; the solution u is not touched), launching its kernels
 * one by one with CUDA events between them on the mesh's stream (every
 * iteration enqueued before one synchronisation; iters in [1, 4096]).  us_out5 =
 * mean microseconds per iteration of the stencil, the vector update, the
 * coarse right-hand side, the coarse step, and (variant 1) the separate
 * search-direction kernel.  variant 0: the stencil forms p = z + W mu +
 * beta p_old as it loads it; variant 1: k_prolong forms p first and the
 * stencil reads it.  nsplit > 0 times the coarse right-hand side with that
 * many shares per group (0: the mesh's own).  Host output. */
int afd_time_dpcg_kernels(afd_mesh* m, int iters, int nsplit, int variant, double* us_out5);

/* Measurement aid for the persistent inner solver (opt.persistent), as seen
 * by its CTA 0 and summed over all iterations since the last reset, in ms:
 * out10[0..4] wall time of the phases between grid barriers -- stencil with
 * the fused search direction, vector update, coarse right-hand side, coarse
 * apply, scalar recurrences; out10[5] the iterations counted; out10[6..9]
 * the part of phases 0..3 that CTA 0 spent waiting in the barrier.  reset = 1
 * zeroes the counters after reading.  Host output. */
int afd_solver_phase_times(afd_mesh* m, double* out10, int reset);

/* Sizes of the mesh. */
int64_t afd_ndof(const afd_mesh* m);
int64_t afd_nelem(const afd_mesh* m);

/* Frees every device buffer, stream, event and graph the mesh owns and the
 * handle itself (null is allowed).  Waits for the mesh's stream first; the
 * handle must not be used afterwards, nor by another thread during the call. */
void afd_destroy(afd_mesh* m);

/* The message of the calling thread's most recent failure (thread-local,
 * owned by the library; the pointer stays valid until that thread's next
 * failing call); "" if none of its calls has failed. */
const char* afd_last_error(void);

/* ---- serving: solve requests of different mesh sizes concurrently ---- */

/* Upper bound of the device bytes a mesh of this size holds after a solve
 * with n_rhs load cases (host only; used for admission). */
size_t afd_mesh_bytes(int nx, int ny, int nz, int n_rhs, const afd_options* opt);

typedef struct afd_server afd_server;

typedef struct {
  int max_slots;         /* requests in flight at once (worker threads, one CUDA stream each) */
  double budget_bytes;   /* device memory the in-flight and cached meshes may hold */
  afd_options opt;       /* options of every mesh the server creates */
} afd_server_config;

/* Start a server on the current device.  Requests are admitted in arrival
 * order as slots and budget free up (continuous batching: a request that
 * arrives while others are on the GPU starts as soon as one of them finishes
 * and leaves room); their kernels overlap on the device through the slots'
 * streams.  Meshes (moduli, vectors, coarse inverse, tuned stencil shape)
 * stay resident in a pool after their request: the next request of the same
 * size takes an idle one without allocating, and idle meshes are destroyed
 * least recently used first only when a new mesh needs the room. */
int afd_server_create(const afd_server_config* cfg, afd_server** out);

/* Queue one solve of K u = f (one load case) on an nx*ny*nz mesh: E
 * (nelem), f (ndof) and the fixed-DOF mask (ndof) are host arrays copied by
 * the call.  *id_out identifies the request.  AFD_ERR_OOM if the mesh alone
 * exceeds the budget. */
int afd_server_submit(afd_server* s, int nx, int ny, int nz, const double* E, const double* f,
                      const uint8_t* fixed_dof_mask, double rel_tol, int64_t* id_out);

/* afd_server_submit within a session (session > 0; 0 = none): a client's
 * successive solves, e.g. the level-set iterations of one design (Sec. 3.8).
 * The session keeps its own mesh; when a request's loads and fixed-DOF mask
 * equal those of the session's previous solve, the solve starts from that
 * solution (afd_solve's warm start) with the new moduli.  Requests of one
 * session run one at a time, in submission order. */
int afd_server_submit_session(afd_server* s, int64_t session, int nx, int ny, int nz, const double* E,
                              const double* f, const uint8_t* fixed_dof_mask, double rel_tol, int64_t* id_out);

/* End a session: its mesh stays resident as an ordinary pooled mesh. */
int afd_server_end_session(afd_server* s, int64_t session);

/* Meshes resident in the pool (busy or idle) and the bytes they hold. */
int afd_server_resident(afd_server* s, int* meshes, double* bytes);

/* Wait for request id and collect its result: stats, compliance J = f^T u,
 * latency from submit to completion (ms), and the displacement (u_out,
 * nullable host array of ndof).  Returns the solve's status code. */
int afd_server_wait(afd_server* s, int64_t id, afd_stats* stats, double* J_out, double* latency_ms,
                    double* u_out);

/* Stop the workers after the queued requests and free every mesh. */
void afd_server_destroy(afd_server* s);

/* ---- augmented-Lagrangian scalars (Eqs. 3.11, 3.12, 3.18), host only ---- */
typedef struct {
  double mu;     /* multiplier, starts at 100 (Sec. 3.8 step 1) */
  double gamma;  /* penalty, starts at 10 (Sec. 3.8 step 1) */
  double g;      /* last normalised constraint value, g = J/J_all - 1 */
  int k;         /* update counter */
} afd_al_state;

void afd_al_init(afd_al_state* s);
/* One update with the new constraint value: mu <- max(mu + gamma g, 0)
 * (Eq. 3.11), then gamma kept if max(g,0) <= 0.25 max(g_prev,0) else
 * gamma <- max(10 gamma, k^2) (Eq. 3.12). */
void afd_al_update(afd_al_state* s, double g_new);
/* Eq. 3.18 weight: mu + gamma g when positive, else 0. */
double afd_al_weight(const afd_al_state* s);

/* ---- the algorithm of Sec. 3.8 (steps 2-9) with Eq. 3.21's constraints ----
 *
 * min |Omega| subject to up to four constraints, each against its value at
 * the initial design (Sec. 3.8 step 1):
 *   AFD_CON_COMPLIANCE  J <= bound J_0          g = J / (bound J_0) - 1
 *   AFD_CON_STRESS      sigma_PN <= bound s_0   g = sigma_PN / (bound s_0) - 1
 *   AFD_CON_EIGEN       lambda_1 >= bound l_0   g = 1 - lambda_1 / (bound l_0)
 *   AFD_CON_BUCKLING    P >= bound P_0          g = 1 - P / (bound P_0)
 * (J and sigma_PN of load case 0, Eqs. 1.3-1.4 and the p-norm of Eq. 3.3;
 * lambda_1 the fundamental eigenvalue of the lumped-mass modal problem; P the
 * smallest positive buckling factor of load case 0).  Every analysis updates
 * each constraint's (mu, gamma) by Eqs. 3.11-3.12; a hard constraint with
 * g > 0 makes the design infeasible.  Steps: a violated hard constraint sends
 * the run back to the last feasible design with the volume step halved (stop
 * when it falls below dv_min); a feasible analysis whose J moved by at most
 * conv since the previous analysis at the same target lowers the target by the
 * volume step (stop when it would fall below v_min); otherwise the target
 * stays.  Each new design is the level set (Eq. 3.17) of the constraints'
 * fields -- strain energy (compliance), the adjoint T_sigma (stress, Eq. 3.3),
 * T_lambda (Eq. 3.4), Eq. 3.5's field (buckling) -- weighted by their Eq. 3.18
 * weights, optionally with the casting scan (Sec. 3.7), cut at the target
 * volume (Eq. 3.6).  The volume objective's sensitivity is constant and does
 * not change the ranking. */
enum { AFD_CON_COMPLIANCE = 0, AFD_CON_STRESS = 1, AFD_CON_EIGEN = 2, AFD_CON_BUCKLING = 3, AFD_CON_COUNT = 4 };
enum { AFD_STOP_MAX_FEA = 0, AFD_STOP_DV_MIN = 1, AFD_STOP_V_MIN = 2 };

typedef struct {
  double bound[AFD_CON_COUNT];  /* alpha per constraint; a constraint is active when bound > 0 */
  int soft[AFD_CON_COUNT];      /* 1: soft (Sec. 3.6: eigenvalue and buckling only) -- steers, never violated */
  double p;                     /* p-norm exponent of the stress constraint */
  double dv0;                   /* first volume step */
  double dv_min;                /* stop when the halved step falls below it (<= 0: 0.1 dv0) */
  double v_min;                 /* lowest target volume fraction */
  double conv;                  /* relative change of J that counts as converged (e.g. 0.01) */
  int max_fea;                  /* cap on analyses */
  double tol;                   /* relative residual of every solve */
  double eig_tol;               /* relative residual of the eigen analyses */
  double rho;                   /* density of the modal analysis */
  int casting_axis;             /* -1: no casting constraint; else 0/1/2 with casting_parting */
  int casting_parting;
} afd_topology_spec;

/* One analysis of the run.  g[c]/mu[c]/gamma[c] are NaN for inactive c, and
 * so is value[c] except J (value[AFD_CON_COMPLIANCE]), analysed every time. */
typedef struct {
  int fea;                          /* analyses so far (1 = the initial design) */
  double v;                         /* volume fraction of the analysed design */
  double target;                    /* target volume fraction after this analysis' decision */
  double dv;                        /* volume step */
  double value[AFD_CON_COUNT];      /* J, sigma_PN, lambda_1, P */
  double g[AFD_CON_COUNT];          /* normalised constraint values */
  int violated;                     /* a hard constraint has g > 0 */
  int iters;                        /* inner iterations of the static solve */
  double rel_residual;              /* its final relative residual */
  double mu[AFD_CON_COUNT], gamma[AFD_CON_COUNT];  /* AL scalars after this analysis' update */
} afd_topology_record;

typedef struct {
  int stop;                         /* AFD_STOP_* */
  int fea;                          /* analyses run */
  int n_records;                    /* records produced (those beyond hist_cap are not stored) */
  double volume_fraction;           /* of the final (last feasible) design */
  double reference[AFD_CON_COUNT];  /* values at the initial design */
} afd_topology_result;

/* The steps above with caller-supplied analyses (the same loop that
 * afd_constrained_topology runs on a mesh; lets any analysis drive it).  Each
 * callback returns AFD_OK or an error code that ends the run with that code.
 *   analyse: analyse the current design (warm: start the solve from the last
 *            solution), fill value[4] for the active constraints, keep their
 *            fields for the next cut, and report the static solve's stats;
 *   save_feasible / restore_feasible: remember / reinstate the current design;
 *   cut:     make the level set of the kept fields with weight[c] (0 for
 *            inactive c) at volume fraction v_target the current design. */
typedef struct {
  int (*analyse)(void* ctx, int warm, double* value, int* iters, double* rel_residual);
  int (*save_feasible)(void* ctx);
  int (*restore_feasible)(void* ctx);
  int (*cut)(void* ctx, const double* weight, double v_target);
} afd_topology_ops;

int afd_topology_run(const afd_topology_spec* spec, const afd_topology_ops* ops, void* ctx,
                     afd_topology_record* hist, int hist_cap, afd_topology_result* res);

/* The Sec. 3.8 algorithm on a mesh, from its current moduli, loads (one load
 * case) and supports: every analysis, field, snapshot and cut stays on the
 * device (afd_solve warm-started, afd_compliance, afd_pnorm_stress,
 * afd_sensitivity, afd_stress_sensitivity, afd_buckling(+_sensitivity),
 * afd_modal + afd_eigen_sensitivity, the level-set cut).  kept_out (host,
 * N_e bytes) and E_out (host, N_e doubles), nullable, receive the final
 * feasible design; the mesh ends holding the last analysed design. */
int afd_constrained_topology(afd_mesh* m, const afd_topology_spec* spec, afd_topology_record* hist, int hist_cap,
                             afd_topology_result* res, uint8_t* kept_out, double* E_out);

/* The compliance-constrained volume minimisation with fixed volume steps
 * (Sec. 3.8 with the Delta-v control replaced by v_k = 1 - k dv): solve for
 * J_0 (J_all = j_factor J_0), then `steps` times take the level set of the
 * AL-weighted field `kind` (AFD_SENS_*) at v_k, solve it warm-started from the
 * previous solution, and update (mu, gamma) with g = J / J_all - 1.  One
 * record per solve (record 0: the initial design), hist holds steps + 1. */
typedef struct {
  int step;
  double volume_fraction;
  double J, J_over_J0, g;
  int iters;
  double rel_residual;
  double ms;                /* wall time of the step (level set + solve + J) */
  double tau;               /* level-set threshold (NaN for step 0) */
  double al_weight;         /* Eq. 3.18 weight used for the cut (before this step's update) */
  double mu, gamma;         /* AL scalars after the step's update */
  long long kept;           /* elements kept by the cut (N_e for step 0) */
} afd_volmin_record;

int afd_volume_minimisation(afd_mesh* m, int steps, double dv, double j_factor, double tol, int kind,
                            afd_volmin_record* hist, uint8_t* kept_out, double* u_out);

#ifdef __cplusplus
}
#endif
#endif /* AFD_H_ */
