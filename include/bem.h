/*
 * bem.h -- C ABI of the GB300 library for acoustic transmission through a
 * penetrable object with nonconforming interior and exterior surface grids
 * (van 't Wout, "The boundary element method for acoustic transmission with
 * nonconforming grids", arXiv 2206.00708).
 *
 * Plain C: pointers, sizes and status codes only.  Every call returns a
 * bem_status; 0 is success and negative values are errors.  The message of the
 * last error on the calling thread is available from bem_last_error().  No call
 * aborts the process and no device code traps.
 *
 * Ownership: inputs are copied during the call and stay owned by the caller.
 * Handles (contexts, grids, matrices, sparse matrices) belong to the library
 * and are released with their *_destroy call.  Output arrays are allocated by
 * the caller with the sizes stated at each call.
 *
 * Conventions (paper Sec. 2): time dependence exp(-i omega t); Green's function
 * G(x,y) = exp(i k |x-y|) / (4 pi |x-y|); triangles are counter-clockwise seen
 * from outside so that the normal (b-a) x (c-a) points outward; P1 degrees of
 * freedom are the grid vertices, in the caller's vertex order.
 *
 * Complex numbers are two doubles (re, im), interleaved.  Dense matrices are
 * row-major: entry (i, j) (test function i, trial function j) is element
 * i * n_cols + j.
 */
#ifndef BEM_GB300_H
#define BEM_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Exported symbols keep default visibility when the library hides the rest. */
#if defined(__GNUC__)
#define BEM_API __attribute__((visibility("default")))
#else
#define BEM_API
#endif

typedef int32_t bem_status;

#define BEM_OK                    0
#define BEM_E_INVALID_ARG        -1  /* a pointer, size, enum or value is not allowed      */
#define BEM_E_OOM                -2  /* device or host allocation failed                   */
#define BEM_E_NOT_CONVERGED      -3  /* GMRES hit maxiter; outputs hold the last iterate   */
#define BEM_E_NONFINITE          -4  /* a NaN or Inf was found in an input or a result     */
#define BEM_E_TIMEOUT            -5  /* a request exceeded its time limit                  */
#define BEM_E_ADMISSION_REFUSED  -6  /* a request can never fit the server's memory budget */
#define BEM_E_BUSY               -7  /* poll: the request is not finished yet              */
#define BEM_E_CUDA               -8  /* a CUDA runtime call failed                         */
#define BEM_E_INTERNAL           -9  /* an internal consistency check failed               */
#define BEM_E_CANCELLED         -10  /* the request was cancelled                          */

typedef struct { double re, im; } bem_c128;

typedef struct bem_context bem_context;
typedef struct bem_grid    bem_grid;
typedef struct bem_matrix  bem_matrix;
typedef struct bem_sparse  bem_sparse;

/* Operators (paper Sec. 2.1, eq. for V, K, T, D; Sec. 3.1 for M). */
#define BEM_OP_V 0   /* single layer:            int int G phi_j theta_i                 */
#define BEM_OP_K 1   /* double layer:            int int dG/dn(y) phi_j theta_i          */
#define BEM_OP_T 2   /* adjoint double layer:    int int dG/dn(x) phi_j theta_i          */
#define BEM_OP_D 3   /* hypersingular (with the paper's minus sign), Maue's weak form     */

/* Arithmetic of assembly and matvec. */
#define BEM_PREC_FP64   0   /* FP64 operators and vectors; the geometry and kernel values of
                               the assembly in FP64; the quadrature sums of the assembly, the
                               products and the Arnoldi inner products and basis updates in
                               double-float arithmetic (pairs of FP32 values, 48 significant
                               bits) on the FP32 pipe, which on GB300 is 64 times the FP64 rate */
#define BEM_PREC_MIXED  1   /* regular pairs assembled in FP32 into complex64 operators;
                               singular pairs (as in FP64 mode), mass and mortar in FP64;
                               solve: GMRES with an FP32 matvec inside iterative refinement
                               whose residual uses the double-float product, with the
                               double-float Arnoldi of the FP64 mode.                          */

/* Sign variant of the multiple-traces system (paper eq. mtf:discrete). */
#define BEM_MTF_DERIVED 0   /* transfer blocks as derived from Sec. 2.2: returns phi_int, psi_int */
#define BEM_MTF_PRINTED 1   /* transfer blocks with the signs printed in eq. mtf:discrete      */

/* Boundary integral formulation of bem_solve_transmission (bem_solve_opts.formulation) */
#define BEM_FORM_MTF        0  /* multiple-traces system of eq. mtf:discrete: 4 unknowns      */
#define BEM_FORM_PMCHWT     1  /* exterior PMCHWT (eq. pmchwt:ext, discretised by eq.
                                  pmchwt:discrete): 2 unknowns on the exterior grid          */
#define BEM_FORM_MULLER     2  /* exterior Mueller (eq. muller:ext)                          */
#define BEM_FORM_PMCHWT_INT 3  /* interior PMCHWT (eq. pmchwt:int): 2 unknowns on the
                                  interior grid                                              */
#define BEM_FORM_MULLER_INT 4  /* interior Mueller (eq. muller:int)                          */
#define BEM_FORM_HC_EXT_NEU 5  /* exterior high-contrast Neumann (eq. highcontrast:ext:neu)    */
#define BEM_FORM_HC_EXT_DIR 6  /* exterior high-contrast Dirichlet (eq. highcontrast:ext:dir)  */
#define BEM_FORM_HC_INT_NEU 7  /* interior high-contrast Neumann (eq. highcontrast:int:neu)    */
#define BEM_FORM_HC_INT_DIR 8  /* interior high-contrast Dirichlet (eq. highcontrast:int:dir)  */

/* Thread-local message of the last failing call (never NULL). */
BEM_API const char* bem_last_error(void);

/* Library version string. */
BEM_API const char* bem_version(void);

/* ---------------------------------------------------------------- autotuner
 * Launch shapes of the iteration's kernels (no counterpart in the paper, which runs
 * on CPUs).  bem_autotune times the candidates on complex64 operators of the two
 * grids' sizes (seeded random values) and on the grids' mass matrices, and keeps the
 * fastest in a process-wide table keyed by (kernel, width, ceil(log2(rows))):
 *   "cheb"    Chebyshev mass-inverse steps, width 1 and 8 columns: block 64/128/256;
 *   "gemm_tc" tensor-core product of min(n_rhs, 64) columns (only if n_rhs > 8),
 *             width = columns padded to 8: variant = K splits (1 or 2).
 * Solves of any later call look their shapes up there (built-in defaults where no
 * entry matches); results do not depend on the shapes beyond rounding.  Takes a
 * few seconds at 10^4 vertices per grid and needs the same device memory as the
 * operators of a mixed-precision solve.  bem_tune_get returns block = 0 when no
 * entry matches (ms: the measured time, may be NULL).  bem_tune_save writes the
 * table as JSON (format "bem-tune-1"); bem_tune_load merges such a file into it
 * (entries with the same key are replaced; malformed files: BEM_E_INVALID_ARG,
 * nothing merged).  The table functions need no GPU.  If the environment variable
 * BEM_TUNE_FILE names such a file when the library is loaded, it is merged then. */
BEM_API bem_status bem_autotune(bem_context* ctx, const bem_grid* ext, const bem_grid* intr, int32_t n_rhs);
BEM_API bem_status bem_tune_get(const char* kernel, int32_t width, int64_t rows, int32_t* block,
                                int32_t* variant, double* ms);
BEM_API int32_t    bem_tune_count(void);
BEM_API void       bem_tune_clear(void);
BEM_API bem_status bem_tune_save(const char* path);
BEM_API bem_status bem_tune_load(const char* path);

/* ---------------------------------------------------------------- context
 * A context binds a CUDA device and a stream.  `stream` is a cudaStream_t
 * passed as void*; NULL makes the context create and own a non-blocking stream.
 * A context is not thread-safe: one caller thread at a time.                 */
BEM_API bem_status bem_context_create(int device, void* stream, bem_context** out);
BEM_API bem_status bem_context_destroy(bem_context* ctx);
/* Block until all work queued on the context's stream has finished. */
BEM_API bem_status bem_context_synchronize(bem_context* ctx);
/* exclusive = 1: the caller guarantees that this context's solves never overlap with
 * other solves on the device, and each mass-matrix inverse then runs as one
 * cooperative launch whose blocks synchronise through a grid barrier (bounded waits).
 * exclusive = 0 (default): one launch per Chebyshev step, replayed as CUDA graphs when
 * cuda_graphs is on (on GB300 this measured faster: a barrier step costs about what a
 * graph node does, and the graph form keeps more parallel work in flight).  The results
 * do not depend on it. */
BEM_API bem_status bem_context_set_exclusive(bem_context* ctx, int exclusive);

/* ---------------------------------------------------------------- grids
 * Grid intake (paper Sec. 2.4 and Sec. 3: a conforming triangular surface grid).
 *   xyz  [nv*3] float64 vertex coordinates; tri [nt*3] int32 vertex indices,
 *   counter-clockwise seen from outside.  With on_device = 1 both pointers are
 *   device pointers on the context's device; otherwise host pointers.
 * Errors: BEM_E_INVALID_ARG for nv < 3, nt < 1, an index outside [0, nv), a
 * triangle with a repeated vertex or zero area; BEM_E_NONFINITE for a NaN/Inf
 * coordinate.                                                                 */
BEM_API bem_status bem_grid_create(bem_context* ctx, const double* xyz, int64_t nv,
                           const int32_t* tri, int64_t nt, int on_device, bem_grid** out);
BEM_API bem_status bem_grid_destroy(bem_grid* g);
BEM_API int64_t    bem_grid_num_vertices(const bem_grid* g);
BEM_API int64_t    bem_grid_num_triangles(const bem_grid* g);

/* ---------------------------------------------------------------- assembly
 * Dense Galerkin matrix of operator `op` (BEM_OP_*) for wavenumber k on one P1
 * space (paper Sec. 2.1 and Sec. 2.4; quadrature of Sec. 5.1: a 6-point
 * degree-4 triangle rule per triangle for pairs without a common vertex,
 * Sauter-Schwab transformations with n_singular Gauss points per axis for
 * coincident, edge- and vertex-adjacent pairs).  test must equal trial (both
 * operators of the method act within one grid).  n_singular in [1, 16].
 * The result is a library-owned device matrix of nv x nv entries: complex128
 * for BEM_PREC_FP64, complex64 (two floats) for BEM_PREC_MIXED.              */
BEM_API bem_status bem_assemble(bem_context* ctx, int op, bem_c128 k, const bem_grid* test,
                        const bem_grid* trial, int precision, int n_singular,
                        bem_matrix** out);
BEM_API bem_status bem_matrix_destroy(bem_matrix* m);
/* Bytes per entry of a matrix: 16 (complex128) or 8 (complex64). */
BEM_API int        bem_matrix_entry_bytes(const bem_matrix* m);
/* Copy a matrix out, row-major, in its own entry type.  dst_bytes must be at least
 * rows*cols*entry_bytes.  on_device = 1: dst is a device pointer (copy on the stream,
 * asynchronous); 0: dst is host memory (the call waits).                      */
BEM_API bem_status bem_matrix_copy_out(bem_context* ctx, const bem_matrix* m, void* dst,
                               int64_t dst_bytes, int on_device);
BEM_API bem_status bem_matrix_shape(const bem_matrix* m, int64_t* rows, int64_t* cols);

/* ---------------------------------------------------------------- sparse
 * Mass matrix of one grid, M_ij = <phi_j, theta_i> (paper Sec. 3.1).         */
BEM_API bem_status bem_mass(bem_context* ctx, const bem_grid* g, bem_sparse** out);
/* Mortar matrix P_ab (paper Sec. 3.1): entry (i, j) is the L2 product of test
 * function i on grid a with basis function j on grid b over the common surface.
 * The common surface of two different polyhedra is read through central
 * projection from `center` ([3] host doubles; NULL means the origin): each
 * triangle of b is projected onto the plane of each triangle of a along rays from
 * the centre, and on that plane basis j is the linear function of the projected
 * triangle.  For coplanar grids this is the plain mortar matrix; for identical
 * grids it is the mass matrix.  Both surfaces must be star-shaped about center.
 * P_ba = P_ab^T (Sec. 5.4).                                                   */
BEM_API bem_status bem_projection(bem_context* ctx, const bem_grid* a, const bem_grid* b,
                          const double* center, bem_sparse** out);
/* bem_projection without any device allocation.  The paper has no counterpart:
 * this entry point exists for callers that must not have a library allocate device
 * memory while they run -- a host program that owns all HBM through its own budgeted
 * pool, or a latency-critical loop that cannot pay for cudaMalloc and its implicit
 * synchronisation.  Its working memory is one fixed ~9.9 MB array in device global
 * memory that every GPU loading the library holds until the process exits.
 *   a, b:        validated grid handles, at most 32768 triangles each (else
 *                BEM_E_INVALID_ARG); center as in bem_projection.
 *   row, col, val: caller-owned DEVICE arrays of `capacity` entries; on return *nnz
 *                holds the number of COO entries (9 per candidate pair, repeated
 *                (row, col) pairs add up).  A capacity below *nnz, or more than
 *                1048576 candidate pairs, returns BEM_E_INVALID_ARG and writes no
 *                entries.  The entries are written asynchronously on the context's
 *                stream: synchronise before reading them.
 * Part-way through, the call waits for the context's stream: it reads the number of
 * candidate pairs back to the host before it launches the clipping kernel.
 * The first call on a device looks up the array's device address (once per device);
 * make that first call before any stream capture.  All calls share the one array and
 * it keeps the last call's contents (the call clears what must start at zero), so
 * calls whose GPU work overlaps -- from several threads, or on several streams of
 * one device -- race; serialise them.                                          */
BEM_API bem_status bem_projection_noalloc(bem_context* ctx, const bem_grid* a, const bem_grid* b,
                                          const double* center, int32_t* row, int32_t* col,
                                          double* val, int64_t capacity, int64_t* nnz);
BEM_API bem_status bem_sparse_destroy(bem_sparse* s);
/* Coordinate (COO) form.  Entries may repeat a (row, col) pair; repeated entries
 * add up.  Query nnz first, then copy into host arrays of at least nnz items.  */
BEM_API bem_status bem_sparse_info(const bem_sparse* s, int64_t* rows, int64_t* cols, int64_t* nnz);
BEM_API bem_status bem_sparse_copy_out(bem_context* ctx, const bem_sparse* s, int32_t* row,
                               int32_t* col, double* val, int64_t capacity);

/* ---------------------------------------------------------------- solve
 * Incident field (paper Sec. 2: u_inc in the exterior medium, data f_j = <u_inc, theta_j>
 * and g_j = <du_inc/dn, theta_j> on the exterior grid, the right-hand side of
 * eq. mtf:discrete), n_rhs of them, of one kind:
 *   BEM_INC_PLANE_WAVE (0, the default of a zeroed struct): amp_r exp(i k_ext x . d_r)
 *     (eq. planewave); dirs [n_rhs*3] unit vectors.
 *   BEM_INC_POINT_SOURCE: amp_r exp(i k_ext |x - s_r|) / (4 pi |x - s_r|), the field of
 *     a monopole at s_r in the exterior medium; sources [n_rhs*3] positions, which the
 *     caller places in the exterior medium and off the surface (not checked).
 *   BEM_INC_USER_TRACES: the weak-form data themselves, f and g [n_rhs*N_ext]
 *     (right-hand side r at offset r*N_ext), on the host, or on the device when the
 *     solve's on_device flag is set.  Any incident field, or any data of the form
 *     (<a, theta_j>, <b, theta_j>), enters this way.
 * amps [n_rhs] (NULL = all 1) scale plane waves and point sources.
 * bem_solve_screen uses g only (the Neumann data of its one grid).  */
#define BEM_INC_PLANE_WAVE   0
#define BEM_INC_POINT_SOURCE 1
#define BEM_INC_USER_TRACES  2
typedef struct {
    int32_t         n_rhs;
    const double*   dirs;     /* BEM_INC_PLANE_WAVE: [n_rhs*3] unit directions              */
    const bem_c128* amps;     /* plane waves and point sources: [n_rhs] or NULL             */
    int32_t         kind;     /* BEM_INC_*                                                   */
    const double*   sources;  /* BEM_INC_POINT_SOURCE: [n_rhs*3] source positions           */
    const bem_c128* f;        /* BEM_INC_USER_TRACES: [n_rhs*N_ext] <u_inc, theta_j>         */
    const bem_c128* g;        /* BEM_INC_USER_TRACES: [n_rhs*N_ext] <du_inc/dn, theta_j>     */
} bem_incident;

typedef struct {
    double  gmres_tol;        /* relative residual of the preconditioned system (default 1e-8)  */
    int32_t gmres_maxiter;    /* default 2000; unrestarted (paper Sec. 5.1)                       */
    int32_t precision;        /* BEM_PREC_*                                                       */
    int32_t n_singular;       /* Gauss points per axis of singular pairs (default 4)             */
    int32_t mtf_variant;      /* BEM_MTF_DERIVED (default) or BEM_MTF_PRINTED                     */
    double  center[3];        /* projection centre for the mortar (default origin)               */
    double  ir_inner_tol;     /* BEM_PREC_MIXED: relative residual reduction asked of each inner
                                 GMRES solve, or the reduction that brings the outer residual to
                                 half the target where that is less.  0 (default)
                                 chooses: 1e-5 where the inner products are FP32 or tensor-core
                                 products throughout (batches, dd_switch = 1: the true inner
                                 residual stalls near their 1e-7 accuracy, so a second short inner
                                 solve on the FP64 residual is cheaper than running the first one
                                 on), 1e-8 where a double-float phase reaches the target in one
                                 inner solve (dd_switch < 1); any value in (0, 1) is used as given */
    int32_t batch_columns;    /* right-hand sides solved together (one Krylov process each, the
                                 operator read once per iteration for all): 0 = default (64 with
                                 BEM_PREC_MIXED and tensor cores, else 8); 1..128                   */
    int32_t tensor_cores;     /* BEM_PREC_MIXED batches of more than 8 right-hand sides: 2 (default)
                                 = products on the tcgen05 tensor cores with an FP16 two-term
                                 split of both operands (pre-tiled operator copy read by TMA bulk
                                 copies, FP32 accumulation), 3 = the same with a BF16 two-term
                                 split (8 + 8 bits: products to ~2e-5, more refinement), 1 =
                                 tensor cores with a TF32 three-term split, 0 = FP32 CUDA cores in
                                 groups of 8 columns                                               */
    int32_t formulation;      /* BEM_FORM_* (default BEM_FORM_MTF); the single-trace and
                                 high-contrast systems are available in bem_solve_transmission
                                 only (bem_solve_many and the server solve the multiple-traces
                                 system); high-contrast products always use the CUDA cores         */
    double  dd_switch;        /* BEM_PREC_MIXED, one right-hand side: the inner GMRES products run
                                 in double-float arithmetic while the inner residual is above
                                 dd_switch of its right-hand side, in FP32 below (default 1: FP32
                                 throughout, with a complex64 Krylov basis and two inner solves;
                                 0: double-float throughout; e.g. 1e-3: double-float to 1e-3, one
                                 inner solve).  bem_solve_many: a lockstep step runs in
                                 double-float while some running instance's residual estimate is
                                 above it.  Every setting refines to the same FP64 residual        */
    int32_t cuda_graphs;      /* 1 (default): the fixed launch sequences of each iteration (the
                                 Chebyshev mass inverses) are captured once per solve and replayed
                                 as CUDA graphs; 0: every kernel is launched on its own.  Results
                                 agree to the run-to-run rounding of the assembly either way.      */
} bem_solve_opts;

typedef struct {
    int32_t iterations;       /* GMRES iterations, summed over right-hand sides (and inner solves) */
    int32_t converged;        /* 1 if every right-hand side met gmres_tol                        */
    double  residual;         /* final relative preconditioned residual (max over RHS)           */
    double  t_assembly_ms;    /* device time of operator assembly (both grids)                   */
    double  t_mortar_ms;      /* device time of mass + mortar matrices                           */
    double  t_solve_ms;       /* device time of right-hand sides + GMRES                         */
    int32_t mtf_variant;      /* sign variant used                                               */
    int32_t outer_iterations; /* refinement steps (1 for BEM_PREC_FP64)                           */
} bem_solve_report;

/* Fill opts with the defaults stated above. */
BEM_API void bem_solve_opts_default(bem_solve_opts* opts);

/* Solve the mass-preconditioned multiple-traces system (paper eq. mtf:discrete
 * with the left preconditioner of Sec. 3.3) for plane-wave incidence from the
 * exterior, on exterior grid `ext` (wavenumber k_ext) and interior grid `intr`
 * (wavenumber k_int), density ratio rho_int / rho_ext.
 * Outputs (caller-owned, host memory unless opts-independent flag on_device=1):
 *   v_ext, w_ext [n_rhs * N_ext]: P1 coefficients of phi_ext = -gamma_D^+ p and
 *                                 psi_ext = -gamma_N^+ p (paper Sec. 2.2);
 *   v_int, w_int [n_rhs * N_int]: phi_int = gamma_D^- p and psi_int = gamma_N^- p
 *                                 (negated for BEM_MTF_PRINTED).
 * Right-hand side r occupies [r*N, (r+1)*N).  rep may be NULL.
 * BEM_E_NOT_CONVERGED still writes the last iterate and the report.
 *
 * Single-trace formulations (paper Sec. 2.2, discretised as eq. pmchwt:discrete;
 * r = rho_i/rho_e, A_g = [[-K_g, V_g], [D_g, T_g]] on grid g):
 *   BEM_FORM_PMCHWT      (A_e + hat_e(A_i^r)) [v_e; w_e] = [-f; -g]
 *   BEM_FORM_MULLER      (M_e + A_e - hat_e(A_i^r)) [v_e; w_e] = [-f; -g]
 *   BEM_FORM_PMCHWT_INT  (A_i + hat_i(A_e^r)) [v_i; w_i] = [P_ie M_e^-1 f; r P_ie M_e^-1 g]
 *   BEM_FORM_MULLER_INT  (M_i + hat_i(A_e^r) - A_i) [v_i; w_i] = (the same)
 * with A_i^r = [[-K_i, r V_i], [D_i / r, T_i]], A_e^r = [[-K_e, V_e / r], [r D_e, T_e]],
 * hat_e(X) = P_ei M_i^-1 X M_i^-1 P_ie and hat_i(X) = P_ie M_e^-1 X M_e^-1 P_ei (the
 * Mueller identity is the mass matrix: the paper's exact projection of the identity),
 * left-preconditioned by the mass inverse of the unknowns' grid.  The hatted operators
 * are never formed: every product applies P, M^-1, the other grid's operators, M^-1
 * and P in turn.  The other grid's potentials follow from the transmission conditions
 * tested on it: v_i = -M_i^-1 P_ie v_e, w_i = -r M_i^-1 P_ie w_e (exterior variants),
 * v_e = -M_e^-1 P_ei v_i, w_e = -(1/r) M_e^-1 P_ei w_i (interior variants), so the
 * four outputs keep the meaning stated above.  mtf_variant is ignored.
 *
 * High-contrast formulations (paper Sec. 2.3), discretised the same way (a mass
 * inverse between two operators and on a data vector an operator acts on; X^ the
 * other grid's operator mapped as above):
 *   BEM_FORM_HC_EXT_NEU  unknowns a = gamma_N^+ p and mu (u_s = V mu), exterior grid:
 *     [M_e/2 - T^_i, -(1/r) D^_i M_e^-1 V_e; M_e, M_e/2 - T_e] = [(1/r) D^_i M_e^-1 f; g]
 *   BEM_FORM_HC_EXT_DIR  unknowns nu (u_s = -K nu) and b = gamma_D^+ p:
 *     [M_e/2 + K_e, M_e; -r V^_i M_e^-1 D_e, M_e/2 + K^_i] = [f; r V^_i M_e^-1 g]
 *   BEM_FORM_HC_INT_NEU  unknowns a = gamma_N^- p and mu (u_int = V mu), interior grid:
 *     [M_i/2 + T^_e, r D^_e M_i^-1 V_i; -M_i, M_i/2 + T_i]
 *       = [r P_ie M_e^-1 (D_e M_e^-1 f + g/2 + T_e M_e^-1 g); 0]
 *   BEM_FORM_HC_INT_DIR  unknowns nu (u_int = -K nu) and b = gamma_D^- p:
 *     [M_i/2 - K_i, -M_i; (1/r) V^_e M_i^-1 D_i, M_i/2 - K^_e]
 *       = [0; P_ie M_e^-1 (V_e M_e^-1 g + f/2 - K_e M_e^-1 f)]
 * left-preconditioned by the mass inverse of the unknowns' grid.  The unknowns' grid
 * traces follow from the representation (e.g. v_e = -M_e^-1 (f + V_e mu)), the other
 * grid's from the transmission conditions; the four outputs keep their meaning.  Their
 * products run on the CUDA cores (tensor_cores is ignored).                   */
BEM_API bem_status bem_solve_transmission(bem_context* ctx, const bem_grid* ext, const bem_grid* intr,
                                  bem_c128 k_int, bem_c128 k_ext, double rho_int_over_rho_ext,
                                  const bem_incident* inc, const bem_solve_opts* opts,
                                  bem_c128* v_ext, bem_c128* w_ext,
                                  bem_c128* v_int, bem_c128* w_int,
                                  int on_device, bem_solve_report* rep);

/* Neumann screen (paper Sec. 4.2, eq. neumannscreen; the benchmark of Sec. 5.7): a
 * sound-hard open surface `screen` (a grid with a boundary: nodes on edges of one
 * triangle), u_s = K phi with phi the jump of the total field across the screen, and
 *     D phi = gamma_N u_inc   on the screen,
 * discretised with the P1 functions of the screen's interior nodes (phi = 0 on its
 * boundary), data g_i = <i k (d . n) exp(i k x . d), theta_i> (n: the triangles' normal),
 * and solved by unrestarted GMRES on the left-preconditioned system
 *   BEM_SCREEN_MASS  M^-1 D phi = M^-1 g,
 *   BEM_SCREEN_OO    M^-1 V^_c M^-1 D phi = M^-1 V^_c M^-1 g  (opposite-order),
 *                    V^_c = P_cs^T M_c^-1 V_c M_c^-1 P_cs: the single layer on the grid
 *                    `coarse` (coplanar, all its nodes) through the mortar matrix,
 * M the screen's mass matrix on its interior nodes.  With a coarse grid V^_c has rank
 * at most its node count, so the OO iterate solves the preconditioned system, not
 * D phi = g itself; coarse = screen gives the conforming preconditioner (same solution
 * as BEM_SCREEN_MASS).  phi: [n_rhs * N_screen] (host, or device with on_device = 1),
 * zero at boundary nodes.  opts: gmres_tol, gmres_maxiter, precision (FP64 or mixed:
 * FP32 assembly, complex64 storage, FP64 refinement), n_singular, batch_columns (1..8,
 * default 8), cuda_graphs; the others are ignored.  rep as for bem_solve_transmission. */
#define BEM_SCREEN_MASS 0
#define BEM_SCREEN_OO   1
BEM_API bem_status bem_solve_screen(bem_context* ctx, const bem_grid* screen, const bem_grid* coarse,
                                    bem_c128 k, const bem_incident* inc, const bem_solve_opts* opts,
                                    int32_t precond, bem_c128* phi, int on_device, bem_solve_report* rep);

/* Field of P1 densities at points off the surface (paper Sec. 2.1, eq.
 * representation):
 *     u(x) = [V psi](x) - [K phi](x)
 *          = int G(x,y) psi(y) dy - int dG/dn(y)(x,y) phi(y) dy,   G = exp(ik|x-y|) / (4 pi |x-y|),
 * integrated with the 6-point degree-4 rule of the regular Galerkin pairs on each
 * triangle of g (points within about one triangle size of the surface get only that
 * rule's accuracy).  With the interior grid, k_int and (v_int, w_int) of
 * bem_solve_transmission this is the interior field; with the exterior grid, k_ext and
 * (v_ext, w_ext) it is the scattered field (add the incident wave for the total field).
 * phi, psi: [N] vertex values (either may be NULL: its term is left out, not both);
 * points: [npts][3]; u: [npts].  All host memory, or all device memory with
 * on_device = 1.  FP64; the result does not depend on scheduling.              */
BEM_API bem_status bem_field(bem_context* ctx, const bem_grid* g, bem_c128 k, const bem_c128* phi,
                             const bem_c128* psi, const double* points, int64_t npts, bem_c128* u,
                             int on_device);

/* Many independent transmission problems of uneven sizes in one call (the batching
 * pattern for uneven instances; no counterpart in the paper, which solves one
 * problem at a time).  Each instance has its own grids, wavenumbers, density ratio
 * and one plane wave; the mixed-precision solve of eq. mtf:discrete runs for all of
 * them together: the regular-pair assembly of all grids is one persistent launch,
 * and every step of the lockstep GMRES / iterative refinement is one launch for all
 * instances, each with its own Krylov process and stopping test, so each result is
 * the one the instance gets alone (up to FP32 rounding of its assembly).
 * opts: as for bem_solve_transmission; precision must be BEM_PREC_MIXED
 * (batch_columns and tensor_cores do not apply).  Outputs per instance as in
 * bem_solve_transmission (host memory unless on_device = 1); reports [count] may be
 * NULL.  Grids may be shared between instances.                                   */
typedef struct {
    const bem_grid* ext;           /* exterior grid                                        */
    const bem_grid* intr;          /* interior grid                                        */
    bem_c128 k_ext, k_int;         /* wavenumbers                                          */
    double rho_int_over_rho_ext;   /* density ratio (> 0)                                  */
    double dir[3];                 /* unit propagation direction of the plane wave         */
    bem_c128 amp;                  /* its amplitude                                        */
    bem_c128 *v_ext, *w_ext;       /* outputs [N_ext]                                      */
    bem_c128 *v_int, *w_int;       /* outputs [N_int]                                      */
} bem_instance;

BEM_API bem_status bem_solve_many(bem_context* ctx, int32_t count, const bem_instance* instances,
                                  const bem_solve_opts* opts, int on_device, bem_solve_report* reports);

/* ---------------------------------------------------------------- serving
 * A request server for streams of transmission solves (continuous batching):
 * submitted requests wait in a FIFO queue; up to max_inflight of them run at once,
 * each on its own CUDA stream, so the GPU work of different requests overlaps.  A
 * request is admitted when a slot is free and its device working set (operators,
 * Krylov basis, workspaces; an upper estimate) fits in what is left of the HBM
 * budget; requests that could never fit are refused at submission.  The head of
 * the queue is never overtaken, so no request starves.  The server is thread-safe.
 * Lockstep groups: when a slot takes a mixed-precision request with one or two plane
 * waves whose operators are small (complex64 tiles of both grids at most 64 MiB, so
 * that a group's operators stay in L2), it also takes requests of the same kind from
 * the first 4 * group_max
 * places of the queue, up to group_max requests, 64 plane waves, 64 MiB of operators
 * and the memory budget; the requests it passes over keep their order and their room
 * in the budget, so the next free slot takes them.  The group's waves are solved
 * together through bem_solve_many's lockstep path: every GMRES step is one launch
 * for the whole group, each wave keeping its own Krylov process and stopping test;
 * cancellation and deadlines stop a member alone.  Members finish together, when
 * the group's last wave converges.  Larger, FP64 and many-wave requests run alone,
 * their waves batched as columns of one product (faster than one lockstep instance
 * per wave, which reads the operators once per wave).
 * dry_run = 1 runs the scheduler without any GPU work (each request "runs" for
 * dry_run_us_per_unknown microseconds per unknown and wave, a group for the longest
 * of its members, and returns zeros): this is the host-side mode used to test
 * admission, ordering, grouping, timeouts and cancellation.                      */
typedef struct bem_server bem_server;

typedef struct {
    int32_t device;                 /* CUDA device (ignored in dry-run mode)                 */
    int32_t max_inflight;           /* concurrent requests, one stream each (default 4)      */
    int64_t hbm_budget_bytes;       /* 0: 80% of the free device memory at creation          */
    int32_t precision;              /* default precision of requests (BEM_PREC_MIXED)        */
    int32_t gmres_maxiter;          /* default 2000                                          */
    double  gmres_tol;              /* default 1e-8                                          */
    int32_t dry_run;                /* 1: no GPU work (scheduler tests)                      */
    int32_t group_max;              /* requests solved together in one lockstep group
                                       (0: default 8; 1: every request alone), see below     */
    double  dry_run_us_per_unknown; /* dry-run service time per unknown (default 1 us)       */
} bem_server_opts;

typedef struct {
    const double*  xyz_ext; int64_t nv_ext; const int32_t* tri_ext; int64_t nt_ext;  /* host */
    const double*  xyz_int; int64_t nv_int; const int32_t* tri_int; int64_t nt_int;  /* host */
    bem_c128 k_ext, k_int;
    double   rho_int_over_rho_ext;
    int32_t  n_rhs;
    int32_t  precision;             /* BEM_PREC_*, or -1 for the server default              */
    const double*   dirs;           /* [n_rhs*3] unit vectors (host)                         */
    const bem_c128* amps;           /* [n_rhs] or NULL                                       */
    double   timeout_ms;            /* 0: none; counted from submission                      */
} bem_request;

typedef struct {
    int32_t status;                 /* outcome: BEM_OK, BEM_E_NOT_CONVERGED, BEM_E_TIMEOUT,
                                       BEM_E_CANCELLED, BEM_E_CUDA, ...                      */
    int32_t iterations;
    double  residual;
    double  queue_ms, run_ms, total_ms;  /* submit->start, start->finish, submit->finish     */
    int64_t nv_ext, nv_int;
    int32_t n_rhs, precision;
    int64_t bytes_reserved;         /* admission estimate charged to the budget              */
    int32_t group_size;             /* requests of the lockstep group it ran in (1: alone)   */
    int32_t group_waves;            /* plane waves of that group                             */
} bem_result;

typedef struct {
    int64_t submitted, completed, refused, cancelled, timed_out, failed;
    int64_t queued, running;
    int64_t hbm_budget_bytes, hbm_reserved_bytes, hbm_high_water_bytes;
    int64_t groups, grouped;        /* lockstep groups of two or more requests; their requests */
} bem_serve_stats;

BEM_API void       bem_serve_opts_default(bem_server_opts* opts);
BEM_API bem_status bem_serve_create(const bem_server_opts* opts, bem_server** out);
/* Cancels queued requests, stops running ones at their next iteration, joins the
 * workers and frees everything (unpolled results included). */
BEM_API bem_status bem_serve_destroy(bem_server* srv);
/* Copies the request (all host arrays) and queues it.  Returns
 * BEM_E_ADMISSION_REFUSED (no ticket) if its working set exceeds the whole budget,
 * BEM_E_INVALID_ARG for malformed input. */
BEM_API bem_status bem_serve_submit(bem_server* srv, const bem_request* req, uint64_t* ticket);
/* BEM_E_BUSY while the request is queued or running.  Once it has finished: fills
 * *info (may be NULL), copies the traces into the non-NULL host arrays
 * ([n_rhs*nv_ext] for v_ext, w_ext; [n_rhs*nv_int] for v_int, w_int), releases the
 * request and returns BEM_OK; info->status holds the request's own outcome.
 * Unknown or already released tickets return BEM_E_INVALID_ARG. */
BEM_API bem_status bem_serve_poll(bem_server* srv, uint64_t ticket, bem_result* info,
                                  bem_c128* v_ext, bem_c128* w_ext, bem_c128* v_int, bem_c128* w_int);
/* Blocks until the request has finished or timeout_ms elapses (BEM_E_BUSY). */
BEM_API bem_status bem_serve_wait(bem_server* srv, uint64_t ticket, double timeout_ms);
/* Queued: removed at once; running: stops at its next GMRES iteration.  Either way
 * its outcome becomes BEM_E_CANCELLED (unless it had already finished). */
BEM_API bem_status bem_serve_cancel(bem_server* srv, uint64_t ticket);
BEM_API bem_status bem_serve_get_stats(bem_server* srv, bem_serve_stats* st);

/* ---------------------------------------------------------------- diagnostics
 * Accounting, self-tests and per-kernel timing used by the tests and the benchmark
 * (no counterpart in the paper). */

/* Number of CUDA kernels the library has launched since it was loaded (all
 * contexts and threads; a monotone counter for profiling and accounting). */
BEM_API uint64_t bem_launch_count(void);

/* Accuracy self-tests of device arithmetic written for this library (no
 * counterpart in the paper).  which = 0: largest absolute difference between the
 * FP32 assembly kernel's sin/cos (Cody-Waite reduction + Taylor series) and CUDA's
 * sincosf on 2^20 evenly spaced arguments in [-64, 64].  which = 1: relative L2
 * difference between the tensor-core multi-column MTF product (TF32 three-term
 * split) and the FP32 CUDA-core product on seeded random complex64 blocks
 * (N_ext = 300, N_int = 170, 24 columns).  which = 2: the same with 8 columns.
 * which = 3: the bounded wait of the grid barrier that the fused mass inverse uses:
 * two cooperative blocks whose barrier can never complete must each give up after
 * about a second and flag it; result = 1000 * flag + elapsed seconds (expected
 * 1000 + ~1).  which = 4..9: relative L2 difference between the tiled operator
 * product (symmetry-packed V, D; K applied as K and K^T) and an FP64 product with
 * dense copies of the same seeded random operators (two grids of 300 and 170
 * vertices): 4 FP32 on complex64, 1 column; 5 the same, 5 columns; 6 double-float on
 * complex64, 1 column; 7 the same, 3 columns; 8 double-float on complex128, 1 column;
 * 9 the same, 8 columns.  which = 10, 11: as 1, for the TMA-fed tensor-core product
 * with the FP16 two-term split of both operands, 24 and 128 columns; 12: the same
 * with the BF16 two-term split, 24 columns. */
BEM_API bem_status bem_selftest(bem_context* ctx, int which, double* result);

/* Per-kernel device timing.  While enabled, each launch of the library is
 * bracketed by CUDA events on its own stream; totals accumulate per kernel
 * name.  bem_profile_count() returns the number of kernel names seen and
 * bem_profile_get(i, ...) the i-th name (NUL-terminated, truncated to name_len),
 * its summed device time in ms and its number of launches.  Collecting waits
 * for the recorded events.  Not meant to be toggled while a solve is running. */
BEM_API void       bem_profile_enable(int on);
/* Restrict the timing to kernels whose names start with one of the comma-separated
 * prefixes (NULL or "": every kernel), so that a few kernels can be timed inside a
 * measured region without bracketing every launch. */
BEM_API void       bem_profile_select(const char* prefixes);
BEM_API void       bem_profile_reset(void);
BEM_API int        bem_profile_count(void);
BEM_API bem_status bem_profile_get(int index, char* name, int name_len, double* total_ms,
                                   int64_t* launches);

#ifdef __cplusplus
}
#endif

#endif /* BEM_GB300_H */
