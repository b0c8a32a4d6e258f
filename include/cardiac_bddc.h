/*
 * cardiac_bddc.h -- C ABI of the GB300 Newton-GMRES-BDDC tangent solver.
 *
 * The library solves the cardiac mechanics problem of Barnafi, Pavarino &
 * Scacchi, "A comparative study of scalable multilevel preconditioners for
 * cardiac mechanics" (arXiv 2208.06191):
 *   - Section 2: Guccione passive law, active stress gamma (Ff)(x)f/|Ff|,
 *     follower endocardial pressure -p J F^{-T} N (Eq. bc endo), weak form
 *     (Eq. mechanics time discrete; the inertia term and the generalized
 *     Robin condition through fem_set_time_state), Newton on the tangent
 *     problem (Eq. tangent problem);
 *   - Section 3.2: two-level and multilevel BDDC with vertex /
 *     edge-average / face-average primal constraints, counting or deluxe
 *     scaling, as preconditioner of GMRES; Section 4: rigid motions as
 *     primal constraints; a Petrov (left and right basis) coarse space for
 *     the nonsymmetric tangent.
 *
 * Conventions shared by every call:
 *   - Return value: 0 (CBDDC_OK) or one of the CBDDC_E* codes below; the
 *     message of the last failure on the calling thread is returned by
 *     cbddc_last_error().  No call aborts or throws across this boundary.
 *   - "dev" pointers are CUDA device memory of the current device and are
 *     borrowed (the caller keeps ownership); "host" pointers are ordinary
 *     host memory, copied during the call unless stated otherwise.
 *   - Vectors cover the free degrees of freedom only: nodes in increasing
 *     id with Dirichlet nodes removed, three interleaved components
 *     (x, y, z) per node (block size 3, Section 4).  n_free = 3 * number
 *     of free nodes.
 *   - Calls are ordered on the given stream and asynchronous unless stated
 *     otherwise.  A handle must not be used from two streams at once.
 *   - All floating point arguments are FP64.
 */
#ifndef CARDIAC_BDDC_H
#define CARDIAC_BDDC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define CBDDC_API __attribute__((visibility("default")))
#else
#define CBDDC_API
#endif

/* cudaStream_t without including the CUDA headers (same type). */
typedef struct CUstream_st* cbddc_stream_t;

enum {
  CBDDC_OK = 0,
  CBDDC_EINVAL = 1,    /* bad argument or unsupported input               */
  CBDDC_ECUDA = 2,     /* a CUDA runtime call failed                      */
  CBDDC_EPIVOT = 3,    /* zero (tiny) pivot in a local factorisation      */
  CBDDC_EINVERTED = 4, /* J = det F <= 0 at a quadrature point            */
  CBDDC_ENOCONV = 5,   /* GMRES or Newton did not converge                */
  CBDDC_ETIMEOUT = 6,  /* a device wait exceeded its iteration budget     */
  CBDDC_ENOMEM = 7     /* device or host allocation failed               */
};

/* Element types (Section 2, "Space discretization"). */
enum {
  CBDDC_HEX_Q1 = 1, /* 8-node trilinear hexahedron, 2x2x2 Gauss points  */
  CBDDC_HEX_Q2 = 2, /* 27-node triquadratic hexahedron, 3x3x3 points   */
  CBDDC_TET_P1 = 3, /* 4-node linear tetrahedron, centroid rule         */
  CBDDC_TET_P2 = 4  /* 10-node quadratic tetrahedron, 4-point rule of
                       degree 2; faces: centroid / 3-point rule          */
};

/* Analytic fibre fields, evaluated at quadrature points. */
enum {
  /* f = (cos a, sin a, 0), s = (-sin a, cos a, 0), n = e_z, with
     a = p[2] + (p[3] - p[2]) (Z - p[0]) / (p[1] - p[0]) and Z the
     reference height; p = fiber_params. */
  CBDDC_FIBER_SLAB_HELIX = 1,
  /* Nodal directions fiber_nodal[node] = (f_x, f_y, f_z, n_x, n_y, n_z),
     interpolated with the shape functions to each quadrature point; there
     f is normalised, n is made orthogonal to f and normalised, and
     s = n x f. */
  CBDDC_FIBER_NODAL = 2
};

/*
 * Problem description (all arrays host memory, copied by
 * fem_problem_create).
 *
 * Hexahedron local numbering is lexicographic: local node a+(k+1)(b+(k+1)c)
 * sits at reference point (-1+2a/k, -1+2b/k, -1+2c/k), k = element order.
 * Local faces: 0 = xi-, 1 = xi+, 2 = eta-, 3 = eta+, 4 = zeta-, 5 = zeta+.
 *
 * Tetrahedron: vertices 0..3 at (0,0,0), (1,0,0), (0,1,0), (0,0,1); P2 adds
 * the midpoints of edges (0,1), (1,2), (0,2), (0,3), (1,3), (2,3) as local
 * nodes 4..9.  Local face f is the face opposite vertex f.  Elements must
 * be positively oriented (det of the reference Jacobian > 0).
 */
typedef struct {
  int elem_type;               /* CBDDC_HEX_* or CBDDC_TET_*                */
  int n_nodes;
  const double* coords;        /* [n_nodes][3] reference coordinates        */
  int n_elems;
  const int32_t* elems;        /* [n_elems][nodes per element]              */
  const int32_t* elem_part;    /* [n_elems] subdomain id in [0, n_parts)    */
  int n_parts;
  int n_dirichlet;
  const int32_t* dirichlet_nodes; /* clamped nodes (all 3 components)        */
  int n_pressure_faces;
  const int32_t* pressure_faces;  /* [n][2] (element, local face) pairs on
                                     which the follower pressure acts      */
  int fiber_kind;              /* CBDDC_FIBER_*                             */
  double fiber_params[8];
  /* Guccione constants C, b_ff, b_ss, b_nn, b_fs, b_fn, b_sn and the
     volumetric coefficient B of B/2 (J-1) log J (Section 2). */
  double material[8];
  double pressure;             /* p at load factor 1 (Pa)                   */
  double gamma;                /* activation gamma at load factor 1 (Pa)    */
  const double* fiber_nodal;   /* [n_nodes][6] for CBDDC_FIBER_NODAL, else
                                  ignored (may be NULL)                     */
  /* Time-dependent terms (Section 2; active with fem_set_time_state).
     rho: density of the inertia term rho (d^n - 2 d^{n-1} + d^{n-2})/dt^2
     (consistent mass; 0 = none).  Robin faces carry the generalized Robin
     condition of Eq. (bc epi): traction -[(N x N)(K_perp d + C_perp v) +
     (I - N x N)(K_par d + C_par v)], N the reference outward normal and
     v = (d^n - d^{n-1})/dt (v = 0 without a time state). */
  double rho;
  int n_robin_faces;
  const int32_t* robin_faces;  /* [n][3] (element, local face, set 0 or 1)  */
  double robin[2][4];          /* per set: K_perp, K_par, C_perp, C_par    */
} fem_problem_desc;

typedef struct fem_problem fem_problem;

typedef struct {
  int64_t n_free;              /* free DoFs                                 */
  int64_t n_block_rows;        /* free nodes                                */
  int64_t nnzb;                /* 3x3 blocks of the tangent                 */
  int n_parts;
  int n_vertices, n_edges, n_faces; /* interface classes (Section 3.2)      */
  int64_t max_local_dofs;      /* largest subdomain (interior + interface)  */
  int64_t sum_local_dofs;
  int64_t device_bytes;        /* device memory held by the problem         */
} fem_problem_info;

/* Builds DoF numbering, the BSR pattern, element-to-slot maps, the
   subdomain maps and the interface classification on the host, then
   uploads everything to the current device.  Interface classes: nodes are
   grouped by the set of subdomains sharing them and split into connected
   pieces; a piece shared by two subdomains is a face, by three or more an
   edge, and single-node edges plus edge nodes on the outer boundary are
   vertices.  *out receives a handle owned by the caller (destroy it with
   fem_problem_destroy).  Synchronous. */
CBDDC_API int fem_problem_create(const fem_problem_desc* desc, fem_problem** out);
CBDDC_API void fem_problem_destroy(fem_problem* P);
CBDDC_API int fem_problem_get_info(const fem_problem* P, fem_problem_info* info);

/* View of the assembled global tangent in block-CSR form (3x3 blocks,
   row-major inside a block).  All pointers are device memory owned by the
   problem; they stay valid until the next fem_assemble_tangent on the
   same problem or its destruction. */
typedef struct {
  const double* vals;          /* [nnzb][3][3]                              */
  const int32_t* row_ptr;      /* [n_block_rows + 1]                        */
  const int32_t* col_idx;      /* [nnzb]                                    */
  int64_t n_block_rows;
  int64_t nnzb;
} fem_tangent;

/* Residual F(d) of the weak form at load factor lambda (pressure and
   activation scaled by lambda), Section 2:
     F(d) = int P(F) : grad d*  +  int_{pressure faces} p J F^{-T} N . d*.
   d, residual: dev, [n_free].  Returns CBDDC_EINVERTED (after writing the
   residual) if J <= 0 at any quadrature point; that status is only known
   once the stream reaches the call, so this call synchronises. */
CBDDC_API int fem_residual(fem_problem* P, const double* d, double load_factor,
                 double* residual, cbddc_stream_t stream);

/* Residual (if residual != NULL) and the exact tangent DF(d) of
   Eq. (tangent problem): material tangent dP/dF plus the follower-pressure
   linearisation (non-symmetric).  Fills *K with a view of the global BSR
   matrix and keeps the element and face matrices for bddc_setup.
   Synchronises (reports CBDDC_EINVERTED like fem_residual). */
CBDDC_API int fem_assemble_tangent(fem_problem* P, const double* d, double load_factor,
                         double* residual, fem_tangent* K,
                         cbddc_stream_t stream);

/* Copies the last assembled tangent into caller-owned device buffers:
   vals [nnzb*9], row_ptr [n_block_rows+1], col_idx [nnzb] (any may be
   NULL to skip it).  Asynchronous. */
CBDDC_API int fem_tangent_copy(const fem_problem* P, double* vals, int32_t* row_ptr,
                               int32_t* col_idx, cbddc_stream_t stream);

/* y = K x with the last assembled tangent.  x, y: dev [n_free]. */
CBDDC_API int fem_spmv(fem_problem* P, const double* x, double* y, cbddc_stream_t stream);

/* Time state of the backward-Euler step (Section 2, time discretization):
   with dt > 0 the residual and tangent gain the inertia term
   rho (d - 2 d_prev + d_prev2)/dt^2 (the printed /dt read as /dt^2) and the
   damping part C v, v = (d - d_prev)/dt, of the Robin traction; dt = 0
   returns to the quasi-static problem (Robin springs only).  d_prev and
   d_prev2: device FP64 [n_free], borrowed: they must stay valid and hold
   their values while the state is set (until dt = 0 or destroy).  Host
   call, no device work. */
CBDDC_API int fem_set_time_state(fem_problem* P, double dt, const double* d_prev,
                                 const double* d_prev2);

/* ---------------------------------------------------------------- BDDC */

enum { CBDDC_FP64 = 0, CBDDC_FP32 = 1 };      /* local operator precision */
/* Interface scaling D_i of the restriction and extension (Section 3.2).
   COUNTING: delta_i^dagger = 1 / #subdomains sharing the DoF.  DELUXE: on
   every edge and face class K (vertex nodes keep counting),
   D_K^(i) = (sum_j S_K^(j))^-1 S_K^(i), with S_K^(j) the class block of
   subdomain j's Schur complement onto its interface; the extension applies
   D_K^(i), the restriction its transpose.  Deluxe is set up per Newton
   step from the local Schur complements (dense, in the local operator
   precision) and applies to the first level of a multilevel method. */
enum { CBDDC_SCALING_COUNTING = 0, CBDDC_SCALING_DELUXE = 1 };
/* Coarse space.  GALERKIN: one basis Phi (the minimum-energy extension of
   the primal constraints for S_i) on both sides, coarse matrix
   sum Phi_i^T S_i Phi_i.  PETROV: the nonsymmetric BDDC, with a left basis
   Psi built the same way for S_i^T: coarse matrix sum Psi_i^T S_i Phi_i and
   coarse right-hand side sum Psi_i^T g_i (equal to GALERKIN for a
   symmetric tangent).  A multilevel method uses it on every level. */
enum { CBDDC_COARSE_GALERKIN = 0, CBDDC_COARSE_PETROV = 1 };
enum { CBDDC_PRIMAL_V = 1, CBDDC_PRIMAL_E = 2, CBDDC_PRIMAL_F = 4, CBDDC_PRIMAL_R = 8 };
/* CBDDC_PRIMAL_R adds, to every edge (E) or face (F) class, constraints on
   the infinitesimal rotations about the class centroid (the rigid motions,
   near-null space of elasticity, taken into the primal space: Section 4):
   the rotation fields e_k x (x - xbar), k = x, y, z, restricted to the class
   nodes, orthonormalised along the principal axes of the class; an axis
   whose principal moment is below 1e-8 of the largest (the axis of a
   straight edge) gives no constraint.  So a planar face carries 6 primal
   DoFs, a straight edge 5.  Two-level method only (levels = 2, not in
   primal2): bddc_setup returns CBDDC_EINVAL otherwise. */

typedef struct {
  int precision;     /* CBDDC_FP64: all local operators in FP64;
                        CBDDC_FP32: local Schur complements, inverses and
                        triangular-solve equivalents in FP32 (inputs and
                        outputs of bddc_apply stay FP64, coarse solve FP64) */
  int primal;        /* OR of CBDDC_PRIMAL_* (Section 6.2: V, VE, VEF ...) */
  double pivot_tol;  /* a pivot below pivot_tol * max|diag| is an error   */
  /* Multilevel BDDC (Section 3.2, last paragraph; Section 7).  levels = 2
     (or 0): the coarse problem S_PiPi is inverted densely in FP64.
     levels = 3: the coarse problem, an unassembled matrix whose elements
     are the subdomains with their local coarse matrices, is approximated by
     one BDDC application on n_parts2 level-2 subdomains (part2[i] is the
     level-2 subdomain of subdomain i, host array, copied), with primal
     space primal2 and local operators in precision2 (CBDDC_FP64, the
     zero default, or CBDDC_FP32); its own (coarsest) problem is inverted
     densely in FP64.  A subdomain may carry at most 512 primal
     constraints. */
  int levels;
  int n_parts2;
  const int32_t* part2;
  int primal2;
  int precision2;
  int scaling;       /* CBDDC_SCALING_COUNTING (0) or CBDDC_SCALING_DELUXE;
                        deluxe allows at most 65535 edge and face classes,
                        of at most 1024 nodes each (CBDDC_EINVAL otherwise) */
  int coarse;        /* CBDDC_COARSE_GALERKIN (0) or CBDDC_COARSE_PETROV */
  int sweep_block;   /* pivot block width of the local Gauss-Jordan sweeps:
                        0 or 64 (default), or 128 (FP32 operators only:
                        half the passes over each local matrix) */
  int tile_order;    /* order of the output tiles of the setup GEMMs: 0 =
                        by subdomain (default), 1 = largest problems first
                        (uneven subdomains: the long ones start first) */
} bddc_options;

typedef struct bddc_ctx bddc_ctx;

typedef struct {
  int n_primal;                /* coarse space dimension                    */
  int n_primal2;               /* level-2 coarse dimension (levels = 3)     */
  int precision;
  int64_t local_bytes;         /* bytes of local operators read per apply   */
  int64_t device_bytes;        /* device memory held by the context         */
  double setup_flops;          /* algorithmic flops of the last setup       */
  int sweep_block;             /* pivot block width of the local sweeps     */
  int tile_order;              /* tile order of the setup GEMMs             */
  float ms_setup_tuned;        /* autotuned contexts: the chosen candidate's
                                  setup time, and that of the default
                                  (64, subdomain order); 0 otherwise        */
  float ms_setup_default;
} bddc_info;

/* BDDC setup for the tangent last assembled on P (Section 3.2): subdomain
   matrices A^(i) from the element matrices; A_II^-1, A_II^-1 A_IG,
   A_GI A_II^-1 and the Schur complement S_i by a block Gauss-Jordan sweep;
   the constrained Neumann solution operator on the interface and the
   minimum-energy coarse basis Phi_i; S_PiPi = sum Phi_i^T S_i Phi_i and its
   FP64 inverse.  If *inout is NULL a context is created (owned by the
   caller, release with bddc_destroy); otherwise it is reused, and must
   have been created for the same P and options.  Synchronises and returns
   CBDDC_EPIVOT on a tiny pivot. */
CBDDC_API int bddc_setup(fem_problem* P, const fem_tangent* K, const bddc_options* opt,
               bddc_ctx** inout, cbddc_stream_t stream);

/* z = M_BDDC^-1 r for the full system: interior correction, interface
   restriction with counting scaling, constrained local solves plus coarse
   correction, averaging, harmonic extension.  r, z: dev [n_free], must not
   alias.  Asynchronous. */
CBDDC_API int bddc_apply(bddc_ctx* C, const double* r, double* z, cbddc_stream_t stream);
CBDDC_API void bddc_destroy(bddc_ctx* C);

/* Same result as bddc_apply, for callers that must not allocate device
   memory while they run: code that is not allowed to call cudaMalloc
   (which synchronises the device and may fail or stall once another
   allocator has reserved the memory), and setups whose memory was
   budgeted up front.  The paper has no counterpart.
   The per-apply work vectors live in one static device array of 4 MiB
   (524288 doubles), held by every device that loads the library until the
   process exits.  A context whose work vectors need more than that is
   rejected with CBDDC_EINVAL (the message gives both sizes); bddc_apply
   serves those.  The call performs no allocation: the context C must
   already exist (bddc_setup allocates it).  The first call on a device
   looks up the array's device address (cudaGetSymbolAddress, no
   allocation); make that first call before any stream capture.  All calls
   on one device share its array (each device has its own): every entry is
   written before it is read within a call, so nothing needs clearing, but
   calls on the same device whose work overlaps on the GPU (for example on
   two streams) race and give wrong results; serialise them.
   r, z: dev [n_free], must not alias.  Asynchronous. */
CBDDC_API int bddc_apply_noalloc(bddc_ctx* C, const double* r, double* z, cbddc_stream_t stream);
CBDDC_API int bddc_get_info(const bddc_ctx* C, bddc_info* info);

/* ---------------------------------------------------- GMRES and Newton */

typedef struct {
  int restart;         /* Krylov dimension per cycle (default 100, <= 1023) */
  int max_iters;       /* total iteration cap                               */
  double rtol;         /* stop when ||b - K x|| <= rtol ||b||               */
} gmres_options;

typedef struct {
  int iterations;
  int converged;
  double rel_residual; /* true relative residual at exit                    */
} gmres_report;

/* Flexible GMRES (right preconditioned by BDDC) for K x = b with the last
   assembled tangent of P.  Arnoldi step in FP64: for n_free <= 10^6 and
   at most 128 basis vectors classical Gram-Schmidt applied twice, else
   modified Gram-Schmidt.  b, x:
   dev [n_free]; x is overwritten (zero initial guess).  Synchronises once
   per iteration to test convergence.  Returns CBDDC_ENOCONV if max_iters
   is reached. */
CBDDC_API int gmres_solve(fem_problem* P, bddc_ctx* C, const double* b, double* x,
                const gmres_options* opt, gmres_report* rep,
                cbddc_stream_t stream);

typedef struct {
  int precision;       /* CBDDC_FP64 or CBDDC_FP32 local operators           */
  int primal;          /* OR of CBDDC_PRIMAL_*                               */
  int load_steps;      /* lambda_k = k / load_steps                          */
  int max_newton;      /* Newton iterations per load step                    */
  int max_halvings;    /* load-increment halvings before giving up           */
  int restart;         /* GMRES restart (default 100, at most 1023)          */
  int max_gmres;       /* GMRES iteration cap per Newton step                */
  double newton_rtol;  /* ||F(d)|| <= newton_rtol ||F(d^{n,0})||             */
  double gmres_rtol;   /* relative residual of each tangent solve            */
  double pivot_tol;
  int levels;          /* as in bddc_options                                 */
  int n_parts2;
  const int32_t* part2;
  int primal2;
  int precision2;
  int scaling;         /* as in bddc_options                                 */
  int coarse;          /* as in bddc_options                                 */
  int sweep_block;     /* as in bddc_options                                 */
  int tile_order;      /* as in bddc_options                                 */
  int autotune;        /* 1: when a Newton step creates the BDDC context, it
                          first times one setup for every candidate (sweep
                          block 64/128 for FP32 operators, tile order 0/1)
                          on the assembled tangent and keeps the fastest;
                          the choice is cached in the problem per precision
                          and reported by bddc_get_info, the tuning time in
                          newton_record.ms_autotune.  sweep_block and
                          tile_order are then ignored. */
} solve_options;

#define CBDDC_MAX_RECORDS 512
typedef struct {
  double load;         /* load factor of this Newton step                    */
  int newton;          /* Newton index within the load step                  */
  int gmres_its;
  double res;          /* ||F(d)|| before the step                           */
  double res0;         /* ||F(d^{n,0})|| of the load step                    */
  float ms_assemble, ms_setup, ms_gmres, ms_total; /* CUDA-event times       */
  double gmres_relres; /* ||b - K delta|| / ||b|| of the tangent solve at exit */
  int gmres_reorth;    /* Arnoldi steps that took a second Gram-Schmidt pass */
  float ms_autotune;   /* time spent tuning the setup in this step (0: none) */
} newton_record;

typedef struct {
  int status;
  int newton_steps;
  int load_steps_done;
  int halvings;
  int total_gmres_its;
  double final_rel_residual;
  int n_records;
  newton_record rec[CBDDC_MAX_RECORDS];
} solve_report;

/* One Newton step at load factor lambda (Eq. tangent problem): residual,
   tangent, BDDC setup (into *ctx, created if NULL), GMRES on
   DF(d) delta = -F(d), then d += delta.  d: dev [n_free], updated in
   place.  rec (host, may be NULL) receives the step's timings.
   Synchronises. */
CBDDC_API int newton_step(fem_problem* P, bddc_ctx** ctx, const solve_options* opt,
                double load_factor, double* d, newton_record* rec,
                cbddc_stream_t stream);

/* Same as newton_step with d in host memory: d is copied to the device,
   the step runs, and the updated d is copied back before returning. */
CBDDC_API int newton_step_host(fem_problem* P, bddc_ctx** ctx, const solve_options* opt,
                     double load_factor, double* d_host, newton_record* rec,
                     cbddc_stream_t stream);

/* Full load-stepped Newton solve (Section 2): for each load level,
   Newton from the previous solution until ||F|| <= newton_rtol ||F_0||;
   the increment is halved on J <= 0 or Newton failure.  d: dev [n_free],
   in: initial guess (usually zero), out: solution.  rep: host,
   caller-allocated.  Synchronises. */
CBDDC_API int newton_gmres_solve(fem_problem* P, const solve_options* opt, double* d,
                       solve_report* rep, cbddc_stream_t stream);

/* ------------------------------------------------------- observability */

/* Number of kernels this library has launched since it was loaded. */
CBDDC_API uint64_t cbddc_kernel_launches(void);

/* Kernel classes that the launch timer can follow. */
enum {
  CBDDC_TIMER_OFF = 0,
  CBDDC_TIMER_SWEEP_GEMM = 1, /* FP32 setup GEMMs: trailing updates of the
                                 Gauss-Jordan sweeps and the E, S, constraint
                                 and coarse-basis products (tensor cores)     */
  CBDDC_TIMER_ELEMENT = 2,    /* element residual/tangent kernel              */
  CBDDC_TIMER_APPLY = 3,      /* one whole BDDC apply (all its launches)      */
  CBDDC_TIMER_SPMV = 4,       /* BSR SpMV                                     */
  CBDDC_TIMER_ORTH = 5,       /* one GMRES Arnoldi step (Gram-Schmidt,
                                 Givens, normalisation)                       */
  CBDDC_TIMER_SETUP = 6,      /* one whole BDDC setup (all levels)            */
  CBDDC_TIMER_LEVEL2_SETUP = 7, /* setup of the level-2 BDDC (multilevel)     */
  CBDDC_TIMER_LEVEL2_APPLY = 8, /* apply of the level-2 BDDC (multilevel)     */
  CBDDC_TIMER_COARSE_SETUP = 9, /* coarsest level: FP64 coarse assembly and
                                   dense inverse                              */
  CBDDC_TIMER_COARSE_APPLY = 10, /* coarsest level: dense FP64 coarse solve   */
  CBDDC_TIMER_SETUP_GEMM_F64 = 11 /* FP64 setup GEMMs (FP64 local operators
                                     and the coarse inverse)                  */
};

/* Selects the kernels of the FP32 setup GEMMs.  mode bit 0 (1): tcgen05
   tensor cores with operands split into TF32 parts (else every FP32 setup
   GEMM on the CUDA cores); bit 1 (2): three parts (six products) for the
   Gauss-Jordan sweep updates, else two (three products); bit 2 (4): the
   same for the other setup products; bit 3 (8): the other products on the
   CUDA cores; bit 4 (16): the sweep updates on the CUDA cores; bit 5 (32):
   the tensor-core sweep updates accumulate a whole 32-wide K block in each
   TMEM slice instead of one K-step of 8; bit 6 (64): the other products
   accumulate one K-step of 8 per slice instead of a 32-wide K block.
   Bits above 6 are ignored.  Default 1
   (tensor cores, two parts).  The enable bits are read at every setup,
   the part counts when a context is created.  Returns the previous mode.
   Host-side state, not thread safe; a diagnostic and comparison switch. */
CBDDC_API int cbddc_set_tensor_cores(int mode);

/* Starts recording CUDA events around every launch of the given class (and
   stops recording every other class), on the stream the launch uses (at
   most 32768 launches per class are recorded).  Each
   recorded launch also adds its algorithmic flops and bytes.  Host-side
   state, not thread safe. */
CBDDC_API int cbddc_timer_start(int kernel_class);

/* Records one more kernel class alongside those already recorded (its
   totals start at zero). */
CBDDC_API int cbddc_timer_enable(int kernel_class);

/* Waits for the events recorded so far for one enabled class and returns
   its summed device time (ms), launches, algorithmic flops and bytes. */
CBDDC_API int cbddc_timer_result(int kernel_class, double* total_ms, int64_t* launches, double* flops,
                                 double* bytes);

/* Stops recording every class, waits for the recorded events and returns
   the totals of the class given to cbddc_timer_start: summed device time
   (ms), the number of launches and their algorithmic flops and bytes. */
CBDDC_API int cbddc_timer_stop(double* total_ms, int64_t* launches, double* flops, double* bytes);

/* Message for the last non-zero status returned on this thread. */
CBDDC_API const char* cbddc_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* CARDIAC_BDDC_H */
