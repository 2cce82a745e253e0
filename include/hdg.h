/*
 * hdg.h -- C ABI of the GB300 (sm_103a) statically condensed HDG library.
 *
 * The library solves the Helmholtz problem  lambda u - laplace u = f  with
 * Dirichlet (u = g_D) or Neumann (n . grad u = g_N) data on the six sides of
 * a Cartesian box (arXiv:2007.11891, Eq. (helmholtz_equation), Sec. 2.1),
 * discretised by the hybridised LDG method (LDG-H) on cuboid elements with
 * a tensor-product Lagrange basis on the Gauss-Lobatto-Legendre points of
 * degree p (Sec. 2.2, Sec. 3.2) and the penalty tau_{i,e} = 2 tau_hat / h_{i,e}.
 * After static condensation the unknowns are the traces u-tilde on the
 * faces, and the global system is  K ut = F  (Eq. (hdg_system)).
 *
 * ---------------------------------------------------------------------------
 * Data layout (all arrays are dense, little-endian, element/face-major)
 * ---------------------------------------------------------------------------
 *   n = p + 1 nodes per direction.  Elements (e1, e2, e3), 0 <= e_d < N_d,
 *   have index e1 + N1 (e2 + N2 e3).
 *
 *   Volume vectors (f, u, gradients): n^3 values per element, node
 *   i + n j + n^2 k (x1 fastest); hdg_volume_size() = n_e n^3 per
 *   right-hand side.
 *
 *   Trace vectors: faces normal to direction d lie on grid planes 0..N_d.
 *   A plane is an unknown unless it is the boundary plane of a Dirichlet
 *   side; unknown planes of direction d are lo_d..hi_d with lo_d = 1 (0 if
 *   the low side is Neumann) and hi_d = N_d - 1 (N_d if the high side is
 *   Neumann).  The vector is the concatenation of the blocks d = 0, 1, 2;
 *   block d holds its unknown planes in order, each with Na x Nb faces
 *   (the other two element counts in increasing axis order, face a + Na b),
 *   each face n x n nodes ordered by its two axes, lower axis fastest.
 *   hdg_trace_size() values per right-hand side.
 *
 *   Boundary data vectors: the six sides 0..5 = (x1-, x1+, x2-, x2+, x3-,
 *   x3+) in order, each with Na x Nb faces of n x n nodes as above; a
 *   Dirichlet side holds nodal values of g_D, a Neumann side nodal values of
 *   g_N = n . grad u (outer normal).  hdg_boundary_size() values.
 *
 *   Batches of nrhs right-hand sides are stored one after the other
 *   (right-hand side r at offset r * size).
 *
 * ---------------------------------------------------------------------------
 * Conventions
 * ---------------------------------------------------------------------------
 *   - Pointers named d_* are device pointers on the current CUDA device;
 *     h_* are host pointers.  The caller owns every buffer it passes; the
 *     context owns its tables and workspaces and frees them in hdg_destroy.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Device work is enqueued on it; calls that return results
 *     to the host (solve info) synchronise that stream.
 *   - Every call returns an hdg_status and never aborts the process.  On an
 *     error, hdg_last_error() returns a message for the calling thread.
 *   - A context may be used by one host thread at a time.
 */
#ifndef HDG_GB300_H
#define HDG_GB300_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hdg_ctx hdg_ctx;

typedef enum {
  HDG_OK = 0,
  HDG_ERR_INVALID_ARG = 1,   /* bad size, pointer, degree or option        */
  HDG_ERR_SINGULAR = 2,      /* lambda = 0 and no Dirichlet side: K singular */
  HDG_ERR_CUDA = 3,          /* a CUDA runtime call failed                  */
  HDG_ERR_OOM = 4,           /* device allocation failed                    */
  HDG_ERR_NOT_CONVERGED = 5, /* iteration limit reached before tolerance    */
  HDG_ERR_BREAKDOWN = 6,     /* CG breakdown: p^T K p <= 0 or non-finite     */
  HDG_ERR_UNSUPPORTED = 7    /* degree outside the supported range, or not an sm_103 device */
} hdg_status;

/* Precision of an operator application or of the inner CG solve.
 *   HDG_FP64: FP64 storage and arithmetic.
 *   HDG_FP32: FP32 storage and arithmetic.
 *   HDG_BF16: BF16 storage of trace vectors, FP32 arithmetic.            */
typedef enum { HDG_FP64 = 0, HDG_FP32 = 1, HDG_BF16 = 2 } hdg_precision;

/* Basis of trace vectors.
 *   HDG_BASIS_NODAL: nodal values on the GLL points (the K of Eq. (hdg_system),
 *     evaluated as in Alg. (hdg_op_3d)).
 *   HDG_BASIS_TRANSFORMED: coefficients in the face eigenbasis of
 *     Sec. 4.2, ut-hat = (S^T M (x) S^T M) ut per face, where the operator is
 *     K-hat = (S^T (x) S^T) K (S (x) S) of Alg. (hdg_op_3d_transformed).
 *     S is fixed uniquely (for distinct eigenvalues) as follows: its columns
 *     solve L s = Lambda M s with s^T M s = 1 (Eq. (generalized_eigenvalue_
 *     decomposition), L = E + D M^-1 D^T); the GLL points are mirror
 *     symmetric, so every column is even or odd under x -> -x; the columns
 *     are ordered even modes first, then odd modes, each group by increasing
 *     eigenvalue; and each column's sign makes B_S[m][0] > 0, with
 *     B_S = S^T B - S^T D M^-1 C of Eq. (hdg_bs).  Face mode (m1, m2) of a
 *     face is stored at m1 + n m2 (the face's lower axis fastest).          */
typedef enum { HDG_BASIS_NODAL = 0, HDG_BASIS_TRANSFORMED = 1 } hdg_basis;

typedef struct {
  int ne[3];               /* elements per direction, each >= 1                */
  const double* h_grid[3]; /* host; ne[d] + 1 strictly increasing coordinates  */
  int bc[6];               /* per side x1-,x1+,x2-,x2+,x3-,x3+: 0 Dirichlet, 1 Neumann */
} hdg_mesh;

typedef struct {
  double tau_hat;          /* penalty on the standard element, > 0 (Sec. 3.2) */
  int mass_lumped;         /* 0: exact mass matrix (default); 1: GLL-lumped     */
} hdg_options;

typedef struct {
  double tol;              /* stop at ||F - K ut||_2 <= tol ||F||_2 (nodal basis) */
  int max_iter;            /* total inner CG iterations allowed per right-hand side */
  int max_outer;           /* iterative-refinement steps allowed (>= 1)           */
  hdg_precision inner;     /* precision of the inner CG (FP64, FP32 or BF16)      */
  double inner_tol;        /* floor of the relative residual reduction asked of one
                              inner solve; each inner solve targets
                              max(floor, tol ||F|| / (2 ||r||)) for the current
                              outer residual r; <= 0 picks 3e-4 (FP32) or 0 (FP64) */
  int precond;             /* 0: plain CG; 1: face-block Jacobi preconditioner of
                              Sec. 5.1 (Alg. hdg_pc_block), diagonal in the
                              transformed basis (the paper's HDG-trans solver)     */
} hdg_solve_opts;

typedef struct {
  int iterations;          /* inner CG iterations                                 */
  int outer;               /* refinement steps taken                              */
  int applies;             /* condensed-operator applications (all precisions)    */
  double rel_residual;     /* final FP64 ||F - K ut||_2 / ||F||_2 in the nodal basis */
  int status;              /* hdg_status of this right-hand side                  */
} hdg_solve_info;

/* Build a context: 1D tables (GLL nodes, mass and stiffness matrices, the
 * generalised eigen-decomposition S^T M S = I, S^T L S = Lambda of
 * Eq. (generalized_eigenvalue_decomposition), the row matrix
 * B_S = S^T B - S^T D M^-1 C of Eq. (hdg_bs) and the 2x2 face matrix
 * G + C^T M^-1 C), computed on the host in FP64 and uploaded to the current
 * device.  p in 1..32: degrees up to 16 run kernels specialised per degree;
 * degrees 17..32 run runtime-degree kernels (the operator recomputes the
 * eigenspace solution along each direction instead of storing it, D_Z^-1 is
 * computed in the kernel; no BF16 storage, nodal applies always face-wise,
 * inner CG as two kernels per iteration).  Errors: INVALID_ARG, UNSUPPORTED,
 * CUDA, OOM.
 * On success *out owns device memory until hdg_destroy.                  */
hdg_status hdg_setup(const hdg_mesh* mesh, int p, const hdg_options* opts, hdg_ctx** out);

/* Free every resource of ctx (NULL is a no-op).  Synchronises the device. */
void hdg_destroy(hdg_ctx* ctx);

size_t hdg_trace_size(const hdg_ctx* ctx);     /* unknown trace values per rhs */
size_t hdg_volume_size(const hdg_ctx* ctx);    /* n_e n^3                      */
size_t hdg_boundary_size(const hdg_ctx* ctx);  /* boundary data values         */

/* Copy the n GLL points of the standard element [-1, 1] to h_nodes[n].   */
hdg_status hdg_get_nodes(const hdg_ctx* ctx, double* h_nodes);

/* y = K x for nrhs trace vectors with homogeneous Dirichlet data
 * (Eq. (hdg_system); Alg. (hdg_op_3d) for HDG_BASIS_NODAL,
 * Alg. (hdg_op_3d_transformed) for HDG_BASIS_TRANSFORMED), lambda_r =
 * h_lambda[r] >= 0.  d_x, d_y: device, nrhs * hdg_trace_size() values of
 * type double (FP64), float (FP32) or bfloat16 (BF16, transformed basis
 * only); they must not overlap.  Both traces sides of a shared face are
 * summed in a fixed order, so results are bitwise reproducible.
 * Errors: INVALID_ARG (NULL pointer, nrhs < 1, lambda < 0, BF16 in the
 * nodal basis), SINGULAR is not reported here, CUDA.                       */
hdg_status hdg_apply(hdg_ctx* ctx, int nrhs, const double* h_lambda, hdg_precision prec,
                     hdg_basis basis, const void* d_x, void* d_y, void* stream);

/* The same product as hdg_apply(ctx, nrhs, h_lambda, HDG_FP64,
 * HDG_BASIS_NODAL, d_x, d_y, stream), for callers that must not allocate
 * device memory.  The paper has no counterpart: this is an interface for
 * such callers, not part of the method.
 *
 * Who needs it: real-time loops that must neither synchronise nor risk an
 * allocation failure once running (cudaFree synchronises the whole device),
 * programs whose device memory belongs to a pooling allocator that forbids
 * allocations made behind its back, and code that must run within a device
 * memory budget set at start-up.  hdg_apply grows internal workspaces with
 * cudaMalloc the first time a size or lambda is seen; this entry point never
 * calls cudaMalloc, cudaFree or any allocating routine.
 *
 * Its temporaries (the face-eigenbasis traces before and after the
 * operator, 2 x nrhs x hdg_trace_size() doubles, and the D_Z^-1 tables of
 * the lambdas, nrhs x n^2 x (n rounded up to even) doubles on a uniform
 * grid, n_e times that on a stretched one) live in one static device array
 * of 2^21 doubles (16 MiB), which every GPU that loads the library reserves
 * until the process exits.  Larger requests are rejected with
 * HDG_ERR_INVALID_ARG and a message giving the size needed (use hdg_apply
 * then).
 *
 * The first call on a device looks up that array's device address with
 * that device current (and may load the library's device code there); make
 * that first call before any stream capture.  The address is cached per
 * device for the life of the process: after cudaDeviceReset it is stale, so
 * do not call this entry point again after a reset.  All calls share the one
 * array, which keeps the previous call's contents (whatever must start at
 * zero is cleared by each call): calls whose work overlaps on the GPU
 * (different streams, or different host threads) race on it and must be
 * serialised by the caller.  The operator's work split is always the
 * automatic one (hdg_set_x1_segment and hdg_set_slots_per_cta are not
 * consulted; every split gives bitwise the same result).  Arguments, layout
 * and results are those of hdg_apply with FP64 nodal traces; the current
 * device must be the context's device.                                    */
hdg_status hdg_apply_static(hdg_ctx* ctx, int nrhs, const double* h_lambda, const double* d_x, double* d_y,
                            void* stream);

/* Solve K ut = F (Alg. (hdg_cg) with the transformed CG of
 * Alg. (hdg_transformed_cg)) for nrhs right-hand sides, in FP64 or with an
 * FP32/BF16 inner CG inside FP64 iterative refinement.
 *   d_f      device, nrhs * hdg_volume_size(): nodal values of f.
 *   d_bdry   device, nrhs * hdg_boundary_size() boundary data, or NULL (zero).
 *   d_x0     device, nrhs * hdg_trace_size() initial traces, or NULL (zero).
 *   d_trace  device, nrhs * hdg_trace_size(): the solution ut (nodal basis).
 *   d_u      device, nrhs * hdg_volume_size(): recovered u, or NULL.
 *   h_info   host array of nrhs, filled on return (the call synchronises).
 * Returns the worst per-rhs status: SINGULAR (lambda = 0 without a
 * Dirichlet side), NOT_CONVERGED, BREAKDOWN, INVALID_ARG, CUDA, OOM.
 * BREAKDOWN: an FP64 CG breakdown, a non-finite residual, or an FP32 inner
 * breakdown after which the FP64 residual did not fall at least twofold (an
 * FP32 inner solve that broke down after one or more iterations keeps its
 * correction, and the refinement goes on).                                */
hdg_status hdg_solve(hdg_ctx* ctx, int nrhs, const double* h_lambda, const double* d_f,
                     const double* d_bdry, const double* d_x0, double* d_trace, double* d_u,
                     const hdg_solve_opts* opts, hdg_solve_info* h_info, void* stream);

/* Adjoint of a solve with homogeneous boundary data.  Given the forward
 * solution d_u and the gradient d_grad_u = dL/du of a loss L(u) (both
 * nrhs * hdg_volume_size()), solve the adjoint system -- the element system
 * of Eq. (ldg_element_operator_threed) is symmetric, so this is the same
 * condensed solve with volume load dL/du -- and return
 *   d_grad_f[r]      = M_e z_{u,e}                   (dL/df, volume layout)
 *   d_grad_lambda[r] = - sum_e z_{u,e}^T M_e u_e     (dL/dlambda, device)
 * where z_u is the adjoint volume solution.  Errors as hdg_solve.          */
hdg_status hdg_solve_adjoint(hdg_ctx* ctx, int nrhs, const double* h_lambda, const double* d_u,
                             const double* d_grad_u, double* d_grad_f, double* d_grad_lambda,
                             const hdg_solve_opts* opts, hdg_solve_info* h_info, void* stream);

/* Tuning (not part of the method): elements per unit of work of the
 * operator kernel.  Element-tile kernel (the default): elements per tile,
 * rounded up to a multiple of the CTA's element groups and reduced to what
 * fits in shared memory; an x1-face between two elements of a tile is summed
 * in shared memory.  Element-run kernels: the elements one CTA slot marches
 * over along x1 (FP64: a segment of one x1-pencil; FP32: a contiguous run in
 * element order that may continue into the next pencil), the x1-face
 * between consecutive elements summed in registers.  Other shared faces take
 * two atomic adds onto zero.  0 restores the automatic choice.  Speed only:
 * every value gives bitwise identical results.  Errors: INVALID_ARG (NULL
 * context, negative length).                                              */
hdg_status hdg_set_x1_segment(hdg_ctx* ctx, int elements);

/* Tuning (not part of the method): number of element slots per CTA of the
 * element-run operator kernels (each slot is n^2 threads, rounded up to
 * whole warps in the FP32 kernel for n = 8, 9 and n >= 11); 0 restores the
 * automatic choice.  Speed only.  Errors: INVALID_ARG (NULL context,
 * negative count, or a count whose CTA would exceed 320 threads); an FP32
 * apply whose CTA would exceed 256 threads (288 at n = 9; n <= 16) fails
 * with CUDA (invalid configuration).                                        */
hdg_status hdg_set_slots_per_cta(hdg_ctx* ctx, int slots);

/* Autotuner (not part of the method): times the operator kernel of `prec`
 * (transformed basis, nrhs right-hand sides with the given lambdas) with
 * CUDA events on `stream` for every candidate pair of x1-segment length and
 * slots per CTA, keeps the fastest pair on the context (as the two setters
 * above would) and returns it with its mean launch time in microseconds.
 * Allocates workspace (two trace vectors of nrhs x hdg_trace_size()) on
 * first use; synchronises the stream.  Errors: INVALID_ARG, CUDA, OOM.    */
hdg_status hdg_autotune(hdg_ctx* ctx, int nrhs, const double* h_lambda, hdg_precision prec, int* h_best_segment,
                        int* h_best_slots, double* h_best_us, void* stream);

/* Tuning (not part of the method): where the FP32 operator takes the
 * inverse eigenvalue scaling D_Z^-1 of Sec. 4.1 from.  0 automatic (uniform
 * grid: the one element class's table; stretched grid: computed in the
 * kernel with the hardware reciprocal), 1 always a table (one per element on
 * a stretched grid), 2 always computed in the kernel (FP32 only; FP64 always
 * uses tables).  Results agree to FP32 rounding.  Errors: INVALID_ARG.     */
hdg_status hdg_set_dz_mode(hdg_ctx* ctx, int mode);

/* Tuning (not part of the method): work split of the operator kernel.
 * 0 automatic, the choice that measured fastest: element tiles for BF16
 * storage, for FP32 at n = 10 and 12..16 and for FP64 with one right-hand
 * side; element runs otherwise; 2 element tiles (CTAs of n^2 G threads take
 * tiles of consecutive elements in element order, one face node / x1-line
 * per thread; hdg_set_x1_segment sets the elements per tile, rounded to a
 * multiple of G); 1 element runs (one thread per x1-line, runs of elements
 * per CTA slot; slots and run length from hdg_set_slots_per_cta and
 * hdg_set_x1_segment).  FP64, FP32 and BF16 storage.  3 the runtime-degree
 * kernel that degrees 17..32 always use (every mode, FP64 and FP32; at lower
 * degrees for comparison).  Same arithmetic per point: FP64 results of 0-2
 * are bitwise equal, FP32 results agree to FP32 rounding (the tile kernel
 * uses packed two-lane FP32 arithmetic); 3 agrees to rounding.
 * Errors: INVALID_ARG (NULL context, variant outside 0..3).               */
hdg_status hdg_set_operator_variant(hdg_ctx* ctx, int variant);

/* Tuning (not part of the method): how an inner CG iteration runs.
 *   3 (default) as 1, two kernels per iteration (measured fastest or within
 *     10 % on the meshes of 8^3 to 32^3 elements tried, in FP32 and FP64);
 *   0 the whole inner CG in one cooperative launch of the element-tile
 *     kernel (every CTA resident; per iteration,
 *     each CTA applies the CG update of the previous iteration to every face
 *     value it reads -- each face value's one owner stores the new x, p, r,
 *     s -- applies the operator to the new search direction, and after one
 *     grid barrier every CTA forms the step scalars from all CTAs' partial
 *     sums in the same order); where a cooperative launch is not possible,
 *     as variant 2;
 *   2 the same fused step, one launch per iteration (the last CTA of each
 *     launch forms the step scalars), launched from a CUDA graph; in the
 *     FP32 element-run kernel (the state of the faces of the next element
 *     staged asynchronously while the current one computes) where the
 *     automatic operator choice is the element runs, else in the tiles;
 *   1 two kernels per iteration: the operator, then the vector update.
 * All compute the same CG iterates in exact arithmetic.  A grid barrier that
 * waits too long (CTAs not co-resident) ends the kernel and the solve
 * returns HDG_ERR_CUDA.  Errors: INVALID_ARG (NULL context, variant outside
 * 0..3).                                                                  */
hdg_status hdg_set_cg_variant(hdg_ctx* ctx, int variant);

/* Which kernel applies K in the nodal basis (hdg_apply with HDG_FP64 and
 * HDG_BASIS_NODAL):
 *   0 (default) face-wise: every unknown face is transformed to the face
 *     eigenbasis once (S^T M (x) S^T M), the transformed operator of
 *     Alg. (hdg_op_3d_transformed) runs, and every face is transformed back
 *     (M S (x) M S): three launches, 49 n^3 flops per element, two trace-
 *     sized temporaries;
 *   1 one kernel per apply, Alg. (hdg_op_3d) (the paper's HDG-TP, Sec. 4.2):
 *     each element transforms its own six faces in and out, 73 n^3 flops
 *     per element (Tab. operator_variants), no temporaries.
 * Both give K x to FP64 rounding.  Other precisions and bases ignore it.
 * Errors: INVALID_ARG (NULL context, variant outside 0..1).               */
hdg_status hdg_set_nodal_variant(hdg_ctx* ctx, int variant);

/* Measurement support (not part of the method).  Kernel classes:
 *   0 condensed operator, FP32 arithmetic   1 condensed operator, FP64
 *   2 face transforms                       3 volume transforms
 *   4 right-hand side / recovery operator   5 CG vector and reduction kernels
 * hdg_profile(ctx, 1) resets the counters and starts recording a CUDA event
 * pair around every launch of classes 0-5 on the launching stream;
 * hdg_profile(ctx, 0) stops recording.  hdg_profile_read synchronises the
 * device and returns, for one class, the summed launch durations (ms) and
 * the number of launches recorded; class -1 returns the number of kernel
 * launches of all classes since the last hdg_profile(ctx, 1) (counted
 * whether or not recording is on; time is then 0).                         */
hdg_status hdg_profile(hdg_ctx* ctx, int enable);
hdg_status hdg_profile_read(hdg_ctx* ctx, int kernel_class, double* total_ms, long long* launches);

/* Measurement support (not part of the method): the fused multiply-add
 * rate of the current device in TFLOP/s (2 flops per FMA), measured with CUDA
 * events over 5 launches (after one warm-up launch) of a kernel in which
 * every thread runs 8 independent register-resident FMA chains, 4 blocks of
 * 256 threads per SM.  prec: HDG_FP64 or HDG_FP32.  Synchronises the
 * stream.  Errors: INVALID_ARG, CUDA.                                     */
hdg_status hdg_measure_fma_peak(hdg_precision prec, double* h_tflops, void* stream);

/* Message of the last failed call on this host thread ("" if none).      */
const char* hdg_last_error(void);
const char* hdg_status_string(hdg_status s);

/* ---- One- and two-dimensional meshes ---------------------------------------
 * The condensed operator K of Eq. (hdg_system) for lambda u - u'' = f on an
 * interval split into ne[0] elements (dim = 1, Alg. (hdg_op_1d), Sec. 2.2),
 * and for lambda u - laplace u = f on a rectangle of ne[0] x ne[1]
 * rectangular elements (dim = 2: Alg. (hdg_op_3d) / (hdg_op_3d_transformed)
 * with one direction fewer).  Same 1D tables, penalty tau = 2 tau_hat / h
 * and mass options as the three-dimensional context; apply only.
 *
 * Trace layout (device, double): faces normal to direction d lie on grid
 * planes 0..ne[d]; a plane is an unknown unless it is a boundary plane of a
 * Dirichlet side.  Block d (d = 0, then 1) holds the unknown planes in
 * order; in 2D each plane holds ne[1-d] faces (one per element along the
 * other axis, in order) of n = p + 1 GLL nodes along that axis; in 1D each
 * plane is one value.  hdg_lowdim_trace_size() values per right-hand side.
 */
typedef struct hdg_lowdim hdg_lowdim;

typedef struct {
  int dim;                 /* 1 or 2                                             */
  int ne[2];               /* elements per direction, >= 1 (ne[1] unused if dim = 1) */
  const double* h_grid[2]; /* host; ne[d] + 1 strictly increasing coordinates    */
  int bc[4];               /* sides x1-, x1+, x2-, x2+ (the last two unused if
                              dim = 1): 0 Dirichlet, 1 Neumann                   */
} hdg_lowdim_mesh;

/* Build a 1D/2D context (opts may be NULL: tau_hat 25, exact mass).  Errors:
 * INVALID_ARG (NULL pointers, dim outside 1..2, empty direction, grid not
 * increasing, bc not 0/1), UNSUPPORTED (p outside 1..16, not sm_103, trace
 * above 2^31 - 1), CUDA, OOM.  *out owns device memory until
 * hdg_lowdim_destroy.                                                      */
hdg_status hdg_lowdim_setup(const hdg_lowdim_mesh* mesh, int p, const hdg_options* opts, hdg_lowdim** out);
size_t hdg_lowdim_trace_size(const hdg_lowdim* ctx);

/* y_r = K(lambda_r) x_r, r < nrhs, FP64, on `stream` (asynchronous; the
 * lambdas are copied before return).  d_x, d_y: device, nrhs blocks of
 * hdg_lowdim_trace_size() values, caller-owned, not overlapping; d_y is
 * overwritten.  basis: HDG_BASIS_NODAL (GLL nodal values on the faces) or
 * HDG_BASIS_TRANSFORMED (face eigenbasis S^-1 x per edge in 2D); in 1D the
 * faces are single points and both give the same K.  Errors: INVALID_ARG
 * (NULL pointers, nrhs outside 1..65535, lambda < 0 or not finite, bad
 * basis), CUDA.                                                            */
hdg_status hdg_lowdim_apply(hdg_lowdim* ctx, int nrhs, const double* h_lambda, hdg_basis basis, const double* d_x,
                            double* d_y, void* stream);
void hdg_lowdim_destroy(hdg_lowdim* ctx);

#ifdef __cplusplus
}
#endif
#endif /* HDG_GB300_H */
