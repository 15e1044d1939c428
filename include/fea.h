/*
 * fea.h - C ABI of libfea, a GB300 (sm_103a) finite element assembly engine
 * for P1/P2 tetrahedra.
 *
 * What the library computes is the assembled linear system of a weak form
 * (Cui, Guo & Liu, "GPU Accelerated Finite Element Assembly with Runtime
 * Compilation", Sec. 4.1):
 *   Eq. 1-2: the weak form  (grad v, sigma grad u) + lambda (v, u) = (v, f)
 *            with sigma = kappa I, kappa constant on each element, and
 *            lambda = mass_coef; and, on vector P1 elements, linear elasticity
 *            a(u, v) = int lambda div u div v + 2 mu eps(u):eps(v) with the
 *            Lame parameters constant on each element;
 *   Eq. 3:   A x = b, where A_ij sums the local entries of every element that
 *            holds dofs i and j, and b_i the local load entries of every
 *            element that holds dof i.
 * The input mesh is what Sec. 5 (Algorithm 1) takes: node coordinates plus
 * the global node indices of every element.  The matrix is returned in CSR
 * form, the compressed counterpart of the N x MAX_NZ sparse layout of the
 * sparse variant of Algorithm 1 (Sec. 5).
 *
 * Conventions that hold for every entry point:
 *  - Array arguments are DEVICE pointers owned by the caller unless a comment
 *    says otherwise.  8-byte arrays must be 8-byte aligned, 4-byte arrays
 *    4-byte aligned.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Calls are stream-ordered and asynchronous unless marked
 *    "synchronises".
 *  - Scalar dof numbering: P1 dofs are node ids; P2 dofs are node ids followed
 *    by one dof per mesh edge, the dof of edge (a, b), a < b, being
 *    n_nodes + the rank of (a, b) in lexicographic order over all edges.
 *    Vector (elasticity) dofs interleave components: dof = 3 * node + c.
 *    Element-local order: vertices v0..v3, then edges (0,1), (0,2), (0,3),
 *    (1,2), (1,3), (2,3).
 *  - CSR: int32 row_ptr[ndof + 1], int32 col_idx[nnz]; columns strictly
 *    ascending in each row; every pair of dofs that share an element is
 *    stored, zeros included.
 *  - Outputs are fully overwritten, never accumulated into.  No boundary
 *    conditions are applied (the paper's Neumann problem, Sec. 4.1).
 *  - The scatter into the CSR values is deterministic: repeated calls on the
 *    same inputs give bitwise identical results, and the matrix is bitwise
 *    symmetric.
 *  - Errors: every entry point returns an fea_status; nothing throws across
 *    the ABI.  fea_last_error() gives a message for the calling thread.
 *    Faults found on the device (an index out of range, det J <= 0, a row too
 *    long for the scatter) are latched in the mesh and returned by the next
 *    synchronising call or by fea_mesh_check.
 *  - A mesh handle is not thread-safe: use it from one host thread and one
 *    stream at a time.
 */
#ifndef FEA_H
#define FEA_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fea_mesh fea_mesh;   /* opaque, library-owned */
typedef struct fea_batch fea_batch; /* opaque, library-owned */

typedef enum {
  FEA_OK = 0,
  FEA_ERR_ARG = 1,        /* bad argument (NULL, size, alignment, unsupported combination) */
  FEA_ERR_INDEX = 2,      /* connectivity entry out of [0, n_nodes) or repeated in an element */
  FEA_ERR_DEGENERATE = 3, /* an element with det J <= 0 (values are still computed with |det J|) */
  FEA_ERR_OVERFLOW = 4,   /* nnz above INT32_MAX, or a row too long for the scatter (> 255 entries
                             per scalar row, or more than 1024 candidate couplings per scalar row) */
  FEA_ERR_NOMEM = 5,      /* device allocation failed */
  FEA_ERR_CUDA = 6,       /* a CUDA runtime call failed */
  FEA_ERR_TIMEOUT = 7,    /* a bounded device-side wait gave up */
  FEA_ERR_STATE = 8       /* call out of order (e.g. assemble before fea_pattern) */
} fea_status;

enum { FEA_P1 = 1, FEA_P2 = 2 };

/* Weak forms (Eq. 2 of the paper with sigma = kappa I, plus elasticity). */
enum {
  FEA_POISSON = 0,        /* -div(kappa grad u) = f                       */
  FEA_DIFFUSION_MASS = 1, /* -div(kappa grad u) + mass_coef u = f          */
  FEA_ELASTICITY = 2      /* -div sigma(u) = f, sigma = lambda tr(eps) I + 2 mu eps; P1 only */
};

/* Arithmetic of the element kernels. */
enum {
  FEA_FP64 = 0,  /* everything in FP64 */
  FEA_MIXED = 1  /* Jacobian, det J, J^{-1} and the CSR accumulation in FP64;
                    quadrature-point products (basis gradients, weights, f) in FP32 */
};

/* Load f. */
enum {
  FEA_LOAD_NONE = 0,    /* f = 0 (rhs written as zeros) */
  FEA_LOAD_CONST = 1,   /* scalar: f = p0; elasticity: f = (p0, p1, p2) */
  FEA_LOAD_SINPROD = 2  /* scalar: f = p0 sin(pi x) sin(pi y) sin(pi z); elasticity: component
                           c is p_c times the same product */
};

typedef struct {
  int32_t kind;      /* FEA_POISSON, FEA_DIFFUSION_MASS or FEA_ELASTICITY */
  int32_t order;     /* FEA_P1 or FEA_P2 */
  double mass_coef;  /* lambda of Eq. 1 (used by FEA_DIFFUSION_MASS) */
} fea_form;

typedef struct {
  const double* kappa;        /* [n_elems] per-element kappa, or NULL to use kappa_const */
  double kappa_const;
  const double* lame_lambda;  /* [n_elems] or NULL to use lambda_const (elasticity) */
  double lambda_const;
  const double* lame_mu;      /* [n_elems] or NULL to use mu_const (elasticity) */
  double mu_const;
  int32_t f_kind;             /* FEA_LOAD_* */
  double f_param[4];
} fea_coeffs;

typedef struct {
  int32_t npts; /* load-vector rule: 1 (centroid), 4 (degree 2) or 11 (Keast, degree 4).  The
                   matrix integrands are polynomials of degree <= 4 on affine elements with
                   element-constant coefficients and are integrated exactly. */
  int32_t prec; /* FEA_FP64 or FEA_MIXED */
} fea_quadrature;

/* Create a mesh handle.  Synchronises.
 *   x, y, z : [n_nodes] FP64 node coordinates (device).  REFERENCED, not
 *             copied: they must stay valid, and may be changed in place
 *             between calls (moving the nodes keeps every pattern valid).
 *   tets    : [4][n_elems] int32 connectivity, structure-of-arrays (vertex a
 *             of element e at tets[a * n_elems + e]); copied.
 * Validates the connectivity (FEA_ERR_INDEX).  *out receives the handle. */
fea_status fea_mesh_create(const double* x, const double* y, const double* z, int64_t n_nodes,
                           const int32_t* tets, int64_t n_elems, void* stream, fea_mesh** out);

/* Create a handle for a 2-D mesh of P1 triangles (the paper's worked example,
 * Sec. 4.1-4.2).  x, y: [n_nodes] FP64 node coordinates (device, referenced);
 * tris: [3][n_elems] int32 SoA connectivity, counter-clockwise (copied).
 * Only fea_pattern(mesh, FEA_P1, 1, ...) and fea_assemble_2d apply to it.
 * Synchronises; validates the connectivity (FEA_ERR_INDEX). */
fea_status fea_mesh_create_tri(const double* x, const double* y, int64_t n_nodes, const int32_t* tris,
                               int64_t n_elems, void* stream, fea_mesh** out);

/* Re-point the referenced coordinate arrays (same n_nodes). */
fea_status fea_mesh_set_coords(fea_mesh* mesh, const double* x, const double* y, const double* z);

/* Number of consecutive element chunks fea_assemble overlaps with the
 * scatter (1 to 16; default 1 = element kernel, then scatter kernel).
 * With k > 1, chunk c's element kernel runs on `stream` while the row tiles
 * completed by chunks < c are scattered on a stream owned by the handle,
 * joined back to `stream` before the call's work completes.  Results are
 * bitwise identical for every setting. */
fea_status fea_mesh_set_stages(fea_mesh* mesh, int32_t stages);

/* Scatter of fea_assemble (stages == 1), fea_assemble_noalloc,
 * fea_assemble_2d and fea_jit_assemble.  3 = the bulk-copy scatter: local rows
 * in the tile-interleaved layout, each row tile streamed into shared memory
 * by cp.async.bulk copies through a ring of mbarrier-completed stages (scalar forms;
 * elasticity falls back to 0).  The incidence-order scatters: 0 = one launch
 * of the two-deep pipelined kernel over all row tiles; 1 = tiles whose CSR
 * span exceeds half the widest in one such launch, the rest in a second
 * launch with a smaller shared-memory size and a one-deep kernel; 2 = one
 * launch of the one-deep kernel.  -1 (default) = automatic: 3 for scalar
 * forms, else 2 when the pattern mixes long and short rows, else 0.
 * Results are bitwise identical for every mode. */
fea_status fea_mesh_set_scatter_classes(fea_mesh* mesh, int32_t mode);

/* Scatter algorithm of fea_assemble (the paper has the shared-memory batch
 * plus global atomicAdd of Sec. 5, Algorithm 1; both algorithms here are
 * deterministic instead):
 *  FEA_SCATTER_LOCAL_ROWS: the element kernel writes every local row to HBM
 *    scratch and a row-gather kernel adds each CSR row's contributions in
 *    element order (all forms; the launch shapes above apply to it);
 *  FEA_SCATTER_CHUNKED: P1 elasticity only.  The elements are grouped into
 *    spatially compact chunks of at most 384; one CTA per chunk adds its
 *    elements' entries into shared memory as 64-bit fixed-point integers,
 *    one scale per node pair set from an exponent bound of the contributing
 *    elements (integer sums are exact, so the order of the additions cannot
 *    change the result), writes the couplings the chunk completes straight to
 *    the CSR values, and one FP64 partial sum per chunk for the couplings it
 *    shares, which a second kernel adds in chunk order.  Values agree with
 *    the local-row scatter to rounding (within the FP64 tolerance of the
 *    oracle), are bitwise reproducible and bitwise symmetric.  An element
 *    with non-finite inputs or det J = 0 makes the entries it touches NaN.
 *    The chunks are built (and the device synchronised) by the first chunked
 *    assembly of a mesh; a mesh whose chunks cannot be built (a grid cell of
 *    more than 1024 elements, a chunk too large for shared memory, a node
 *    pair in more than 128 elements of one chunk) reports FEA_ERR_OVERFLOW
 *    when this mode is requested;
 *  FEA_SCATTER_AUTO (default): chunked for P1 elasticity when its chunks can
 *    be built, the local-row scatter otherwise. */
enum { FEA_SCATTER_AUTO = 0, FEA_SCATTER_LOCAL_ROWS = 1, FEA_SCATTER_CHUNKED = 2 };
fea_status fea_mesh_set_scatter(fea_mesh* mesh, int32_t mode);

/* Shared-memory stages per CTA of the bulk-copy scatter (scatter mode 3):
 * 2, 3 or 4 steps of the row tile in flight per CTA; 0 (default) =
 * automatic, per launch the most resident CTAs per SM given the
 * accumulator's shared memory, and the fewest stages at that count.
 * Results are bitwise identical for every count. */
fea_status fea_mesh_set_scatter_stages(fea_mesh* mesh, int32_t stages);

/* Element launch of fea_assemble for scalar forms with a load vector (stages
 * == 1): 0 = one kernel computes the local matrix and the local load; 1 = a
 * matrix kernel, then a load kernel; 2 = the load kernel on a stream owned
 * by the handle, concurrent with the matrix kernel (joined back to
 * `stream`); 3 = one kernel whose blocks hold matrix warps and load warps of
 * the same elements (FP64; the mixed path takes 0); -1 (default) =
 * automatic: 3 for FP64 P2 with the sine load, 0 elsewhere (the fastest
 * measured).  Results are bitwise identical for every mode. */
fea_status fea_mesh_set_load_split(fea_mesh* mesh, int32_t mode);

/* Release the handle and everything it owns.  Synchronises the device. */
fea_status fea_mesh_destroy(fea_mesh* mesh);

/* Synchronise `stream` and return (then clear) any fault latched on the
 * device by earlier calls on this mesh. */
fea_status fea_mesh_check(fea_mesh* mesh, void* stream);

/* Build (once; cached in the handle) the global CSR sparsity pattern of the
 * given element order and dofs per node (1 for scalar forms, 3 for
 * elasticity), with the structures the deterministic scatter needs.
 * Synchronises.  Returns the number of dofs and nonzeros. */
fea_status fea_pattern(fea_mesh* mesh, int32_t order, int32_t dofs_per_node, int64_t* ndof,
                       int64_t* nnz, void* stream);

/* Copy a built pattern out: row_ptr [ndof + 1], col_idx [nnz] (device). */
fea_status fea_pattern_copy(fea_mesh* mesh, int32_t order, int32_t dofs_per_node,
                            int32_t* row_ptr, int32_t* col_idx, void* stream);

/* Copy the element -> scalar dof table of an order whose pattern is built:
 * [nb][n_elems] int32 SoA, nb = 4 (P1) or 10 (P2), local order as above. */
fea_status fea_dof_table_copy(fea_mesh* mesh, int32_t order, int32_t* edof, void* stream);

/* Assemble the CSR values and the load vector of a weak form (Eq. 3).
 *   values : [nnz] FP64 (device), overwritten; may not be NULL.
 *   rhs    : [ndof] FP64 (device), overwritten; may be NULL to skip the load.
 * The pattern of (form->order, 1 or 3 dofs per node) must have been built
 * with fea_pattern.  Asynchronous.  Per-call device scratch is owned by the
 * handle (allocated on first use, which synchronises once). */
fea_status fea_assemble(fea_mesh* mesh, const fea_form* form, const fea_coeffs* coeffs,
                        const fea_quadrature* quad, double* values, double* rhs, void* stream);

/* The 2-D weak form of Eq. 2 on P1 triangles:
 *   (grad v, sigma grad u) + lambda (v, u) = (v, f),
 *   sigma(x, y) = sigma0 + x sigma_x + y sigma_y  (2 x 2, row-major; need not
 *                 be symmetric - the paper's example is [[1, -x-y], [x+y, 1]]),
 *   f(x, y) = f0 + f1 x + f2 y + f3 x^2 + f4 x y + f5 y^2. */
typedef struct {
  double sigma0[4], sigma_x[4], sigma_y[4];
  double lambda;
  double f[6];
  int32_t npts; /* load rule on triangles: 1, 3 (degree 2) or 6 (degree 4) */
} fea_form2d;

/* Assemble the 2-D system (Eq. 3) on a triangle mesh: values [nnz], rhs
 * [n_nodes] (may be NULL) in FP64.  The stiffness and mass integrals are
 * exact (constant gradients, affine sigma); the load uses the rule npts.  A is
 * not symmetric when sigma is not; the scatter is the same deterministic one
 * as fea_assemble.  Asynchronous. */
fea_status fea_assemble_2d(fea_mesh* mesh, const fea_form2d* form, double* values, double* rhs,
                           void* stream);

/* fea_assemble without any device allocation (the paper has no counterpart;
 * this is a deployment variant).  For callers that cannot let a library
 * call cudaMalloc - a process whose device memory is reserved by another
 * allocator, or a latency-critical loop that cannot afford the device
 * synchronisation cudaMalloc/cudaFree imply.  Same arguments, argument
 * checks and results as fea_assemble with the local-row scatter (values
 * within the FP64 tolerance of the oracle, bitwise equal to fea_assemble
 * whenever fea_assemble uses the same element and scatter launches).  It
 * always runs the fused element kernel and the automatic local-row scatter:
 * the load-split, stage and scatter-algorithm settings of the mesh do not
 * apply to it.  The per-call scratch (local rows and local loads) lives in
 * one fixed 32 MiB device array inside the library instead of the mesh
 * handle: about 200 K P1 scalar elements, 32 K P2 elements or 25 K P1
 * elasticity elements in FP64.  Larger meshes are rejected with FEA_ERR_ARG
 * before anything runs, as are misaligned or NULL arguments.
 *  - The array is taken on a device by the first call there (CUDA loads the
 *    library's module lazily), when its address is looked up with
 *    cudaGetSymbolAddress, with that device current; make that first call
 *    before any stream capture and before another allocator reserves the
 *    device's memory (FEA_ERR_NOMEM otherwise).  The device then holds it
 *    until the process exits.
 *  - Every call shares the array and it keeps the last call's contents;
 *    nothing in it needs clearing (every value is written before it is read).
 *    Calls whose kernels overlap on the GPU (other streams, other threads)
 *    race on it: serialise them.
 *  - The pattern must have been built with fea_pattern beforehand. */
fea_status fea_assemble_noalloc(fea_mesh* mesh, const fea_form* form, const fea_coeffs* coeffs,
                                const fea_quadrature* quad, double* values, double* rhs, void* stream);

/* The paper's own sparse assembly (Sec. 5, Algorithm 1, sparse variant) as a
 * comparison point: same arguments and element arithmetic as fea_assemble
 * (FP64 only), but every local entry is added into the global CSR row with a
 * global FP64 atomicAdd after a linear search of the row for its column, and
 * every load entry into rhs the same way; values and rhs are zeroed first.
 * Allocates nothing.  The order of the additions depends on scheduling, so
 * results agree with fea_assemble to rounding only and are not reproducible
 * bit for bit. */
fea_status fea_assemble_atomic(fea_mesh* mesh, const fea_form* form, const fea_coeffs* coeffs,
                               const fea_quadrature* quad, double* values, double* rhs, void* stream);

/* Reverse mode of fea_assemble for the scalar forms (FEA_POISSON,
 * FEA_DIFFUSION_MASS; P1 or P2; FP64).  For a scalar loss L with
 * grad_values = dL/dvalues [nnz] and grad_rhs = dL/drhs [ndof] (either may be
 * NULL = zero), writes
 *   grad_kappa [n_elems] = dL/dkappa per element (may be NULL; needs a
 *                          per-element kappa to be meaningful);
 *   grad_x     [3][n_nodes] = dL/d(x, y, z) per node, SoA (may be NULL).
 * Local matrices are recomputed, never stored.  Deterministic. */
fea_status fea_assemble_backward(fea_mesh* mesh, const fea_form* form, const fea_coeffs* coeffs,
                                 const fea_quadrature* quad, const double* grad_values,
                                 const double* grad_rhs, double* grad_kappa, double* grad_x,
                                 void* stream);

/* ---- Batched assembly of many independent meshes (no counterpart in the
 * paper; it batches the per-mesh work of Eq. 3 / Algorithm 1).
 *
 * Create a batch over n mesh handles (which stay owned by the caller and
 * must outlive the batch).  forms[k], quads[k] give mesh k's scalar form
 * (FEA_POISSON or FEA_DIFFUSION_MASS, P1 or P2, FP64); every P1 mesh must use
 * the same rule and every P2 mesh the same rule, with (P1, P2) rules in
 * {(4, 11), (11, 11), (4, 4)}; f_kind is the load kind shared by all meshes.
 * Builds each mesh's pattern if needed and allocates the batch's scratch.
 * Synchronises. */
fea_status fea_batch_create(fea_mesh* const* meshes, int32_t n, const fea_form* forms,
                            const fea_quadrature* quads, int32_t f_kind, void* stream,
                            fea_batch** out);

/* Bind per-mesh coefficients and outputs.  coeffs: host array [n] (kappa
 * pointers are device arrays); values, rhs: HOST arrays [n] of DEVICE
 * pointers ([nnz_k] and [ndof_k] doubles; rhs may be NULL, or hold NULL
 * entries, to skip loads).  Copies the descriptors to the device;
 * synchronises.  The bound pointers are used by every later
 * fea_batch_assemble until the next bind. */
fea_status fea_batch_bind(fea_batch* batch, const fea_coeffs* coeffs, double* const* values,
                          double* const* rhs);

/* Assemble every mesh of the batch: one launch of an internal CUDA graph
 * with two branches that may run concurrently, one for the P2 meshes and one
 * for the P1 meshes, each a persistent element kernel over all of its meshes
 * followed by the row-tile scatter kernels.  Asynchronous on `stream`;
 * allocates nothing.  Each mesh's values and rhs are bitwise those of
 * fea_assemble. */
fea_status fea_batch_assemble(fea_batch* batch, void* stream);

/* Autotune the batch's launch: times candidate (elements per work item,
 * P2 element-kernel CTAs) pairs on the device, then, per order, the element
 * kernel's variant with its CTA count; keeps the fastest and rebuilds the
 * graph.  params (may be NULL) receives int32_t[6]: the
 * chosen elements per item, P2 and P1 element-kernel CTAs, the scatter CTA
 * count (one per row tile), and the P2 and P1 element-kernel variants (0: the
 * compiler's register count; 1: capped for the single-mesh residency; 2, P2
 * with the sine load only: matrix warps and load warps in one CTA).
 * Synchronises; overwrites the bound outputs. */
fea_status fea_batch_tune(fea_batch* batch, void* stream, int32_t* params);

/* Release the batch (not the meshes).  Synchronises the device. */
fea_status fea_batch_destroy(fea_batch* batch);

/* Measurement hooks (no counterpart in the paper; used by the benchmark).
 * When enabled, every fea_assemble on this mesh records CUDA events on its
 * stream before the element kernel, between the element kernel and the
 * scatter kernel, and after the scatter kernel. */
fea_status fea_profile_enable(fea_mesh* mesh, int32_t enable);

/* Wait for the events of the last profiled fea_assemble and return the
 * durations (ms) of its element kernel and of its scatter kernel.
 * FEA_ERR_STATE if no profiled call was made. */
fea_status fea_profile_last(fea_mesh* mesh, float* elem_ms, float* scatter_ms);

/* Self-check of the FP64-accurate sin(pi x) helpers (no counterpart in the
 * paper): for x [n] (device) writes the helper's value to mine [n] and CUDA's
 * sinpi to lib [n].  variant 0: the fixed-point evaluation the element
 * kernels use (sinpi_fx); 1: the FP64-pipe polynomial (its fallback for tiny,
 * huge and non-finite arguments, and the sinpi_fp64 of runtime-compiled
 * expressions); 2: the fixed-point value with 62 fractional bits the FP64
 * load vectors multiply and sum on the integer pipes (sinpi_q62), converted;
 * 3: the same value from x in fixed point, x 2^(61 - s) with s set by |x|
 * (to_fx, sinpi_q62_fx: the path of the FP64 sine loads, whose quadrature
 * points are formed in fixed point), for |x| < 2^58.  Asynchronous. */
fea_status fea_diag_sinpi(const double* x, int64_t n, int32_t variant, double* mine, double* lib, void* stream);

/* Self-check of the FP64 reciprocal the element kernels scale their
 * gradient products with (no counterpart in the paper; 1 / (6 |det J|) of
 * Eq. 3's |T| grad phi_a . grad phi_b): for x [n] (device) writes the helper's
 * 1 / x (an FP32 seed and one third-order Newton step; within one ulp) to
 * mine [n] and CUDA's division 1.0 / x to lib [n].  Asynchronous;
 * FEA_ERR_ARG for n < 0 or NULL arrays with n > 0. */
fea_status fea_diag_rcp(const double* x, int64_t n, double* mine, double* lib, void* stream);

/* Failure-path check of the bounded device waits: one warp waits, with the
 * bulk-copy scatter's bounded mbarrier wait, on a barrier whose expected
 * arrival never comes, gives up after `polls` polls (1 to 2^20) and raises
 * the timeout bit in the mesh's device error word; the next fea_mesh_check
 * returns FEA_ERR_TIMEOUT and clears it.  Nothing else is touched and the
 * context stays usable.  Asynchronous. */
fea_status fea_diag_wait_timeout(fea_mesh* mesh, int32_t polls, void* stream);

/* Failure-path check of the bounds-checked build (libfea_checked.so, built
 * with -DFEA_CHECKED; see build_lib.py): *checked receives 1 for that build,
 * 0 otherwise.  In the checked build one thread reads src[idx] (device) into
 * out[0] (device) through the same check as the library's gathers: with idx
 * outside [0, n) nothing is read, out[0] receives -1 and DEV_ERR_INDEX is
 * latched in the mesh's error word (the next fea_mesh_check returns
 * FEA_ERR_INDEX and clears it).  The normal build launches nothing (it would
 * read unchecked).  Asynchronous. */
fea_status fea_diag_checked_gather(fea_mesh* mesh, const double* src, int64_t n, int64_t idx, double* out,
                                   int32_t* checked, void* stream);

/* Measure the device's sustained FP64 FMA throughput (flop/s, FMA = 2)
 * with independent DFMA chains on every SM.  Synchronises. */
fea_status fea_diag_fp64_rate(double* flops_per_s, void* stream);

/* ---------------------------------------------------------------- runtime specialisation
 * Sec. 5 (runtime compilation): the paper turns the user's weak form into
 * kernel source and compiles it with NVRTC while the program runs.  Here the
 * user gives two CUDA C++ expressions of type double in the variables x, y, z
 * (the physical point), the parameters p0..p3 (fea_coeffs.f_param at
 * assembly time) and the constant pi, using CUDA's device math functions
 * (sin, exp, pow, sinpi, ...) and the library's sin(pi v) helpers sinpi_fx (on
 * the integer pipes, within 0.51 ulp) and sinpi_fp64 (on the FP64 pipe):
 *   kappa_expr : k(x) inside the stiffness integral, -div(kappa_T k(x) grad u)
 *                with kappa_T from fea_coeffs (per element or constant);
 *                NULL means k = 1;
 *   f_expr     : the load f(x); NULL means no load vector.
 * Expressions may not contain ; { } # quotes, backslashes or comments.
 * Integrals use the rule quad->npts: the stiffness as
 * sum_q w_q |T| kappa_T k(x_q) grad phi_a . grad phi_b (exact, whatever the
 * rule, when k is NULL), the load as sum_q w_q |T| f(x_q) phi_a; the mass
 * term (FEA_DIFFUSION_MASS, form->mass_coef) is exact.  quad->prec selects
 * FP64 or the mixed split (quadrature products in FP32).  Scalar forms only
 * (FEA_POISSON, FEA_DIFFUSION_MASS), P1 or P2 tetrahedra. */
typedef struct fea_jit fea_jit;

/* Compile (NVRTC, host only: no GPU needed) the element kernel for the
 * expressions and return a handle owning its sm_103a cubin.  Compiled
 * sources are cached per process: the same specialisation compiles once.
 * FEA_ERR_ARG with the compiler log in fea_last_error if they do not compile. */
fea_status fea_jit_compile(const fea_form* form, const fea_quadrature* quad, const char* kappa_expr,
                           const char* f_expr, fea_jit** out);

/* Wall time of the fea_jit_compile call (ms), cubin size, and whether it was
 * served from the process cache (1) or compiled (0).  NULL outputs skipped. */
fea_status fea_jit_info(const fea_jit* jit, double* compile_ms, int64_t* cubin_bytes, int32_t* cache_hit);

/* Generated kernel source and NVRTC log of a handle (owned by the handle). */
const char* fea_jit_source(const fea_jit* jit);
const char* fea_jit_log(const fea_jit* jit);

/* Assemble with a compiled handle: CSR values [nnz] and, iff the handle has
 * an f expression, the load rhs [ndof] (both FP64, device, overwritten).
 * The pattern of (order, 1) must be built.  The first call loads the cubin
 * (synchronises once); later calls are asynchronous. */
fea_status fea_jit_assemble(fea_mesh* mesh, fea_jit* jit, const fea_coeffs* coeffs, double* values, double* rhs,
                            void* stream);

/* Release a handle (and its loaded module). */
fea_status fea_jit_destroy(fea_jit* jit);

/* ---------------------------------------------------------------- solving
 * The step after assembly (the paper assembles the pure Neumann operator and
 * leaves solving out, Sec. 2).  Both calls work on the CSR pattern of
 * (order, dofs_per_node), which must be built. */

/* Dirichlet conditions u_d = g_d by symmetric elimination, in place:
 *   dofs   : [n] int32 dof ids (device), any order, repeats allowed; an id
 *            outside [0, ndof) latches FEA_ERR_INDEX (fea_mesh_check);
 *   g      : [n] FP64 values (device), or NULL for zero;
 *   values : [nnz] CSR values (device): row d becomes the identity row,
 *            column d of every other row is zeroed (A stays symmetric);
 *   rhs    : [ndof] (device): rhs_d = g_d, rhs_i -= A_id g_d for the other
 *            rows; may be NULL.
 * Asynchronous.  Scratch (ndof doubles + bytes) is owned by the handle. */
fea_status fea_dirichlet(fea_mesh* mesh, int32_t order, int32_t dofs_per_node, const int32_t* dofs, int64_t n,
                         const double* g, double* values, double* rhs, void* stream);

/* Solve A x = b with conjugate gradients and the Jacobi preconditioner
 * (A symmetric positive definite, e.g. after fea_dirichlet).
 *   values : [nnz] CSR values, b : [ndof], x : [ndof] (device, FP64); x holds
 *            the initial guess and receives the solution;
 *   stops at ||b - A x||_2 <= rtol ||b||_2 (rtol ||.|| of 1 when b = 0) or
 *   after max_iter iterations; *iters and *rel_res (= ||r|| / ||b||) may be NULL.
 * Every reduction has a fixed order: the same inputs give bitwise the same x.
 * Runs on the handle's own stream after the work queued on `stream`, and
 * synchronises (the host checks convergence every 16 iterations).
 * FEA_ERR_ARG if p.Ap <= 0 occurs (A not positive definite). */
fea_status fea_cg(fea_mesh* mesh, int32_t order, int32_t dofs_per_node, const double* values, const double* b,
                  double* x, double rtol, int32_t max_iter, int32_t* iters, double* rel_res, void* stream);

/* ---------------------------------------------------------------- several GPUs
 * Row partition of a P1 tetrahedral mesh (the paper assembles one mesh on one
 * GPU, Sec. 5; this splits the same element-parallel assembly by rows).  Part
 * `part` of `nparts` owns the nodes [lo, hi), lo = floor(part N / nparts),
 * hi = floor((part + 1) N / nparts) (for node ids that run z-slowest, as on
 * the cube meshes, a z-slab), and takes every element with a vertex in that
 * range: its own elements and the ghost layer it shares with its neighbours.
 * Assembled on its own, that sub-mesh gives the complete rows of every owned
 * node - the rows of the whole mesh's matrix, with no exchange between parts:
 * nodes are renumbered in ascending global order (so each row's columns stay
 * in the same order) and elements keep their ascending order (so the
 * local-row scatter adds each entry's contributions in the same order and
 * the owned rows are bitwise those of the whole mesh).  P1 patterns only
 * (scalar or 3 dofs per node); the owned rows of the sub-mesh are those of
 * its local nodes [a, b) with nodes[a] = lo, nodes[b - 1] = hi - 1.
 *   tets       : [4][n_elems] int32 connectivity, HOST memory;
 *   node_lo/hi : receive lo, hi;  n_sub_elems / n_sub_nodes: the sub-mesh sizes;
 *   elems      : [n_sub_elems] the global ids of its elements, ascending, or NULL;
 *   nodes      : [n_sub_nodes] the global ids of its nodes, ascending (the
 *                nodes of its elements and every owned node), or NULL;
 *   sub_tets   : [4][n_sub_elems] its connectivity in local node numbers, or NULL.
 * All arrays are host memory owned by the caller: call once with NULL arrays
 * for the sizes, then with arrays of those sizes.  Host only (no CUDA call,
 * no GPU needed); deterministic.  FEA_ERR_INDEX for a node id out of range. */
fea_status fea_partition(const int32_t* tets, int64_t n_elems, int64_t n_nodes, int32_t nparts, int32_t part,
                         int64_t* node_lo, int64_t* node_hi, int64_t* n_sub_elems, int64_t* n_sub_nodes,
                         int32_t* elems, int32_t* nodes, int32_t* sub_tets);

/* Independent meshes of a batch (the batched assembly of fea_batch_create)
 * spread over `nparts` GPUs with no exchange: no mesh is split, each part
 * assembles its own meshes as a batch of its own.  The paper has no batched
 * form; this is longest processing time first (Graham's list scheduling):
 * the meshes in order of decreasing cost (equal costs by index), each to the
 * part whose total cost is lowest so far (equal totals: the lowest part), so
 * the largest total is at most 4/3 of the best possible.
 *   cost    : [n] the caller's cost estimate of each mesh (for example its
 *             element count weighted by the element order), finite, >= 0;
 *   part_of : [n] receives the part of each mesh;
 *   load    : [nparts] receives each part's total cost, or NULL.
 * Host memory owned by the caller; host only (no CUDA call); deterministic.
 * FEA_ERR_ARG for n < 0, nparts < 1, a NULL array or a negative or
 * non-finite cost. */
fea_status fea_partition_batch(const double* cost, int32_t n, int32_t nparts, int32_t* part_of, double* load);

/* Message for the last error on the calling thread ("" if none). */
const char* fea_last_error(void);

/* Name of a status code. */
const char* fea_status_string(fea_status status);

#ifdef __cplusplus
}
#endif

#endif /* FEA_H */
