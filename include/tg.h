/*
 * tg.h — C ABI of the GB300 Galerkin-assembly library (libtg.so).
 *
 * The library computes the two stages of TensorGalerkin's assembly on one
 * GPU: the Map (per-element local matrices and vectors by quadrature,
 * Eq. (kloc1), Algorithm 1, concrete form Eq. (matlclquad) of SM A.2) and the
 * Reduce (sum of the local entries into a CSR matrix and a vector over the
 * mesh-induced sparsity graph, Algorithm 2), plus the reverse-mode gradients
 * of the assembled values (the adjoint relations of Eq. (adj)).
 *
 * Conventions shared by every call
 * --------------------------------
 * - Array arguments are DEVICE pointers owned by the caller, unless a
 *   parameter says "host".  Outputs are overwritten, never accumulated
 *   (except where a flag says so).  Element arrays are row-major:
 *   cells[e][a], coords[node][d], kappa[e][q].
 * - Floating-point arrays use the dtype argument (TG_F32: float,
 *   TG_F64: double) for coordinates, coefficients and outputs alike.
 * - Calls are asynchronous on the given stream (a cudaStream_t; NULL is the
 *   legacy default stream) unless documented as synchronising.  Nothing
 *   allocates or synchronises on the assembly path, so those calls may be
 *   captured in a CUDA graph.
 * - Host-side validation (null pointers, sizes, enum values, a pattern of
 *   another element kind) returns an error before any GPU work.
 *   Data-dependent problems found on the device (an index outside
 *   [0, n_nodes), a degenerate element with |det J| ~ 0) are recorded in the
 *   pattern's device status word and read with tg_get_device_status().
 *   No call aborts, traps or prints.
 * - Reference elements: the triangle {x, y >= 0, x + y <= 1} of SM A.2 and
 *   its 3D analogue.  Quadrature: 3-point degree-2 rule for P1 triangles,
 *   6-point degree-4 (Dunavant) rule for P2 triangles, 4-point degree-2 rule
 *   for tetrahedra; per-point coefficient arrays follow those rules' point
 *   order (documented in the design notes and in tg_quadrature()).
 * - P2 triangles carry 6 nodes per element: the 3 vertices, then the edge
 *   nodes of edges (0,1), (1,2), (2,0).  Geometry uses the vertices only
 *   (straight-sided elements).
 * - Vector elasticity numbers DoFs as 3 * node + component.
 * - The CSR pattern holds every pair (i, j) of nodes sharing an element,
 *   columns sorted ascending, structural zeros kept, int32 indices.
 * - Determinism: for a fixed pattern every forward and backward call is
 *   bitwise reproducible from run to run (each output is summed in a fixed
 *   order that the pattern determines: incident elements by increasing
 *   element index, or, for P1 triangle meshes whose every node has a single
 *   fan of triangles, the order of that fan, each off-diagonal entry being
 *   the sum of its two terms).  The only exception is
 *   tg_assemble_bilinear_atomic, the atomicAdd comparison variant.
 */
#ifndef TG_H_
#define TG_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* A CUDA stream (identical to cudaStream_t / CUstream). */
typedef struct CUstream_st* tg_stream;

typedef enum {
  TG_OK = 0,
  TG_ERR_INVALID_ARG = 1,        /* null pointer, bad size or enum, mismatched pattern */
  TG_ERR_INDEX_RANGE = 2,        /* a cell index outside [0, n_nodes) */
  TG_ERR_DEGENERATE_ELEMENT = 3, /* repeated vertex or |det J| below the dtype's threshold */
  TG_ERR_INDEX_OVERFLOW = 4,     /* nnz or an index would exceed 2^31 - 1 */
  TG_ERR_OUT_OF_MEMORY = 5,      /* a device allocation inside a pattern/batch build failed */
  TG_ERR_CUDA = 6,               /* a CUDA runtime call failed; see tg_last_error_message() */
  TG_ERR_TIMEOUT = 7,            /* a bounded device-side wait ran out */
  TG_ERR_UNSUPPORTED = 8         /* a limit of this implementation (e.g. row length > 255) */
} tg_status;

typedef enum {
  TG_P1_TRI = 0,      /* linear triangle,      3 nodes, d = 2 */
  TG_P2_TRI = 1,      /* quadratic triangle,   6 nodes, d = 2 */
  TG_P1_TET = 2,      /* linear tetrahedron,   4 nodes, d = 3 */
  TG_P1_TET_VEC3 = 3, /* linear tetrahedron, 3 DoF per node (elasticity), d = 3 */
  TG_Q1_QUAD_VEC2 = 4  /* bilinear quadrilateral, 2 DoF per node (plane stress), d = 2 */
} tg_element;

typedef enum { TG_F32 = 0, TG_F64 = 1 } tg_dtype;

typedef enum {
  TG_PER_ELEMENT = 0, /* one value per element:           [E]      */
  TG_PER_QP = 1,      /* one value per quadrature point:  [E][Q]   */
  TG_PER_NODE = 2,    /* one value per node:              [N]      */
  TG_CONSTANT = 3     /* one value for the whole mesh:    [1]      */
} tg_layout;

typedef struct tg_pattern tg_pattern; /* opaque; owns its device buffers */
typedef struct tg_batch tg_batch;     /* opaque; owns its device buffers */
typedef struct tg_facets tg_facets;   /* opaque; owns its device buffers */

/* ------------------------------------------------------------------------
 * Status and diagnostics
 * ---------------------------------------------------------------------- */

/* Human-readable name of a status code (static storage). */
const char* tg_status_string(tg_status s);

/* Text of the last TG_ERR_CUDA raised on the calling host thread. */
const char* tg_last_error_message(void);

/* Number of quadrature points of an element kind and, when w / xhat are
 * non-NULL (host arrays of Q and Q*d doubles), the weights and reference
 * points in the order per-point coefficient arrays use. */
int32_t tg_quadrature(tg_element el, double* w, double* xhat);

/* ------------------------------------------------------------------------
 * Stage II routing: the sparsity pattern (Algorithm 2's routing matrices
 * S_mat, S_vec and CSR indices "precomputed based solely on mesh topology").
 * ---------------------------------------------------------------------- */

/* Build the pattern of a mesh on the device.
 *   cells     device int32 [n_elems][nv] (nv = 3, 6, 4, 4 by element kind);
 *             copied, so the caller may free it afterwards.
 *   n_elems   >= 0 (an empty mesh gives an empty pattern); n_nodes >= 1.
 *   out       receives a new pattern; release it with tg_pattern_destroy().
 * Allocates device memory and SYNCHRONISES the stream.  Index errors and
 * repeated vertices are returned directly (TG_ERR_INDEX_RANGE,
 * TG_ERR_DEGENERATE_ELEMENT, *out stays NULL); tg_last_error_message()
 * names the smallest offending element.
 * Rows longer than 255 entries return TG_ERR_UNSUPPORTED. */
tg_status tg_build_pattern(const int32_t* cells, int64_t n_elems, int64_t n_nodes, tg_element el,
                           tg_stream stream, tg_pattern** out);

/* Borrowed device views of a pattern (valid until tg_pattern_destroy).
 *   n_rows, nnz   CSR size (DoF level for TG_P1_TET_VEC3: 3N rows, 9 nnz_node)
 *   row_ptr       int32 [n_rows + 1];  col_idx  int32 [nnz]
 *   elem_slot     int32 [E][nv][nv]: CSR position of local entry (a, b); for
 *                 TG_P1_TET_VEC3 the position of DoF entry (3a+0, 3b+0), the
 *                 entry (3a+i, 3b+j) sits at elem_slot + i*3*len(g_a) + j with
 *                 len(g_a) the node-row length (row_ptr[3g+1]-row_ptr[3g])/3.
 *   slot_stride   nv * nv.
 * Any output pointer may be NULL. */
tg_status tg_pattern_info(const tg_pattern* p, int64_t* n_rows, int64_t* nnz, const int32_t** row_ptr,
                          const int32_t** col_idx, const int32_t** elem_slot, int32_t* slot_stride);

/* Shape of a pattern: element kind, element and node counts, the longest
 * node row and the largest number of elements sharing a node. */
tg_status tg_pattern_shape(const tg_pattern* p, tg_element* el, int64_t* n_elems, int64_t* n_nodes,
                           int32_t* max_row_len, int32_t* max_degree);

/* Row blocks of a pattern (the data layout of the element-once kernels, no
 * counterpart in the paper).  *rows_per_block receives the rows a block owns
 * and *n_blocks the block count; both are 0 when the pattern has none (an
 * empty mesh, rows longer than 16 entries (32 for P2), or a block whose
 * vertex ids span 2^16 or more, e.g. a random node numbering), in which case
 * the generic row-owner kernels serve every call.  Either pointer may be NULL. */
tg_status tg_pattern_row_blocks(const tg_pattern* p, int32_t* rows_per_block, int64_t* n_blocks);

/* The optional layouts a pattern was built with (no counterpart in the
 * paper), as the OR of these flags in *flags: row blocks (see above); fans,
 * the fan-ordered Reduce of P1 and P2 triangles (built with row blocks when
 * every node's triangles form one fan); packed positions (elem_pos, the
 * backward's upstream-weight gather); elasticity edge masks (the two-pass
 * FP32 elasticity forward).  They select the kernels that serve a call;
 * results do not depend on them beyond the documented summation orders.
 * Returns TG_ERR_INVALID_ARG for a NULL argument. */
#define TG_LAYOUT_ROW_BLOCKS 1u
#define TG_LAYOUT_FANS 2u
#define TG_LAYOUT_ELEM_POS 4u
#define TG_LAYOUT_EDGE_MASKS 8u
tg_status tg_pattern_layouts(const tg_pattern* p, uint32_t* flags);

/* Read and clear the device status word of a pattern.  SYNCHRONISES the
 * device.  Returns TG_OK or the first recorded data error; *first_bad_elem
 * (may be NULL) gets the smallest offending element index, or -1. */
tg_status tg_get_device_status(const tg_pattern* p, int64_t* first_bad_elem);

void tg_pattern_destroy(tg_pattern* p);

/* ------------------------------------------------------------------------
 * Forward assembly: fused Map + deterministic Reduce (Eq. (matlclquad),
 * Algorithms 1 and 2).
 * ---------------------------------------------------------------------- */

/* Scalar bilinear form a(u, v) = int kappa grad u . grad v + c u v
 * (Eq. (matlclquad) with the mass term of SM A.1):
 *   vals[s] = sum over elements e and local pairs (a, b) routed to slot s of
 *             sum_q w_q |det J_e| ( kappa_eq G_qa . G_qb + c phi_a(x_q) phi_b(x_q) ).
 *   coords      [N][d]; kappa per kappa_layout (PER_QP, PER_ELEMENT or
 *               CONSTANT); vals_out [nnz] (node-level CSR of the pattern).
 * Element kinds TG_P1_TRI, TG_P2_TRI, TG_P1_TET.  On meshes of at least
 * 65,536 elements, FP64 calls on P1 elements and FP32 calls on P1
 * tetrahedra go through the pattern's per-element scratch (each element
 * evaluated once, then reduced; the same bits as one pass): such calls on
 * one pattern that overlap (several streams) race, as do the corresponding
 * tg_assemble_system calls. */
tg_status tg_assemble_bilinear(const tg_pattern* p, tg_dtype dtype, const void* coords, const void* kappa,
                               tg_layout kappa_layout, double c, void* vals_out, tg_stream stream);

/* Same result through the classic scatter-add with atomicAdd (Eq.
 * (scatter_add)): one thread per element, atomics into vals_out after a
 * clear.  Kept as the comparison point; summation order, hence the last
 * bits, vary from run to run. */
tg_status tg_assemble_bilinear_atomic(const tg_pattern* p, tg_dtype dtype, const void* coords,
                                      const void* kappa, tg_layout kappa_layout, double c, void* vals_out,
                                      tg_stream stream);

/* Vector P1 linear elasticity, int lambda div u div v + 2 mu eps(u):eps(v)
 * (Hooke's law, SM B.1 Benchmark II):
 *   K[(a,i),(b,j)] = sum_q w_q |det J| ( lam_q g_ai g_bj + mu_q g_aj g_bi + mu_q delta_ij g_a . g_b ).
 *   lam, mu     per layout (PER_ELEMENT, PER_QP or CONSTANT); vals_out [9 nnz_node]
 *               in the DoF-level CSR.  Pattern kind TG_P1_TET_VEC3.
 * The element terms go through the pattern's per-element scratch (computed
 * once per element) in FP64, and in both precisions when the mesh's rows
 * hold at most 16 nodes and its nodes at most 32 elements: such calls on one
 * pattern that overlap (several streams) race. */
tg_status tg_assemble_elasticity(const tg_pattern* p, tg_dtype dtype, const void* coords, const void* lam,
                                 const void* mu, tg_layout layout, void* vals_out, tg_stream stream);

/* The linear system of one scalar problem in one pass: the CSR values of
 * tg_assemble_bilinear and the load vector of tg_assemble_load (ncomp = 1)
 * together, as the Map of Algorithm 1 computes an element's local matrix and
 * load vector together.  Same arguments as those two calls, same outputs,
 * bitwise; on P1 meshes with row blocks one kernel shares the geometry and
 * the streams of both, otherwise the two assemblies run one after the other.
 * vals_out [nnz], F_out [N]. */
tg_status tg_assemble_system(const tg_pattern* p, tg_dtype dtype, const void* coords, const void* kappa,
                             tg_layout kappa_layout, double c, const void* f, tg_layout f_layout, void* vals_out,
                             void* F_out, tg_stream stream);

/* Load vector (second line of Eq. (matlclquad)):
 *   F[g(a) * ncomp + k] = sum_e sum_q w_q |det J_e| f_k(x_q) phi_a(x_q).
 *   f layouts: PER_NODE [N][ncomp] (f is its finite-element interpolant),
 *   PER_QP [E][Q][ncomp], CONSTANT [ncomp].  ncomp = 1 or 3.
 *   F_out [N * ncomp]. */
tg_status tg_assemble_load(const tg_pattern* p, tg_dtype dtype, const void* coords, const void* f,
                           tg_layout f_layout, int32_t ncomp, void* F_out, tg_stream stream);

/* Matrix-free residual of the Galerkin system, the vector inside the
 * physics-informed loss of Eq. (res1), without storing K:
 *   y[i] = sum_e sum_b K_e[a][b] x[g(b)] - F[i]        (i = g(a)),
 * with K_e the local matrix of tg_assemble_bilinear (kappa, kappa_layout, c)
 * and F the load vector of tg_assemble_load (f, f_layout, ncomp = 1); with
 * f == NULL there is no load term (y = K x).
 *   dirichlet  uint8 [N] or NULL: y[i] = 0 where dirichlet[i] != 0 (the rows
 *              the reduced system drops; x holds the boundary values there).
 *   loss       device scalar of dtype, or NULL: sum_i y[i]^2, summed in FP64
 *              in a fixed order.
 *   x, y [N]   distinct buffers (TG_ERR_INVALID_ARG otherwise).
 * Elements P1_TRI, P2_TRI, P1_TET; the load term on P1 only
 * (TG_ERR_UNSUPPORTED for P2 with f).  Deterministic: every y[i] sums its
 * element results in increasing element order.  Uses the pattern's per-
 * element scratch and partial-sum buffers (the latter like
 * tg_assemble_backward): calls on one pattern that overlap (several
 * streams) race.
 * Reverse mode, for an upstream gradient gy of y that is zero on Dirichlet
 * rows: dL/dx = K gy (this call with x = gy, f = NULL; K is symmetric);
 * dL/dkappa, dL/dc and the K part of dL/dcoords from tg_assemble_backward
 * with lam = gy, U = x; dL/df and the F part of dL/dcoords from
 * tg_assemble_load_backward with grad_F = -gy. */
tg_status tg_residual(const tg_pattern* p, tg_dtype dtype, const void* coords, const void* kappa,
                      tg_layout kappa_layout, double c, const void* x, const void* f, tg_layout f_layout,
                      const uint8_t* dirichlet, void* y, void* loss, tg_stream stream);

/* The residual of a semilinear time step (method of lines, SM: M dU/dt +
 * K U + F_nonlin(U) = F_ext), tg_residual plus a reaction term:
 *   y[i] = (K x)[i] + N[i] - F[i],
 *   N[i] = sum_e sum_q w_q |det J_e| s_q phi_a(x_q),   u_q = sum_b phi_b(x_q) x_b,
 * with s_q = r(u_q), r(u) = reaction[0] + reaction[1] u + reaction[2] u^2 +
 * reaction[3] u^3 (host array of 4), when x_react is NULL; with x_react
 * ([N], the state of a linearisation) s_q = r'(ur_q) u_q, ur_q the same
 * interpolation of x_react: the reaction's Jacobian at x_react applied to
 * x.  The element's own rule (the points of tg_quadrature) integrates both.
 * Backward Euler for du/dt = div(a^2 grad u) - r(u):
 *   (1/dt) M (U1 - U0) + a^2 K U1 + N(U1) = this call with kappa = a^2,
 *   c = 1/dt, x = U1, f = U0 / dt (PER_NODE: F = M f).
 * Reverse mode: dL/dx = K gy + J(x) gy (this call with x = gy, f = NULL,
 * x_react = x).  Other arguments, errors and determinism as tg_residual. */
tg_status tg_semilinear_residual(const tg_pattern* p, tg_dtype dtype, const void* coords, const void* kappa,
                                 tg_layout kappa_layout, double c, const void* x, const void* f, tg_layout f_layout,
                                 const double* reaction, const void* x_react, const uint8_t* dirichlet, void* y,
                                 void* loss, tg_stream stream);

/* r(u_q) at the quadrature points of every element, out [E][Q] (the
 * element's rule), u_q = sum_b phi_b(x_q) x[g(b)], r as in
 * tg_semilinear_residual.  As the per-point load f of
 * tg_assemble_load_backward (grad_F = the upstream gradient of y) it gives
 * the reaction term's coordinate gradient: only |det J| depends on the
 * coordinates. */
tg_status tg_reaction_points(const tg_pattern* p, tg_dtype dtype, const void* x, const double* reaction, void* out,
                             tg_stream stream);

/* ------------------------------------------------------------------------
 * Backward (reverse mode) of the scalar bilinear assembly.
 * For an upstream gradient W of the assembled values, either
 *   grad_vals [nnz]  (W_ab^e = grad_vals[slot(e, a, b)], the transpose of the
 *                     routing, S_mat^T), or
 *   lam, U    [N]    (W_ab^e = lam[g_a] U[g_b]: the adjoint outer product
 *                     dGamma/dK = lam U^T of Eq. (adj)) when grad_vals is NULL,
 * computes the gradients of L = sum_s W_s vals_s:
 *   grad_kappa  same layout as kappa (PER_QP, PER_ELEMENT or CONSTANT), or NULL;
 *   grad_coords [N][d], or NULL;
 *   grad_c      device scalar of dtype, or NULL.
 * All outputs are overwritten; sums run in a fixed order (deterministic).
 * Uses the pattern's partial-sum buffers and, for tetrahedra and in FP64,
 * its per-element scratch: calls on one pattern that overlap (several
 * streams) race. */
tg_status tg_assemble_backward(const tg_pattern* p, tg_dtype dtype, const void* coords, const void* kappa,
                               tg_layout kappa_layout, double c, const void* grad_vals, const void* lam,
                               const void* U, void* grad_kappa, void* grad_coords, void* grad_c,
                               tg_stream stream);

/* Backward of the vector P1 elasticity assembly (tg_assemble_elasticity;
 * the SM form with lambda div u div v + 2 mu eps(u):eps(v)).  For an upstream
 * gradient W of the DoF-level values, either
 *   grad_vals [nnz of the DoF-level CSR], or
 *   lam_adj, U [3 N]  (W = lam_adj U^T, Eq. (adj)) when grad_vals is NULL,
 * computes the gradients of L = sum_s W_s vals_s:
 *   grad_lam, grad_mu  in the layout of lam and mu (PER_ELEMENT [E] or
 *                      PER_QP [E][4]), or NULL;
 *   grad_coords        [N][3], or NULL.
 * All outputs are overwritten; sums run in a fixed order (deterministic):
 * one thread per element writes its terms to the pattern's per-element
 * scratch, then every node sums its elements' terms in increasing element
 * order.  Calls on one pattern that overlap (several streams) race. */
tg_status tg_assemble_elasticity_backward(const tg_pattern* p, tg_dtype dtype, const void* coords, const void* lam,
                                          const void* mu, tg_layout layout, const void* grad_vals,
                                          const void* lam_adj, const void* U, void* grad_lam, void* grad_mu,
                                          void* grad_coords, tg_stream stream);

/* Backward of the load vector (second line of Eq. (matlclquad)).  For an
 * upstream gradient grad_F [N * ncomp] of F, computes
 *   grad_f       same layout as f (PER_NODE, PER_QP or CONSTANT), or NULL;
 *   grad_coords  [N][d] (only |det J| depends on the coordinates), or NULL.
 * accumulate != 0 adds to grad_f / grad_coords instead of overwriting them
 * (used to sum the load and bilinear contributions of one objective). */
tg_status tg_assemble_load_backward(const tg_pattern* p, tg_dtype dtype, const void* coords, const void* f,
                                    tg_layout f_layout, int32_t ncomp, const void* grad_F, void* grad_f,
                                    void* grad_coords, int32_t accumulate, tg_stream stream);

/* ------------------------------------------------------------------------
 * Support: CSR products and the conjugate-gradient solve of the condensed
 * system (SM B.1 solver configuration; used by the adjoint of Eq. (adj)).
 * ---------------------------------------------------------------------- */

/* y = K x over the pattern's CSR (DoF level for elasticity).  A pattern
 * with no rows does nothing; vals may be NULL when it has no entries. */
tg_status tg_spmv(const tg_pattern* p, tg_dtype dtype, const void* vals, const void* x, void* y, tg_stream stream);

/* out[s] = alpha * lam[row(s)] * U[col(s)] for every CSR slot s: the adjoint
 * outer product dGamma/dK = lam U^T of Eq. (adj) on the pattern (DoF level
 * for elasticity).  lam, U [n_rows]; out [nnz].  A pattern with no entries
 * does nothing. */
tg_status tg_csr_outer(const tg_pattern* p, tg_dtype dtype, const void* lam, const void* U, double alpha, void* out,
                       tg_stream stream);

/* out[i] = alpha * x[i] on the rows where dirichlet[i] == 0 (uint8 [n], or
 * NULL for none) and out[i] = 0 on the others; out may be x itself.  The
 * adjoint relations of Eq. (adj) carry signs (dGamma/dF = -lam) and the
 * condensed system of SM B.1 drops the Dirichlet rows: this call applies
 * both to an upstream gradient before it enters the assembly backward
 * calls.  n = 0 does nothing. */
tg_status tg_scale_masked(tg_dtype dtype, const void* x, const uint8_t* dirichlet, double alpha, void* out,
                          int64_t n, tg_stream stream);

/* Conjugate gradients on K x = F restricted to the rows/columns where
 * dirichlet[i] == 0 (uint8 [n_rows], or NULL for none); entries of x on
 * Dirichlet rows are set to 0.  x holds the initial guess on entry (its
 * Dirichlet entries are set to 0 before the initial residual is formed).
 * Stops when ||F_I - K_II x_I|| <= rtol ||F_I|| or after maxit iterations.
 * The residual norm is checked every 8 iterations and at maxit.
 * iters / relres are HOST outputs (may be NULL).  SYNCHRONISES the stream.
 * Allocates and frees its work vectors.  Systems of up to 8 x (SM count) x
 * 256 rows run all iterations in one cooperative launch when its CTAs can
 * be resident together (bounded grid barriers: TG_ERR_TIMEOUT if one runs
 * out); otherwise each 8 iterations run as one launch of a CUDA graph
 * captured for the call.  Both forms give the iterates bit for bit. */
tg_status tg_cg_solve(const tg_pattern* p, tg_dtype dtype, const void* vals, const void* F,
                      const uint8_t* dirichlet, void* x, double rtol, int32_t maxit, int32_t* iters,
                      double* relres, tg_stream stream);

/* Bytes of the fixed device scratch of tg_cg_solve_noalloc (16 MiB): 4 KB of
 * scalars and partial sums, then four work vectors of n_rows values each
 * (each rounded up to 256 bytes).  That admits up to 1,048,320 rows in
 * TG_F32 and 524,160 rows in TG_F64. */
#define TG_CG_NOALLOC_SCRATCH_BYTES (16u << 20)

/* tg_cg_solve without any device allocation.  The paper has no counterpart:
 * it is a library variant of the solver above for callers that cannot
 * allocate device memory at solve time, e.g. a caller whose device memory is
 * held by a framework's caching allocator (cudaMalloc would fail or force
 * that cache to be emptied), or one solving inside a latency-critical loop
 * such as the adjoint solve of every optimisation step, where cudaMalloc and
 * cudaFree would synchronise the whole device and stall work queued on other
 * streams.  Same arguments, arithmetic and results (bitwise) as tg_cg_solve.
 *
 * The work vectors live in one fixed array of TG_CG_NOALLOC_SCRATCH_BYTES in
 * the library's device memory (one per device, allocated when the module is
 * loaded).  Consequences:
 * - A system whose work vectors do not fit returns TG_ERR_UNSUPPORTED before
 *   any GPU work (message in tg_last_error_message()).
 * - Calls that overlap on the same device (from several host threads, or on
 *   several streams) share the scratch and race; the caller serialises them.
 * - The first call on each device looks up the scratch address
 *   (cudaGetSymbolAddress, checked) and may load the module; make that first
 *   call outside any stream capture.  Like tg_cg_solve, every call
 *   SYNCHRONISES the stream. */
tg_status tg_cg_solve_noalloc(const tg_pattern* p, tg_dtype dtype, const void* vals, const void* F,
                              const uint8_t* dirichlet, void* x, double rtol, int32_t maxit, int32_t* iters,
                              double* relres, tg_stream stream);

/* ------------------------------------------------------------------------
 * Batched assembly: many independent instances in one persistent launch
 * (SM B.1, "Efficient Batch Data Generation": many-query use).
 * ---------------------------------------------------------------------- */

/* Group n_inst patterns of one element kind (TG_P1_TRI, TG_P2_TRI or
 * TG_P1_TET).  The patterns must outlive the batch.  Allocates device
 * memory and SYNCHRONISES the device. */
tg_status tg_batch_create(const tg_pattern* const* pats, int32_t n_inst, tg_batch** out);

/* Scalar bilinear assembly of every instance in ONE launch of a persistent
 * kernel.  coords, kappa, vals_out: HOST arrays of n_inst device pointers;
 * c: HOST array of n_inst values.  Same per-instance result, bit for bit, as
 * tg_assemble_bilinear on that instance.  Captured-graph safe. */
tg_status tg_batch_assemble(tg_batch* b, tg_dtype dtype, const void* const* coords, const void* const* kappa,
                            tg_layout kappa_layout, const double* c, void* const* vals_out, tg_stream stream);

/* The schedule of the persistent launch: threads per CTA, rows per work
 * item (a multiple of the thread count), CTAs per SM (0 = as many as fit).
 * When every instance's pattern has element-once row blocks (the element
 * kinds and meshes the single-instance element-once kernels take), the
 * batch walks (instance, row block) items with 128-thread CTAs and only
 * ctas_per_sm applies. */
tg_status tg_batch_set_schedule(tg_batch* b, int32_t threads, int32_t rows_per_item, int32_t ctas_per_sm);
tg_status tg_batch_get_schedule(const tg_batch* b, int32_t* threads, int32_t* rows_per_item,
                                int32_t* ctas_per_sm);

/* Autotuner: times every candidate schedule on the given inputs with CUDA
 * events (reps launches each, after a warm-up), keeps the fastest, and
 * returns its time per launch in *best_ms (host, may be NULL).  Overwrites
 * vals_out.  SYNCHRONISES the stream; not for use under graph capture. */
tg_status tg_batch_autotune(tg_batch* b, tg_dtype dtype, const void* const* coords, const void* const* kappa,
                            tg_layout kappa_layout, const double* c, void* const* vals_out, int32_t reps,
                            float* best_ms, tg_stream stream);

void tg_batch_destroy(tg_batch* b);

/* ------------------------------------------------------------------------
 * Boundary facets: the Neumann and Robin terms of a scalar problem, routed
 * into the same CSR values and load vector as the element terms (the
 * mixed-boundary-condition Poisson benchmark of the SM; the Map over
 * boundary quadrature and a boundary routing into Sparse-Reduce).  With the
 * Robin condition kappa du/dn + alpha u = g_R on Gamma_R and the Neumann
 * condition kappa du/dn = g_N on Gamma_N, the weak form gains
 *   sum_f int_f alpha u v ds   (matrix)  and  sum_f int_f g v ds   (load).
 * Facets of P1 triangles are boundary edges (2 vertices; 2-point Gauss
 * rule on the edge), of P1 tetrahedra boundary faces (3 vertices; the
 * 3-point rule of the triangle).  P2 is not supported.
 * ---------------------------------------------------------------------- */

/* Routing of a facet set on a pattern (P1_TRI or P1_TET).
 *   facets  device int32 [n_facets][d] (d = 2 for triangles, 3 for
 *           tetrahedra): node ids; copied.  Every facet's vertex pairs must
 *           share an element of the pattern (a facet of the mesh).
 * Errors: TG_ERR_INDEX_RANGE (node id outside [0, N)), TG_ERR_DEGENERATE_
 * ELEMENT (repeated vertex), TG_ERR_INVALID_ARG (a pair that shares no
 * element); tg_last_error_message() names the facet.  SYNCHRONISES.  The
 * facet set reads the pattern's row pointers: destroy it before the
 * pattern. */
tg_status tg_build_facets(const tg_pattern* p, const int32_t* facets, int64_t n_facets, tg_stream stream,
                          tg_facets** out);

/* Adds the facet terms to assembled values, one facet at a time in
 * increasing facet order (deterministic):
 *   vals_inout[slot(g_a, g_b)] += sum_q w_q |J_f| alpha_q phi_a phi_b
 *   F_inout[g_a]               += sum_q w_q |J_f| g_q phi_a
 * |J_f| = the edge length or twice the face area; quadrature on the
 * reference facet (weights sum to 1 on the edge, 1/2 on the face).
 *   alpha  layouts PER_ELEMENT (one per facet, [n_facets]), PER_QP
 *          ([n_facets][2 or 3]) or CONSTANT; NULL = no matrix term.
 *   g      layouts PER_NODE ([N], the facet interpolant), PER_QP or
 *          CONSTANT; NULL = no load term.
 *   vals_inout [nnz] (the pattern's CSR), F_inout [N]; either may be NULL
 *          when its term is absent.
 * A facet of zero measure is recorded as TG_ERR_DEGENERATE_ELEMENT (facet
 * index) in the pattern's device status. */
tg_status tg_assemble_facets(const tg_facets* fc, tg_dtype dtype, const void* coords, const void* alpha,
                             tg_layout alpha_layout, const void* g, tg_layout g_layout, void* vals_inout,
                             void* F_inout, tg_stream stream);

/* Number of facets and of nodes that carry at least one. */
tg_status tg_facets_shape(const tg_facets* fc, int64_t* n_facets, int64_t* n_boundary_nodes);

void tg_facets_destroy(tg_facets* fc);

/* ------------------------------------------------------------------------
 * Plane-stress bilinear quadrilaterals with the SIMP law (the SM's
 * topology-optimisation benchmark; element kind TG_Q1_QUAD_VEC2, cells
 * [E][4] counter-clockwise, DoF = 2 node + component).
 *   E(rho_e) = e_min + rho_e^penal (e_max - e_min),
 *   K(rho)   = sum_e E(rho_e) K0_e,  K0_e the unit-modulus element matrix
 *              by the 2 x 2 Gauss rule (tg_quadrature(TG_Q1_QUAD_VEC2)),
 *              plane-stress Lame constants nu / (1 - nu^2), 1 / (2 (1 + nu)).
 * ---------------------------------------------------------------------- */

/* vals_out [nnz of the DoF-level CSR of tg_pattern_info]; rho [E];
 * -1 < nu < 1/2.  Each node's two DoF rows sum their elements in increasing
 * element order (deterministic).  A non-positive Jacobian determinant at a
 * Gauss point flags TG_ERR_DEGENERATE_ELEMENT. */
tg_status tg_assemble_simp(const tg_pattern* p, tg_dtype dtype, const void* coords, const void* rho, double e_min,
                           double e_max, double penal, double nu, void* vals_out, tg_stream stream);

/* Compliance sensitivity (SM): dc_out[e] = -penal rho_e^(penal-1)
 * (e_max - e_min) u_e^T K0_e u_e for the displacement u [2 N] of
 * K(rho) u = F (the compliance C = F^T u is self-adjoint). */
tg_status tg_simp_sensitivity(const tg_pattern* p, tg_dtype dtype, const void* coords, const void* rho, double e_min,
                              double e_max, double penal, double nu, const void* u, void* dc_out, tg_stream stream);

/* ------------------------------------------------------------------------
 * Measurement helper (no counterpart in the paper): sustained rate of
 * dependent-free fused multiply-adds in the given dtype across the whole
 * GPU, in FLOP/s (2 per FMA), written to *flops (host).  SYNCHRONISES. */
tg_status tg_diag_fma_rate(tg_dtype dtype, double* flops, tg_stream stream);

/* Accuracy check (no counterpart in the paper): y[i] = the FP64 reciprocal
 * that the P1 forward kernels take of |det J| (Newton's iteration from an
 * FP32 seed, within one unit in the last place of 1 / x[i]), for n values;
 * x and y are device arrays of n doubles, n = 0 does nothing.  Asynchronous
 * on the stream. */
tg_status tg_diag_recip(const double* x, double* y, int64_t n, tg_stream stream);

/* Failure-path check (no counterpart in the paper): one CTA waits, bounded
 * by max_tries polls (1 .. 2^22), on a shared-memory barrier that nothing
 * completes, exactly as the pipelined kernels wait for their bulk copies;
 * the wait gives up and records TG_ERR_TIMEOUT in p's device status, which
 * tg_get_device_status then returns (and clears).  Nothing hangs or
 * faults. */
tg_status tg_diag_wait_timeout(const tg_pattern* p, int32_t max_tries, tg_stream stream);

/* Failure-path check of the grid barrier of tg_cg_solve's one-launch loop
 * (no counterpart in the paper): a cooperative launch of two CTAs in which
 * one leaves without arriving, so the barrier never completes; the other
 * polls at most max_polls times (1 .. 2^22, the CG's own limit), gives up,
 * and the call returns TG_ERR_TIMEOUT, as tg_cg_solve does when its barrier
 * gives up.  Nothing hangs or faults.  Synchronises the stream; allocates 16
 * bytes of device memory for the call. */
tg_status tg_diag_grid_barrier_timeout(int32_t max_polls, tg_stream stream);

#ifdef __cplusplus
}
#endif

#endif /* TG_H_ */
