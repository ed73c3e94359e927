// Internal declarations of libtg.so (GB300 / sm_103a Galerkin assembly).
//
// Data layout of a pattern in HBM (all int32 unless noted):
//   cells    [E][nv]          copy of the connectivity
//   inc_ptr  [N+1]            node -> incident (element, local index) list
//   inc_e    [E*nv]           e * 8 + a, sorted by e within each node
//   inc_pos  [E*nv][npw] u32  8-bit positions of the element's nv nodes in
//                             the row of the owning node (npw = 1 for nv <= 4,
//                             2 for P2); this is the routing S_mat of
//                             Algorithm 2 in compressed, row-owned form
//   row_ptr  [N+1], col_idx [nnz]   node-level CSR
//   elem_slot [E][nv][nv]     CSR slot of each local entry (API view)
//   row_ptr_dof [nc N+1], col_idx_dof [nc^2 nnz]  DoF-level CSR of the vector kinds
//                         (nc DoFs per node: 3 tetrahedral elasticity, 2 plane-stress quads)
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>

#include "tg.h"

#define TG_MAX_ROW 255  // positions are stored in 8 bits

struct tg_pattern {
  tg_element el;
  int nv = 0, dim = 0, nq = 0, ngeo = 0, npw = 1;
  int64_t E = 0, N = 0, nnz = 0;
  int device = 0;
  int max_row_len = 0, max_deg = 0;
  int32_t* cells = nullptr;
  int32_t* inc_ptr = nullptr;
  int32_t* inc_e = nullptr;
  uint32_t* inc_pos = nullptr;
  int32_t* row_ptr = nullptr;
  int32_t* col_idx = nullptr;
  int32_t* elem_slot = nullptr;
  int32_t* row_ptr_dof = nullptr;
  int32_t* col_idx_dof = nullptr;
  // Row blocks of the element-once kernels (scalar kinds only, built when
  // the packed fields fit; bel == NULL otherwise).  The kernels walk the
  // rows in an internal order: iperm[i] is the node of internal row i
  // (nodes by smallest incident element, then each block of blk_rows rows
  // in ascending node id); iinc and irp are the incidence and CSR-value
  // prefix sums in that order, urp[i] = row_ptr[iperm[i]].  Block b owns the internal rows [b*blk_rows,
  // (b+1)*blk_rows) and hence the internal incidences [J0, J1) =
  // [iinc[b*blk_rows], iinc[min((b+1)*blk_rows, N)]).
  //   bel + boff[b]: the block's distinct elements (nbe = bel_cnt[b] of
  //     them, ascending): (nbe + 3) & ~3 words of element ids (bit 31 set in
  //     the one block that owns the element, the block of its smallest
  //     vertex), then nv rows of (nbe + 7) & ~7 16-bit vertex offsets from
  //     bvbase[b] (built only when every block's vertex ids span < 2^16).
  //   brec[j], j in [J0, J1), per incidence (row i, element e, local vertex
  //     a), rows in internal order, each row's incidences in element order.
  //     nv <= 4: 4-bit fields [4c, 4c+4) the position in row i of the column
  //     of vertex (a + c) mod nv (c < nv; field 0 is the diagonal), then a
  //     (2 bits), then the local index of e in the block's list (the rest).
  //     P2 (two words): six 5-bit fields in the same rotated order, then a
  //     (3 bits) and the local index in the second word.
  //   elem_pos[e] (64 bit): position of vertex b's column in vertex a's row
  //     at bits [4(a*nv + b), ...).
  //   fan (P1 triangles whose every node has a single fan of triangles
  //     around it): per block b, a region of 16-bit words at fan + fan_off[b]
  //     (kf = (fan_off[b + 1] - fan_off[b]) / fan_rs - 5 fan steps, fan_rs =
  //     blk_rows rounded up to a multiple of 8):
  //       4 * fan_rs words: per row t, a 64-bit word of 4-bit CSR positions of
  //         the row's neighbours j_0, j_1, ... in the order of the fan;
  //       fan_rs words: per row t, deg (bits 0-4), open fan (bit 5), CSR
  //         position of the diagonal (bits 6-9);
  //       kf * fan_rs words: record [k][t] of the k-th triangle of row t's fan
  //         (the triangle between neighbours j_k and j_{k+1}): its index in the
  //         block's element list (bits 0-10), the row's local vertex a in it
  //         (bits 11-12), and whether j_k is vertex a + 2 rather than a + 1
  //         (bit 13).
  //     NULL when some node's triangles do not form one fan (or a block
  //     holds more than 2048 elements); the row-owner Reduce serves then.
  //     P2 triangles: per block, 32-bit words: info[t] (deg bits 0-4, edge
  //     node bit 5, open fan bit 6, diagonal position bits 7-11, then two
  //     5-bit positions: an open fan's last vertex neighbour and edge node,
  //     or an edge node's endpoints u and w), then records [k][t]: the
  //     element's list index (bits 0-10), the row's local node a (bits 11-13),
  //     a swap bit (14) and three 5-bit positions (bits 15-29).
  uint16_t* fan = nullptr;
  // emask[s] (vector elasticity with rows of at most 16 nodes and at most 32
  // incident elements per node): bit m set when the m-th incident element
  // of the row's node (inc_e order) also holds the column node of node-level
  // CSR entry s; 0 on the diagonal.  NULL otherwise.
  uint32_t* emask = nullptr;
  int64_t* fan_off = nullptr;
  int fan_rs = 0, fan_kmax = 0, fan_maxw = 0;  // fan_maxw: largest region, 16-bit words
  int blk_rows = 0, blk_pb = 0;
  int blk_max_elems = 0, blk_max_inc = 0, blk_max_nz = 0;  // per-block maxima
  int64_t n_blk = 0;
  int32_t* iperm = nullptr;
  int32_t* urp = nullptr;
  int32_t* iinc = nullptr;
  int32_t* irp = nullptr;
  uint32_t* bel = nullptr;
  int64_t* boff = nullptr;
  int32_t* bvbase = nullptr;
  int32_t* bel_cnt = nullptr;
  uint32_t* brec = nullptr;
  uint64_t* elem_pos = nullptr;
  // device status: [0] error code (first one wins), [1] smallest bad element
  unsigned long long* status = nullptr;
  // per-CTA partial sums of global reductions (backward of c / constant kappa)
  double* partials = nullptr;
  int64_t n_partials = 0;
  // arrival counter of the element-once backward's CTAs (zero between
  // launches: the last CTA to arrive wraps it back to zero)
  unsigned int* arrivals = nullptr;
  // per-element results of the two-pass kernels (residual: nv values;
  // backward: nv x dim coordinate gradients), up to 8 bytes each (scalar
  // element kinds)
  void* elem_scratch = nullptr;
};

namespace tg {

// ------------------------------------------------------------------ errors
void set_error(const std::string& msg);
tg_status cuda_fail(cudaError_t err, const char* what, const char* file, int line);

#define TG_CK(call)                                                         \
  do {                                                                      \
    cudaError_t err__ = (call);                                             \
    if (err__ != cudaSuccess) return tg::cuda_fail(err__, #call, __FILE__, __LINE__); \
  } while (0)

#define TG_CK_LAUNCH(what) TG_CK(cudaGetLastError())

// ------------------------------------------------------------------ element traits
template <int EL>
struct Elem;
template <>
struct Elem<TG_P1_TRI> {
  static constexpr int nv = 3, dim = 2, nq = 3, ngeo = 3, npw = 1;
};
template <>
struct Elem<TG_P2_TRI> {
  static constexpr int nv = 6, dim = 2, nq = 6, ngeo = 3, npw = 2;
};
template <>
struct Elem<TG_P1_TET> {
  static constexpr int nv = 4, dim = 3, nq = 4, ngeo = 4, npw = 1;
};

template <>
struct Elem<TG_Q1_QUAD_VEC2> {
  static constexpr int nv = 4, dim = 2, nq = 4, ngeo = 4, npw = 1;
};

inline int nv_of(tg_element el) { return el == TG_P1_TRI ? 3 : el == TG_P2_TRI ? 6 : 4; }
inline int dim_of(tg_element el) { return (el == TG_P1_TRI || el == TG_P2_TRI || el == TG_Q1_QUAD_VEC2) ? 2 : 3; }
inline int nq_of(tg_element el) { return el == TG_P1_TRI ? 3 : el == TG_P2_TRI ? 6 : 4; }
// DoFs per node: 3 for tetrahedral elasticity, 2 for plane-stress quads, 1 otherwise
inline int ncomp_of(tg_element el) { return el == TG_P1_TET_VEC3 ? 3 : el == TG_Q1_QUAD_VEC2 ? 2 : 1; }
// the scalar element kinds (the Poisson-type assembly, load, residual, backward)
inline bool scalar_kind(tg_element el) { return el == TG_P1_TRI || el == TG_P2_TRI || el == TG_P1_TET; }

// Reference tables of one element kind, built on the host from the
// quadrature rule and the reference basis, passed to kernels by value.
template <typename T>
struct RefTab {
  T w[6];          // quadrature weights (sum = reference measure)
  T phi[6][6];     // phi[q][a]   basis value at point q
  T gh[6][6][3];   // gh[q][a][s] reference gradient at point q
  T M[6][6];       // sum_q w_q phi_a phi_b  (reference mass matrix)
  T m1[6];         // sum_q w_q phi_a
  T wsum;          // sum_q w_q
};

// Host-side: rule and tables of an element kind (kernel side of the code,
// independent of the oracle).
int quadrature_rule(tg_element el, double* w, double* x);
template <typename T>
RefTab<T> ref_table(tg_element el);

// ------------------------------------------------------------------ device helpers
__device__ __forceinline__ void record_error(unsigned long long* status, int code, long long e) {
  atomicCAS(status, 0ull, (unsigned long long)code);
  atomicMin(status + 1, (unsigned long long)e);
}

template <typename T>
struct Vec2;
template <>
struct Vec2<float> {
  using type = float2;
};
template <>
struct Vec2<double> {
  using type = double2;
};

template <typename T>
__device__ __forceinline__ T ldg(const T* p) {
  return __ldg(p);
}

template <typename T>
__host__ __device__ constexpr T det_tiny();
template <>
__host__ __device__ constexpr float det_tiny<float>() {
  return 1e-37f;
}
template <>
__host__ __device__ constexpr double det_tiny<double>() {
  return 1e-300;
}

// A 32-bit pattern carried in a T slot of shared memory, and back.
template <typename T>
__device__ __forceinline__ T bits_as(uint32_t b) {
  if constexpr (sizeof(T) == 4) return __uint_as_float(b);
  else return __longlong_as_double((long long)b);
}
template <typename T>
__device__ __forceinline__ uint32_t as_bits(T x) {
  if constexpr (sizeof(T) == 4) return __float_as_uint(x);
  else return (uint32_t)__double_as_longlong(x);
}

// 1 / x rounded to nearest (IEEE), bitwise the quotient T(1) / x.
__device__ __forceinline__ float recip(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double recip(double x) { return __drcp_rn(x); }

// FP32: recip.  FP64: 1 / x within one unit in the last place, by Newton's
// iteration for the reciprocal, y <- y + y (1 - x y), from the FP32
// approximate reciprocal of x rounded to FP32 as the seed (relative error
// below 2^-21): two steps take it below 2^-84 before the last rounding.
// Four FP64 fused multiply-adds and two conversions, fewer FP64-pipe
// operations than the correctly rounded quotient; the P1 forward, bound by
// that pipe in FP64, takes its 1 / |det J| here.  |x| outside [2^-120,
// 2^120] (no normal FP32 seed), zero, infinities and NaN take the quotient
// 1.0 / x.
__device__ __forceinline__ float recip_fast(float x) { return recip(x); }
__device__ __forceinline__ double recip_fast(double x) {
  const uint32_t ex = ((uint32_t)(__double_as_longlong(x) >> 52)) & 0x7ffu;
  if (ex < 1023u - 120u || ex > 1023u + 119u) return 1.0 / x;
  float yf;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(yf) : "f"(__double2float_rn(x)));
  double y = (double)yf;
  y = fma(y, fma(-x, y, 1.0), y);
  return fma(y, fma(-x, y, 1.0), y);
}

// Coefficient sum over quadrature points with the rule's weights.
template <typename T, int NQ>
__device__ __forceinline__ T weighted_coef(const T* __restrict__ v, int layout, int64_t e, const T (&w)[6], T wsum) {
  if (layout == TG_PER_QP) {
    T s = T(0);
#pragma unroll
    for (int q = 0; q < NQ; ++q) s += w[q] * ldg(v + e * NQ + q);
    return s;
  } else if (layout == TG_PER_ELEMENT) {
    return wsum * ldg(v + e);
  }
  return wsum * ldg(v);
}

template <typename T, int NQ>
__device__ __forceinline__ T coef_q(const T* __restrict__ v, int layout, int64_t e, int q) {
  if (layout == TG_PER_QP) return ldg(v + e * NQ + q);
  if (layout == TG_PER_ELEMENT) return ldg(v + e);
  return ldg(v);
}

inline int grid_for(int64_t n, int threads) { return (int)((n + threads - 1) / threads); }

int sm_count();

}  // namespace tg
