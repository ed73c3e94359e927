// Vector P1 linear elasticity, forward: the DoF-level CSR values of
//   K[(a,i),(b,j)] = sum_q w_q |det J| (lam_q g_ai g_bj + mu_q g_aj g_bi + mu_q delta_ij g_a . g_b)
// (the SM form lam div u div v + 2 mu eps(u) : eps(v)), one thread per node
// row, summing the node's incidences in increasing element order.
#include <algorithm>
#include <cstdint>

#include "blk_bilinear.cuh"

namespace {

constexpr int EB = 64;  // node rows per CTA (9 * row length accumulators per thread)

using tg::FwdArgs;
using tg::absv;

// Store the n values acc[p * stride] to out[0, n) (out aligned to T):
// scalar stores up to the first 16-byte boundary, then 16-byte vectors, then
// the tail.  Rows written by one thread each land in different lines across
// a warp, so every vector store moves four (FP32) values per sector written
// instead of one.
template <typename T>
__device__ __forceinline__ void store_row(T* __restrict__ out, const T* acc, int stride, int n) {
  using V = typename tg::Vec16<T>::type;
  constexpr int VN = tg::Vec16<T>::n;
  const int head = (int)(((16u - ((unsigned)(uintptr_t)out & 15u)) & 15u) / sizeof(T));
  int p = 0;
  for (; p < head && p < n; ++p) out[p] = acc[p * stride];
  for (; p + VN <= n; p += VN) {
    T x[VN];
#pragma unroll
    for (int k = 0; k < VN; ++k) x[k] = acc[(p + k) * stride];
    *reinterpret_cast<V*>(out + p) = tg::Vec16<T>::make(x);
  }
  for (; p < n; ++p) out[p] = acc[p * stride];
}

// Vector P1 elasticity, one thread per node: the node's three DoF rows are
// consecutive in the DoF CSR and together hold 9 * len entries in the order
// [component i][column node p][component j], accumulated in shared memory
// over the node's incidences in increasing element order:
//   block (a, b) = L n_a n_b^T + M n_b n_a^T + M (n_a.n_b) I,
// n_c = |det J| grad(phi_c), L = sum_q w_q lam_q / |det J|, M likewise.
// The row goes out in 16-byte stores (every thread writes its own 9 * len
// values, so scalar stores would write one value per sector).
// In FP64 the element terms are computed once per element by
// k_elastic_geom into geo[16 e + 4 c + r] = n_c[r], geo[16 e + 3] = L,
// geo[16 e + 7] = M (zeros for a degenerate element, which is flagged and
// adds nothing); in FP32 every thread computes them from the gathered
// coordinates, which is cheaper than the records' extra L1 footprint.
template <typename T>
__global__ void __launch_bounds__(128) k_elastic_geom(const FwdArgs<T> a, const __grid_constant__ tg::RefTab<T> tab,
                                                      int64_t E, T* __restrict__ geo) {
  using V = typename tg::Vec16<T>::type;
  constexpr int VN = tg::Vec16<T>::n;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < E; e += (int64_t)gridDim.x * blockDim.x) {
    const int32_t* cl = a.cells + e * 4;
    tg::Geom<3, T> g;
    tg::tet_geom(a.coords, __ldg(cl), __ldg(cl + 1), __ldg(cl + 2), __ldg(cl + 3), g);
    const T adet = absv(g.det);
    T o[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) o[k] = T(0);
    if (!(adet > tg::det_tiny<T>())) {
      tg::record_error(a.status, TG_ERR_DEGENERATE_ELEMENT, e);
    } else {
      const T inv = tg::recip(adet);
#pragma unroll
      for (int c = 0; c < 4; ++c)
#pragma unroll
        for (int r = 0; r < 3; ++r) o[4 * c + r] = g.n[c][r];
      o[3] = tg::weighted_coef<T, 4>(a.coef, a.layout, e, tab.w, tab.wsum) * inv;
      o[7] = tg::weighted_coef<T, 4>(a.coef2, a.layout, e, tab.w, tab.wsum) * inv;
    }
    V* dst = reinterpret_cast<V*>(geo + 16 * e);
#pragma unroll
    for (int k = 0; k < 16 / VN; ++k) dst[k] = tg::Vec16<T>::make(o + k * VN);
  }
}

template <typename T, bool GEO>
__global__ void __launch_bounds__(EB) k_elastic_gather(const FwdArgs<T> a, const __grid_constant__ tg::RefTab<T> tab,
                                                       const T* __restrict__ geo) {
  using V = typename tg::Vec16<T>::type;
  constexpr int VN = tg::Vec16<T>::n;
  extern __shared__ __align__(16) unsigned char smem[];
  T* acc = reinterpret_cast<T*>(smem) + threadIdx.x;
  const int64_t i = (int64_t)blockIdx.x * EB + threadIdx.x;
  if (i >= a.n) return;
  const int r0 = __ldg(a.row_ptr + i), len = __ldg(a.row_ptr + i + 1) - r0;
  for (int p = 0; p < 9 * len; ++p) acc[p * EB] = T(0);
  const int j0 = __ldg(a.inc_ptr + i), j1 = __ldg(a.inc_ptr + i + 1);
  for (int j = j0; j < j1; ++j) {
    const int ea = __ldg(a.inc_e + j);
    const int64_t e = ea >> 3;
    const int la = ea & 7;
    const uint32_t w0 = __ldg(a.inc_pos + j);
    T o[16];
    if constexpr (GEO) {
      const V* src = reinterpret_cast<const V*>(geo + 16 * e);
#pragma unroll
      for (int k = 0; k < 16 / VN; ++k) {
        const V x = __ldg(src + k);
#pragma unroll
        for (int q = 0; q < VN; ++q) o[k * VN + q] = tg::Vec16<T>::get(x, q);
      }
    } else {
      const int32_t* cl = a.cells + e * 4;
      tg::Geom<3, T> g;
      tg::tet_geom(a.coords, __ldg(cl), __ldg(cl + 1), __ldg(cl + 2), __ldg(cl + 3), g);
      const T adet = absv(g.det);
      if (!(adet > tg::det_tiny<T>())) {
        tg::record_error(a.status, TG_ERR_DEGENERATE_ELEMENT, e);
        continue;
      }
      const T inv = tg::recip(adet);
#pragma unroll
      for (int c = 0; c < 4; ++c)
#pragma unroll
        for (int r = 0; r < 3; ++r) o[4 * c + r] = g.n[c][r];
      o[3] = tg::weighted_coef<T, 4>(a.coef, a.layout, e, tab.w, tab.wsum) * inv;
      o[7] = tg::weighted_coef<T, 4>(a.coef2, a.layout, e, tab.w, tab.wsum) * inv;
    }
    const T L = o[3], M = o[7];
    T na[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const T col[4] = {o[r], o[4 + r], o[8 + r], o[12 + r]};
      na[r] = tg::sel(la, col);
    }
    // each entry accumulates by two fused multiply-adds onto the running
    // sum (the FP64 pipe bounds the FP64 kernel)
    T Lna[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) Lna[r] = L * na[r];
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int pos = tg::pos_of(w0, 0u, b);
      const T nb[3] = {o[4 * b], o[4 * b + 1], o[4 * b + 2]};
      const T Md = M * (na[0] * nb[0] + na[1] * nb[1] + na[2] * nb[2]);
#pragma unroll
      for (int ii = 0; ii < 3; ++ii) {
        const T Mnb = M * nb[ii];
#pragma unroll
        for (int jj = 0; jj < 3; ++jj) {
          T* q = acc + ((ii * len + pos) * 3 + jj) * EB;
          T v = fma(Mnb, na[jj], fma(Lna[ii], nb[jj], *q));
          if (ii == jj) v += Md;
          *q = v;
        }
      }
    }
  }
  store_row<T>(a.out + 9ll * r0, acc, EB, 9 * len);
}

// Two passes for rows of at most 16 nodes and 32 incident elements per node
// (the pattern's emask).  Pass 1, one thread per element: the record
//   rec[20 e + 4 c + r] = n_c[r] (c < 4, r < 3),  rec[20 e + 4 c + 3] = L,
//   rec[20 e + 16] = M,
// with n_c = |det J| grad(phi_c), L = sum_q w_q lam_q / |det J| and M
// likewise (zeros for a degenerate element, which is flagged).
// The CTA's 128 consecutive records go through shared memory, so that the
// stores to HBM are contiguous 16-byte vectors across the warp.
template <typename T>
__global__ void __launch_bounds__(128) k_elastic_rec(const FwdArgs<T> a, const __grid_constant__ tg::RefTab<T> tab,
                                                     int64_t E, T* __restrict__ rec) {
  using V = typename tg::Vec16<T>::type;
  constexpr int VN = tg::Vec16<T>::n;
  constexpr int NVR = 20 / VN;  // 16-byte vectors per record
  __shared__ V buf[128 * NVR];
  for (int64_t e0 = (int64_t)blockIdx.x * 128; e0 < E; e0 += (int64_t)gridDim.x * 128) {
    const int64_t e = e0 + threadIdx.x;
    T o[20];
#pragma unroll
    for (int k = 0; k < 20; ++k) o[k] = T(0);
    if (e < E) {
      const int32_t* cl = a.cells + e * 4;
      tg::Geom<3, T> g;
      tg::tet_geom(a.coords, __ldg(cl), __ldg(cl + 1), __ldg(cl + 2), __ldg(cl + 3), g);
      const T adet = absv(g.det);
      if (!(adet > tg::det_tiny<T>())) {
        tg::record_error(a.status, TG_ERR_DEGENERATE_ELEMENT, e);
      } else {
        const T inv = tg::recip(adet);
        const T L = tg::weighted_coef<T, 4>(a.coef, a.layout, e, tab.w, tab.wsum) * inv;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
#pragma unroll
          for (int r = 0; r < 3; ++r) o[4 * c + r] = g.n[c][r];
          o[4 * c + 3] = L;
        }
        o[16] = tg::weighted_coef<T, 4>(a.coef2, a.layout, e, tab.w, tab.wsum) * inv;
      }
    }
#pragma unroll
    for (int k = 0; k < NVR; ++k) buf[threadIdx.x * NVR + k] = tg::Vec16<T>::make(o + k * VN);
    __syncthreads();
    const int64_t nv = (E - e0 < 128 ? E - e0 : 128) * NVR;  // vectors of this CTA's records
    V* dst = reinterpret_cast<V*>(rec + 20 * e0);
    for (int k = threadIdx.x; k < nv; k += 128) dst[k] = buf[k];
    __syncthreads();
  }
}

// Pass 2: 16 lanes per node row i (two rows per warp), lane p owning the
// 3 x 3 block of the row's p-th column node j in registers.  The block is
// summed over the elements around edge (i, j) (the bits of emask,
// increasing element order), each entry by two fused multiply-adds onto its
// running sum:
//   L n_a n_b^T + M n_b n_a^T + M (n_a . n_b) I,
// a, b the local indices of i and j.  An element's diagonal-block terms
// (L + M) n_a n_a^T + M |n_a|^2 I are added by the lane of its neighbour of
// smallest position; the row's 16 partial diagonal blocks are summed by a
// fixed butterfly over its lanes and written by the diagonal lane.  The
// segments of consecutive lanes of each DoF row are contiguous (48 values
// per half-warp).
constexpr int ELR = 16;  // lanes per node row

template <typename T>
__device__ __forceinline__ void ld_vec4(const T* __restrict__ r, T (&x)[4]) {
  if constexpr (sizeof(T) == 4) {
    const float4 q = __ldg(reinterpret_cast<const float4*>(r));
    x[0] = q.x;
    x[1] = q.y;
    x[2] = q.z;
    x[3] = q.w;
  } else {
    const double2 q0 = __ldg(reinterpret_cast<const double2*>(r));
    const double2 q1 = __ldg(reinterpret_cast<const double2*>(r) + 1);
    x[0] = q0.x;
    x[1] = q0.y;
    x[2] = q1.x;
    x[3] = q1.y;
  }
}

template <typename T>
__global__ void __launch_bounds__(128) k_elastic_lanes(const FwdArgs<T> a, const T* __restrict__ rec,
                                                       const uint32_t* __restrict__ emask) {
  const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t i = gt / ELR;
  const int p = (int)(gt % ELR);
  const bool row = i < a.n;
  int r0 = 0, len = 0, j0 = 0;
  if (row) {
    r0 = __ldg(a.row_ptr + i);
    len = __ldg(a.row_ptr + i + 1) - r0;
    j0 = __ldg(a.inc_ptr + i);
  }
  const bool live = row && p < len;
  uint32_t mask = live ? __ldg(emask + r0 + p) : 0u;
  T B[3][3], D[6];  // D: xx, yy, zz, xy, xz, yz
#pragma unroll
  for (int u = 0; u < 3; ++u)
#pragma unroll
    for (int v = 0; v < 3; ++v) B[u][v] = T(0);
#pragma unroll
  for (int k = 0; k < 6; ++k) D[k] = T(0);
  while (mask) {
    const int m = __ffs(mask) - 1;
    mask &= mask - 1;
    const int ea = __ldg(a.inc_e + j0 + m);
    const int64_t e = ea >> 3;
    const int la = ea & 7;
    const uint32_t w = __ldg(a.inc_pos + j0 + m);
    int lb = 0, pmin = 16;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int pc = (int)((w >> (8 * c)) & 15u);
      if (c != la) {
        if (pc == p) lb = c;
        pmin = pc < pmin ? pc : pmin;
      }
    }
    const T* re = rec + 20 * e;
    T na[4], nb[4];
    ld_vec4(re + 4 * la, na);
    ld_vec4(re + 4 * lb, nb);
    const T L = na[3], M = __ldg(re + 16);
    const T Md = M * (na[0] * nb[0] + na[1] * nb[1] + na[2] * nb[2]);
#pragma unroll
    for (int u = 0; u < 3; ++u) {
      const T Lna = L * na[u], Mnb = M * nb[u];
#pragma unroll
      for (int v = 0; v < 3; ++v) {
        const T x = fma(Mnb, na[v], fma(Lna, nb[v], B[u][v]));
        B[u][v] = u == v ? x + Md : x;
      }
    }
    if (p == pmin) {
      const T S = L + M, q = M * (na[0] * na[0] + na[1] * na[1] + na[2] * na[2]);
      D[0] += S * na[0] * na[0] + q;
      D[1] += S * na[1] * na[1] + q;
      D[2] += S * na[2] * na[2] + q;
      D[3] += S * na[0] * na[1];
      D[4] += S * na[0] * na[2];
      D[5] += S * na[1] * na[2];
    }
  }
  // the row's diagonal block: a fixed butterfly over its 16 lanes
#pragma unroll
  for (int o = ELR / 2; o >= 1; o >>= 1)
#pragma unroll
    for (int k = 0; k < 6; ++k) D[k] += __shfl_xor_sync(0xffffffffu, D[k], o, ELR);
  if (!live) return;
  // the diagonal's position: that of the row's node in its first element
  const int ea0 = __ldg(a.inc_e + j0);
  if ((int)((__ldg(a.inc_pos + j0) >> (8 * (ea0 & 7))) & 15u) == p) {
    B[0][0] = D[0];
    B[1][1] = D[1];
    B[2][2] = D[2];
    B[0][1] = B[1][0] = D[3];
    B[0][2] = B[2][0] = D[4];
    B[1][2] = B[2][1] = D[5];
  }
  T* out = a.out + 9ll * r0 + 3 * p;
#pragma unroll
  for (int u = 0; u < 3; ++u)
#pragma unroll
    for (int v = 0; v < 3; ++v) out[3 * len * u + v] = B[u][v];
}

// ---------------------------------------------------------------- host side
template <typename T>
FwdArgs<T> el_args(const tg_pattern* p, const void* coords) {
  FwdArgs<T> a{};
  a.row_ptr = p->row_ptr;
  a.inc_ptr = p->inc_ptr;
  a.inc_e = p->inc_e;
  a.inc_pos = p->inc_pos;
  a.cells = p->cells;
  a.elem_slot = p->elem_slot;
  a.coords = static_cast<const T*>(coords);
  a.n = p->N;
  a.status = p->status;
  return a;
}

template <typename T>
tg_status elastic(const tg_pattern* p, const void* coords, const void* lam, const void* mu, tg_layout l, void* vals,
                  cudaStream_t s) {
  FwdArgs<T> a = el_args<T>(p, coords);
  a.coef = static_cast<const T*>(lam);
  a.coef2 = static_cast<const T*>(mu);
  a.layout = l;
  a.out = static_cast<T*>(vals);
  if (p->N == 0) return TG_OK;
  T* rec = static_cast<T*>(p->elem_scratch);  // 20 values per element
  if (p->emask && rec && sizeof(T) == 4) {
    const tg::RefTab<T>& tab = tg::table<T>(TG_P1_TET);
    if (p->E > 0) {
      const int g1 = (int)std::min<int64_t>(tg::grid_for(p->E, 128), 32ll * tg::sm_count());
      k_elastic_rec<T><<<g1, 128, 0, s>>>(a, tab, p->E, rec);
      TG_CK_LAUNCH("k_elastic_rec");
    }
    k_elastic_lanes<T><<<tg::grid_for(p->N * ELR, 128), 128, 0, s>>>(a, rec, p->emask);
    TG_CK_LAUNCH("k_elastic_lanes");
    return TG_OK;
  }
  constexpr bool use_geo = sizeof(T) == 8;
  T* geo = static_cast<T*>(p->elem_scratch);  // 16 values per element
  if constexpr (use_geo) {
    if (p->E > 0) {
      if (!geo) return TG_ERR_UNSUPPORTED;
      k_elastic_geom<T><<<tg::grid_for(p->E, 128), 128, 0, s>>>(a, tg::table<T>(TG_P1_TET), p->E, geo);
      TG_CK_LAUNCH("k_elastic_geom");
    }
  }
  const size_t smem = (size_t)EB * 9 * p->max_row_len * sizeof(T);
  auto kern = k_elastic_gather<T, use_geo>;
  const tg_status st = tg::set_smem((const void*)kern, smem);
  if (st != TG_OK) return st;
  kern<<<tg::grid_for(p->N, EB), EB, smem, s>>>(a, tg::table<T>(TG_P1_TET), geo);
  TG_CK_LAUNCH("k_elastic_gather");
  return TG_OK;
}

}  // namespace

extern "C" tg_status tg_assemble_elasticity(const tg_pattern* p, tg_dtype dtype, const void* coords,
                                            const void* lam, const void* mu, tg_layout layout, void* vals_out,
                                            tg_stream stream) {
  if (!p || (dtype != TG_F32 && dtype != TG_F64) || p->el != TG_P1_TET_VEC3) return TG_ERR_INVALID_ARG;
  if ((p->N > 0 && !coords) || ((uintptr_t)coords % (dtype == TG_F32 ? 4 : 8)) != 0) return TG_ERR_INVALID_ARG;
  if (!(layout == TG_PER_ELEMENT || layout == TG_PER_QP || layout == TG_CONSTANT) || !lam || !mu ||
      (p->nnz > 0 && !vals_out))
    return TG_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  return dtype == TG_F32 ? elastic<float>(p, coords, lam, mu, layout, vals_out, s)
                         : elastic<double>(p, coords, lam, mu, layout, vals_out, s);
}
