// Backward (reverse mode) of the vector P1 elasticity assembly: dL/dlam,
// dL/dmu and dL/dcoords for an upstream gradient of the DoF-level values
// (a CSR array) or the adjoint outer product lam U^T of Eq. (adj).
#include <cstdint>

#include "blocks.cuh"

namespace {

constexpr int BB = 128;

// In two passes: each element evaluated once, then a per-node sum.  With
// G = grad(phi) (G[:, a] = n_a / det J) and the upstream weights W of one
// element (12 x 12, DoF (a, i) = 3a + i), the element's
//   L_e = |det J| (sl T1 + sm (T2 + T3)),  sl = sum_q w_q lam_q, sm likewise,
//   T1 = sum W_{ai,bj} G_ia G_jb,  T2 = sum W_{ai,bj} G_ja G_ib,
//   T3 = sum_ab (sum_i W_{ai,bi}) G_a . G_b,
// give dL/dlam_q = w_q |det J| T1, dL/dmu_q = w_q |det J| (T2 + T3), and,
// from d|det J| = |det J| tr(J^{-1} dJ) and dG = -J^{-T} dJ^T G,
//   dL/dx_c = P G[:, c],  P = L_e I - G Gam^T,  Gam = |det J| (sl dT1 + sm (dT2 + dT3))
// for every vertex c (dT = derivatives of T with respect to G).  W is
// streamed one 3 x 3 vertex-pair block at a time: the DoF-level CSR keeps
// block (a, b) at 9 row_ptr[v_a] + 3 (i len_a + pos_ab) + j.
template <typename T>
struct ElBwdArgs {
  const T* __restrict__ coords;
  const T* __restrict__ lam;
  const T* __restrict__ mu;
  int layout;
  const T* __restrict__ gvals;
  const T* __restrict__ lam_adj;
  const T* __restrict__ U;
  T* __restrict__ grad_lam;
  T* __restrict__ grad_mu;
  T* __restrict__ grad_coords;
  unsigned long long* status;
};

// The contractions of one element's upstream blocks with G: T1, T2, T3 and
// their derivatives dT/dG (d1, d2, d3, zero on entry).  wblk(p, q, w)
// yields the 3 x 3 block of vertex pair (p, q).  Every term below is linear
// in the block and the pair (q, p) contributes with W_qp^T exactly what the
// pair (p, q) contributes with W_pq, so FP64 (bound by the FP64 pipe)
// evaluates each unordered pair once with W_pq + W_qp^T (10 evaluations
// instead of 16: 3.19 -> 2.37 ms on 64^3); FP32 keeps the 16 (the sums
// take 8 more registers, which costs a CTA per SM and 3%).
template <typename T, typename WBlk>
__device__ __forceinline__ void el_bwd_sums(const T (&G)[3][4], WBlk wblk, T& t1, T& t2, T& t3, T (&d1)[3][4],
                                            T (&d2)[3][4], T (&d3)[3][4]) {
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int q = (sizeof(T) == 8 ? p : 0); q < 4; ++q) {
      T w[3][3];
      wblk(p, q, w);
      if (sizeof(T) == 8 && q != p) {
        T w2[3][3];
        wblk(q, p, w2);
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
          for (int j = 0; j < 3; ++j) w[i][j] += w2[j][i];
      }
      // w G_q, w^T G_q, w G_p, w^T G_p
      T wGq[3], wtGq[3], wGp[3], wtGp[3];
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        wGq[i] = w[i][0] * G[0][q] + w[i][1] * G[1][q] + w[i][2] * G[2][q];
        wtGq[i] = w[0][i] * G[0][q] + w[1][i] * G[1][q] + w[2][i] * G[2][q];
        wGp[i] = w[i][0] * G[0][p] + w[i][1] * G[1][p] + w[i][2] * G[2][p];
        wtGp[i] = w[0][i] * G[0][p] + w[1][i] * G[1][p] + w[2][i] * G[2][p];
      }
      const T cpq = w[0][0] + w[1][1] + w[2][2];
      const T gpq = G[0][p] * G[0][q] + G[1][p] * G[1][q] + G[2][p] * G[2][q];
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        t1 += G[i][p] * wGq[i];
        t2 += G[i][q] * wGp[i];
        d1[i][p] += wGq[i];
        d1[i][q] += wtGp[i];
        d2[i][p] += wtGq[i];
        d2[i][q] += wGp[i];
        d3[i][p] += cpq * G[i][q];
        d3[i][q] += cpq * G[i][p];
      }
      t3 += cpq * gpq;
    }
}

// The same sums in FP64 from the symmetrised blocks U_pq = W_pq + W_qp^T of
// each unordered pair (U_qp = U_pq^T; U_pp = W_pp + W_pp^T):
//   dT1/dG_p = sum_q U_pq G_q,  dT2/dG_p = sum_q U_pq^T G_q,
//   dT3/dG_p = sum_q tr(U_pq) G_q,  T_k = (1/2) sum_p G_p . dT_k/dG_p,
// each derivative accumulated by fused multiply-adds onto its running sum
// (pairs in the order of el_bwd_sums): about 40% fewer FP64 operations than
// accumulating every term of each pair separately.
template <typename T, typename WBlk>
__device__ __forceinline__ void el_bwd_sums_sym(const T (&G)[3][4], WBlk wblk, T& t1, T& t2, T& t3, T (&d1)[3][4],
                                                T (&d2)[3][4], T (&d3)[3][4]) {
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int q = p; q < 4; ++q) {
      T u[3][3];
      wblk(p, q, u);
      if (q != p) {
        T w2[3][3];
        wblk(q, p, w2);
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
          for (int j = 0; j < 3; ++j) u[i][j] += w2[j][i];
        const T tr = u[0][0] + u[1][1] + u[2][2];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          T a1 = d1[i][p], b1 = d1[i][q], a2 = d2[i][p], b2 = d2[i][q];
#pragma unroll
          for (int j = 0; j < 3; ++j) {
            a1 = fma(u[i][j], G[j][q], a1);  // U G_q
            b1 = fma(u[j][i], G[j][p], b1);  // U^T G_p
            a2 = fma(u[j][i], G[j][q], a2);  // U^T G_q
            b2 = fma(u[i][j], G[j][p], b2);  // U G_p
          }
          d1[i][p] = a1;
          d1[i][q] = b1;
          d2[i][p] = a2;
          d2[i][q] = b2;
          d3[i][p] = fma(tr, G[i][q], d3[i][p]);
          d3[i][q] = fma(tr, G[i][p], d3[i][q]);
        }
      } else {
        // U_pp is symmetric: U_pp G_p serves both derivatives
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
          for (int j = i + 1; j < 3; ++j) u[i][j] = u[j][i] = u[i][j] + u[j][i];
        const T tr = u[0][0] + u[1][1] + u[2][2];  // half the trace of U_pp
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          T v = u[i][0] * G[0][p];
          v = fma(u[i][1], G[1][p], v);
          v = fma(u[i][2], G[2][p], v);
          // the diagonal of U_pp is 2 W_pp[i][i]: v holds U_pp G_p minus W_pp[i][i] G_ip
          v = fma(u[i][i], G[i][p], v);
          d1[i][p] += v;
          d2[i][p] += v;
          d3[i][p] = fma(tr + tr, G[i][p], d3[i][p]);
        }
      }
    }
  T s1 = T(0), s2 = T(0), s3 = T(0);
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      s1 = fma(G[i][p], d1[i][p], s1);
      s2 = fma(G[i][p], d2[i][p], s2);
      s3 = fma(G[i][p], d3[i][p], s3);
    }
  t1 = T(0.5) * s1;
  t2 = T(0.5) * s2;
  t3 = T(0.5) * s3;
}

// dL/dx_c = P G[:, c] of one element from the sums of el_bwd_sums.
template <typename T>
__device__ __forceinline__ void el_bwd_gx(const T (&G)[3][4], T adet, T sl, T sm, T t1, T t2, T t3,
                                          const T (&d1)[3][4], const T (&d2)[3][4], const T (&d3)[3][4],
                                          T (&gx)[4][3]) {
  const T Le = adet * (sl * t1 + sm * (t2 + t3));
  T P[3][3];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int s2 = 0; s2 < 3; ++s2) {
      T acc = T(0);
#pragma unroll
      for (int c = 0; c < 4; ++c) acc += G[r][c] * (adet * (sl * d1[s2][c] + sm * (d2[s2][c] + d3[s2][c])));
      P[r][s2] = (r == s2 ? Le : T(0)) - acc;
    }
#pragma unroll
  for (int c = 0; c < 4; ++c)
#pragma unroll
    for (int r = 0; r < 3; ++r) gx[c][r] = P[r][0] * G[0][c] + P[r][1] * G[1][c] + P[r][2] * G[2][c];
}

// The element's vertices, coordinates and quadrature sums of lam and mu.
template <typename T>
__device__ __forceinline__ void el_bwd_coefs(const ElBwdArgs<T>& a, const tg::RefTab<T>& tab, int64_t e, T& sl,
                                             T& sm) {
  sl = T(0);
  sm = T(0);
  if (a.layout == TG_PER_QP) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      sl += tab.w[q] * __ldg(a.lam + 4 * e + q);
      sm += tab.w[q] * __ldg(a.mu + 4 * e + q);
    }
  } else {
    const T l0 = __ldg(a.lam + e), m0 = __ldg(a.mu + e);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      sl += tab.w[q] * l0;
      sm += tab.w[q] * m0;
    }
  }
}

// dL/dlam and dL/dmu of element e (written by one thread per element).
template <typename T>
__device__ __forceinline__ void el_bwd_write_coef(const ElBwdArgs<T>& a, const tg::RefTab<T>& tab, int64_t e,
                                                  T adet, T t1, T t23) {
  if (a.layout == TG_PER_QP) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if (a.grad_lam) a.grad_lam[4 * e + q] = tab.w[q] * adet * t1;
      if (a.grad_mu) a.grad_mu[4 * e + q] = tab.w[q] * adet * t23;
    }
  } else {
    if (a.grad_lam) a.grad_lam[e] = tab.wsum * adet * t1;
    if (a.grad_mu) a.grad_mu[e] = tab.wsum * adet * t23;
  }
}

template <typename T>
__device__ __forceinline__ void el_bwd_zero_coef(const ElBwdArgs<T>& a, int64_t e) {
  const int nc = a.layout == TG_PER_QP ? 4 : 1;
  for (int q = 0; q < nc; ++q) {
    if (a.grad_lam) a.grad_lam[e * nc + q] = T(0);
    if (a.grad_mu) a.grad_mu[e * nc + q] = T(0);
  }
}

// One element of the elasticity backward: writes dL/dlam, dL/dmu and
// returns the vertex terms gx.  FUSED: W = lam_adj U^T on the element's DoFs;
// otherwise the blocks are read from grad_vals at
// base(p, q) + 3 i len_p + j, base(p, q) = 9 row_ptr[v_p] + 3 pos_pq.
template <typename T, bool FUSED, typename Base>
__device__ __forceinline__ void el_bwd_element(const ElBwdArgs<T>& a, const tg::RefTab<T>& tab, int64_t e,
                                               const int (&vid)[4], const int (&lena)[4], Base base,
                                               T (&gx)[4][3]) {
  T x[4][3];
#pragma unroll
  for (int c = 0; c < 4; ++c) tg::load_x<3, T>(a.coords, vid[c], x[c]);
  T sl, sm;
  el_bwd_coefs<T>(a, tab, e, sl, sm);
  T la[4][3], ua[4][3];
  if constexpr (FUSED) {
#pragma unroll
    for (int c = 0; c < 4; ++c)
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        la[c][i] = __ldg(a.lam_adj + 3ll * vid[c] + i);
        ua[c][i] = __ldg(a.U + 3ll * vid[c] + i);
      }
  }
  tg::Geom<3, T> gm;
  tg::tet_geom_x(x[0], x[1], x[2], x[3], gm);
  const T adet = tg::absv(gm.det);
  if (!(adet > tg::det_tiny<T>())) {
    tg::record_error(a.status, TG_ERR_DEGENERATE_ELEMENT, e);
    el_bwd_zero_coef<T>(a, e);
#pragma unroll
    for (int c = 0; c < 4; ++c)
#pragma unroll
      for (int r = 0; r < 3; ++r) gx[c][r] = T(0);
    return;
  }
  const T id = tg::recip(gm.det);
  T G[3][4];  // G[r][c] = d phi_c / d x_r
#pragma unroll
  for (int c = 0; c < 4; ++c)
#pragma unroll
    for (int r = 0; r < 3; ++r) G[r][c] = gm.n[c][r] * id;
  T t1 = T(0), t2 = T(0), t3 = T(0);
  T d1[3][4], d2[3][4], d3[3][4];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) d1[r][c] = d2[r][c] = d3[r][c] = T(0);
  auto wblk = [&](int p, int q, T (&w)[3][3]) {
    if constexpr (FUSED) {
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int jj = 0; jj < 3; ++jj) w[i][jj] = la[p][i] * ua[q][jj];
    } else {
      const T* b = a.gvals + base(p, q);
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int jj = 0; jj < 3; ++jj) w[i][jj] = __ldg(b + 3ll * i * lena[p] + jj);
    }
  };
  if constexpr (sizeof(T) == 8) el_bwd_sums_sym<T>(G, wblk, t1, t2, t3, d1, d2, d3);
  else el_bwd_sums<T>(G, wblk, t1, t2, t3, d1, d2, d3);
  el_bwd_write_coef<T>(a, tab, e, adet, t1, t2 + t3);
  el_bwd_gx<T>(G, adet, sl, sm, t1, t2, t3, d1, d2, d3, gx);
}

// Pass 1: one thread per element writes dL/dlam, dL/dmu and the element's
// vertex terms gxe[e][c][r]; pass 2 (k_elastic_backward_node) sums every
// node's terms in increasing element order.  The blocks of W are found
// through the packed positions (elem_pos, rows of at most 16 nodes) or the
// slot map (elem_slot[e][p][q] = 9 row_ptr[v_p] + 3 pos_pq).
// Row blocks would evaluate an element once per block holding one of its
// vertices, about three times on tetrahedral grids; here the 24 incident
// tetrahedra of a node cost one pass over an E x 12 scratch instead.
template <typename T, bool FUSED, bool POS>
__global__ void __launch_bounds__(BB) k_elastic_backward_map(const ElBwdArgs<T> a,
                                                             const __grid_constant__ tg::RefTab<T> tab,
                                                             const int32_t* __restrict__ cells,
                                                             const int32_t* __restrict__ elem_slot,
                                                             const uint64_t* __restrict__ elem_pos,
                                                             const int32_t* __restrict__ row_ptr, int64_t E,
                                                             T* __restrict__ gxe) {
  for (int64_t e = (int64_t)blockIdx.x * BB + threadIdx.x; e < E; e += (int64_t)gridDim.x * BB) {
    int vid[4], rpa[4] = {0, 0, 0, 0}, lena[4] = {0, 0, 0, 0};
#pragma unroll
    for (int c = 0; c < 4; ++c) vid[c] = __ldg(cells + 4 * e + c);
    uint64_t ep = 0;
    if constexpr (!FUSED) {
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        rpa[c] = __ldg(row_ptr + vid[c]);
        lena[c] = __ldg(row_ptr + vid[c] + 1) - rpa[c];
      }
      if constexpr (POS) ep = __ldg(reinterpret_cast<const unsigned long long*>(elem_pos) + e);
    }
    auto base = [&](int p, int q) -> int64_t {
      if constexpr (POS) return 9ll * rpa[p] + 3ll * (int)((ep >> (4 * (p * 4 + q))) & 15u);
      else return (int64_t)__ldg(elem_slot + 16 * e + 4 * p + q);
    };
    T gx[4][3];
    el_bwd_element<T, FUSED>(a, tab, e, vid, lena, base, gx);
    if (gxe) {
#pragma unroll
      for (int c = 0; c < 4; ++c)
#pragma unroll
        for (int r = 0; r < 3; ++r) gxe[(4 * e + c) * 3 + r] = gx[c][r];
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(BB) k_elastic_backward_node(const int32_t* __restrict__ inc_ptr,
                                                              const int32_t* __restrict__ inc_e, int64_t N,
                                                              const T* __restrict__ gxe, T* __restrict__ grad_coords) {
  const int64_t i = (int64_t)blockIdx.x * BB + threadIdx.x;
  if (i >= N) return;
  T gs[3] = {T(0), T(0), T(0)};
  const int j1 = __ldg(inc_ptr + i + 1);
  for (int j = __ldg(inc_ptr + i); j < j1; ++j) {
    const int ea = __ldg(inc_e + j);
    const T* gp = gxe + ((int64_t)(ea >> 3) * 4 + (ea & 7)) * 3;
#pragma unroll
    for (int r = 0; r < 3; ++r) gs[r] += gp[r];
  }
#pragma unroll
  for (int r = 0; r < 3; ++r) grad_coords[3 * i + r] = gs[r];
}

}  // namespace

extern "C" tg_status tg_assemble_elasticity_backward(const tg_pattern* p, tg_dtype dtype, const void* coords,
                                                     const void* lam, const void* mu, tg_layout layout,
                                                     const void* grad_vals, const void* lam_adj, const void* U,
                                                     void* grad_lam, void* grad_mu, void* grad_coords,
                                                     tg_stream stream) {
  if (!p || (dtype != TG_F32 && dtype != TG_F64) || p->el != TG_P1_TET_VEC3) return TG_ERR_INVALID_ARG;
  if (!(layout == TG_PER_ELEMENT || layout == TG_PER_QP) || (p->N > 0 && !coords) || !lam || !mu)
    return TG_ERR_INVALID_ARG;
  if (!grad_vals && (!lam_adj || !U)) return TG_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if (p->E == 0) {
    if (grad_coords && p->N > 0) TG_CK(cudaMemsetAsync(grad_coords, 0, 3 * p->N * (dtype == TG_F32 ? 4 : 8), s));
    return TG_OK;
  }
  if (!grad_lam && !grad_mu && !grad_coords) return TG_OK;
  if (!p->elem_scratch) {
    tg::set_error("tg_assemble_elasticity_backward: the pattern has no element scratch");
    return TG_ERR_UNSUPPORTED;
  }
  auto run = [&](auto zero) -> tg_status {
    using T = decltype(zero);
    ElBwdArgs<T> a;
    a.coords = static_cast<const T*>(coords);
    a.lam = static_cast<const T*>(lam);
    a.mu = static_cast<const T*>(mu);
    a.layout = layout;
    a.gvals = static_cast<const T*>(grad_vals);
    a.lam_adj = static_cast<const T*>(lam_adj);
    a.U = static_cast<const T*>(U);
    a.grad_lam = static_cast<T*>(grad_lam);
    a.grad_mu = static_cast<T*>(grad_mu);
    a.grad_coords = static_cast<T*>(grad_coords);
    a.status = p->status;
    const tg::RefTab<T>& tab = tg::table<T>(TG_P1_TET);
    T* gxe = grad_coords ? static_cast<T*>(p->elem_scratch) : nullptr;
    const int grid = tg::grid_for(p->E, BB);
    if (!grad_vals)
      k_elastic_backward_map<T, true, false>
          <<<grid, BB, 0, s>>>(a, tab, p->cells, p->elem_slot, nullptr, p->row_ptr, p->E, gxe);
    else if (p->elem_pos)
      k_elastic_backward_map<T, false, true>
          <<<grid, BB, 0, s>>>(a, tab, p->cells, p->elem_slot, p->elem_pos, p->row_ptr, p->E, gxe);
    else
      k_elastic_backward_map<T, false, false>
          <<<grid, BB, 0, s>>>(a, tab, p->cells, p->elem_slot, nullptr, p->row_ptr, p->E, gxe);
    TG_CK_LAUNCH("k_elastic_backward_map");
    if (grad_coords) {
      k_elastic_backward_node<T><<<tg::grid_for(p->N, BB), BB, 0, s>>>(p->inc_ptr, p->inc_e, p->N, gxe,
                                                                       static_cast<T*>(grad_coords));
      TG_CK_LAUNCH("k_elastic_backward_node");
    }
    return TG_OK;
  };
  return dtype == TG_F32 ? run(0.0f) : run(0.0);
}
