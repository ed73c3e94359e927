// Row-owner gather shared by the single-instance and batched kernels:
// the fused Map (Algorithm 1) and the deterministic Reduce (Algorithm 2) of
// a block of CSR rows.  See forward.cu for the design.
#pragma once

#include <algorithm>
#include <cstdint>

#include "elements.cuh"

namespace tg {

template <typename T>
struct FwdArgs {
  const int32_t* __restrict__ row_ptr;
  const int32_t* __restrict__ inc_ptr;
  const int32_t* __restrict__ inc_e;
  const uint32_t* __restrict__ inc_pos;
  const int32_t* __restrict__ cells;
  const int32_t* __restrict__ elem_slot;
  const T* __restrict__ coords;
  const T* __restrict__ coef;   // kappa, f or lambda
  const T* __restrict__ coef2;  // mu
  int layout;
  T c;
  T* __restrict__ out;
  int64_t n;  // rows (gather kernels) or elements (atomic kernel)
  unsigned long long* status;
  const T* __restrict__ f;  // load of the fused system assembly (NULL otherwise)
  int f_layout;
  T* __restrict__ F;
  // per-element K_e (packed upper triangles, scr) and F_e (scrF), written
  // by a first pass (FP64 two-pass assembly; NULL otherwise)
  const T* __restrict__ scr;
  const T* __restrict__ scrF;
};

template <typename T>
__host__ __device__ constexpr size_t tab_bytes() {
  return (sizeof(RefTab<T>) + 15) & ~size_t(15);
}

template <typename T>
__device__ __forceinline__ void copy_table(RefTab<T>& dst, const RefTab<T>& src) {
  constexpr int n = sizeof(RefTab<T>) / sizeof(T);
  for (int k = threadIdx.x; k < n; k += blockDim.x) reinterpret_cast<T*>(&dst)[k] = reinterpret_cast<const T*>(&src)[k];
  __syncthreads();
}

template <typename T>
__device__ __forceinline__ T absv(T x) {
  return x < T(0) ? -x : x;
}

template <typename T, int NQ>
__device__ __forceinline__ void load_kq(const T* __restrict__ v, int layout, int64_t e, T (&kq)[6]) {
  if (layout == TG_PER_QP) {
#pragma unroll
    for (int q = 0; q < NQ; ++q) kq[q] = __ldg(v + e * NQ + q);
  } else {
    const T k = layout == TG_PER_ELEMENT ? __ldg(v + e) : __ldg(v);
#pragma unroll
    for (int q = 0; q < NQ; ++q) kq[q] = k;
  }
}

// Element inputs of the scalar Map, loaded in two dependent levels so that
// several elements can be in flight per thread: ids (vertex indices), then
// data (vertex coordinates and the coefficient at the points).
template <int EL, typename T>
struct ElemIn {
  static constexpr int NG = Elem<EL>::ngeo, D = Elem<EL>::dim, NQ = Elem<EL>::nq;
  int v[NG];
  T x[NG][D];
  T kq[NQ];
};

template <int EL, typename T>
__device__ __forceinline__ void elem_ids(const FwdArgs<T>& a, int64_t e, ElemIn<EL, T>& in) {
  const int32_t* cl = a.cells + e * Elem<EL>::nv;
#pragma unroll
  for (int k = 0; k < ElemIn<EL, T>::NG; ++k) in.v[k] = __ldg(cl + k);
}

template <int EL, typename T>
__device__ __forceinline__ void elem_data(const FwdArgs<T>& a, int64_t e, ElemIn<EL, T>& in) {
  constexpr int NG = ElemIn<EL, T>::NG, D = ElemIn<EL, T>::D, NQ = ElemIn<EL, T>::NQ;
#pragma unroll
  for (int k = 0; k < NG; ++k) {
    if constexpr (D == 2) {
      const auto p = ldg2(a.coords, in.v[k]);
      in.x[k][0] = p.x;
      in.x[k][1] = p.y;
    } else {
#pragma unroll
      for (int r = 0; r < 3; ++r) in.x[k][r] = __ldg(a.coords + 3ll * in.v[k] + r);
    }
  }
  if (a.layout == TG_PER_QP) {
#pragma unroll
    for (int q = 0; q < NQ; ++q) in.kq[q] = __ldg(a.coef + e * NQ + q);
  } else {
    const T k = a.layout == TG_PER_ELEMENT ? __ldg(a.coef + e) : __ldg(a.coef);
#pragma unroll
    for (int q = 0; q < NQ; ++q) in.kq[q] = k;
  }
}

// Scales of a P1 matrix: sc = (sum_q w_q kappa_q) / |det J| and mc = c |det J|
// (fixed-order fused multiply-adds).
template <int NQ, typename T>
__device__ __forceinline__ void p1_scales(const T (&kq)[NQ], const RefTab<T>& ts, T adet, T c, T& sc, T& mc) {
  T s = ts.w[0] * kq[0];
#pragma unroll
  for (int q = 1; q < NQ; ++q) s = fma(ts.w[q], kq[q], s);
  sc = s * recip_fast(adet);
  mc = c * adet;
}

// Coordinates of node v.
template <int D, typename T>
__device__ __forceinline__ void load_x(const T* __restrict__ coords, int v, T (&x)[D]) {
  if constexpr (D == 2) {
    const auto p = ldg2(coords, v);
    x[0] = p.x;
    x[1] = p.y;
  } else {
#pragma unroll
    for (int r = 0; r < 3; ++r) x[r] = __ldg(coords + 3ll * v + r);
  }
}

// Upper triangle (row by row) of the P2 triangle matrix with kappa at the 6
// points (the quantity of p2_row for all rows at once):
//   K[a][b] = (1/|det|) sum_q w_q kappa_q gh_q,a^T C gh_q,b + c |det| M[a][b],
// the per-point transformed gradients h_a = w_q kappa_q C gh_q,a shared by
// the row.  All table reads have compile-time indices (tc: the kernel's
// constant parameter).  False for a degenerate element.
template <typename T>
__device__ __forceinline__ bool p2_elem_sym(const ElemIn<TG_P2_TRI, T>& in, T c, const RefTab<T>& tc, T (&K)[21],
                                            T* adet_out = nullptr) {
  Geom<2, T> g;
  tri_geom_x(in.x[0], in.x[1], in.x[2], g);
  const T adet = absv(g.det);
  if (adet_out) *adet_out = adet;
  if (!(adet > det_tiny<T>())) return false;
  const T c00 = g.n[1][0] * g.n[1][0] + g.n[1][1] * g.n[1][1];
  const T c01 = g.n[1][0] * g.n[2][0] + g.n[1][1] * g.n[2][1];
  const T c11 = g.n[2][0] * g.n[2][0] + g.n[2][1] * g.n[2][1];
  // 1/|det J| enters the per-point scale w_q kappa_q / |det J| of C, and
  // every product accumulates by fused multiply-adds
  const T inv = recip(adet), mc = c * adet;
#pragma unroll
  for (int k = 0; k < 21; ++k) K[k] = T(0);
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    const T wk = (tc.w[q] * in.kq[q]) * inv;
    const T w00 = wk * c00, w01 = wk * c01, w11 = wk * c11;
    T hx[6], hy[6];
#pragma unroll
    for (int a = 0; a < 6; ++a) {
      const T g0 = tc.gh[q][a][0], g1 = tc.gh[q][a][1];
      hx[a] = fma(w00, g0, w01 * g1);
      hy[a] = fma(w01, g0, w11 * g1);
    }
    int k = 0;
#pragma unroll
    for (int a = 0; a < 6; ++a)
#pragma unroll
      for (int b = a; b < 6; ++b, ++k) K[k] = fma(hx[a], tc.gh[q][b][0], fma(hy[a], tc.gh[q][b][1], K[k]));
  }
  int k = 0;
#pragma unroll
  for (int a = 0; a < 6; ++a)
#pragma unroll
    for (int b = a; b < 6; ++b, ++k) K[k] = fma(mc, tc.M[a][b], K[k]);
  return true;
}

// Load values f of a P1 element as its F_e needs them: at the vertices
// (PER_NODE), at the points (PER_QP; NQ == NV for P1) or one constant.
template <int NV, typename T>
__device__ __forceinline__ void p1_load_f(const T* __restrict__ f, int layout, int64_t e, const int (&vid)[NV],
                                          T (&fv)[NV]) {
  if (layout == TG_PER_NODE) {
#pragma unroll
    for (int c = 0; c < NV; ++c) fv[c] = __ldg(f + vid[c]);
  } else if (layout == TG_PER_QP) {
#pragma unroll
    for (int q = 0; q < NV; ++q) fv[q] = __ldg(f + e * NV + q);
  } else {
    fv[0] = __ldg(f);
#pragma unroll
    for (int q = 1; q < NV; ++q) fv[q] = fv[0];
  }
}

// F_e[c] = sum_q w_q |det J| f(x_q) phi_c(x_q) (second line of Eq.
// (matlclquad)); for nodal f the interpolant, F_e = |det J| M f_e.
template <int NV, typename T>
__device__ __forceinline__ T p1_load_entry(int layout, T adet, const T (&fv)[NV], const RefTab<T>& ts, int c) {
  if (layout == TG_PER_NODE) {
    T s2 = T(0);
#pragma unroll
    for (int b = 0; b < NV; ++b) s2 = fma(ts.M[c][b], fv[b], s2);
    return adet * s2;
  }
  if (layout == TG_PER_QP) {
    T s2 = T(0);
#pragma unroll
    for (int q = 0; q < NV; ++q) s2 = fma(ts.w[q] * ts.phi[q][c], fv[q], s2);
    return adet * s2;
  }
  return adet * ts.m1[c] * fv[0];
}

// All NV entries of F_e (the values of p1_load_entry).  In FP64 (bound by
// the FP64 pipe) the nodal case instead uses that the P1 mass matrix has
// one value m_d on the diagonal and one m_o off it:
//   F_c = (|det J| m_o) sum_b f_b + |det J| (m_d - m_o) f_c,
// the common terms formed once per element.
template <int NV, typename T>
__device__ __forceinline__ void p1_load_entries(int layout, T adet, const T (&fv)[NV], const RefTab<T>& ts,
                                                T (&F)[NV]) {
  if constexpr (sizeof(T) == 8 && NV <= 4) {
    if (layout == TG_PER_NODE) {
      T fs = fv[0];
#pragma unroll
      for (int b = 1; b < NV; ++b) fs += fv[b];
      const T base = (adet * ts.M[0][1]) * fs, ad = adet * (ts.M[0][0] - ts.M[0][1]);
#pragma unroll
      for (int c = 0; c < NV; ++c) F[c] = fma(ad, fv[c], base);
      return;
    }
  }
#pragma unroll
  for (int c = 0; c < NV; ++c) F[c] = p1_load_entry<NV, T>(layout, adet, fv, ts, c);
}

// Row la of the local matrix from loaded inputs; false for a degenerate
// element.  Same arithmetic, operation for operation, as scalar_row.
template <int EL, typename T>
__device__ __forceinline__ bool elem_row(const ElemIn<EL, T>& in, T c, const RefTab<T>& ts, const RefTab<T>& tc, int la,
                                         T (&Krow)[Elem<EL>::nv]) {
  if constexpr (EL == TG_P1_TRI || EL == TG_P2_TRI) {
    Geom<2, T> g;
    tri_geom_x(in.x[0], in.x[1], in.x[2], g);
    const T adet = absv(g.det);
    if (!(adet > det_tiny<T>())) return false;
    if constexpr (EL == TG_P1_TRI) {
      T sc, mc;
      p1_scales<3, T>(in.kq, ts, adet, c, sc, mc);
      p1_row<2, T>(g, la, sc, mc, ts.M, Krow);
    } else {
      p2_row<T>(g, la, in.kq, recip(adet), c * adet, ts, tc, Krow);
    }
  } else {
    Geom<3, T> g;
    tet_geom_x(in.x[0], in.x[1], in.x[2], in.x[3], g);
    const T adet = absv(g.det);
    if (!(adet > det_tiny<T>())) return false;
    T sc, mc;
    p1_scales<4, T>(in.kq, ts, adet, c, sc, mc);
    p1_row<3, T>(g, la, sc, mc, ts.M, Krow);
  }
  return true;
}

// Upper triangle (row by row) of the P1 local matrix of an element; false
// for a degenerate element.  Entry for entry the arithmetic of elem_row.
template <int EL, typename T>
__device__ __forceinline__ bool p1_elem_sym(const ElemIn<EL, T>& in, T c, const RefTab<T>& ts,
                                            T (&K)[Elem<EL>::nv * (Elem<EL>::nv + 1) / 2], T* adet_out = nullptr) {
  constexpr int D = Elem<EL>::dim, NV = D + 1;
  Geom<D, T> g;
  if constexpr (D == 2) tri_geom_x(in.x[0], in.x[1], in.x[2], g);
  else tet_geom_x(in.x[0], in.x[1], in.x[2], in.x[3], g);
  const T adet = absv(g.det);
  if (adet_out) *adet_out = adet;
  if (!(adet > det_tiny<T>())) return false;
  T sc, mc;
  p1_scales<Elem<EL>::nq, T>(in.kq, ts, adet, c, sc, mc);
  int k = 0;
  if constexpr (sizeof(T) == 8) {
    // the P1 mass matrix has one value on the diagonal and one off it
    T d[NV * (NV + 1) / 2];
    p1_dots<D, T>(g, d);
    const T md = mc * ts.M[0][0], mo = mc * ts.M[0][1];
#pragma unroll
    for (int a = 0; a < NV; ++a)
#pragma unroll
      for (int b = a; b < NV; ++b, ++k) K[k] = fma(sc, d[k], a == b ? md : mo);
  } else {
#pragma unroll
    for (int a = 0; a < NV; ++a)
#pragma unroll
      for (int b = a; b < NV; ++b, ++k) K[k] = p1_entry<T>(dot_n<D, T>(g.n[a], g.n[b]), sc, mc, ts.M[a][b]);
  }
  return true;
}

// Local row la of element e for the scalar form; false for a degenerate element.
template <int EL, typename T>
__device__ __forceinline__ bool scalar_row(const FwdArgs<T>& a, const RefTab<T>& ts, const RefTab<T>& tc, int64_t e, int la,
                                           T (&Krow)[Elem<EL>::nv]) {
  ElemIn<EL, T> in;
  elem_ids<EL, T>(a, e, in);
  elem_data<EL, T>(a, e, in);
  return elem_row<EL, T>(in, a.c, ts, tc, la, Krow);
}

// Accumulate and store CSR rows.
//
// Staged form used by every scalar forward kernel: a CTA owns the rows
// [r0, r1) (R = blockDim.x of them) and therefore the contiguous incidence
// range [inc_ptr[r0], inc_ptr[r1]) and the contiguous CSR value range
// [row_ptr[r0], row_ptr[r1]).
//   phase 1: all threads stride over the incidence range, UB incidences in
//            flight per thread, and evaluate the element rows (independent
//            loads: high memory-level parallelism); the rows and their
//            column positions go to shared memory;
//   phase 2: thread t sums the incidences of row r0 + t from shared memory
//            in increasing element order into the row's slice of a CSR-local
//            shared copy of the CTA's values;
//   store:   the CTA writes its value range with coalesced stores.
// Every slot is summed in the order of the one-thread-per-row formulation,
// so the results are bitwise reproducible and independent of R.
//
// Shared buffer: contrib [NV][cap] T | posw [NPW][cap] u32 | owner [cap] u8 |
// acc [R * max_row] T, with cap >= R * max_degree.
template <typename T, int NV, int NPW>
__host__ __device__ constexpr size_t staged_head(int cap) {
  return ((size_t)NV * cap * sizeof(T) + (size_t)NPW * cap * 4 + (size_t)cap + 15) & ~size_t(15);
}

template <typename T, int NV, int NPW>
__host__ __device__ constexpr size_t staged_bytes(int R, int cap, int max_row) {
  return staged_head<T, NV, NPW>(cap) + (size_t)max_row * R * sizeof(T);
}

// Phase 2 and the coalesced store, shared by both phase-1 variants.
template <typename T, int NV, int NPW>
__device__ __forceinline__ void reduce_rows(const FwdArgs<T>& a, const T* contrib, const uint32_t* posw, T* acc,
                                            int cap, int64_t r0, int64_t r1, int J0) {
  const int R = blockDim.x;
  const int64_t i = r0 + threadIdx.x;
  const int rbase = __ldg(a.row_ptr + r0);
  if (i < r1) {
    const int rs = __ldg(a.row_ptr + i) - rbase, len = __ldg(a.row_ptr + i + 1) - rbase - rs;
    T* row = acc + rs;
    for (int p = 0; p < len; ++p) row[p] = T(0);
    const int js = __ldg(a.inc_ptr + i) - J0, je = __ldg(a.inc_ptr + i + 1) - J0;
    for (int k = js; k < je; ++k) {
      const uint32_t w0 = posw[k];
      const uint32_t w1 = NPW == 2 ? posw[cap + k] : 0u;
#pragma unroll
      for (int b = 0; b < NV; ++b) row[pos_of(w0, w1, b)] += contrib[b * cap + k];
    }
  }
  __syncthreads();
  const int nz = __ldg(a.row_ptr + r1) - rbase;
  T* out = a.out + rbase;
  for (int k = threadIdx.x; k < nz; k += R) out[k] = acc[k];
  __syncthreads();  // the buffer is reused by the next row block
}

// Incidences in flight per thread in phase 1 (bounded by registers).
template <int EL, typename T>
__host__ __device__ constexpr int ub_of() {
  return EL == TG_P1_TRI ? 4 : EL == TG_P2_TRI ? 2 : (sizeof(T) == 4 ? 3 : 2);
}

// SCR (P1, FP64 two passes): the incidences' rows come from the per-element
// K_e of a first pass (a.scr, packed upper triangles of NV (NV + 1) / 2
// values), the values elem_row would compute.
template <int EL, typename T, bool SCR = false>
__device__ __forceinline__ void assemble_rows(const FwdArgs<T>& a, const RefTab<T>& ts, const RefTab<T>& tc, unsigned char* buf, int cap,
                                              int64_t r0, int64_t r1) {
  using El = Elem<EL>;
  constexpr int NV = El::nv, NPW = El::npw;
  const int R = blockDim.x;
  T* contrib = reinterpret_cast<T*>(buf);
  uint32_t* posw = reinterpret_cast<uint32_t*>(contrib + (size_t)NV * cap);
  T* acc = reinterpret_cast<T*>(buf + staged_head<T, NV, NPW>(cap));
  const int J0 = __ldg(a.inc_ptr + r0), J1 = __ldg(a.inc_ptr + r1);
  if constexpr (SCR) {
    constexpr int NS = NV * (NV + 1) / 2;
    for (int j = J0 + (int)threadIdx.x; j < J1; j += R) {
      const int ea = __ldg(a.inc_e + j);
      posw[j - J0] = __ldg(a.inc_pos + (int64_t)j * NPW);
      if (NPW == 2) posw[cap + j - J0] = __ldg(a.inc_pos + (int64_t)j * NPW + 1);
      const T* src = a.scr + (int64_t)(ea >> 3) * NS;
      const int la = ea & 7;
#pragma unroll
      for (int b = 0; b < NV; ++b) {
        // entry (la, b) of the packed triangle, la chosen at run time
        contrib[b * cap + (j - J0)] = __ldg(src + (la <= b ? la * NV - la * (la - 1) / 2 + (b - la)
                                                              : b * NV - b * (b - 1) / 2 + (la - b)));
      }
    }
    __syncthreads();
    reduce_rows<T, NV, NPW>(a, contrib, posw, acc, cap, r0, r1, J0);
    return;
  }
  // UB incidences per thread in flight: every load of one dependency level
  // (incidence record, then vertex ids, then coordinates and coefficients)
  // is issued for all of them before any is used.
  constexpr int UB = ub_of<EL, T>();
  for (int base = J0 + (int)threadIdx.x; base < J1; base += UB * R) {
    int ea[UB];
#pragma unroll
    for (int u = 0; u < UB; ++u) {
      const int j = base + u * R;
      ea[u] = j < J1 ? __ldg(a.inc_e + j) : 0;
      if (j < J1) {
        posw[j - J0] = __ldg(a.inc_pos + (int64_t)j * NPW);
        if (NPW == 2) posw[cap + j - J0] = __ldg(a.inc_pos + (int64_t)j * NPW + 1);
      }
    }
    ElemIn<EL, T> in[UB];
#pragma unroll
    for (int u = 0; u < UB; ++u) elem_ids<EL, T>(a, ea[u] >> 3, in[u]);
#pragma unroll
    for (int u = 0; u < UB; ++u) elem_data<EL, T>(a, ea[u] >> 3, in[u]);
#pragma unroll
    for (int u = 0; u < UB; ++u) {
      const int j = base + u * R;
      if (j < J1) {
        T Krow[NV];
        if (!elem_row<EL, T>(in[u], a.c, ts, tc, ea[u] & 7, Krow)) {
          record_error(a.status, TG_ERR_DEGENERATE_ELEMENT, ea[u] >> 3);
#pragma unroll
          for (int b = 0; b < NV; ++b) Krow[b] = T(0);
        }
#pragma unroll
        for (int b = 0; b < NV; ++b) contrib[b * cap + (j - J0)] = Krow[b];
      }
    }
  }
  __syncthreads();
  reduce_rows<T, NV, NPW>(a, contrib, posw, acc, cap, r0, r1, J0);
}

// One row block of the batched kernel.
template <int EL, typename T>
__device__ __forceinline__ void assemble_block(const FwdArgs<T>& a, const RefTab<T>& ts, const RefTab<T>& tc, unsigned char* buf, int cap,
                                               int64_t r0, int64_t r1) {
  assemble_rows<EL, T>(a, ts, tc, buf, cap, r0, r1);
}

// Host: reference tables of each element kind, built once per process.
template <typename T>
inline const RefTab<T>& table(tg_element el) {
  static const RefTab<T> t0 = ref_table<T>(TG_P1_TRI);
  static const RefTab<T> t1 = ref_table<T>(TG_P2_TRI);
  static const RefTab<T> t2 = ref_table<T>(TG_P1_TET);
  static const RefTab<T> t3 = ref_table<T>(TG_Q1_QUAD_VEC2);
  return el == TG_P1_TRI ? t0 : el == TG_P2_TRI ? t1 : el == TG_Q1_QUAD_VEC2 ? t3 : t2;
}

// Host: rows per CTA of the staged kernels and the shared-memory bytes of the
// stage (without the reference table): the largest R in {128, 64, 32}
// whose stage fits in 64 KB, else the largest that fits in 200 KB.
template <typename T, int NV, int NPW>
inline int staged_rows(int max_deg, int max_row, size_t* bytes) {
  const int cands[3] = {128, 64, 32};
  for (int lim : {64 * 1024, 200 * 1024})
    for (int R : cands) {
      const size_t b = staged_bytes<T, NV, NPW>(R, std::max(1, R * max_deg), max_row);
      if (b <= (size_t)lim) {
        *bytes = b;
        return R;
      }
    }
  *bytes = 0;
  return 0;
}

// Host: allow a kernel the dynamic shared memory it needs (<= 227 KB).
inline tg_status set_smem(const void* func, size_t bytes) {
  if (bytes > 227 * 1024) {
    set_error("row too long for the shared-memory accumulators");
    return TG_ERR_UNSUPPORTED;
  }
  // The 48 KB default covers static plus dynamic shared memory; kernels here
  // keep at most a few KB static, so the limit is raised above 40 KB dynamic.
  if (bytes > 40 * 1024) TG_CK(cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  return TG_OK;
}

}  // namespace tg
