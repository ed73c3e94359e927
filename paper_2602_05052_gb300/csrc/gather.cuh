// Row-owner gather shared by the single-instance and batched kernels:
// the fused Map (Algorithm 1) and the deterministic Reduce (Algorithm 2) of
// one CSR row.  See forward.cu for the design.
#pragma once

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

// Local row la of element e for the scalar form; false for a degenerate element.
template <int EL, typename T>
__device__ __forceinline__ bool scalar_row(const FwdArgs<T>& a, const RefTab<T>& ts, int64_t e, int la,
                                           T (&Krow)[Elem<EL>::nv]) {
  using El = Elem<EL>;
  const int32_t* cl = a.cells + e * El::nv;
  if constexpr (EL == TG_P1_TRI) {
    Geom<2, T> g;
    tri_geom(a.coords, __ldg(cl), __ldg(cl + 1), __ldg(cl + 2), g);
    const T adet = absv(g.det);
    if (!(adet > det_tiny<T>())) return false;
    const T inv = T(1) / adet;
    const T s = weighted_coef<T, El::nq>(a.coef, a.layout, e, ts.w, ts.wsum) * inv;
    p1_row<2, T>(g, la, s, a.c * adet, ts.M[la], Krow);
  } else if constexpr (EL == TG_P1_TET) {
    Geom<3, T> g;
    tet_geom(a.coords, __ldg(cl), __ldg(cl + 1), __ldg(cl + 2), __ldg(cl + 3), g);
    const T adet = absv(g.det);
    if (!(adet > det_tiny<T>())) return false;
    const T inv = T(1) / adet;
    const T s = weighted_coef<T, El::nq>(a.coef, a.layout, e, ts.w, ts.wsum) * inv;
    p1_row<3, T>(g, la, s, a.c * adet, ts.M[la], Krow);
  } else {
    Geom<2, T> g;
    tri_geom(a.coords, __ldg(cl), __ldg(cl + 1), __ldg(cl + 2), g);
    const T adet = absv(g.det);
    if (!(adet > det_tiny<T>())) return false;
    T kq[6];
    load_kq<T, 6>(a.coef, a.layout, e, kq);
    p2_row<T>(g, la, kq, T(1) / adet, a.c * adet, ts, Krow);
  }
  return true;
}


// Accumulate and store CSR row i.  acc points at this thread's column of
// the shared accumulators (stride BSZ).
template <int EL, typename T, int BSZ>
__device__ __forceinline__ void gather_row(const FwdArgs<T>& a, const RefTab<T>& ts, T* acc, int64_t i) {
  using El = Elem<EL>;
  const int r0 = __ldg(a.row_ptr + i), len = __ldg(a.row_ptr + i + 1) - r0;
  for (int p = 0; p < len; ++p) acc[p * BSZ] = T(0);
  const int j0 = __ldg(a.inc_ptr + i), j1 = __ldg(a.inc_ptr + i + 1);
  for (int j = j0; j < j1; ++j) {
    const int ea = __ldg(a.inc_e + j);
    const int64_t e = ea >> 3;
    const int la = ea & 7;
    const uint32_t w0 = __ldg(a.inc_pos + (int64_t)j * El::npw);
    const uint32_t w1 = El::npw == 2 ? __ldg(a.inc_pos + (int64_t)j * El::npw + 1) : 0u;
    T Krow[El::nv];
    if (!scalar_row<EL, T>(a, ts, e, la, Krow)) {
      record_error(a.status, TG_ERR_DEGENERATE_ELEMENT, e);
      continue;
    }
#pragma unroll
    for (int b = 0; b < El::nv; ++b) acc[pos_of(w0, w1, b) * BSZ] += Krow[b];
  }
  T* out = a.out + r0;
  for (int p = 0; p < len; ++p) out[p] = acc[p * BSZ];
}

// Host: reference tables of each element kind, built once per process.
template <typename T>
inline const RefTab<T>& table(tg_element el) {
  static const RefTab<T> t0 = ref_table<T>(TG_P1_TRI);
  static const RefTab<T> t1 = ref_table<T>(TG_P2_TRI);
  static const RefTab<T> t2 = ref_table<T>(TG_P1_TET);
  return el == TG_P1_TRI ? t0 : el == TG_P2_TRI ? t1 : t2;
}

// Host: allow a kernel the dynamic shared memory it needs (<= 227 KB).
inline tg_status set_smem(const void* func, size_t bytes) {
  if (bytes > 227 * 1024) {
    set_error("row too long for the shared-memory accumulators");
    return TG_ERR_UNSUPPORTED;
  }
  if (bytes > 48 * 1024) TG_CK(cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  return TG_OK;
}

}  // namespace tg
