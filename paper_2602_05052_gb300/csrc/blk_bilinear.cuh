// Map and Reduce of one element-once row block for the scalar bilinear form
// (and, with LOAD, the load vector): shared by the single-instance kernel
// (block views staged in shared memory) and the batched kernel (block
// views reading the pattern arrays in global memory).
#pragma once

#include "blocks.cuh"

namespace tg {

// 16-byte vector of T (the unit of the Map's output rows).
template <typename T>
struct Vec16;
template <>
struct Vec16<float> {
  using type = float4;
  static constexpr int n = 4;
  __device__ static float get(const float4& v, int k) { return k == 0 ? v.x : k == 1 ? v.y : k == 2 ? v.z : v.w; }
  __device__ static float4 make(const float* x) { return make_float4(x[0], x[1], x[2], x[3]); }
};
template <>
struct Vec16<double> {
  using type = double2;
  static constexpr int n = 2;
  __device__ static double get(const double2& v, int k) { return k == 0 ? v.x : v.y; }
  __device__ static double2 make(const double* x) { return make_double2(x[0], x[1]); }
};

// 16-byte vectors per (element, local vertex a) output row of the Map: row a
// of K_e in rotated column order K[a][a], K[a][a+1 mod NV], ..., then (with
// LOAD) F_e[a], zero-padded.
template <int NV, typename T, bool LOAD>
__host__ __device__ constexpr int kf_vecs() {
  return ((NV + (LOAD ? 1 : 0)) * (int)sizeof(T) + 15) / 16;
}

// Shared bytes of the Map's output rows and of the Reduce's accumulators
// (max_row_len positions x rs threads).
template <int NV, typename T, bool LOAD>
size_t blk_bilinear_work_bytes(int capE, int max_row_len, int rs) {
  return (size_t)NV * kf_vecs<NV, T, LOAD>() * capE * 16 + (size_t)max_row_len * rs * sizeof(T);
}

// Column order of output row r of the Map.  Rotated (the row-owner Reduce
// and the P1 fans): column c is local node (r + c) mod NV.  P2 fan order: a
// vertex row r as (r, r+1, r+2, edge(r, r+1), edge(r+2, r), opposite edge);
// the edge row of edge e = r - 3 from vertex e to e + 1 as (r, e, e+1, e+2,
// edge(e+1, e+2), edge(e+2, e)) (vertices mod 3; edge(v, v+1) is local
// node 3 + v).
template <int NV, bool FANP2>
__host__ __device__ constexpr int map_col(int r, int c) {
  if constexpr (!FANP2) {
    return (r + c) % NV;
  } else {
    if (r < 3) {
      const int o[6] = {r, (r + 1) % 3, (r + 2) % 3, 3 + r, 3 + (r + 2) % 3, 3 + (r + 1) % 3};
      return o[c];
    }
    const int e = r - 3;
    const int o[6] = {r, e, (e + 1) % 3, (e + 2) % 3, 3 + (e + 1) % 3, 3 + (e + 2) % 3};
    return o[c];
  }
}

// The Map of a block (any view with nbe, be[] and vtx(c, k)): every
// distinct element's output rows into KF, columns in map_col order.  SCR:
// the element's K_e (a.scr, NS values per element) and, with LOAD, F_e
// (a.scrF, NV per element) come from a first pass instead of being computed
// here.
template <int EL, typename T, int UB, bool LOAD, bool FANP2 = false, bool SCR = false, typename View>
__device__ __forceinline__ void blk_bilinear_map(const FwdArgs<T>& a, const RefTab<T>& tab, int capE, const View& v,
                                                 void* kf_buf) {
  constexpr int NV = Elem<EL>::nv, NG = Elem<EL>::ngeo, NS = NV * (NV + 1) / 2;
  constexpr int NW = kf_vecs<NV, T, LOAD>(), VN = Vec16<T>::n;
  using V = typename Vec16<T>::type;
  V* KF = reinterpret_cast<V*>(kf_buf);
  const int NT = blockDim.x;
  if constexpr (SCR) {
    for (int j0 = threadIdx.x; j0 < v.nbe; j0 += UB * NT) {
      T K[UB][NS], fe[UB][LOAD ? NV : 1];
#pragma unroll
      for (int u = 0; u < UB; ++u) {
        const int j = j0 + u * NT < v.nbe ? j0 + u * NT : 0;
        const int64_t e = bel_elem(v.be[j]);
        const T* src = a.scr + e * NS;
#pragma unroll
        for (int k = 0; k < NS; ++k) K[u][k] = __ldg(src + k);
        if constexpr (LOAD) {
#pragma unroll
          for (int r = 0; r < NV; ++r) fe[u][r] = __ldg(a.scrF + e * NV + r);
        }
      }
#pragma unroll
      for (int u = 0; u < UB; ++u) {
        const int j = j0 + u * NT;
        if (j >= v.nbe) continue;
#pragma unroll
        for (int r = 0; r < NV; ++r) {
          T row[NW * VN];
#pragma unroll
          for (int c = 0; c < NV; ++c) {
            const int b = map_col<NV, FANP2>(r, c), lo = r < b ? r : b, hi = r < b ? b : r;
            row[c] = K[u][lo * NV - lo * (lo - 1) / 2 + (hi - lo)];
          }
#pragma unroll
          for (int c = NV; c < NW * VN; ++c) row[c] = T(0);
          if constexpr (LOAD) row[NV] = fe[u][r];
#pragma unroll
          for (int w = 0; w < NW; ++w) KF[(r * NW + w) * capE + j] = Vec16<T>::make(row + w * VN);
        }
      }
    }
    return;
  }
  for (int j0 = threadIdx.x; j0 < v.nbe; j0 += UB * NT) {
    int e[UB];
    ElemIn<EL, T> in[UB];
#pragma unroll
    for (int u = 0; u < UB; ++u) {
      const int j = j0 + u * NT < v.nbe ? j0 + u * NT : 0;  // idle slots load element 0 of the list
      e[u] = (int)bel_elem(v.be[j]);
#pragma unroll
      for (int c = 0; c < NG; ++c) in[u].v[c] = v.vtx(c, j);
    }
#pragma unroll
    for (int u = 0; u < UB; ++u) elem_data<EL, T>(a, e[u], in[u]);
    T fv[LOAD ? UB : 1][NV];
    if constexpr (LOAD) {
#pragma unroll
      for (int u = 0; u < UB; ++u) p1_load_f<NV, T>(a.f, a.f_layout, e[u], in[u].v, fv[u]);
    }
#pragma unroll
    for (int u = 0; u < UB; ++u) {
      const int j = j0 + u * NT;
      if (j >= v.nbe) continue;
      T K[NS];
      T adet;
      bool ok;
      if constexpr (EL == TG_P2_TRI) ok = p2_elem_sym<T>(in[u], a.c, tab, K, &adet);
      else ok = p1_elem_sym<EL, T>(in[u], a.c, tab, K, &adet);
      if (!ok) {
        record_error(a.status, TG_ERR_DEGENERATE_ELEMENT, e[u]);
#pragma unroll
        for (int q = 0; q < NS; ++q) K[q] = T(0);
      }
      // FP64: the element's load entries at once (shared terms); FP32: row by
      // row, the same values with fewer live registers
      constexpr bool FE = LOAD && sizeof(T) == 8;
      T fe[FE ? NV : 1];
      if constexpr (FE) tg::p1_load_entries<NV, T>(a.f_layout, adet, fv[u], tab, fe);
#pragma unroll
      for (int r = 0; r < NV; ++r) {
        T row[NW * VN];
#pragma unroll
        for (int c = 0; c < NV; ++c) {
          const int b = map_col<NV, FANP2>(r, c), lo = r < b ? r : b, hi = r < b ? b : r;
          row[c] = K[lo * NV - lo * (lo - 1) / 2 + (hi - lo)];  // K_sym[lo][hi], rows packed upper
        }
#pragma unroll
        for (int c = NV; c < NW * VN; ++c) row[c] = T(0);
        if constexpr (FE) row[NV] = ok ? fe[r] : T(0);
        else if constexpr (LOAD) row[NV] = ok ? p1_load_entry<NV, T>(a.f_layout, adet, fv[u], tab, r) : T(0);
#pragma unroll
        for (int w = 0; w < NW; ++w) KF[(r * NW + w) * capE + j] = Vec16<T>::make(row + w * VN);
      }
    }
  }
}

//   Map    - every distinct element of the block computes K_e (and with
//            LOAD F_e) once (UB elements per thread, one round when
//            UB * blockDim.x >= the block's element count) and stores its
//            NV output rows: vector w of row a of element j at
//            KF[(a * NW + w) * capE + j];
//   Reduce - thread t owns row i = r0 + t; for each incidence (e, a) in
//            increasing e it adds row a of K_e: the diagonal entry (rotated
//            column 0) in a register, the others into acc[pos * rs + t]
//            (pos = the column's position in the row; the records hold the
//            positions in the same rotated order).  The row is then written
//            to its node's CSR row and acc cleared for the next block; with
//            LOAD also F of the node.  Ends with a CTA barrier.
// Every CSR entry is the sum of its contributions in increasing element
// order, starting from the first one.
template <int EL, typename T, int UB, bool LOAD, bool SCR = false>
__device__ __forceinline__ void blk_bilinear_block(const FwdArgs<T>& a, const RefTab<T>& tab, int capE,
                                                   const BlkView& v, void* kf_buf, T* acc) {
  constexpr int NV = Elem<EL>::nv;
  constexpr int NW = kf_vecs<NV, T, LOAD>(), VN = Vec16<T>::n;
  using V = typename Vec16<T>::type;
  const V* KF = reinterpret_cast<const V*>(kf_buf);
  const int NT = blockDim.x;
  blk_bilinear_map<EL, T, UB, LOAD, false, SCR>(a, tab, capE, v, kf_buf);
  __syncthreads();
  // Reduce
  {
    const int t = (int)threadIdx.x, i = v.r0 + t;
    if (i < v.r1) {
      const int je = v.ip[i + 1];
      T diag = T(0), fs = T(0);
      int dpos = -1;
      for (int j = v.ip[i]; j < je; ++j) {
        const auto r = blk_rec<NV>(v.rc, j);
        const V* src = KF + r.a() * NW * capE + r.le();
        V x[NW];
#pragma unroll
        for (int w = 0; w < NW; ++w) x[w] = src[w * capE];
        T kv[NW * VN];
#pragma unroll
        for (int k = 0; k < NW * VN; ++k) kv[k] = Vec16<T>::get(x[k / VN], k % VN);
        diag += kv[0];
        dpos = r.pos(0);
        // the NV - 1 off-diagonal columns of one incidence are distinct: loads first
        T cur[NV - 1];
#pragma unroll
        for (int c = 1; c < NV; ++c) cur[c - 1] = acc[r.pos(c) * NT + t];
#pragma unroll
        for (int c = 1; c < NV; ++c) acc[r.pos(c) * NT + t] = cur[c - 1] + kv[c];
        if constexpr (LOAD) fs += kv[NV];
      }
      if (dpos >= 0) acc[dpos * NT + t] = diag;
      if constexpr (LOAD) a.F[v.pm[i]] = fs;
      const int len = v.rp[i + 1] - v.rp[i];
      T* out = a.out + v.up[i];
      if constexpr (EL == TG_P2_TRI) {
        // P2 rows are long (up to 19 entries): 16-byte stores from the first
        // 16-byte boundary on, so that a warp's stores (one row per thread,
        // each in its own lines) write four FP32 values per sector
        const int head = (int)(((16u - ((unsigned)(uintptr_t)out & 15u)) & 15u) / sizeof(T));
        int q = 0;
        for (; q < head && q < len; ++q) {
          out[q] = acc[q * NT + t];
          acc[q * NT + t] = T(0);
        }
        for (; q + VN <= len; q += VN) {
          T x[VN];
#pragma unroll
          for (int k = 0; k < VN; ++k) {
            x[k] = acc[(q + k) * NT + t];
            acc[(q + k) * NT + t] = T(0);
          }
          *reinterpret_cast<V*>(out + q) = Vec16<T>::make(x);
        }
        for (; q < len; ++q) {
          out[q] = acc[q * NT + t];
          acc[q * NT + t] = T(0);
        }
      } else {
        for (int q = 0; q < len; ++q) {
          out[q] = acc[q * NT + t];
          acc[q * NT + t] = T(0);
        }
      }
    }
    __syncthreads();  // stage s and the work buffers are free again
  }
}

}  // namespace tg
