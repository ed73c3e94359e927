// Map and Reduce of one element-once row block for the scalar bilinear form
// (and, with LOAD, the load vector): shared by the single-instance kernel
// (block views staged in shared memory) and the batched kernel (block
// views reading the pattern arrays in global memory).
#pragma once

#include "blocks.cuh"

namespace tg {

//   Map    - the local matrix K_e of every distinct element of the block into
//            Ke[NV*NV][capE] (UB elements per thread, one round when
//            UB * blockDim.x >= the block's element count), and with LOAD
//            F_e into Fe[NV][capE];
//   Reduce - row i adds, for each incidence (e, a) in increasing e, row a of
//            K_e into its CSR-local slice of acc and writes the slice to its
//            node's CSR row (clearing acc for the next block); with LOAD also
//            F of the node.  Ends with a CTA barrier.
template <int EL, typename T, int UB, bool LOAD>
__device__ __forceinline__ void blk_bilinear_block(const FwdArgs<T>& a, const RefTab<T>& tab, int capE,
                                                   const BlkView& v, T* Ke, T* Fe, T* acc) {
  constexpr int NV = Elem<EL>::nv, NG = Elem<EL>::ngeo, NS = NV * (NV + 1) / 2;
  const int NT = blockDim.x;
  // Map
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
      if constexpr (LOAD) {
#pragma unroll
        for (int c = 0; c < NV; ++c) Fe[c * capE + j] = ok ? p1_load_entry<NV, T>(a.f_layout, adet, fv[u], tab, c) : T(0);
      }
      int q = 0;
#pragma unroll
      for (int r = 0; r < NV; ++r)
#pragma unroll
        for (int c = r; c < NV; ++c, ++q) {
          Ke[(r * NV + c) * capE + j] = K[q];
          if (c != r) Ke[(c * NV + r) * capE + j] = K[q];
        }
    }
  }
  __syncthreads();
  // Reduce: rows summed in increasing element order, each row's values
  // written to its node's CSR row (acc cleared on the way for the next block)
  {
    const int i = v.r0 + (int)threadIdx.x;
    if (i < v.r1) {
      T* row = acc + (v.rp[i] - v.rp[v.r0]);
      const int je = v.ip[i + 1];
      T fs = T(0);
      for (int j = v.ip[i]; j < je; ++j) {
        const auto r = blk_rec<NV>(v.rc, j);
        const T* kr = Ke + r.a() * NV * capE + r.le();
        // the NV columns of one incidence are distinct: all loads first
        T cur[NV], add[NV];
#pragma unroll
        for (int c = 0; c < NV; ++c) {
          cur[c] = row[r.pos(c)];
          add[c] = kr[c * capE];
        }
#pragma unroll
        for (int c = 0; c < NV; ++c) row[r.pos(c)] = cur[c] + add[c];
        if constexpr (LOAD) fs += Fe[r.a() * capE + r.le()];
      }
      if constexpr (LOAD) a.F[v.pm[i]] = fs;
      const int len = v.rp[i + 1] - v.rp[i];
      T* out = a.out + v.up[i];
      for (int q = 0; q < len; ++q) {
        out[q] = row[q];
        row[q] = T(0);
      }
    }
    __syncthreads();  // stage s and the work buffers are free again
  }
}

}  // namespace tg
