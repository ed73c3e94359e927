// Forward assembly kernels: fused Map (Algorithm 1) + deterministic Reduce
// (Algorithm 2) as a row-owner gather.
//
// Design.  Algorithm 2 sums local entries into CSR slots through the
// routing matrices S_mat / S_vec.  Here every CSR row (mesh node) is owned by
// one thread, which walks the node's incident elements in increasing element
// order, evaluates the element's local row for that node directly from the
// vertex coordinates and coefficients (Map fused in), and accumulates it into
// a per-thread strip of shared memory at the column positions the pattern
// stored (the row-owned form of S_mat).  Each row is then written to HBM
// exactly once, contiguously.  There are no atomics, no intermediate
// K_local array in HBM, and the summation order of every slot is fixed, so
// results are bitwise reproducible.  The price is that an element's geometry
// is evaluated once per vertex (nv times), which is cheap in FP32 next to
// the memory traffic.
#include <cstdint>

#include "fan.cuh"

namespace {

constexpr int BS = 128;  // rows per CTA (scalar kernels)
constexpr int BT = 128;  // threads per CTA of the element-once kernels (>= rows per block)
// Largest shared memory of an element-once CTA (two CTAs per SM); patterns
// that need more use the generic kernels.
constexpr size_t kBlkSmemMax = 113 * 1024;

using tg::FwdArgs;
using tg::tab_bytes;
using tg::copy_table;
using tg::absv;
using tg::load_kq;
using tg::scalar_row;

// One CTA per block of R consecutive rows (staged gather, gather.cuh).
// Shared memory: the reference tables, then the stage buffer.
// SCR: the rows come from k_p1_map's per-element K_e (FP64 two passes).
template <int EL, typename T, bool SCR = false>
__global__ void __launch_bounds__(BS) k_bilinear_gather(const FwdArgs<T> a, const __grid_constant__ tg::RefTab<T> tab,
                                                        int cap) {
  extern __shared__ __align__(16) unsigned char smem[];
  auto& ts = *reinterpret_cast<tg::RefTab<T>*>(smem);
  copy_table(ts, tab);
  const int64_t r0 = (int64_t)blockIdx.x * blockDim.x;
  const int64_t r1 = r0 + blockDim.x < a.n ? r0 + blockDim.x : a.n;
  tg::assemble_rows<EL, T, SCR>(a, ts, tab, smem + tab_bytes<T>(), cap, r0, r1);
}


// Resident CTAs per SM the element-once kernels are compiled for (register
// budget 64K / (128 * n)): 7 for FP32 triangles with up to 4 elements per
// thread (70-72 registers, no spills), fewer where more live values need
// more registers.
template <int EL, typename T, int UB>
constexpr int blk_min_ctas() {
  return EL == TG_P1_TET ? 2 : EL == TG_P2_TRI ? 4 : sizeof(T) == 8 ? 4 : UB <= 4 ? 7 : 5;
}

// The same register budget for CTAs of BT threads (LOAD keeps one CTA of
// 128 threads less).
template <int EL, typename T, int UB, bool LOAD>
constexpr int blk_min_ctas_bt() {
  const int n = (blk_min_ctas<EL, T, UB>() - (LOAD ? 1 : 0)) * 128 / BT;
  return n < 1 ? 1 : n;
}

// Scalar forward over element-once row blocks (blocks.cuh): the Map and
// Reduce of blk_bilinear_block per row block.  LOAD also assembles the load
// vector F (a.f, a.f_layout -> a.F), entry for entry the arithmetic of
// k_load_blk: the system (K, F) in one pass.  acc_n = the accumulator count
// (the longest row x BS), cleared here once and by every block after use.
// SCR: the Map takes each element's K_e and F_e from k_p1_map (FP64 two
// passes).
template <int EL, typename T, int UB, bool LOAD, bool SCR = false>
__global__ void __launch_bounds__(BT, blk_min_ctas_bt<EL, T, UB, LOAD>()) k_bilinear_blk(
    const FwdArgs<T> a, const __grid_constant__ tg::RefTab<T> tab, const tg::BlkArgs g, int acc_n) {
  constexpr int NV = tg::Elem<EL>::nv;
  static_assert(!LOAD || EL != TG_P2_TRI, "the one-pass system is built for P1");
  extern __shared__ __align__(16) unsigned char smem[];
  tg::BlkPipe pipe;
  unsigned char* kf = pipe.init(smem, g);
  T* acc = reinterpret_cast<T*>(kf + (size_t)NV * tg::kf_vecs<NV, T, LOAD>() * g.capE * 16);
  for (int q = threadIdx.x; q < acc_n; q += blockDim.x) acc[q] = T(0);
  __syncthreads();  // publishes the mbarrier initialisation and the cleared acc
  TG_BLK_PIPELINE_BEGIN(pipe, g, a.status)
  tg::blk_bilinear_block<EL, T, UB, LOAD, SCR>(a, tab, g.capE, v, kf, acc);
  TG_BLK_PIPELINE_END
}

template <int NV, typename T, bool LOAD>
size_t bilinear_blk_smem(const tg_pattern* p) {
  const tg::BlkArgs g = tg::blk_args(p);
  return tg::blk_stage_bytes(p->blk_rows, g.capJ, g.capE, NV) +
         tg::blk_bilinear_work_bytes<NV, T, LOAD>(g.capE, p->max_row_len, BT);
}

// Map of the P1 load vector over a block (any view with nbe, be[] and
// vtx(c, k)): F_e of every distinct element into Fe[c * capE + j].
template <int D, typename T, int UB, typename View>
__device__ __forceinline__ void blk_load_map(const FwdArgs<T>& a, const tg::RefTab<T>& ts, int capE, const View& v,
                                             T* Fe) {
  constexpr int NV = D + 1;
  const int NT = blockDim.x;
  for (int j0 = threadIdx.x; j0 < v.nbe; j0 += UB * NT) {
    int e[UB];
    int vid[UB][NV];
#pragma unroll
    for (int u = 0; u < UB; ++u) {
      const int j = j0 + u * NT < v.nbe ? j0 + u * NT : 0;
      e[u] = tg::bel_elem(v.be[j]);
#pragma unroll
      for (int c = 0; c < NV; ++c) vid[u][c] = v.vtx(c, j);
    }
    T x[UB][NV][D];
    T fv[UB][NV];
#pragma unroll
    for (int u = 0; u < UB; ++u) {
#pragma unroll
      for (int c = 0; c < NV; ++c) tg::load_x<D, T>(a.coords, vid[u][c], x[u][c]);
      tg::p1_load_f<NV, T>(a.coef, a.layout, e[u], vid[u], fv[u]);
    }
#pragma unroll
    for (int u = 0; u < UB; ++u) {
      const int j = j0 + u * NT;
      if (j >= v.nbe) continue;
      tg::Geom<D, T> gm;
      if constexpr (D == 2) tg::tri_geom_x(x[u][0], x[u][1], x[u][2], gm);
      else tg::tet_geom_x(x[u][0], x[u][1], x[u][2], x[u][3], gm);
      const T adet = absv(gm.det);
      const bool ok = adet > tg::det_tiny<T>();
      if (!ok) tg::record_error(a.status, TG_ERR_DEGENERATE_ELEMENT, e[u]);
      if constexpr (sizeof(T) == 8) {  // the element's entries at once (shared terms)
        T fe[NV];
        tg::p1_load_entries<NV, T>(a.layout, adet, fv[u], ts, fe);
#pragma unroll
        for (int c = 0; c < NV; ++c) Fe[c * capE + j] = ok ? fe[c] : T(0);
      } else {  // the same values entry by entry, fewer live registers
#pragma unroll
        for (int c = 0; c < NV; ++c) Fe[c * capE + j] = ok ? tg::p1_load_entry<NV, T>(a.layout, adet, fv[u], ts, c) : T(0);
      }
    }
  }
}

// P1 load vector over element-once row blocks: Map F_e (NV values) per
// distinct element, Reduce F[i] = sum of the incidences' entries in
// increasing element order (second line of Eq. (matlclquad)).
template <int D, typename T, int UB>
__global__ void __launch_bounds__(BT) k_load_blk(const FwdArgs<T> a, const __grid_constant__ tg::RefTab<T> tab,
                                                 const tg::BlkArgs g) {
  constexpr int NV = D + 1;
  extern __shared__ __align__(16) unsigned char smem[];
  tg::BlkPipe pipe;
  T* Fe = reinterpret_cast<T*>(pipe.init(smem, g));
  __syncthreads();  // publishes the mbarrier initialisation
  TG_BLK_PIPELINE_BEGIN(pipe, g, a.status)
  blk_load_map<D, T, UB>(a, tab, g.capE, v, Fe);
  __syncthreads();
  {
    const int i = v.r0 + (int)threadIdx.x;
    if (i < v.r1) {
      T f = T(0);
      const int je = v.ip[i + 1];
      for (int j = v.ip[i]; j < je; ++j) {
        const auto r = tg::blk_rec<NV>(v.rc, j);
        f += Fe[r.a() * g.capE + r.le()];
      }
      a.out[v.pm[i]] = f;
    }
    __syncthreads();
  }
  TG_BLK_PIPELINE_END
}

// The fan-ordered kernels (P1 triangles, fan.cuh): the same Map, the Reduce
// along each row's fan in registers.  LOAD assembles the system (K, F).
// SCR: the Map takes each element's K_e and F_e from k_p1_map (the FP64
// two-pass form), the same values as computing them here.
template <typename T, int UB, bool LOAD, bool SCR = false>
__global__ void __launch_bounds__(BT, blk_min_ctas_bt<TG_P1_TRI, T, UB, LOAD>()) k_bilinear_fan(
    const FwdArgs<T> a, const __grid_constant__ tg::RefTab<T> tab, const tg::FanArgs g) {
  extern __shared__ __align__(16) unsigned char smem[];
  tg::FanPipe pipe;
  unsigned char* kf = pipe.init(smem, g);
  __syncthreads();  // publishes the mbarrier initialisation
  TG_FAN_PIPELINE_BEGIN(pipe, g, a.status)
  tg::blk_bilinear_map<TG_P1_TRI, T, UB, LOAD, false, SCR>(a, tab, g.capE, v, kf);
  __syncthreads();
  tg::fan_reduce_bilinear<T, LOAD>(a, g.capE, v, kf);
  __syncthreads();  // stage s and the Map's rows are free again
  TG_FAN_PIPELINE_END
}

// P2 triangles over the fans: the Map in the P2 fan column order, the
// Reduce of fan_reduce_p2.
template <typename T, int UB>
__global__ void __launch_bounds__(BT, blk_min_ctas_bt<TG_P2_TRI, T, UB, false>()) k_bilinear_fan_p2(
    const FwdArgs<T> a, const __grid_constant__ tg::RefTab<T> tab, const tg::FanArgs g) {
  extern __shared__ __align__(16) unsigned char smem[];
  tg::FanPipe pipe;
  unsigned char* kf = pipe.init(smem, g);
  __syncthreads();  // publishes the mbarrier initialisation
  TG_FAN_PIPELINE_BEGIN(pipe, g, a.status)
  tg::blk_bilinear_map<TG_P2_TRI, T, UB, false, true>(a, tab, g.capE, v, kf);
  __syncthreads();
  tg::fan_reduce_p2<T>(a, g.capE, v, kf);
  __syncthreads();  // stage s and the Map's rows are free again
  TG_FAN_PIPELINE_END
}

template <typename T, bool LOAD, int NV = 3>
size_t bilinear_fan_smem(const tg_pattern* p) {
  const tg::FanArgs g = tg::fan_args(p);
  return tg::fan_stage_bytes(g.R, g.capF, g.capE, NV) + (size_t)NV * tg::kf_vecs<NV, T, LOAD>() * g.capE * 16;
}

template <typename T, int UB>
__global__ void __launch_bounds__(BT) k_load_fan(const FwdArgs<T> a, const __grid_constant__ tg::RefTab<T> tab,
                                                 const tg::FanArgs g) {
  extern __shared__ __align__(16) unsigned char smem[];
  tg::FanPipe pipe;
  T* Fe = reinterpret_cast<T*>(pipe.init(smem, g));
  __syncthreads();  // publishes the mbarrier initialisation
  TG_FAN_PIPELINE_BEGIN(pipe, g, a.status)
  blk_load_map<2, T, UB>(a, tab, g.capE, v, Fe);
  __syncthreads();
  tg::fan_reduce_load<T>(a.out, g.capE, v, Fe);
  __syncthreads();
  TG_FAN_PIPELINE_END
}

template <typename T>
size_t load_fan_smem(const tg_pattern* p) {
  const tg::FanArgs g = tg::fan_args(p);
  return tg::fan_stage_bytes(g.R, g.capF, g.capE, 3) + (size_t)3 * g.capE * sizeof(T);
}

template <int D, typename T>
size_t load_blk_smem(const tg_pattern* p) {
  const tg::BlkArgs g = tg::blk_args(p);
  return tg::blk_stage_bytes(p->blk_rows, g.capJ, g.capE, D + 1) + (size_t)(D + 1) * g.capE * sizeof(T);
}

// Elements per thread of a Map round: enough for one round over the largest
// block where registers allow (FP32), else a smaller batch over several
// rounds.
template <typename T>
int blk_ub(const tg_pattern* p) {
  const int need = (p->blk_max_elems + BT - 1) / BT;
  if (p->el == TG_P2_TRI) return need <= 1 ? 1 : 2;
  if (sizeof(T) == 8) return need <= 2 ? 2 : 3;
  return need <= 2 ? 2 : need <= 3 ? 3 : need <= 4 ? 4 : need <= 5 ? 5 : 6;
}

// Threads per CTA of the element-once kernels (rows per block <= BT).
inline int blk_threads(const tg_pattern*) { return BT; }

// Persistent launch of an element-once kernel: one CTA per resident slot,
// at most one per row block.
template <typename K>
tg_status launch_blk(K kern, size_t smem, const tg_pattern* p, dim3* grid_out) {
  tg_status st = tg::set_smem((const void*)kern, smem);
  if (st != TG_OK) return st;
  int per_sm = 0;
  TG_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, blk_threads(p), smem));
  *grid_out = dim3((unsigned)std::min<int64_t>(p->n_blk, (int64_t)std::max(per_sm, 1) * tg::sm_count()));
  return TG_OK;
}

// Whether the element-once kernels serve this pattern at this precision.
template <typename T>
bool use_blk(const tg_pattern* p, size_t smem) {
  return p->bel != nullptr && smem <= kBlkSmemMax;
}

// Whether the fan-ordered kernels serve this pattern.
inline bool use_fan(const tg_pattern* p, size_t smem) {
  return p->fan != nullptr && p->bel != nullptr && smem <= kBlkSmemMax;
}

// The fan kernel for ub elements per thread (as k_bilinear_blk picks them).
template <typename T, bool LOAD, typename Go>
void fan_dispatch(int ub, Go&& go) {
  if constexpr (sizeof(T) == 8) {
    if (ub <= 2) go(k_bilinear_fan<T, 2, LOAD>);
    else go(k_bilinear_fan<T, 3, LOAD>);
  } else {
    if (ub <= 2) go(k_bilinear_fan<T, 2, LOAD>);
    else if (ub <= 3) go(k_bilinear_fan<T, 3, LOAD>);
    else if (ub <= 4) go(k_bilinear_fan<T, 4, LOAD>);
    else go(k_bilinear_fan<T, 6, LOAD>);
  }
}

// P1 simplices, pass 1 of 2 (FP64, bound by the FP64 pipe, where the row
// blocks would evaluate an element 1.23 times on triangles and about 3
// times on tetrahedra; FP32 tetrahedra): one thread per element computes
// K_e (packed upper triangle, NS = NV (NV + 1) / 2 values) into
// rec[NS e ...] and, with LOAD, F_e into recF[NV e ...], once, exactly as
// the block Map does; a degenerate element is flagged and gets zeros.  A
// CTA's 128 K records go to HBM as contiguous 16-byte vectors through
// shared memory.
template <int EL, typename T, bool LOAD>
__global__ void __launch_bounds__(128) k_p1_map(const FwdArgs<T> a, const __grid_constant__ tg::RefTab<T> tab,
                                               int64_t E, T* __restrict__ rec, T* __restrict__ recF) {
  constexpr int NV = tg::Elem<EL>::nv, NS = NV * (NV + 1) / 2;
  using V = typename tg::Vec16<T>::type;
  constexpr int VN = tg::Vec16<T>::n;
  __shared__ V buf[(128 * NS + VN - 1) / VN];
  T* bd = reinterpret_cast<T*>(buf);
  for (int64_t e0 = (int64_t)blockIdx.x * 128; e0 < E; e0 += (int64_t)gridDim.x * 128) {
    const int64_t e = e0 + threadIdx.x;
    T o[NS];
#pragma unroll
    for (int k = 0; k < NS; ++k) o[k] = T(0);
    if (e < E) {
      tg::ElemIn<EL, T> in;
      tg::elem_ids<EL, T>(a, e, in);
      tg::elem_data<EL, T>(a, e, in);
      T fv[NV], fe[NV];
      if constexpr (LOAD) tg::p1_load_f<NV, T>(a.f, a.f_layout, e, in.v, fv);
      T adet;
      if (!tg::p1_elem_sym<EL, T>(in, a.c, tab, o, &adet)) {
        tg::record_error(a.status, TG_ERR_DEGENERATE_ELEMENT, e);
#pragma unroll
        for (int k = 0; k < NS; ++k) o[k] = T(0);
#pragma unroll
        for (int r = 0; r < NV; ++r) fe[r] = T(0);
      } else if constexpr (LOAD) {
        tg::p1_load_entries<NV, T>(a.f_layout, adet, fv, tab, fe);
      }
      if constexpr (LOAD) {
#pragma unroll
        for (int r = 0; r < NV; ++r) recF[e * NV + r] = fe[r];
      }
    }
#pragma unroll
    for (int k = 0; k < NS; ++k) bd[threadIdx.x * NS + k] = o[k];
    __syncthreads();
    const int64_t nd = (E - e0 < 128 ? E - e0 : 128) * NS;  // values of this CTA's records
    T* dst0 = rec + NS * e0;  // 16-byte aligned: NS * 128 values are
    V* dst = reinterpret_cast<V*>(dst0);
    for (int64_t k = threadIdx.x; k < nd / VN; k += 128) dst[k] = buf[k];
    for (int64_t k = (nd / VN) * VN + threadIdx.x; k < nd; k += 128) dst0[k] = bd[k];
    __syncthreads();
  }
}

// P1, pass 2 of the load vector: F[i] = the sum of F_e[a] over node i's
// incidences (e, a) in increasing element order, starting from the first
// (the order and the values of the row-block load kernel).
template <int EL, typename T>
__global__ void __launch_bounds__(128) k_p1_load_reduce(const FwdArgs<T> a, const T* __restrict__ recF) {
  constexpr int NV = tg::Elem<EL>::nv;
  const int64_t i = (int64_t)blockIdx.x * 128 + threadIdx.x;
  if (i >= a.n) return;
  T fs = T(0);
  const int j1 = __ldg(a.inc_ptr + i + 1);
  for (int j = __ldg(a.inc_ptr + i); j < j1; ++j) {
    const int ea = __ldg(a.inc_e + j);
    fs += __ldg(recF + (int64_t)(ea >> 3) * NV + (ea & 7));
  }
  a.F[i] = fs;
}

// Comparison point: classic scatter-add (Eq. (scatter_add)) with atomics,
// one thread per element, output cleared beforehand.
template <int EL, typename T>
__global__ void __launch_bounds__(BS) k_bilinear_atomic(const FwdArgs<T> a, const __grid_constant__ tg::RefTab<T> tab) {
  using El = tg::Elem<EL>;
  extern __shared__ __align__(16) unsigned char smem[];
  auto& ts = *reinterpret_cast<tg::RefTab<T>*>(smem);
  copy_table(ts, tab);
  const int64_t e = (int64_t)blockIdx.x * BS + threadIdx.x;
  if (e >= a.n) return;
  const int32_t* slot = a.elem_slot + e * El::nv * El::nv;
#pragma unroll 1
  for (int la = 0; la < El::nv; ++la) {
    T Krow[El::nv];
    if (!scalar_row<EL, T>(a, ts, tab, e, la, Krow)) {
      tg::record_error(a.status, TG_ERR_DEGENERATE_ELEMENT, e);
      return;
    }
#pragma unroll
    for (int b = 0; b < El::nv; ++b) atomicAdd(a.out + __ldg(slot + la * El::nv + b), Krow[b]);
  }
}

// Load vector, staged like the bilinear kernel: phase 1 evaluates one
// (element, local node) visit per thread into contrib [NC][cap], phase 2
// sums each node's visits in increasing element order.
template <int EL, typename T, int NC>
__global__ void __launch_bounds__(BS) k_load_gather(const FwdArgs<T> a, const __grid_constant__ tg::RefTab<T> tab,
                                                    int cap) {
  using El = tg::Elem<EL>;
  extern __shared__ __align__(16) unsigned char smem[];
  auto& ts = *reinterpret_cast<tg::RefTab<T>*>(smem);
  T* contrib = reinterpret_cast<T*>(smem + tab_bytes<T>());
  copy_table(ts, tab);
  const int R = blockDim.x;
  const int64_t r0 = (int64_t)blockIdx.x * R;
  const int64_t r1 = r0 + R < a.n ? r0 + R : a.n;
  const int J0 = __ldg(a.inc_ptr + r0), J1 = __ldg(a.inc_ptr + r1);
#pragma unroll 2
  for (int j = J0 + (int)threadIdx.x; j < J1; j += R) {
    const int ea = __ldg(a.inc_e + j);
    const int64_t e = ea >> 3;
    const int la = ea & 7;
    const int32_t* cl = a.cells + e * El::nv;
    T F[NC];
#pragma unroll
    for (int k = 0; k < NC; ++k) F[k] = T(0);
    T det;
    if constexpr (El::dim == 2) det = tg::tri_det(a.coords, __ldg(cl), __ldg(cl + 1), __ldg(cl + 2));
    else det = tg::tet_det(a.coords, __ldg(cl), __ldg(cl + 1), __ldg(cl + 2), __ldg(cl + 3));
    const T adet = absv(det);
    if (!(adet > tg::det_tiny<T>())) {
      tg::record_error(a.status, TG_ERR_DEGENERATE_ELEMENT, e);
    } else if (a.layout == TG_PER_NODE) {
      int v[El::nv];
#pragma unroll
      for (int b = 0; b < El::nv; ++b) v[b] = __ldg(cl + b);
#pragma unroll
      for (int k = 0; k < NC; ++k) {
        T s = T(0);
#pragma unroll
        for (int b = 0; b < El::nv; ++b) s += ts.M[la][b] * __ldg(a.coef + (int64_t)v[b] * NC + k);
        F[k] += adet * s;
      }
    } else if (a.layout == TG_PER_QP) {
#pragma unroll
      for (int k = 0; k < NC; ++k) {
        T s = T(0);
#pragma unroll
        for (int q = 0; q < El::nq; ++q) s += ts.w[q] * ts.phi[q][la] * __ldg(a.coef + (e * El::nq + q) * NC + k);
        F[k] += adet * s;
      }
    } else {
#pragma unroll
      for (int k = 0; k < NC; ++k) F[k] += adet * ts.m1[la] * __ldg(a.coef + k);
    }
#pragma unroll
    for (int k = 0; k < NC; ++k) contrib[k * cap + (j - J0)] = F[k];
  }
  __syncthreads();
  const int64_t i = r0 + threadIdx.x;
  if (i >= r1) return;
  const int js = __ldg(a.inc_ptr + i) - J0, je = __ldg(a.inc_ptr + i + 1) - J0;
#pragma unroll
  for (int k = 0; k < NC; ++k) {
    T s = T(0);
    for (int m = js; m < je; ++m) s += contrib[k * cap + m];
    a.out[i * NC + k] = s;
  }
}

// ---------------------------------------------------------------- host side
using tg::table;
using tg::set_smem;

template <typename T>
FwdArgs<T> base_args(const tg_pattern* p, const void* coords) {
  FwdArgs<T> a;
  a.row_ptr = p->row_ptr;
  a.inc_ptr = p->inc_ptr;
  a.inc_e = p->inc_e;
  a.inc_pos = p->inc_pos;
  a.cells = p->cells;
  a.elem_slot = p->elem_slot;
  a.coords = static_cast<const T*>(coords);
  a.coef = nullptr;
  a.coef2 = nullptr;
  a.layout = 0;
  a.c = T(0);
  a.out = nullptr;
  a.n = p->N;
  a.status = p->status;
  a.f = nullptr;
  a.f_layout = 0;
  a.F = nullptr;
  a.scr = nullptr;
  a.scrF = nullptr;
  return a;
}

bool aligned(const void* ptr, size_t a) { return ((uintptr_t)ptr % a) == 0; }

// P1 simplices with row blocks in two passes through the pattern's element
// scratch (FP64 triangles and tetrahedra, FP32 tetrahedra): k_p1_map
// evaluates every element once, then the block kernel (triangles: the fan
// kernel) reduces the stored K_e (and F_e).  The same values and summation
// order as the one-pass kernels, hence the same bits; overlapping calls on
// one pattern share the scratch.  Below kTwoPassMinElems elements one pass
// is faster (a second launch costs more than the repeated element work).
constexpr int64_t kTwoPassMinElems = 1 << 16;

template <typename T, int EL>
bool two_pass_applies(const tg_pattern* p) {
  return p->elem_scratch && p->E >= kTwoPassMinElems && (sizeof(T) == 8 || EL == TG_P1_TET);
}

template <int EL, typename T, bool LOAD>
tg_status two_pass(const tg_pattern* p, FwdArgs<T> a, cudaStream_t s) {
  const tg::RefTab<T>& tab = table<T>(p->el);
  constexpr int NV = tg::Elem<EL>::nv, NS = NV * (NV + 1) / 2;
  T* rec = static_cast<T*>(p->elem_scratch);
  T* recF = rec + p->E * NS;
  if (p->E > 0) {
    const int g1 = (int)std::min<int64_t>(tg::grid_for(p->E, 128), 32ll * tg::sm_count());
    k_p1_map<EL, T, LOAD><<<g1, 128, 0, s>>>(a, tab, p->E, rec, recF);
    TG_CK_LAUNCH("k_p1_map");
  }
  a.scr = rec;
  a.scrF = recF;
  dim3 grid;
  if constexpr (EL == TG_P1_TRI) {
    const size_t sb = bilinear_fan_smem<T, LOAD>(p);
    auto kern = k_bilinear_fan<T, 3, LOAD, true>;
    tg_status st = launch_blk(kern, sb, p, &grid);
    if (st != TG_OK) return st;
    kern<<<grid, blk_threads(p), sb, s>>>(a, tab, tg::fan_args(p));
    TG_CK_LAUNCH("k_bilinear_fan<scratch>");
  } else {
    const size_t sb = bilinear_blk_smem<tg::Elem<EL>::nv, T, LOAD>(p);
    auto kern = k_bilinear_blk<EL, T, sizeof(T) == 8 ? 2 : 4, LOAD, true>;
    tg_status st = launch_blk(kern, sb, p, &grid);
    if (st != TG_OK) return st;
    kern<<<grid, blk_threads(p), sb, s>>>(a, tab, tg::blk_args(p), p->max_row_len * BT);
    TG_CK_LAUNCH("k_bilinear_blk<scratch>");
  }
  return TG_OK;
}

template <int EL, typename T>
tg_status launch_bilinear(const tg_pattern* p, FwdArgs<T> a, cudaStream_t s, bool atomic) {
  const tg::RefTab<T>& tab = table<T>(p->el);
  if (atomic) {
    a.n = p->E;
    if (p->nnz) TG_CK(cudaMemsetAsync(a.out, 0, p->nnz * sizeof(T), s));
    if (p->E == 0) return TG_OK;
    const size_t smem = tab_bytes<T>();
    k_bilinear_atomic<EL, T><<<tg::grid_for(p->E, BS), BS, smem, s>>>(a, tab);
    TG_CK_LAUNCH("k_bilinear_atomic");
    return TG_OK;
  }
  using El = tg::Elem<EL>;
  size_t stage = 0;
  const int R = tg::staged_rows<T, El::nv, El::npw>(p->max_deg, p->max_row_len, &stage);
  if (R == 0) {
    tg::set_error("mesh degree too large for the staged gather");
    return TG_ERR_UNSUPPORTED;
  }
  const size_t smem = tab_bytes<T>() + stage;
  const int cap = std::max(1, R * p->max_deg);
  if constexpr (EL == TG_P2_TRI) {
    const size_t sb = bilinear_fan_smem<T, false, 6>(p);
    if (use_fan(p, sb)) {
      tg_status st = TG_OK;
      auto go = [&](auto kern) {
        dim3 grid;
        if ((st = launch_blk(kern, sb, p, &grid)) != TG_OK) return;
        kern<<<grid, blk_threads(p), sb, s>>>(a, tab, tg::fan_args(p));
      };
      if (blk_ub<T>(p) <= 1) go(k_bilinear_fan_p2<T, 1>);
      else go(k_bilinear_fan_p2<T, 2>);
      if (st != TG_OK) return st;
      TG_CK_LAUNCH("k_bilinear_fan_p2");
      return TG_OK;
    }
  }
  if constexpr (EL == TG_P1_TRI) {
    const size_t sb = bilinear_fan_smem<T, false>(p);
    if (use_fan(p, sb)) {
      if constexpr (sizeof(T) == 8) {
        if (two_pass_applies<T, TG_P1_TRI>(p)) return two_pass<TG_P1_TRI, T, false>(p, a, s);
      }
      tg_status st = TG_OK;
      auto go = [&](auto kern) {
        dim3 grid;
        if ((st = launch_blk(kern, sb, p, &grid)) != TG_OK) return;
        kern<<<grid, blk_threads(p), sb, s>>>(a, tab, tg::fan_args(p));
      };
      fan_dispatch<T, false>(blk_ub<T>(p), go);
      if (st != TG_OK) return st;
      TG_CK_LAUNCH("k_bilinear_fan");
      return TG_OK;
    }
  }
  {
    const size_t sb = bilinear_blk_smem<El::nv, T, false>(p);
    if (use_blk<T>(p, sb)) {
      if constexpr (EL == TG_P1_TET) {
        if (two_pass_applies<T, TG_P1_TET>(p)) return two_pass<TG_P1_TET, T, false>(p, a, s);
      }
      const int ub = blk_ub<T>(p);
      tg_status st = TG_OK;
      auto go = [&](auto kern) {
        dim3 grid;
        if ((st = launch_blk(kern, sb, p, &grid)) != TG_OK) return;
        kern<<<grid, blk_threads(p), sb, s>>>(a, tab, tg::blk_args(p), p->max_row_len * BT);
      };
      if constexpr (EL == TG_P2_TRI) {
        if (ub <= 1) go(k_bilinear_blk<EL, T, 1, false>);
        else go(k_bilinear_blk<EL, T, 2, false>);
      } else if constexpr (sizeof(T) == 8) {
        if (ub == 2) go(k_bilinear_blk<EL, T, 2, false>);
        else go(k_bilinear_blk<EL, T, 3, false>);
      } else {
        if (ub == 2) go(k_bilinear_blk<EL, T, 2, false>);
        else if (ub == 3) go(k_bilinear_blk<EL, T, 3, false>);
        else if (ub == 4) go(k_bilinear_blk<EL, T, 4, false>);
        else if (ub == 5) go(k_bilinear_blk<EL, T, 5, false>);
        else go(k_bilinear_blk<EL, T, 6, false>);
      }
      if (st != TG_OK) return st;
      TG_CK_LAUNCH("k_bilinear_blk");
      return TG_OK;
    }
  }
  if constexpr (EL != TG_P2_TRI) {
    if (two_pass_applies<T, EL>(p)) {  // P1: every element once, then the rows' sums
      const int g1 = (int)std::min<int64_t>(tg::grid_for(p->E, 128), 32ll * tg::sm_count());
      k_p1_map<EL, T, false><<<g1, 128, 0, s>>>(a, tab, p->E, static_cast<T*>(p->elem_scratch), nullptr);
      TG_CK_LAUNCH("k_p1_map");
      a.scr = static_cast<const T*>(p->elem_scratch);
      tg_status st = set_smem((const void*)k_bilinear_gather<EL, T, true>, smem);
      if (st != TG_OK) return st;
      k_bilinear_gather<EL, T, true><<<tg::grid_for(p->N, R), R, smem, s>>>(a, tab, cap);
      TG_CK_LAUNCH("k_bilinear_gather<scratch>");
      return TG_OK;
    }
  }
  tg_status st = set_smem((const void*)k_bilinear_gather<EL, T>, smem);
  if (st != TG_OK) return st;
  k_bilinear_gather<EL, T><<<tg::grid_for(p->N, R), R, smem, s>>>(a, tab, cap);
  TG_CK_LAUNCH("k_bilinear_gather");
  return TG_OK;
}

template <typename T>
tg_status bilinear(const tg_pattern* p, const void* coords, const void* kappa, tg_layout kl, double c, void* vals,
                   cudaStream_t s, bool atomic) {
  FwdArgs<T> a = base_args<T>(p, coords);
  a.coef = static_cast<const T*>(kappa);
  a.layout = kl;
  a.c = (T)c;
  a.out = static_cast<T*>(vals);
  switch (p->el) {
    case TG_P1_TRI: return launch_bilinear<TG_P1_TRI, T>(p, a, s, atomic);
    case TG_P2_TRI: return launch_bilinear<TG_P2_TRI, T>(p, a, s, atomic);
    default: return launch_bilinear<TG_P1_TET, T>(p, a, s, atomic);
  }
}

tg_status check_common(const tg_pattern* p, tg_dtype dtype, const void* coords) {
  if (!p || (dtype != TG_F32 && dtype != TG_F64)) return TG_ERR_INVALID_ARG;
  if (p->N > 0 && !coords) return TG_ERR_INVALID_ARG;
  const size_t es = dtype == TG_F32 ? 4 : 8;
  if (!aligned(coords, p->dim == 2 ? 2 * es : es)) {
    tg::set_error("coords must be aligned to 2 * sizeof(dtype) for 2D meshes");
    return TG_ERR_INVALID_ARG;
  }
  return TG_OK;
}

template <typename T>
tg_status load(const tg_pattern* p, const void* coords, const void* f, tg_layout fl, int ncomp, void* F,
               cudaStream_t s) {
  FwdArgs<T> a = base_args<T>(p, coords);
  a.coef = static_cast<const T*>(f);
  a.layout = fl;
  a.out = static_cast<T*>(F);
  const tg_element el = p->el == TG_P1_TET_VEC3 ? TG_P1_TET : p->el;
  const tg::RefTab<T>& tab = table<T>(el);
  if (ncomp == 1 && el == TG_P1_TRI && use_fan(p, load_fan_smem<T>(p))) {
    const size_t sb = load_fan_smem<T>(p);
    tg_status st = TG_OK;
    auto go = [&](auto kern) {
      dim3 grid;
      if ((st = launch_blk(kern, sb, p, &grid)) != TG_OK) return;
      kern<<<grid, blk_threads(p), sb, s>>>(a, tab, tg::fan_args(p));
    };
    if constexpr (sizeof(T) == 8) go(k_load_fan<T, 2>);
    else if (blk_ub<T>(p) <= 4) go(k_load_fan<T, 4>);
    else go(k_load_fan<T, 6>);
    if (st != TG_OK) return st;
    TG_CK_LAUNCH("k_load_fan");
    return TG_OK;
  }
  if (ncomp == 1 && (el == TG_P1_TRI || el == TG_P1_TET) && p->bel) {
    const bool tri = el == TG_P1_TRI;
    const size_t sb = tri ? load_blk_smem<2, T>(p) : load_blk_smem<3, T>(p);
    if (use_blk<T>(p, sb)) {
      const int ub = sizeof(T) == 8 ? 2 : blk_ub<T>(p) <= 4 ? 4 : 6;
      tg_status st = TG_OK;
      auto go = [&](auto kern) {
        dim3 grid;
        if ((st = launch_blk(kern, sb, p, &grid)) != TG_OK) return;
        kern<<<grid, blk_threads(p), sb, s>>>(a, tab, tg::blk_args(p));
      };
      if constexpr (sizeof(T) == 8) {
        if (tri) go(k_load_blk<2, T, 2>);
        else go(k_load_blk<3, T, 2>);
      } else {
        if (tri) {
          if (ub == 4) go(k_load_blk<2, T, 4>);
          else go(k_load_blk<2, T, 6>);
        } else {
          if (ub == 4) go(k_load_blk<3, T, 4>);
          else go(k_load_blk<3, T, 6>);
        }
      }
      if (st != TG_OK) return st;
      TG_CK_LAUNCH("k_load_blk");
      return TG_OK;
    }
  }
  // rows per CTA: the largest R in {128, 64, 32} whose stage fits in 64 KB
  int R = BS;
  while (R > 32 && (size_t)ncomp * R * p->max_deg * sizeof(T) > 64 * 1024) R /= 2;
  const int cap = std::max(1, R * p->max_deg);
  const size_t smem = tab_bytes<T>() + (size_t)ncomp * cap * sizeof(T);
  const int grid = tg::grid_for(p->N, R);
  tg_status st = TG_OK;
  auto go = [&](auto kern) {
    if ((st = set_smem((const void*)kern, smem)) != TG_OK) return;
    kern<<<grid, R, smem, s>>>(a, tab, cap);
  };
  if (el == TG_P1_TRI) {
    if (ncomp == 1) go(k_load_gather<TG_P1_TRI, T, 1>);
    else go(k_load_gather<TG_P1_TRI, T, 3>);
  } else if (el == TG_P2_TRI) {
    if (ncomp == 1) go(k_load_gather<TG_P2_TRI, T, 1>);
    else go(k_load_gather<TG_P2_TRI, T, 3>);
  } else {
    if (ncomp == 1) go(k_load_gather<TG_P1_TET, T, 1>);
    else go(k_load_gather<TG_P1_TET, T, 3>);
  }
  if (st != TG_OK) return st;
  TG_CK_LAUNCH("k_load_gather");
  return TG_OK;
}

// The system (K, F) in one pass where the element-once kernels apply, else
// the two assemblies one after the other (same values either way).
template <typename T>
tg_status system_asm(const tg_pattern* p, const void* coords, const void* kappa, tg_layout kl, double c,
                     const void* f, tg_layout fl, void* vals, void* F, cudaStream_t s) {
  if ((p->el == TG_P1_TRI || p->el == TG_P1_TET) && p->bel) {
    FwdArgs<T> a = base_args<T>(p, coords);
    a.coef = static_cast<const T*>(kappa);
    a.layout = kl;
    a.c = (T)c;
    a.out = static_cast<T*>(vals);
    a.f = static_cast<const T*>(f);
    a.f_layout = fl;
    a.F = static_cast<T*>(F);
    const bool tri = p->el == TG_P1_TRI;
    if (tri && use_fan(p, bilinear_fan_smem<T, true>(p))) {
      if constexpr (sizeof(T) == 8) {
        if (two_pass_applies<T, TG_P1_TRI>(p)) return two_pass<TG_P1_TRI, T, true>(p, a, s);
      }
      const size_t sb = bilinear_fan_smem<T, true>(p);
      const tg::RefTab<T>& tab = table<T>(p->el);
      tg_status st = TG_OK;
      auto go = [&](auto kern) {
        dim3 grid;
        if ((st = launch_blk(kern, sb, p, &grid)) != TG_OK) return;
        kern<<<grid, blk_threads(p), sb, s>>>(a, tab, tg::fan_args(p));
      };
      fan_dispatch<T, true>(blk_ub<T>(p), go);
      if (st != TG_OK) return st;
      TG_CK_LAUNCH("k_bilinear_fan<load>");
      return TG_OK;
    }
    const size_t sb = tri ? bilinear_blk_smem<3, T, true>(p) : bilinear_blk_smem<4, T, true>(p);
    if (use_blk<T>(p, sb)) {
      if (!tri && two_pass_applies<T, TG_P1_TET>(p)) return two_pass<TG_P1_TET, T, true>(p, a, s);
      const int ub = blk_ub<T>(p);
      const tg::RefTab<T>& tab = table<T>(p->el);
      tg_status st = TG_OK;
      auto go = [&](auto kern) {
        dim3 grid;
        if ((st = launch_blk(kern, sb, p, &grid)) != TG_OK) return;
        kern<<<grid, blk_threads(p), sb, s>>>(a, tab, tg::blk_args(p), p->max_row_len * BT);
      };
      if constexpr (sizeof(T) == 8) {
        if (tri) go(k_bilinear_blk<TG_P1_TRI, T, 2, true>);
        else go(k_bilinear_blk<TG_P1_TET, T, 2, true>);
      } else {
        if (tri) {
          if (ub <= 2) go(k_bilinear_blk<TG_P1_TRI, T, 2, true>);
          else if (ub <= 3) go(k_bilinear_blk<TG_P1_TRI, T, 3, true>);
          else if (ub <= 4) go(k_bilinear_blk<TG_P1_TRI, T, 4, true>);
          else go(k_bilinear_blk<TG_P1_TRI, T, 6, true>);
        } else {
          if (ub <= 4) go(k_bilinear_blk<TG_P1_TET, T, 4, true>);
          else go(k_bilinear_blk<TG_P1_TET, T, 6, true>);
        }
      }
      if (st != TG_OK) return st;
      TG_CK_LAUNCH("k_bilinear_blk<load>");
      return TG_OK;
    }
  }
  {
    if ((p->el == TG_P1_TRI && two_pass_applies<T, TG_P1_TRI>(p)) ||
        (p->el == TG_P1_TET && two_pass_applies<T, TG_P1_TET>(p))) {
      // P1 in two passes: every element's K_e and F_e once, then the rows'
      // and the nodes' sums (the values and orders of the one-pass kernels)
      FwdArgs<T> a = base_args<T>(p, coords);
      a.coef = static_cast<const T*>(kappa);
      a.layout = kl;
      a.c = (T)c;
      a.out = static_cast<T*>(vals);
      a.f = static_cast<const T*>(f);
      a.f_layout = fl;
      a.F = static_cast<T*>(F);
      const bool tri = p->el == TG_P1_TRI;
      const int NS = tri ? 6 : 10;
      T* rec = static_cast<T*>(p->elem_scratch);
      T* recF = rec + p->E * NS;
      const tg::RefTab<T>& tab = table<T>(p->el);
      const int g1 = (int)std::min<int64_t>(tg::grid_for(p->E, 128), 32ll * tg::sm_count());
      if (tri) k_p1_map<TG_P1_TRI, T, true><<<g1, 128, 0, s>>>(a, tab, p->E, rec, recF);
      else k_p1_map<TG_P1_TET, T, true><<<g1, 128, 0, s>>>(a, tab, p->E, rec, recF);
      TG_CK_LAUNCH("k_p1_map<load>");
      a.scr = rec;
      using El3 = tg::Elem<TG_P1_TRI>;
      using El4 = tg::Elem<TG_P1_TET>;
      size_t stage = 0;
      const int R = tri ? tg::staged_rows<T, El3::nv, El3::npw>(p->max_deg, p->max_row_len, &stage)
                        : tg::staged_rows<T, El4::nv, El4::npw>(p->max_deg, p->max_row_len, &stage);
      if (R == 0) {
        tg::set_error("mesh degree too large for the staged gather");
        return TG_ERR_UNSUPPORTED;
      }
      const size_t smem = tab_bytes<T>() + stage;
      const int cap = std::max(1, R * p->max_deg);
      const void* kern = tri ? (const void*)k_bilinear_gather<TG_P1_TRI, T, true>
                             : (const void*)k_bilinear_gather<TG_P1_TET, T, true>;
      tg_status st = set_smem(kern, smem);
      if (st != TG_OK) return st;
      if (tri) k_bilinear_gather<TG_P1_TRI, T, true><<<tg::grid_for(p->N, R), R, smem, s>>>(a, tab, cap);
      else k_bilinear_gather<TG_P1_TET, T, true><<<tg::grid_for(p->N, R), R, smem, s>>>(a, tab, cap);
      TG_CK_LAUNCH("k_bilinear_gather<scratch>");
      if (tri) k_p1_load_reduce<TG_P1_TRI, T><<<tg::grid_for(p->N, 128), 128, 0, s>>>(a, recF);
      else k_p1_load_reduce<TG_P1_TET, T><<<tg::grid_for(p->N, 128), 128, 0, s>>>(a, recF);
      TG_CK_LAUNCH("k_p1_load_reduce");
      return TG_OK;
    }
  }
  tg_status st = bilinear<T>(p, coords, kappa, kl, c, vals, s, false);
  if (st != TG_OK) return st;
  return load<T>(p, coords, f, fl, 1, F, s);
}

bool layout_ok(tg_layout l, bool allow_node) {
  return l == TG_PER_ELEMENT || l == TG_PER_QP || l == TG_CONSTANT || (allow_node && l == TG_PER_NODE);
}

tg_status bilinear_entry(const tg_pattern* p, tg_dtype dtype, const void* coords, const void* kappa, tg_layout kl,
                         double c, void* vals, tg_stream stream, bool atomic) {
  tg_status st = check_common(p, dtype, coords);
  if (st != TG_OK) return st;
  if (!tg::scalar_kind(p->el) || !layout_ok(kl, false) || !kappa || (p->nnz > 0 && !vals)) return TG_ERR_INVALID_ARG;
  if (p->N == 0) return TG_OK;
  cudaStream_t s = (cudaStream_t)stream;
  return dtype == TG_F32 ? bilinear<float>(p, coords, kappa, kl, c, vals, s, atomic)
                         : bilinear<double>(p, coords, kappa, kl, c, vals, s, atomic);
}

}  // namespace

extern "C" {

tg_status tg_assemble_bilinear(const tg_pattern* p, tg_dtype dtype, const void* coords, const void* kappa,
                               tg_layout kappa_layout, double c, void* vals_out, tg_stream stream) {
  return bilinear_entry(p, dtype, coords, kappa, kappa_layout, c, vals_out, stream, false);
}

tg_status tg_assemble_bilinear_atomic(const tg_pattern* p, tg_dtype dtype, const void* coords, const void* kappa,
                                      tg_layout kappa_layout, double c, void* vals_out, tg_stream stream) {
  return bilinear_entry(p, dtype, coords, kappa, kappa_layout, c, vals_out, stream, true);
}

tg_status tg_assemble_system(const tg_pattern* p, tg_dtype dtype, const void* coords, const void* kappa,
                             tg_layout kappa_layout, double c, const void* f, tg_layout f_layout, void* vals_out,
                             void* F_out, tg_stream stream) {
  tg_status st = check_common(p, dtype, coords);
  if (st != TG_OK) return st;
  if (!tg::scalar_kind(p->el) || !layout_ok(kappa_layout, false) || !kappa || (p->nnz > 0 && !vals_out) || !f ||
      !F_out || !(f_layout == TG_PER_NODE || f_layout == TG_PER_QP || f_layout == TG_CONSTANT))
    return TG_ERR_INVALID_ARG;
  if (p->N == 0) return TG_OK;
  cudaStream_t s = (cudaStream_t)stream;
  return dtype == TG_F32 ? system_asm<float>(p, coords, kappa, kappa_layout, c, f, f_layout, vals_out, F_out, s)
                         : system_asm<double>(p, coords, kappa, kappa_layout, c, f, f_layout, vals_out, F_out, s);
}

tg_status tg_assemble_load(const tg_pattern* p, tg_dtype dtype, const void* coords, const void* f, tg_layout f_layout,
                           int32_t ncomp, void* F_out, tg_stream stream) {
  tg_status st = check_common(p, dtype, coords);
  if (st != TG_OK) return st;
  if ((ncomp != 1 && ncomp != 3) || !f || !F_out || !(f_layout == TG_PER_NODE || f_layout == TG_PER_QP ||
                                                       f_layout == TG_CONSTANT) || p->el == TG_Q1_QUAD_VEC2)
    return TG_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  return dtype == TG_F32 ? load<float>(p, coords, f, f_layout, ncomp, F_out, s)
                         : load<double>(p, coords, f, f_layout, ncomp, F_out, s);
}

}  // extern "C"
