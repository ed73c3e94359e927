// Matrix-free residual of the Galerkin system, the quantity of the
// physics-informed loss of Eq. (res1):
//   y = K(kappa, c) x - F(f),  loss = sum_i y_i^2 over the free rows,
// computed element by element without storing K: the Map of Algorithm 1
// evaluates K_e and F_e and contracts K_e with the element's values of x;
// the Reduce sums the NV element results of every node in increasing
// element order (the node-level routing S_vec of Algorithm 2).
//
// With a reaction polynomial r (the semilinear forms of the method of lines,
// e.g. the Allen-Cahn reaction), the Map also integrates r(u_h) phi_i (or,
// for the Jacobian action, r'(u_h) v_h phi_i) with the element's rule.
//
// Two forms, with the same per-element arithmetic and the same summation
// order, hence identical bits:
//   k_residual_blk    - element-once row blocks (blocks.cuh): each distinct
//                       element of a block is evaluated once (FP32);
//   k_residual_map +  - two passes through a per-element scratch array:
//   k_residual_reduce   every element evaluated exactly once (FP64, and
//                       patterns without row blocks);
// A mesh without elements has y = 0.
// The loss is summed in FP64: per thread in row order, per CTA in a fixed
// tree, then the last CTA to finish adds the CTA partials in CTA order.
#include <algorithm>
#include <cstdint>
#include <cstring>

#include "blocks.cuh"

namespace {

constexpr int RT = 128;    // threads per CTA (rows per CTA of the gather kernel)
constexpr int kSlots = 4;  // doubles per CTA in the pattern's partials array

template <typename T>
struct ResArgs {
  tg::FwdArgs<T> fa;  // coords, coef (kappa), layout, c, f, f_layout, status, cells, inc_ptr, inc_e
  const T* __restrict__ x;
  const T* __restrict__ xr;  // state of the reaction's Jacobian (NL == 2)
  T r[4];                    // reaction r(u) = r0 + r1 u + r2 u^2 + r3 u^3
  const uint8_t* __restrict__ dir;
  T* __restrict__ y;
  T* loss;
  double* __restrict__ partials;
  unsigned int* arrivals;
};

// Row a of the element's result: sum_b K_e[a][b] x_b (b ascending, first
// product then fused multiply-adds) minus F_e[a] with the load term.
template <int NV, typename T>
__device__ __forceinline__ T kx_row(const T (&K)[NV * (NV + 1) / 2], const T (&xv)[NV], int a) {
  T s = T(0);
#pragma unroll
  for (int b = 0; b < NV; ++b) {
    const int lo = a < b ? a : b, hi = a < b ? b : a;
    const T kab = K[lo * NV - lo * (lo - 1) / 2 + (hi - lo)];
    s = b == 0 ? kab * xv[0] : fma(kab, xv[b], s);
  }
  return s;
}

// Inputs of one element's result: geometry and coefficient (ElemIn), the
// values of x at its NV nodes and, with the load term, f as F_e needs it.
template <int EL, typename T>
struct ResIn {
  tg::ElemIn<EL, T> in;
  T xv[tg::Elem<EL>::nv];
  T fv[tg::Elem<EL>::nv];
  T xr[tg::Elem<EL>::nv];
};

template <int EL, typename T, bool LOADF, int NL>
__device__ __forceinline__ void result_inputs(const ResArgs<T>& r, int64_t e, const int (&vid)[tg::Elem<EL>::nv],
                                              ResIn<EL, T>& d) {
  constexpr int NV = tg::Elem<EL>::nv, NG = tg::Elem<EL>::ngeo;
#pragma unroll
  for (int c = 0; c < NG; ++c) d.in.v[c] = vid[c];
  tg::elem_data<EL, T>(r.fa, e, d.in);
#pragma unroll
  for (int c = 0; c < NV; ++c) d.xv[c] = __ldg(r.x + vid[c]);
  if constexpr (LOADF) tg::p1_load_f<NV, T>(r.fa.f, r.fa.f_layout, e, vid, d.fv);
  if constexpr (NL == 2) {
#pragma unroll
    for (int c = 0; c < NV; ++c) d.xr[c] = __ldg(r.xr + vid[c]);
  }
}

// Reaction term of the element at local node a, |det J| sum_q w_q s_q
// phi_a(x_q): NL == 1, s_q = r(u_q) with u_q = sum_b phi_b(x_q) x_b (the
// semilinear load of the reaction); NL == 2, s_q = r'(ur_q) v_q with ur_q
// from the state xr and v_q from x (its Jacobian applied to x).
template <int EL, typename T, int NL>
__device__ __forceinline__ void reaction_rows(const ResArgs<T>& r, const tg::RefTab<T>& tab, T adet,
                                              const ResIn<EL, T>& d, T (&out)[tg::Elem<EL>::nv]) {
  constexpr int NV = tg::Elem<EL>::nv, NQ = tg::Elem<EL>::nq;
  T sq[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    T u = T(0), v = T(0);
#pragma unroll
    for (int b = 0; b < NV; ++b) {
      u = fma(tab.phi[q][b], NL == 2 ? d.xr[b] : d.xv[b], u);
      if constexpr (NL == 2) v = fma(tab.phi[q][b], d.xv[b], v);
    }
    if constexpr (NL == 1) {
      sq[q] = tab.w[q] * fma(fma(fma(r.r[3], u, r.r[2]), u, r.r[1]), u, r.r[0]);
    } else {
      const T dr = fma(fma(T(3) * r.r[3], u, T(2) * r.r[2]), u, r.r[1]);
      sq[q] = tab.w[q] * dr * v;
    }
  }
#pragma unroll
  for (int a = 0; a < NV; ++a) {
    T s = T(0);
#pragma unroll
    for (int q = 0; q < NQ; ++q) s = fma(sq[q], tab.phi[q][a], s);
    out[a] = adet * s;
  }
}

// The NV results of element e; zeros and a recorded error for a degenerate
// element.
template <int EL, typename T, bool LOADF, int NL>
__device__ __forceinline__ void result_compute(const ResArgs<T>& r, const tg::RefTab<T>& tab, int64_t e,
                                               const ResIn<EL, T>& d, T (&ye)[tg::Elem<EL>::nv]) {
  constexpr int NV = tg::Elem<EL>::nv;
  T K[NV * (NV + 1) / 2];
  T adet;
  bool ok;
  if constexpr (EL == TG_P2_TRI) ok = tg::p2_elem_sym<T>(d.in, r.fa.c, tab, K, &adet);
  else ok = tg::p1_elem_sym<EL, T>(d.in, r.fa.c, tab, K, &adet);
  if (!ok) {
    tg::record_error(r.fa.status, TG_ERR_DEGENERATE_ELEMENT, e);
#pragma unroll
    for (int a = 0; a < NV; ++a) ye[a] = T(0);
    return;
  }
  T nr[NV];
  if constexpr (NL != 0) reaction_rows<EL, T, NL>(r, tab, adet, d, nr);
  T fe[LOADF ? NV : 1];
  if constexpr (LOADF) tg::p1_load_entries<NV, T>(r.fa.f_layout, adet, d.fv, tab, fe);
#pragma unroll
  for (int a = 0; a < NV; ++a) {
    T s = kx_row<NV, T>(K, d.xv, a);
    if constexpr (NL != 0) s += nr[a];
    if constexpr (LOADF) s -= fe[a];
    ye[a] = s;
  }
}

// Fixed-order block sum (warp tree, then warp 0 over the warps); the result
// is valid in thread 0.
__device__ __forceinline__ double block_sum(double v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();  // red may still be read by a previous call
  if (lane == 0) red[wid] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    v = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += red[w];
  }
  return v;
}

// CTA partial, then the last CTA to arrive sums all partials in CTA order
// and writes the loss (no CTA waits for another).
template <typename T>
__device__ __forceinline__ void finish_loss(const ResArgs<T>& r, double part) {
  __shared__ double red[RT / 32];
  __shared__ bool s_last;
  part = block_sum(part, red);
  if (threadIdx.x == 0) {
    r.partials[kSlots * blockIdx.x] = part;
    __threadfence();
    s_last = atomicInc(r.arrivals, gridDim.x - 1) == gridDim.x - 1;  // wraps to 0 for the next launch
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  double s = 0.0;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) s += __ldcg(r.partials + kSlots * b);
  s = block_sum(s, red);
  if (threadIdx.x == 0) *r.loss = (T)s;
}

// Element-once row blocks: Map the block's distinct elements into
// Ye[NV][capE], Reduce the rows (increasing element order), apply the
// Dirichlet mask, write y and add y^2 to this thread's loss term.
// FP32 triangles run two elements per thread at eight CTAs per SM (64
// registers): 51 against 53 us for three elements at six CTAs (1024^2).
template <int EL, typename T, int UB>
constexpr int res_min_ctas() {
  return (EL == TG_P1_TRI && sizeof(T) == 4 && UB == 2) ? 8 : 1;
}

template <int EL, typename T, int UB, bool LOADF, int NL>
__global__ void __launch_bounds__(RT, res_min_ctas<EL, T, UB>()) k_residual_blk(const ResArgs<T> r, const __grid_constant__ tg::RefTab<T> tab,
                                                    const tg::BlkArgs g) {
  constexpr int NV = tg::Elem<EL>::nv;
  extern __shared__ __align__(16) unsigned char smem[];
  tg::BlkPipe pipe;
  T* Ye = reinterpret_cast<T*>(pipe.init(smem, g));
  __syncthreads();  // publishes the mbarrier initialisation
  double part = 0.0;
  TG_BLK_PIPELINE_BEGIN(pipe, g, r.fa.status)
  for (int j0 = threadIdx.x; j0 < v.nbe; j0 += UB * NT_) {
    // all loads of the thread's UB elements first, then the arithmetic
    int64_t e[UB];
    ResIn<EL, T> d[UB];
#pragma unroll
    for (int u = 0; u < UB; ++u) {
      const int j = j0 + u * NT_ < v.nbe ? j0 + u * NT_ : 0;  // idle slots load element 0 of the list
      int vid[NV];
#pragma unroll
      for (int c = 0; c < NV; ++c) vid[c] = v.vtx(c, j);
      e[u] = tg::bel_elem(v.be[j]);
      result_inputs<EL, T, LOADF, NL>(r, e[u], vid, d[u]);
    }
#pragma unroll
    for (int u = 0; u < UB; ++u) {
      const int j = j0 + u * NT_;
      if (j >= v.nbe) continue;
      T ye[NV];
      result_compute<EL, T, LOADF, NL>(r, tab, e[u], d[u], ye);
#pragma unroll
      for (int a = 0; a < NV; ++a) Ye[a * g.capE + j] = ye[a];
    }
  }
  __syncthreads();
  {
    const int i = v.r0 + (int)threadIdx.x;
    if (i < v.r1) {
      T s = T(0);
      const int je = v.ip[i + 1];
      for (int j = v.ip[i]; j < je; ++j) {
        const auto rc = tg::blk_rec<NV>(v.rc, j);
        s += Ye[rc.a() * g.capE + rc.le()];
      }
      const int node = v.pm[i];
      if (r.dir && r.dir[node]) s = T(0);
      r.y[node] = s;
      part += (double)s * (double)s;
    }
    __syncthreads();  // stage s and Ye are free again
  }
  TG_BLK_PIPELINE_END
  if (r.loss) finish_loss(r, part);
}

// Two passes.  Map: one thread per element writes its NV results to
// ye[e][a] (each element evaluated exactly once; consecutive threads write
// consecutive elements).  Reduce: one thread per node sums its incidences'
// results in increasing element order (the incidence lists are sorted by
// element), so every y[i] carries the bits of the one-pass kernels.
template <int EL, typename T, bool LOADF, int NL, int EPT>
__global__ void __launch_bounds__(RT) k_residual_map(const ResArgs<T> r, const __grid_constant__ tg::RefTab<T> tab,
                                                    int64_t E, T* __restrict__ ye) {
  constexpr int NV = tg::Elem<EL>::nv;
  const int64_t e0 = (int64_t)blockIdx.x * (RT * EPT) + threadIdx.x;
  int64_t e[EPT];
  ResIn<EL, T> d[EPT];
#pragma unroll
  for (int u = 0; u < EPT; ++u) {
    e[u] = e0 + u * RT;
    const int64_t ee = e[u] < E ? e[u] : E - 1;
    int vid[NV];
#pragma unroll
    for (int c = 0; c < NV; ++c) vid[c] = __ldg(r.fa.cells + ee * NV + c);
    result_inputs<EL, T, LOADF, NL>(r, ee, vid, d[u]);
  }
#pragma unroll
  for (int u = 0; u < EPT; ++u) {
    if (e[u] >= E) break;
    T out[NV];
    result_compute<EL, T, LOADF, NL>(r, tab, e[u], d[u], out);
#pragma unroll
    for (int a = 0; a < NV; ++a) ye[e[u] * NV + a] = out[a];
  }
}

template <int NV, typename T>
__global__ void __launch_bounds__(RT) k_residual_reduce(const ResArgs<T> r, const T* __restrict__ ye) {
  const int64_t i = (int64_t)blockIdx.x * RT + threadIdx.x;
  double part = 0.0;
  if (i < r.fa.n) {
    const int j0 = __ldg(r.fa.inc_ptr + i), j1 = __ldg(r.fa.inc_ptr + i + 1);
    T s = T(0);
    for (int j = j0; j < j1; ++j) {
      const int ea = __ldg(r.fa.inc_e + j);
      s += ye[(int64_t)(ea >> 3) * NV + (ea & 7)];
    }
    if (r.dir && r.dir[i]) s = T(0);
    r.y[i] = s;
    part = (double)s * (double)s;
  }
  if (r.loss) finish_loss(r, part);
}

template <int EL, typename T, bool LOADF, int NL>
tg_status launch_two_pass(const tg_pattern* p, const ResArgs<T>& r, cudaStream_t s) {
  constexpr int NV = tg::Elem<EL>::nv, EPT = 2;
  const tg::RefTab<T>& tab = tg::table<T>((tg_element)EL);
  T* ye = static_cast<T*>(p->elem_scratch);
  const int64_t gm = (p->E + RT * EPT - 1) / (RT * EPT);
  k_residual_map<EL, T, LOADF, NL, EPT><<<(unsigned)gm, RT, 0, s>>>(r, tab, p->E, ye);
  TG_CK_LAUNCH("k_residual_map");
  const int64_t gr = tg::grid_for(p->N, RT);
  if (gr > (p->n_partials - 4) / kSlots) return TG_ERR_UNSUPPORTED;
  k_residual_reduce<NV, T><<<(unsigned)gr, RT, 0, s>>>(r, ye);
  TG_CK_LAUNCH("k_residual_reduce");
  return TG_OK;
}

template <int EL, typename T, bool LOADF, int NL>
tg_status launch_el(const tg_pattern* p, const ResArgs<T>& r, cudaStream_t s) {
  // FP32 triangles run on the row blocks.  Tetrahedra, FP64 and patterns
  // without row blocks take the two passes, which evaluate each element
  // once: the row blocks evaluate it 1.2 times on Hilbert-ordered triangles
  // but about 3 times on tetrahedral grids, and FP64 is bound by the FP64
  // pipe.
  constexpr int NV = tg::Elem<EL>::nv;
  if constexpr (sizeof(T) == 4 && EL != TG_P1_TET) {
    const tg::RefTab<T>& tab = tg::table<T>((tg_element)EL);
    const int64_t cap_ctas = (p->n_partials - 4) / kSlots;  // partial slots of the pattern
    const tg::BlkArgs g = tg::blk_args(p);
    const size_t smem = p->bel ? tg::blk_stage_bytes(p->blk_rows, g.capJ, g.capE, NV) + (size_t)NV * g.capE * sizeof(T)
                               : 0;
    if (p->bel && p->blk_rows <= RT && smem <= 113 * 1024) {
      tg_status st = TG_OK;
      auto go = [&](auto kern) {
        if ((st = tg::set_smem((const void*)kern, smem)) != TG_OK) return;
        // the most shared memory per SM, so that eight CTAs fit
        cudaError_t ce = cudaFuncSetAttribute((const void*)kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        if (ce != cudaSuccess) {
          st = tg::cuda_fail(ce, "cudaFuncSetAttribute", __FILE__, __LINE__);
          return;
        }
        int per_sm = 0;
        ce = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, RT, smem);
        if (ce != cudaSuccess) {
          st = tg::cuda_fail(ce, "cudaOccupancyMaxActiveBlocksPerMultiprocessor", __FILE__, __LINE__);
          return;
        }
        const int grid =
            (int)std::min<int64_t>({p->n_blk, (int64_t)std::max(per_sm, 1) * tg::sm_count(), cap_ctas});
        kern<<<grid, RT, smem, s>>>(r, tab, g);
      };
      go(k_residual_blk<EL, T, 2, LOADF, NL>);
      if (st != TG_OK) return st;
      TG_CK_LAUNCH("k_residual_blk");
      return TG_OK;
    }
  }
  if (p->elem_scratch) return launch_two_pass<EL, T, LOADF, NL>(p, r, s);
  // no elements: y = 0 and loss = 0
  TG_CK(cudaMemsetAsync(r.y, 0, (size_t)p->N * sizeof(T), s));
  if (r.loss) TG_CK(cudaMemsetAsync(r.loss, 0, sizeof(T), s));
  return TG_OK;
}

// r(u_q) at every quadrature point of every element, u_q = sum_b phi_b(x_q)
// x_b: the same interpolation and Horner evaluation as reaction_rows.  With
// these values as a per-point load, the load backward gives the reaction
// term's coordinate gradient (only |det J| depends on the coordinates).
template <int EL, typename T>
__global__ void __launch_bounds__(RT) k_reaction_points(const int32_t* __restrict__ cells, const T* __restrict__ x,
                                                       const __grid_constant__ tg::RefTab<T> tab, T r0, T r1, T r2,
                                                       T r3, int64_t E, T* __restrict__ out) {
  constexpr int NV = tg::Elem<EL>::nv, NQ = tg::Elem<EL>::nq;
  const int64_t e = (int64_t)blockIdx.x * RT + threadIdx.x;
  if (e >= E) return;
  T xv[NV];
#pragma unroll
  for (int b = 0; b < NV; ++b) xv[b] = __ldg(x + __ldg(cells + e * NV + b));
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    T u = T(0);
#pragma unroll
    for (int b = 0; b < NV; ++b) u = fma(tab.phi[q][b], xv[b], u);
    out[e * NQ + q] = fma(fma(fma(r3, u, r2), u, r1), u, r0);
  }
}

template <typename T>
tg_status reaction_points(const tg_pattern* p, const void* x, const double* rc, void* out, cudaStream_t s) {
  const unsigned grid = (unsigned)tg::grid_for(p->E, RT);
  const T r0 = (T)rc[0], r1 = (T)rc[1], r2 = (T)rc[2], r3 = (T)rc[3];
  const T* xx = static_cast<const T*>(x);
  T* o = static_cast<T*>(out);
  switch (p->el) {
    case TG_P1_TRI:
      k_reaction_points<TG_P1_TRI, T><<<grid, RT, 0, s>>>(p->cells, xx, tg::table<T>(TG_P1_TRI), r0, r1, r2, r3, p->E, o);
      break;
    case TG_P2_TRI:
      k_reaction_points<TG_P2_TRI, T><<<grid, RT, 0, s>>>(p->cells, xx, tg::table<T>(TG_P2_TRI), r0, r1, r2, r3, p->E, o);
      break;
    default:
      k_reaction_points<TG_P1_TET, T><<<grid, RT, 0, s>>>(p->cells, xx, tg::table<T>(TG_P1_TET), r0, r1, r2, r3, p->E, o);
  }
  TG_CK_LAUNCH("k_reaction_points");
  return TG_OK;
}

template <typename T, int NL>
tg_status dispatch(const tg_pattern* p, const ResArgs<T>& r, bool lf, cudaStream_t s) {
  switch (p->el) {
    case TG_P1_TRI:
      return lf ? launch_el<TG_P1_TRI, T, true, NL>(p, r, s) : launch_el<TG_P1_TRI, T, false, NL>(p, r, s);
    case TG_P1_TET:
      return lf ? launch_el<TG_P1_TET, T, true, NL>(p, r, s) : launch_el<TG_P1_TET, T, false, NL>(p, r, s);
    default:
      return launch_el<TG_P2_TRI, T, false, NL>(p, r, s);
  }
}

template <typename T>
tg_status residual(const tg_pattern* p, const void* coords, const void* kappa, tg_layout kl, double c, const void* x,
                   const void* f, tg_layout fl, const double* reaction, const void* x_react, const uint8_t* dir,
                   void* y, void* loss, cudaStream_t s) {
  ResArgs<T> r;
  std::memset(&r, 0, sizeof(r));
  r.fa.inc_ptr = p->inc_ptr;
  r.fa.inc_e = p->inc_e;
  r.fa.cells = p->cells;
  r.fa.coords = static_cast<const T*>(coords);
  r.fa.coef = static_cast<const T*>(kappa);
  r.fa.layout = kl;
  r.fa.c = (T)c;
  r.fa.n = p->N;
  r.fa.status = p->status;
  r.fa.f = static_cast<const T*>(f);
  r.fa.f_layout = fl;
  r.x = static_cast<const T*>(x);
  r.xr = static_cast<const T*>(x_react);
  if (reaction)
    for (int k = 0; k < 4; ++k) r.r[k] = (T)reaction[k];
  r.dir = dir;
  r.y = static_cast<T*>(y);
  r.loss = static_cast<T*>(loss);
  r.partials = p->partials;
  r.arrivals = p->arrivals;
  const bool lf = f != nullptr;
  if (!reaction) return dispatch<T, 0>(p, r, lf, s);
  return x_react ? dispatch<T, 2>(p, r, lf, s) : dispatch<T, 1>(p, r, lf, s);
}

bool aligned_to(const void* ptr, size_t a) { return ((uintptr_t)ptr % a) == 0; }

tg_status entry(const tg_pattern* p, tg_dtype dtype, const void* coords, const void* kappa, tg_layout kappa_layout,
                double c, const void* x, const void* f, tg_layout f_layout, const double* reaction,
                const void* x_react, const uint8_t* dirichlet, void* y, void* loss, tg_stream stream) {
  if (!p || (dtype != TG_F32 && dtype != TG_F64)) return TG_ERR_INVALID_ARG;
  if (!tg::scalar_kind(p->el)) return TG_ERR_INVALID_ARG;
  if (!(kappa_layout == TG_PER_QP || kappa_layout == TG_PER_ELEMENT || kappa_layout == TG_CONSTANT)) return TG_ERR_INVALID_ARG;
  if (f && !(f_layout == TG_PER_NODE || f_layout == TG_PER_QP || f_layout == TG_CONSTANT)) return TG_ERR_INVALID_ARG;
  if (f && p->el == TG_P2_TRI) {
    tg::set_error("tg_residual: the load term is built for P1 elements");
    return TG_ERR_UNSUPPORTED;
  }
  if (x_react && !reaction) return TG_ERR_INVALID_ARG;
  const size_t es = dtype == TG_F32 ? 4 : 8;
  if (p->N > 0 && (!coords || !kappa || !x || !y)) return TG_ERR_INVALID_ARG;
  if (x && x == y) {
    tg::set_error("tg_residual: x and y must be distinct buffers");
    return TG_ERR_INVALID_ARG;
  }
  if ((f && f == y) || (x_react && x_react == y)) return TG_ERR_INVALID_ARG;
  if (coords && !aligned_to(coords, tg::dim_of(p->el) == 2 ? 2 * es : es)) {
    tg::set_error("coords must be aligned to 2 * sizeof(dtype) for 2D meshes");
    return TG_ERR_INVALID_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  if (p->N == 0) {
    if (loss) TG_CK(cudaMemsetAsync(loss, 0, es, s));
    return TG_OK;
  }
  return dtype == TG_F32
             ? residual<float>(p, coords, kappa, kappa_layout, c, x, f, f_layout, reaction, x_react, dirichlet, y, loss, s)
             : residual<double>(p, coords, kappa, kappa_layout, c, x, f, f_layout, reaction, x_react, dirichlet, y, loss,
                                s);
}

}  // namespace

extern "C" {

tg_status tg_residual(const tg_pattern* p, tg_dtype dtype, const void* coords, const void* kappa,
                      tg_layout kappa_layout, double c, const void* x, const void* f, tg_layout f_layout,
                      const uint8_t* dirichlet, void* y, void* loss, tg_stream stream) {
  return entry(p, dtype, coords, kappa, kappa_layout, c, x, f, f_layout, nullptr, nullptr, dirichlet, y, loss, stream);
}

tg_status tg_reaction_points(const tg_pattern* p, tg_dtype dtype, const void* x, const double* reaction, void* out,
                             tg_stream stream) {
  if (!p || (dtype != TG_F32 && dtype != TG_F64) || !tg::scalar_kind(p->el) || !reaction) return TG_ERR_INVALID_ARG;
  if (p->E == 0) return TG_OK;
  if (!x || !out) return TG_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  return dtype == TG_F32 ? reaction_points<float>(p, x, reaction, out, s) : reaction_points<double>(p, x, reaction, out, s);
}

tg_status tg_semilinear_residual(const tg_pattern* p, tg_dtype dtype, const void* coords, const void* kappa,
                                 tg_layout kappa_layout, double c, const void* x, const void* f, tg_layout f_layout,
                                 const double* reaction, const void* x_react, const uint8_t* dirichlet, void* y,
                                 void* loss, tg_stream stream) {
  if (!reaction) return TG_ERR_INVALID_ARG;
  return entry(p, dtype, coords, kappa, kappa_layout, c, x, f, f_layout, reaction, x_react, dirichlet, y, loss,
               stream);
}

}  // extern "C"
