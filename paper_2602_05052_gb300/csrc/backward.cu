// Backward (reverse mode) of the scalar bilinear assembly.
//
// Given the upstream gradient W of the assembled values (either a CSR array
// gathered through the element-to-slot map, i.e. S_mat^T of Algorithm 2, or
// the adjoint outer product lam U^T of Eq. (adj)), the gradients of
// L = sum_e sum_ab W_ab K^e_ab are, with W_s = (W + W^T)/2, det-scaled
// gradients n_b (elements.cuh) and Nd = [n_1 ... n_d]:
//
//   R_q   = Ghat_q W_s Ghat_q^T                    (reference d x d, per point)
//   dL/dkappa_eq = w_q <R_q, Nd^T Nd> / |det J|    (= w_q |det J| tr(G_q W_s G_q^T))
//   dL/dc       = sum_e |det J| <W_s, Mhat>
//   dL/dx_a     = sign(det J) [ (1/det^2)(<Rbar, Nd^T Nd> n_a - 2 Nd Rbar Nd^T n_a) + c <W_s, Mhat> n_a ]
//                 for the vertices a, with Rbar = sum_q w_q kappa_q R_q,
//
// from d|det J| = |det J| tr(J^{-1} dJ) and dG = -J^{-T} dJ^T G.  For P1,
// Nd Ghat = N (the matrix of all n_b), so Nd R Nd^T = N W_s N^T.
//
// Layout of the work: one thread per node (row owner), as in the forward.
// Each node sums the coordinate gradients of its incident elements in
// increasing element order; the coefficient gradient of element e is written
// by the visit with local index 0 (exactly one per element); the global sums
// (dL/dc, constant kappa) go through per-CTA partials summed in a fixed tree
// order by a second kernel.  Everything is deterministic.
#include <cstdint>

#include "gather.cuh"

namespace {

constexpr int BB = 128;

template <typename T>
struct BwdArgs {
  const int32_t* __restrict__ inc_ptr;
  const int32_t* __restrict__ inc_e;
  const int32_t* __restrict__ cells;
  const int32_t* __restrict__ elem_slot;
  const T* __restrict__ coords;
  const T* __restrict__ kappa;
  int layout;
  T c;
  const T* __restrict__ gvals;
  const T* __restrict__ lam;
  const T* __restrict__ U;
  T* __restrict__ grad_kappa;
  T* __restrict__ grad_coords;
  double* __restrict__ partials;
  int64_t N;
  unsigned long long* status;
};

// Fixed-order block sum of two doubles (warp tree, then warp 0 over warps).
__device__ __forceinline__ void block_sum2(double& a, double& b, double (*red)[BB / 32]) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, o);
    b += __shfl_down_sync(0xffffffffu, b, o);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    red[0][wid] = a;
    red[1][wid] = b;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    a = 0;
    b = 0;
    for (int w = 0; w < BB / 32; ++w) {
      a += red[0][w];
      b += red[1][w];
    }
  }
}

template <int EL, typename T, bool FUSED>
__global__ void __launch_bounds__(BB) k_backward_gather(const BwdArgs<T> a, const __grid_constant__ tg::RefTab<T> tab) {
  using El = tg::Elem<EL>;
  constexpr int NV = El::nv, D = El::dim, NQ = El::nq;
  __shared__ tg::RefTab<T> ts;
  __shared__ double red[2][BB / 32];
  tg::copy_table(ts, tab);
  const int64_t i = (int64_t)blockIdx.x * BB + threadIdx.x;
  double pc = 0.0, pk = 0.0;
  if (i < a.N) {
    T gx[D];
#pragma unroll
    for (int r = 0; r < D; ++r) gx[r] = T(0);
    const int j0 = __ldg(a.inc_ptr + i), j1 = __ldg(a.inc_ptr + i + 1);
    for (int j = j0; j < j1; ++j) {
      const int ea = __ldg(a.inc_e + j);
      const int64_t e = ea >> 3;
      const int la = ea & 7;
      const int32_t* cl = a.cells + e * NV;
      int v[NV];
#pragma unroll
      for (int b = 0; b < NV; ++b) v[b] = __ldg(cl + b);
      tg::Geom<D, T> g;
      if constexpr (D == 2) tg::tri_geom(a.coords, v[0], v[1], v[2], g);
      else tg::tet_geom(a.coords, v[0], v[1], v[2], v[3], g);
      const T adet = tg::absv(g.det);
      if (!(adet > tg::det_tiny<T>())) {
        tg::record_error(a.status, TG_ERR_DEGENERATE_ELEMENT, e);
        if (la == 0 && a.grad_kappa) {
          if (a.layout == TG_PER_QP)
            for (int q = 0; q < NQ; ++q) a.grad_kappa[e * NQ + q] = T(0);
          else if (a.layout == TG_PER_ELEMENT) a.grad_kappa[e] = T(0);
        }
        continue;
      }
      // symmetric part of the upstream weights of this element
      T Ws[NV][NV];
      if constexpr (FUSED) {
        T l[NV], u[NV];
#pragma unroll
        for (int b = 0; b < NV; ++b) {
          l[b] = __ldg(a.lam + v[b]);
          u[b] = __ldg(a.U + v[b]);
        }
#pragma unroll
        for (int p = 0; p < NV; ++p)
#pragma unroll
          for (int q = 0; q < NV; ++q) Ws[p][q] = T(0.5) * (l[p] * u[q] + l[q] * u[p]);
      } else {
        const int32_t* sl = a.elem_slot + e * NV * NV;
        T W[NV][NV];
#pragma unroll
        for (int p = 0; p < NV; ++p)
#pragma unroll
          for (int q = 0; q < NV; ++q) W[p][q] = __ldg(a.gvals + __ldg(sl + p * NV + q));
#pragma unroll
        for (int p = 0; p < NV; ++p)
#pragma unroll
          for (int q = 0; q < NV; ++q) Ws[p][q] = T(0.5) * (W[p][q] + W[q][p]);
      }
      T wm = T(0);
#pragma unroll
      for (int p = 0; p < NV; ++p)
#pragma unroll
        for (int q = 0; q < NV; ++q) wm += Ws[p][q] * ts.M[p][q];
      const T inv = T(1) / adet;
      const T sgn = g.det > T(0) ? T(1) : T(-1);
      // Q = Nd Rbar Nd^T (d x d) and t = <Rbar, Nd^T Nd>; gk[q] = <R_q, Nd^T Nd>
      T Q[D][D], t;
      T gk[NQ];
      if constexpr (EL != TG_P2_TRI) {
        // P1: R_q identical for all points; Q = N W_s N^T, scaled by S = sum_q w_q kappa_q
        T y[NV][D];
#pragma unroll
        for (int b = 0; b < NV; ++b)
#pragma unroll
          for (int r = 0; r < D; ++r) {
            T s = T(0);
#pragma unroll
            for (int p = 0; p < NV; ++p) s += Ws[p][b] * g.n[p][r];
            y[b][r] = s;
          }
        T trq = T(0);
#pragma unroll
        for (int r = 0; r < D; ++r)
#pragma unroll
          for (int s2 = 0; s2 < D; ++s2) {
            T s = T(0);
#pragma unroll
            for (int b = 0; b < NV; ++b) s += y[b][r] * g.n[b][s2];
            Q[r][s2] = s;
          }
#pragma unroll
        for (int r = 0; r < D; ++r) trq += Q[r][r];
        const T S = tg::weighted_coef<T, NQ>(a.kappa, a.layout, e, ts.w, ts.wsum);
#pragma unroll
        for (int q = 0; q < NQ; ++q) gk[q] = ts.w[q] * trq * inv;
#pragma unroll
        for (int r = 0; r < D; ++r)
#pragma unroll
          for (int s2 = 0; s2 < D; ++s2) Q[r][s2] *= S;
        t = S * trq;
      } else {
        const T c00 = g.n[1][0] * g.n[1][0] + g.n[1][1] * g.n[1][1];
        const T c01 = g.n[1][0] * g.n[2][0] + g.n[1][1] * g.n[2][1];
        const T c11 = g.n[2][0] * g.n[2][0] + g.n[2][1] * g.n[2][1];
        T kq[6];
        tg::load_kq<T, 6>(a.kappa, a.layout, e, kq);
        T rb00 = T(0), rb01 = T(0), rb11 = T(0);
#pragma unroll
        for (int q = 0; q < 6; ++q) {
          T z0[6], z1[6];
#pragma unroll
          for (int p = 0; p < 6; ++p) {
            T s0 = T(0), s1 = T(0);
#pragma unroll
            for (int b = 0; b < 6; ++b) {
              s0 += Ws[p][b] * ts.gh[q][b][0];
              s1 += Ws[p][b] * ts.gh[q][b][1];
            }
            z0[p] = s0;
            z1[p] = s1;
          }
          T r00 = T(0), r01 = T(0), r11 = T(0);
#pragma unroll
          for (int p = 0; p < 6; ++p) {
            r00 += ts.gh[q][p][0] * z0[p];
            r01 += ts.gh[q][p][0] * z1[p];
            r11 += ts.gh[q][p][1] * z1[p];
          }
          gk[q] = ts.w[q] * (r00 * c00 + T(2) * r01 * c01 + r11 * c11) * inv;
          const T wk = ts.w[q] * kq[q];
          rb00 += wk * r00;
          rb01 += wk * r01;
          rb11 += wk * r11;
        }
        t = rb00 * c00 + T(2) * rb01 * c01 + rb11 * c11;
        // Q = Nd Rbar Nd^T with Nd = [n1 n2]
#pragma unroll
        for (int r = 0; r < 2; ++r)
#pragma unroll
          for (int s2 = 0; s2 < 2; ++s2)
            Q[r][s2] = g.n[1][r] * (rb00 * g.n[1][s2] + rb01 * g.n[2][s2]) +
                       g.n[2][r] * (rb01 * g.n[1][s2] + rb11 * g.n[2][s2]);
      }
      if (la == 0) {
        if (a.grad_kappa) {
          if (a.layout == TG_PER_QP) {
#pragma unroll
            for (int q = 0; q < NQ; ++q) a.grad_kappa[e * NQ + q] = gk[q];
          } else {
            T s = T(0);
#pragma unroll
            for (int q = 0; q < NQ; ++q) s += gk[q];
            if (a.layout == TG_PER_ELEMENT) a.grad_kappa[e] = s;
            else pk += (double)s;
          }
        }
        pc += (double)(adet * wm);
      }
      if (a.grad_coords && la <= D) {
        T na[D];
#pragma unroll
        for (int r = 0; r < D; ++r) {
          T col[D + 1];
#pragma unroll
          for (int b = 0; b <= D; ++b) col[b] = g.n[b][r];
          na[r] = tg::sel(la, col);
        }
        const T inv2 = inv * inv;
        const T cw = a.c * wm;
#pragma unroll
        for (int r = 0; r < D; ++r) {
          T qn = T(0);
#pragma unroll
          for (int s2 = 0; s2 < D; ++s2) qn += Q[r][s2] * na[s2];
          gx[r] += sgn * (inv2 * (t * na[r] - T(2) * qn) + cw * na[r]);
        }
      }
    }
    if (a.grad_coords) {
#pragma unroll
      for (int r = 0; r < D; ++r) a.grad_coords[i * D + r] = gx[r];
    }
  }
  block_sum2(pc, pk, red);
  if (threadIdx.x == 0) {
    a.partials[2 * blockIdx.x] = pc;
    a.partials[2 * blockIdx.x + 1] = pk;
  }
}

// Sum the per-CTA partials in a fixed order and write the global gradients.
template <typename T>
__global__ void __launch_bounds__(256) k_backward_final(const double* __restrict__ partials, int nblocks,
                                                        T* __restrict__ grad_c, T* __restrict__ grad_kappa_const) {
  __shared__ double s[2][256];
  double a = 0.0, b = 0.0;
  for (int k = threadIdx.x; k < nblocks; k += 256) {
    a += partials[2 * k];
    b += partials[2 * k + 1];
  }
  s[0][threadIdx.x] = a;
  s[1][threadIdx.x] = b;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      s[0][threadIdx.x] += s[0][threadIdx.x + w];
      s[1][threadIdx.x] += s[1][threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    if (grad_c) *grad_c = (T)s[0][0];
    if (grad_kappa_const) *grad_kappa_const = (T)s[1][0];
  }
}

template <int EL, typename T>
tg_status launch(const tg_pattern* p, const BwdArgs<T>& a, bool fused, T* grad_c, cudaStream_t s) {
  const int grid = tg::grid_for(p->N, BB);
  const tg::RefTab<T>& tab = tg::table<T>(p->el);
  if (fused) k_backward_gather<EL, T, true><<<grid, BB, 0, s>>>(a, tab);
  else k_backward_gather<EL, T, false><<<grid, BB, 0, s>>>(a, tab);
  TG_CK_LAUNCH("k_backward_gather");
  T* gk_const = (a.layout == TG_CONSTANT) ? a.grad_kappa : nullptr;
  if (grad_c || gk_const) {
    k_backward_final<T><<<1, 256, 0, s>>>(a.partials, grid, grad_c, gk_const);
    TG_CK_LAUNCH("k_backward_final");
  }
  return TG_OK;
}

template <typename T>
tg_status backward(const tg_pattern* p, const void* coords, const void* kappa, tg_layout kl, double c,
                   const void* gvals, const void* lam, const void* U, void* grad_kappa, void* grad_coords,
                   void* grad_c, cudaStream_t s) {
  BwdArgs<T> a;
  a.inc_ptr = p->inc_ptr;
  a.inc_e = p->inc_e;
  a.cells = p->cells;
  a.elem_slot = p->elem_slot;
  a.coords = static_cast<const T*>(coords);
  a.kappa = static_cast<const T*>(kappa);
  a.layout = kl;
  a.c = (T)c;
  a.gvals = static_cast<const T*>(gvals);
  a.lam = static_cast<const T*>(lam);
  a.U = static_cast<const T*>(U);
  a.grad_kappa = static_cast<T*>(grad_kappa);
  a.grad_coords = static_cast<T*>(grad_coords);
  a.partials = p->partials;
  a.N = p->N;
  a.status = p->status;
  const bool fused = gvals == nullptr;
  T* gc = static_cast<T*>(grad_c);
  switch (p->el) {
    case TG_P1_TRI: return launch<TG_P1_TRI, T>(p, a, fused, gc, s);
    case TG_P2_TRI: return launch<TG_P2_TRI, T>(p, a, fused, gc, s);
    default: return launch<TG_P1_TET, T>(p, a, fused, gc, s);
  }
}

}  // namespace

extern "C" tg_status tg_assemble_backward(const tg_pattern* p, tg_dtype dtype, const void* coords, const void* kappa,
                                          tg_layout kappa_layout, double c, const void* grad_vals, const void* lam,
                                          const void* U, void* grad_kappa, void* grad_coords, void* grad_c,
                                          tg_stream stream) {
  if (!p || (dtype != TG_F32 && dtype != TG_F64)) return TG_ERR_INVALID_ARG;
  if (p->el == TG_P1_TET_VEC3 || !kappa || (p->N > 0 && !coords)) return TG_ERR_INVALID_ARG;
  if (!(kappa_layout == TG_PER_QP || kappa_layout == TG_PER_ELEMENT || kappa_layout == TG_CONSTANT))
    return TG_ERR_INVALID_ARG;
  if (!grad_vals && !(lam && U)) return TG_ERR_INVALID_ARG;
  const size_t es = dtype == TG_F32 ? 4 : 8;
  if (((uintptr_t)coords % (p->dim == 2 ? 2 * es : es)) != 0) return TG_ERR_INVALID_ARG;
  if (p->N == 0) return TG_OK;
  cudaStream_t s = (cudaStream_t)stream;
  return dtype == TG_F32 ? backward<float>(p, coords, kappa, kappa_layout, c, grad_vals, lam, U, grad_kappa,
                                           grad_coords, grad_c, s)
                         : backward<double>(p, coords, kappa, kappa_layout, c, grad_vals, lam, U, grad_kappa,
                                            grad_coords, grad_c, s);
}
