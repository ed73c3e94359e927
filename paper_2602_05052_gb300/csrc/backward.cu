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

#include "fan.cuh"

namespace {

constexpr int BB = 128;
constexpr int kSlots = 4;  // partial sums per CTA (must match the pattern allocation)

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
  // element-once kernel: arrival counter and the global sums' outputs
  // (dL/dc, constant-kappa gradient; NULL = not requested)
  unsigned int* arrivals;
  T* sum_out[2];
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
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      a += red[0][w];
      b += red[1][w];
    }
  }
}

// Staged like the forward (gather.cuh): a CTA owns R = blockDim.x rows; in
// phase 1 its threads stride over the rows' contiguous incidence range, one
// incidence each, and leave the coordinate-gradient contribution of the
// visit in shared memory (contrib [D][cap]); in phase 2 each row sums its
// contributions in increasing element order.
template <int EL, typename T, bool FUSED>
__global__ void __launch_bounds__(BB) k_backward_gather(const BwdArgs<T> a, const __grid_constant__ tg::RefTab<T> tab,
                                                        int cap) {
  using El = tg::Elem<EL>;
  constexpr int NV = El::nv, D = El::dim, NQ = El::nq;
  __shared__ tg::RefTab<T> ts;
  __shared__ double red[2][BB / 32];
  extern __shared__ __align__(16) unsigned char dsm[];
  T* contrib = reinterpret_cast<T*>(dsm);
  tg::copy_table(ts, tab);
  const int R = blockDim.x;
  const int64_t r0 = (int64_t)blockIdx.x * R;
  const int64_t r1 = r0 + R < a.N ? r0 + R : a.N;
  double pc = 0.0, pk = 0.0;
  {
    const int J0 = __ldg(a.inc_ptr + r0), J1 = __ldg(a.inc_ptr + r1);
    for (int j = J0 + (int)threadIdx.x; j < J1; j += R) {
      const int ea = __ldg(a.inc_e + j);
      const int64_t e = ea >> 3;
      const int la = ea & 7;
      const int kk = j - J0;
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
#pragma unroll
        for (int r = 0; r < D; ++r) contrib[r * cap + kk] = T(0);
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
      const T inv = tg::recip(adet);
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
      T gxc[D];
#pragma unroll
      for (int r = 0; r < D; ++r) gxc[r] = T(0);
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
          gxc[r] = sgn * (inv2 * (t * na[r] - T(2) * qn) + cw * na[r]);
        }
      }
#pragma unroll
      for (int r = 0; r < D; ++r) contrib[r * cap + kk] = gxc[r];
    }
  }
  __syncthreads();
  const int64_t i = r0 + threadIdx.x;
  if (a.grad_coords && i < r1) {
    const int J0 = __ldg(a.inc_ptr + r0);
    const int js = __ldg(a.inc_ptr + i) - J0, je = __ldg(a.inc_ptr + i + 1) - J0;
    T gx[D];
#pragma unroll
    for (int r = 0; r < D; ++r) gx[r] = T(0);
    for (int k = js; k < je; ++k)
#pragma unroll
      for (int r = 0; r < D; ++r) gx[r] += contrib[r * cap + k];
#pragma unroll
    for (int r = 0; r < D; ++r) a.grad_coords[i * D + r] = gx[r];
  }
  block_sum2(pc, pk, red);
  if (threadIdx.x == 0) {
    a.partials[kSlots * blockIdx.x] = pc;
    a.partials[kSlots * blockIdx.x + 1] = pk;
  }
}

// Global sums: this CTA's partials, then the last CTA to arrive adds all
// CTAs' partials in CTA order and writes the outputs (no CTA waits for
// another).  Every thread of the CTA calls it.
template <typename T>
__device__ __forceinline__ void finish_sums(const BwdArgs<T>& a, double pc, double pk, double (*red)[BB / 32]) {
  block_sum2(pc, pk, red);
  __shared__ bool s_last;
  if (threadIdx.x == 0) {
    a.partials[kSlots * blockIdx.x] = pc;
    a.partials[kSlots * blockIdx.x + 1] = pk;
    __threadfence();
    s_last = atomicInc(a.arrivals, gridDim.x - 1) == gridDim.x - 1;  // wraps to 0 for the next launch
  }
  __syncthreads();
  if (s_last && (a.sum_out[0] || a.sum_out[1])) {
    __threadfence();
    double c0 = 0.0, c1 = 0.0;
    for (int b0 = threadIdx.x; b0 < (int)gridDim.x; b0 += 8 * blockDim.x) {
      double2 q[8];  // independent loads first, then the adds in order
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int b2 = b0 + u * blockDim.x;
        q[u] = b2 < (int)gridDim.x ? __ldcg(reinterpret_cast<const double2*>(a.partials + kSlots * b2))
                                   : make_double2(0.0, 0.0);
      }
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (b0 + u * (int)blockDim.x < (int)gridDim.x) {
          c0 += q[u].x;
          c1 += q[u].y;
        }
    }
    block_sum2(c0, c1, red);
    if (threadIdx.x == 0) {
      if (a.sum_out[0]) *a.sum_out[0] = (T)c0;
      if (a.sum_out[1]) *a.sum_out[1] = (T)c1;
    }
  }
}

// Backward of one P1 element for upstream weights W: the coordinate
// gradient of every vertex, dL/dx_c = A n_c with
//   A = sgn [ (S tr Q / det^2 + c <W,M>) I - (2 S / det^2) Q ],
// Q the symmetric part of P = N W N^T and S = sum_q w_q kappa_q; the
// coefficient gradient at the points gk[q] = w_q tr Q / |det|; and the
// element's dL/dc term |det| <W, M>.  <W, M> and tr(N W N^T) only see the
// symmetric part of W.  False (outputs zero) for a degenerate element.
template <int D, typename T>
__device__ __forceinline__ bool bwd_p1_element(const T (&x)[D + 1][D], const T (&kq)[D == 2 ? 3 : 4],
                                               const T (&W)[D + 1][D + 1], T c, const tg::RefTab<T>& tab,
                                               T (&gx)[D + 1][D], T (&gk)[D == 2 ? 3 : 4], T& cterm) {
  constexpr int NV = D + 1, NQ = D == 2 ? 3 : 4;
  tg::Geom<D, T> gm;
  if constexpr (D == 2) tg::tri_geom_x(x[0], x[1], x[2], gm);
  else tg::tet_geom_x(x[0], x[1], x[2], x[3], gm);
  const T adet = tg::absv(gm.det);
  if (!(adet > tg::det_tiny<T>())) {
#pragma unroll
    for (int cc = 0; cc < NV; ++cc)
#pragma unroll
      for (int r = 0; r < D; ++r) gx[cc][r] = T(0);
#pragma unroll
    for (int q = 0; q < NQ; ++q) gk[q] = T(0);
    cterm = T(0);
    return false;
  }
  T wm = T(0);
#pragma unroll
  for (int p = 0; p < NV; ++p)
#pragma unroll
    for (int q = 0; q < NV; ++q) wm += W[p][q] * tab.M[p][q];
  const T inv = tg::recip(adet);
  T y[NV][D];  // y[b][r] = sum_p W[p][b] n[p][r]
#pragma unroll
  for (int b2 = 0; b2 < NV; ++b2)
#pragma unroll
    for (int r = 0; r < D; ++r) {
      T sacc = T(0);
#pragma unroll
      for (int p = 0; p < NV; ++p) sacc += W[p][b2] * gm.n[p][r];
      y[b2][r] = sacc;
    }
  T P[D][D];  // P^T = N W N^T
#pragma unroll
  for (int r = 0; r < D; ++r)
#pragma unroll
    for (int s2 = 0; s2 < D; ++s2) {
      T sacc = T(0);
#pragma unroll
      for (int b2 = 0; b2 < NV; ++b2) sacc += y[b2][r] * gm.n[b2][s2];
      P[r][s2] = sacc;
    }
  T trq = T(0);
#pragma unroll
  for (int r = 0; r < D; ++r) trq += P[r][r];
  T S = T(0);
#pragma unroll
  for (int q = 0; q < NQ; ++q) S += tab.w[q] * kq[q];
  const T ti = trq * inv;
#pragma unroll
  for (int q = 0; q < NQ; ++q) gk[q] = tab.w[q] * ti;
  cterm = adet * wm;
  // A = sgn [(S tr Q / det^2 + c <W,M>) I - (2 S / det^2) Q] with 2 Q = P + P^T;
  // the sign of det enters by negation, not by a multiply
  const T Si2 = S * (inv * inv);
  const T d0u = fma(Si2, trq, c * wm), f2u = -Si2;
  const bool pos = gm.det > T(0);
  const T d0 = pos ? d0u : -d0u, f2 = pos ? f2u : -f2u;
  T A[D][D];
#pragma unroll
  for (int r = 0; r < D; ++r) {
    A[r][r] = fma(f2 + f2, P[r][r], d0);
#pragma unroll
    for (int s2 = r + 1; s2 < D; ++s2) A[r][s2] = A[s2][r] = f2 * (P[r][s2] + P[s2][r]);
  }
  // dL/dx_c = A n_c; the n_c sum to zero, so the first is minus the others' sum
#pragma unroll
  for (int cc = 1; cc < NV; ++cc)
#pragma unroll
    for (int r = 0; r < D; ++r) {
      T sacc = A[r][0] * gm.n[cc][0];
#pragma unroll
      for (int s2 = 1; s2 < D; ++s2) sacc = fma(A[r][s2], gm.n[cc][s2], sacc);
      gx[cc][r] = sacc;
    }
#pragma unroll
  for (int r = 0; r < D; ++r) {
    T sacc = gx[1][r];
#pragma unroll
    for (int cc = 2; cc < NV; ++cc) sacc += gx[cc][r];
    gx[0][r] = -sacc;
  }
  return true;
}

// Shared-memory layout of the Map's coordinate-gradient contributions: one
// D-vector per (vertex c, element slot j), at Gx[(c * capE + j) * D]
// (triangles: one 8- or 16-byte load per incidence in the Reduce).
template <int D, typename T>
__device__ __forceinline__ void gx_store(T* Gx, int capE, int c, int j, const T (&g)[D]) {
  T* q = Gx + ((size_t)c * capE + j) * D;
  if constexpr (D == 2) {
    *reinterpret_cast<typename tg::Vec2<T>::type*>(q) = {g[0], g[1]};
  } else {
#pragma unroll
    for (int r = 0; r < D; ++r) q[r] = g[r];
  }
}

// The Map of the P1 backward over one block (any view with nbe, be[] and
// vtx(c, k)).  Each distinct element of the block gathers its upstream
// weights W (through row_ptr and the element's packed column positions, or
// from lam and U) and computes the coordinate-gradient contributions of all
// its vertices into Gx (gx_store); the block that owns the element also
// writes its coefficient gradient and adds its dL/dc and constant-kappa
// terms to bc and bk.
template <int D, typename T, bool FUSED, int UB, typename View>
__device__ __forceinline__ void bwd_blk_map(const BwdArgs<T>& a, const tg::RefTab<T>& tab, int capE, const View& v,
                                            const uint64_t* __restrict__ elem_pos,
                                            const int32_t* __restrict__ row_ptr, T* Gx, T& bc, T& bk) {
  constexpr int NV = D + 1, NQ = D == 2 ? 3 : 4;
  const int NT = blockDim.x;
  for (int j0 = threadIdx.x; j0 < v.nbe; j0 += UB * NT) {
    int e[UB], vid[UB][NV];
    bool own[UB];
#pragma unroll
    for (int u = 0; u < UB; ++u) {
      const bool live = j0 + u * NT < v.nbe;
      const int j = live ? j0 + u * NT : 0;
      const uint32_t w0 = v.be[j];
      e[u] = (int)tg::bel_elem(w0);
      own[u] = live && tg::bel_owner(w0);
#pragma unroll
      for (int c = 0; c < NV; ++c) vid[u][c] = v.vtx(c, j);
    }
    T x[UB][NV][D], kq[UB][NQ], W[UB][NV][NV];
    uint64_t ep[UB];
    int rpv[UB][NV];
#pragma unroll
    for (int u = 0; u < UB; ++u) {
#pragma unroll
      for (int c = 0; c < NV; ++c) tg::load_x<D, T>(a.coords, vid[u][c], x[u][c]);
      if (a.layout == TG_PER_QP) {
#pragma unroll
        for (int q = 0; q < NQ; ++q) kq[u][q] = __ldg(a.kappa + (int64_t)e[u] * NQ + q);
      } else {
        const T k = a.layout == TG_PER_ELEMENT ? __ldg(a.kappa + e[u]) : __ldg(a.kappa);
#pragma unroll
        for (int q = 0; q < NQ; ++q) kq[u][q] = k;
      }
      if constexpr (FUSED) {
        T l[NV], uu[NV];
#pragma unroll
        for (int c = 0; c < NV; ++c) {
          l[c] = __ldg(a.lam + vid[u][c]);
          uu[c] = __ldg(a.U + vid[u][c]);
        }
#pragma unroll
        for (int p = 0; p < NV; ++p)
#pragma unroll
          for (int q = 0; q < NV; ++q) W[u][p][q] = l[p] * uu[q];
      } else {
        ep[u] = __ldg(reinterpret_cast<const unsigned long long*>(elem_pos) + e[u]);
#pragma unroll
        for (int c = 0; c < NV; ++c) rpv[u][c] = __ldg(row_ptr + vid[u][c]);
      }
    }
    if constexpr (!FUSED) {
#pragma unroll
      for (int u = 0; u < UB; ++u) {
        const uint32_t lo = (uint32_t)ep[u], hi = (uint32_t)(ep[u] >> 32);
#pragma unroll
        for (int p = 0; p < NV; ++p) {
          const T* row = a.gvals + rpv[u][p];
#pragma unroll
          for (int q = 0; q < NV; ++q) {
            const int sh = 4 * (p * NV + q);
            W[u][p][q] = __ldg(row + ((sh < 32 ? lo >> sh : hi >> (sh - 32)) & 15u));
          }
        }
      }
    }
#pragma unroll
    for (int u = 0; u < UB; ++u) {
      const int j = j0 + u * NT;
      if (j >= v.nbe) continue;
      tg::Geom<D, T> gm;
      if constexpr (D == 2) tg::tri_geom_x(x[u][0], x[u][1], x[u][2], gm);
      else tg::tet_geom_x(x[u][0], x[u][1], x[u][2], x[u][3], gm);
      const T adet = tg::absv(gm.det);
      T gx[NV][D];
      if (!(adet > tg::det_tiny<T>())) {
        tg::record_error(a.status, TG_ERR_DEGENERATE_ELEMENT, e[u]);
        if (own[u] && a.grad_kappa) {
          if (a.layout == TG_PER_QP)
            for (int q = 0; q < NQ; ++q) a.grad_kappa[(int64_t)e[u] * NQ + q] = T(0);
          else if (a.layout == TG_PER_ELEMENT) a.grad_kappa[e[u]] = T(0);
        }
#pragma unroll
        for (int c = 0; c < NV; ++c)
#pragma unroll
          for (int r = 0; r < D; ++r) gx[c][r] = T(0);
      } else {
        // <W, M> = <W_s, M> and tr(N W N^T) = tr(N W_s N^T): only the
        // symmetric part of P = N W N^T needs W_s.
        T wm = T(0);
#pragma unroll
        for (int p = 0; p < NV; ++p)
#pragma unroll
          for (int q = 0; q < NV; ++q) wm += W[u][p][q] * tab.M[p][q];
        const T inv = tg::recip(adet);
        const T sgn = gm.det > T(0) ? T(1) : T(-1);
        T y[NV][D];  // y[b][r] = sum_p W[p][b] n[p][r]
#pragma unroll
        for (int b2 = 0; b2 < NV; ++b2)
#pragma unroll
          for (int r = 0; r < D; ++r) {
            T sacc = T(0);
#pragma unroll
            for (int p = 0; p < NV; ++p) sacc += W[u][p][b2] * gm.n[p][r];
            y[b2][r] = sacc;
          }
        T P[D][D];  // P[s][r] = sum_b n[b][s] y[b][r] = (N W^T-ish) contraction, P^T = N W N^T
#pragma unroll
        for (int r = 0; r < D; ++r)
#pragma unroll
          for (int s2 = 0; s2 < D; ++s2) {
            T sacc = T(0);
#pragma unroll
            for (int b2 = 0; b2 < NV; ++b2) sacc += y[b2][r] * gm.n[b2][s2];
            P[r][s2] = sacc;
          }
        T trq = T(0);
#pragma unroll
        for (int r = 0; r < D; ++r) trq += P[r][r];
        T S = T(0);
#pragma unroll
        for (int q = 0; q < NQ; ++q) S += tab.w[q] * kq[u][q];
        if (own[u]) {
          T gk[NQ];
#pragma unroll
          for (int q = 0; q < NQ; ++q) gk[q] = tab.w[q] * trq * inv;
          if (a.grad_kappa) {
            if (a.layout == TG_PER_QP) {
#pragma unroll
              for (int q = 0; q < NQ; ++q) a.grad_kappa[(int64_t)e[u] * NQ + q] = gk[q];
            } else {
              T sg = T(0);
#pragma unroll
              for (int q = 0; q < NQ; ++q) sg += gk[q];
              if (a.layout == TG_PER_ELEMENT) a.grad_kappa[e[u]] = sg;
              else bk += sg;
            }
          }
          bc += adet * wm;
        }
        // dL/dx_c = A n_c with A = sgn [ (S tr Q / det^2 + c <W,M>) I - (2 S / det^2) Q ],
        // Q = (P + P^T) / 2
        const T inv2 = inv * inv;
        const T d0 = sgn * (S * trq * inv2 + a.c * wm);
        const T f2 = -sgn * S * inv2;  // times 2 Q = P + P^T
        T A[D][D];
#pragma unroll
        for (int r = 0; r < D; ++r)
#pragma unroll
          for (int s2 = 0; s2 < D; ++s2) A[r][s2] = f2 * (P[r][s2] + P[s2][r]) + (r == s2 ? d0 : T(0));
#pragma unroll
        for (int c = 0; c < NV; ++c)
#pragma unroll
          for (int r = 0; r < D; ++r) {
            T sacc = T(0);
#pragma unroll
            for (int s2 = 0; s2 < D; ++s2) sacc += A[r][s2] * gm.n[c][s2];
            gx[c][r] = sacc;
          }
      }
#pragma unroll
      for (int c = 0; c < NV; ++c)
#pragma unroll
        for (int r = 0; r < D; ++r) gx_store<D>(Gx, capE, c, j, gx[c]);
    }
  }
}

// P1 backward over element-once row blocks (blocks.cuh): the Map of
// bwd_blk_map, then rows sum their incidences' contributions in increasing
// element order.  Per-CTA FP64 partials of the global sums are added by the
// last CTA to finish (finish_sums).
template <int D, typename T, bool FUSED, int UB>
__global__ void __launch_bounds__(BB, (D == 2 && sizeof(T) == 4) ? (UB >= 3 ? 5 : 6) : 2) k_backward_blk(const BwdArgs<T> a, const __grid_constant__ tg::RefTab<T> tab,
                                                     const tg::BlkArgs g, const uint64_t* __restrict__ elem_pos,
                                                     const int32_t* __restrict__ row_ptr) {
  constexpr int NV = D + 1;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double red[2][BB / 32];
  tg::BlkPipe pipe;
  T* Gx = reinterpret_cast<T*>(pipe.init(smem, g));
  __syncthreads();  // publishes the mbarrier initialisation
  double pc = 0.0, pk = 0.0;
  TG_BLK_PIPELINE_BEGIN(pipe, g, a.status)
  T bc = T(0), bk = T(0);  // this thread's terms of the block, added to pc, pk once per block
  bwd_blk_map<D, T, FUSED, UB>(a, tab, g.capE, v, elem_pos, row_ptr, Gx, bc, bk);
  pc += (double)bc;
  pk += (double)bk;
  __syncthreads();
  if (a.grad_coords) {
    const int i = v.r0 + (int)threadIdx.x;
    if (i < v.r1) {
      T gs[D];
#pragma unroll
      for (int r = 0; r < D; ++r) gs[r] = T(0);
      const int je = v.ip[i + 1];
      for (int j = v.ip[i]; j < je; ++j) {
        const auto rr = tg::blk_rec<NV>(v.rc, j);
        const T* gp = Gx + ((size_t)rr.a() * g.capE + rr.le()) * D;
#pragma unroll
        for (int r = 0; r < D; ++r) gs[r] += gp[r];
      }
#pragma unroll
      for (int r = 0; r < D; ++r) a.grad_coords[(int64_t)v.pm[i] * D + r] = gs[r];
    }
  }
  __syncthreads();  // stage s and Gx are free again
  TG_BLK_PIPELINE_END
  finish_sums(a, pc, pk, red);
}

// P1 triangle backward with the fan-ordered Reduce (fan.cuh): the same Map;
// each row sums its fan triangles' contributions in fan order.
template <typename T, bool FUSED, int UB>
__global__ void __launch_bounds__(BB, sizeof(T) == 4 ? (UB >= 3 ? 5 : 6) : 2) k_backward_fan(
    const BwdArgs<T> a, const __grid_constant__ tg::RefTab<T> tab, const tg::FanArgs g,
    const uint64_t* __restrict__ elem_pos, const int32_t* __restrict__ row_ptr) {
  using T2 = typename tg::Vec2<T>::type;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double red[2][BB / 32];
  tg::FanPipe pipe;
  T* Gx = reinterpret_cast<T*>(pipe.init(smem, g));
  __syncthreads();  // publishes the mbarrier initialisation
  double pc = 0.0, pk = 0.0;
  TG_FAN_PIPELINE_BEGIN(pipe, g, a.status)
  T bc = T(0), bk = T(0);
  bwd_blk_map<2, T, FUSED, UB>(a, tab, g.capE, v, elem_pos, row_ptr, Gx, bc, bk);
  pc += (double)bc;
  pk += (double)bk;
  __syncthreads();
  if (a.grad_coords) {
    const int t = (int)threadIdx.x;
    if (v.r0 + t < v.r1) {
      const int deg = (int)(v.info[t] & 31u);
      const T2* G2 = reinterpret_cast<const T2*>(Gx);
      T gx0 = T(0), gx1 = T(0);
      for (int k = 0; k < deg; ++k) {
        const unsigned r = v.rec[k * v.rs + t];
        const T2 q = G2[tg::fan_a(r) * g.capE + tg::fan_le(r)];
        gx0 += q.x;
        gx1 += q.y;
      }
      reinterpret_cast<T2*>(a.grad_coords)[v.pm[t]] = T2{gx0, gx1};
    }
  }
  __syncthreads();  // stage s and Gx are free again
  TG_FAN_PIPELINE_END
  finish_sums(a, pc, pk, red);
}

// Two passes, every element evaluated once (the FP64 path: bound by the
// FP64 pipe, it gains from evaluating each element once instead of about
// 1.2 times; in FP32 the row blocks are faster).  Map: one thread per element
// gathers its upstream weights and writes its coefficient gradient and the
// coordinate gradients of its vertices, gxe[(e * NV + c) * D + r]; the
// global sums go through the per-CTA partials.  Node: one thread per node
// sums its incidences' gradients in increasing element order (the order of
// the row-block kernel, so grad_coords carries the same bits).
template <int D, typename T, bool FUSED, int EPT>
__global__ void __launch_bounds__(BB) k_backward_map(const BwdArgs<T> a, const __grid_constant__ tg::RefTab<T> tab,
                                                    const uint64_t* __restrict__ elem_pos,
                                                    const int32_t* __restrict__ row_ptr, int64_t E,
                                                    T* __restrict__ gxe) {
  constexpr int NV = D + 1, NQ = D == 2 ? 3 : 4;
  __shared__ double red[2][BB / 32];
  double pc = 0.0, pk = 0.0;
  for (int64_t base = (int64_t)blockIdx.x * (BB * EPT); base < E; base += (int64_t)gridDim.x * (BB * EPT)) {
    int64_t e[EPT];
    T x[EPT][NV][D], kq[EPT][NQ], W[EPT][NV][NV];
#pragma unroll
    for (int u = 0; u < EPT; ++u) {
      e[u] = base + threadIdx.x + u * BB;
      const int64_t ee = e[u] < E ? e[u] : E - 1;
      int vid[NV];
#pragma unroll
      for (int c = 0; c < NV; ++c) vid[c] = __ldg(a.cells + ee * NV + c);
#pragma unroll
      for (int c = 0; c < NV; ++c) tg::load_x<D, T>(a.coords, vid[c], x[u][c]);
      if (a.layout == TG_PER_QP) {
#pragma unroll
        for (int q = 0; q < NQ; ++q) kq[u][q] = __ldg(a.kappa + ee * NQ + q);
      } else {
        const T k = a.layout == TG_PER_ELEMENT ? __ldg(a.kappa + ee) : __ldg(a.kappa);
#pragma unroll
        for (int q = 0; q < NQ; ++q) kq[u][q] = k;
      }
      if constexpr (FUSED) {
        T l[NV], uu[NV];
#pragma unroll
        for (int c = 0; c < NV; ++c) {
          l[c] = __ldg(a.lam + vid[c]);
          uu[c] = __ldg(a.U + vid[c]);
        }
#pragma unroll
        for (int p = 0; p < NV; ++p)
#pragma unroll
          for (int q = 0; q < NV; ++q) W[u][p][q] = l[p] * uu[q];
      } else {
        const uint64_t ep = __ldg(reinterpret_cast<const unsigned long long*>(elem_pos) + ee);
        int rpv[NV];
#pragma unroll
        for (int c = 0; c < NV; ++c) rpv[c] = __ldg(row_ptr + vid[c]);
#pragma unroll
        for (int p = 0; p < NV; ++p)
#pragma unroll
          for (int q = 0; q < NV; ++q)
            W[u][p][q] = __ldg(a.gvals + rpv[p] + (int)((ep >> (4 * (p * NV + q))) & 15u));
      }
    }
    T bc = T(0), bk = T(0);
#pragma unroll
    for (int u = 0; u < EPT; ++u) {
      if (e[u] >= E) break;
      T gx[NV][D], gk[NQ], cterm;
      if (!bwd_p1_element<D, T>(x[u], kq[u], W[u], a.c, tab, gx, gk, cterm))
        tg::record_error(a.status, TG_ERR_DEGENERATE_ELEMENT, e[u]);
      if (a.grad_kappa) {
        if (a.layout == TG_PER_QP) {
#pragma unroll
          for (int q = 0; q < NQ; ++q) a.grad_kappa[e[u] * NQ + q] = gk[q];
        } else {
          T sg = T(0);
#pragma unroll
          for (int q = 0; q < NQ; ++q) sg += gk[q];
          if (a.layout == TG_PER_ELEMENT) a.grad_kappa[e[u]] = sg;
          else bk += sg;
        }
      }
      bc += cterm;
      if (gxe) {
#pragma unroll
        for (int c = 0; c < NV; ++c)
#pragma unroll
          for (int r = 0; r < D; ++r) gxe[(e[u] * NV + c) * D + r] = gx[c][r];
      }
    }
    pc += (double)bc;
    pk += (double)bk;
  }
  finish_sums(a, pc, pk, red);
}

template <int D, typename T>
__global__ void __launch_bounds__(BB) k_backward_node(const BwdArgs<T> a, const T* __restrict__ gxe) {
  constexpr int NV = D + 1;
  const int64_t i = (int64_t)blockIdx.x * BB + threadIdx.x;
  if (i >= a.N) return;
  const int j0 = __ldg(a.inc_ptr + i), j1 = __ldg(a.inc_ptr + i + 1);
  T gs[D];
#pragma unroll
  for (int r = 0; r < D; ++r) gs[r] = T(0);
  for (int j = j0; j < j1; ++j) {
    const int ea = __ldg(a.inc_e + j);
    const T* gp = gxe + ((int64_t)(ea >> 3) * NV + (ea & 7)) * D;
#pragma unroll
    for (int r = 0; r < D; ++r) gs[r] += gp[r];
  }
#pragma unroll
  for (int r = 0; r < D; ++r) a.grad_coords[i * D + r] = gs[r];
}

// Sum the per-CTA partials (kSlots doubles per CTA) in a fixed order and
// write (or add to) the global gradients out[k], k < nslots (NULL = skip).
struct FinalOut {
  void* out[kSlots];
  int nslots;
  int accumulate;
};

constexpr int kFinal = 256;

// One CTA; FP64 adds are slow on this part, so every thread adds only
// partials that exist (in a fixed order), then a fixed shared-memory tree.
template <typename T>
__global__ void __launch_bounds__(kFinal) k_backward_final(const double* __restrict__ partials, int nblocks,
                                                           const FinalOut o) {
  __shared__ double s[kSlots][kFinal];
  double acc[kSlots] = {0.0, 0.0, 0.0, 0.0};
  const int ns = o.nslots;
  for (int b = threadIdx.x; b < nblocks; b += kFinal)
#pragma unroll
    for (int k = 0; k < kSlots; ++k)
      if (k < ns) acc[k] += partials[kSlots * b + k];
#pragma unroll
  for (int k = 0; k < kSlots; ++k) s[k][threadIdx.x] = acc[k];
  __syncthreads();
  for (int w = kFinal / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w)
#pragma unroll
      for (int k = 0; k < kSlots; ++k)
        if (k < ns) s[k][threadIdx.x] += s[k][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int k = 0; k < ns; ++k)
      if (o.out[k]) {
        T* d = static_cast<T*>(o.out[k]);
        *d = o.accumulate ? *d + (T)s[k][0] : (T)s[k][0];
      }
}

// Rows per CTA of the staged backward kernels: the largest R in {128, 64, 32}
// whose stage (nval values per incidence) fits in 64 KB, else in 160 KB.
template <typename T>
int bwd_rows(const tg_pattern* p, int nval, size_t* bytes) {
  for (size_t lim : {64u * 1024u, 160u * 1024u})
    for (int R : {128, 64, 32}) {
      const size_t b = (size_t)nval * std::max(1, R * p->max_deg) * sizeof(T);
      if (b <= lim) {
        *bytes = b;
        return R;
      }
    }
  return 0;
}

// Element-once launch (P1 with row blocks and packed positions); false in
// *used when the pattern or the shared-memory budget does not allow it.
template <int D, typename T>
tg_status launch_blk(const tg_pattern* p, const BwdArgs<T>& a, bool fused, int* grid_out, bool* used,
                     cudaStream_t s) {
  *used = false;
  if (!p->bel || !p->elem_pos) return TG_OK;
  if constexpr (D == 2) {
    if (p->fan) {
      const tg::FanArgs gf = tg::fan_args(p);
      const size_t smem = tg::fan_stage_bytes(gf.R, gf.capF, gf.capE, 3) + (size_t)3 * 2 * gf.capE * sizeof(T);
      if (smem <= 113 * 1024 && p->blk_rows <= BB) {
        const tg::RefTab<T>& tab = tg::table<T>(p->el);
        const int need = (p->blk_max_elems + BB - 1) / BB;
        tg_status st = TG_OK;
        auto go = [&](auto kern) {
          if ((st = tg::set_smem((const void*)kern, smem)) != TG_OK) return;
          int per_sm = 0;
          cudaError_t ce = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, BB, smem);
          if (ce != cudaSuccess) {
            st = tg::cuda_fail(ce, "cudaOccupancyMaxActiveBlocksPerMultiprocessor", __FILE__, __LINE__);
            return;
          }
          const int64_t cap_ctas = (p->n_partials - 4) / kSlots;
          const int grid =
              (int)std::min<int64_t>({p->n_blk, (int64_t)std::max(per_sm, 1) * tg::sm_count(), cap_ctas});
          kern<<<grid, BB, smem, s>>>(a, tab, gf, p->elem_pos, p->row_ptr);
          *grid_out = grid;
        };
        if constexpr (sizeof(T) == 8) {
          if (fused) go(k_backward_fan<T, true, 1>);
          else go(k_backward_fan<T, false, 1>);
        } else {
          if (need >= 3 && !fused) go(k_backward_fan<T, false, 3>);
          else if (fused) go(k_backward_fan<T, true, 2>);
          else go(k_backward_fan<T, false, 2>);
        }
        if (st != TG_OK) return st;
        TG_CK_LAUNCH("k_backward_fan");
        *used = true;
        return TG_OK;
      }
    }
  }
  const tg::BlkArgs g = tg::blk_args(p);
  const size_t smem = tg::blk_stage_bytes(p->blk_rows, g.capJ, g.capE, D + 1) +
                      (size_t)(D + 1) * D * g.capE * sizeof(T);
  if (smem > 113 * 1024) return TG_OK;
  const int nt = BB;
  if (p->blk_rows > BB) return TG_OK;
  const tg::RefTab<T>& tab = tg::table<T>(p->el);
  const int need = (p->blk_max_elems + BB - 1) / BB;  // elements per thread for one Map round
  tg_status st = TG_OK;
  auto go = [&](auto kern) {
    if ((st = tg::set_smem((const void*)kern, smem)) != TG_OK) return;
    int per_sm = 0;
    cudaError_t ce = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, nt, smem);
    if (ce != cudaSuccess) {
      st = tg::cuda_fail(ce, "cudaOccupancyMaxActiveBlocksPerMultiprocessor", __FILE__, __LINE__);
      return;
    }
    const int64_t cap_ctas = (p->n_partials - 4) / kSlots;  // partial slots of the pattern
    const int grid = (int)std::min<int64_t>({p->n_blk, (int64_t)std::max(per_sm, 1) * tg::sm_count(), cap_ctas});
    kern<<<grid, nt, smem, s>>>(a, tab, g, p->elem_pos, p->row_ptr);
    *grid_out = grid;
  };
  if constexpr (sizeof(T) == 8) {
    if (fused) go(k_backward_blk<D, T, true, 1>);
    else go(k_backward_blk<D, T, false, 1>);
  } else {
    // the fused adjoint path (lam U^T, no gvals gather) runs faster with two
    // elements per thread and one CTA more per SM (61 against 67 us at
    // 1024^2); the gvals path with three (69 against 70)
    if (need >= 3 && !fused) {
      go(k_backward_blk<D, T, false, 3>);
    } else {
      if (fused) go(k_backward_blk<D, T, true, 2>);
      else go(k_backward_blk<D, T, false, 2>);
    }
  }
  if (st != TG_OK) return st;
  TG_CK_LAUNCH("k_backward_blk");
  *used = true;
  return TG_OK;
}

// Two-pass launch (k_backward_map, then k_backward_node when the coordinate
// gradient is wanted).
template <int D, typename T>
tg_status launch_two_pass(const tg_pattern* p, const BwdArgs<T>& a, bool fused, cudaStream_t s) {
  constexpr int EPT = 2;
  T* gxe = a.grad_coords ? static_cast<T*>(p->elem_scratch) : nullptr;
  const tg::RefTab<T>& tab = tg::table<T>(p->el);
  const int64_t cap_ctas = (p->n_partials - 4) / kSlots;  // partial slots of the pattern
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((p->E + BB * EPT - 1) / (BB * EPT), cap_ctas));
  if (fused) k_backward_map<D, T, true, EPT><<<grid, BB, 0, s>>>(a, tab, p->elem_pos, p->row_ptr, p->E, gxe);
  else k_backward_map<D, T, false, EPT><<<grid, BB, 0, s>>>(a, tab, p->elem_pos, p->row_ptr, p->E, gxe);
  TG_CK_LAUNCH("k_backward_map");
  if (a.grad_coords) {
    k_backward_node<D, T><<<tg::grid_for(p->N, BB), BB, 0, s>>>(a, gxe);
    TG_CK_LAUNCH("k_backward_node");
  }
  return TG_OK;
}

template <int EL, typename T>
tg_status launch(const tg_pattern* p, const BwdArgs<T>& a, bool fused, T* grad_c, cudaStream_t s) {
  if constexpr (EL == TG_P1_TRI || EL == TG_P1_TET) {
    bool used = false;
    int grid = 0;
    BwdArgs<T> ab = a;
    ab.arrivals = p->arrivals;
    ab.sum_out[0] = grad_c;
    ab.sum_out[1] = (a.layout == TG_CONSTANT) ? a.grad_kappa : nullptr;
    // Two passes evaluate each element once, row blocks once per block
    // holding one of its vertices: 1.2 times on the Hilbert-ordered
    // triangles, where FP32 runs on the row blocks, about 3 times on
    // tetrahedral grids.  FP64 is bound by the FP64 pipe and always takes
    // the two passes.
    if constexpr (sizeof(T) == 8 || EL == TG_P1_TET) {
      if (p->elem_scratch && p->elem_pos && p->E > 0) return launch_two_pass<tg::Elem<EL>::dim, T>(p, ab, fused, s);
    }
    tg_status st = launch_blk<tg::Elem<EL>::dim, T>(p, ab, fused, &grid, &used, s);
    if (st != TG_OK) return st;
    if (used) return TG_OK;
  }
  size_t smem = 0;
  const int R = bwd_rows<T>(p, tg::Elem<EL>::dim, &smem);
  if (R == 0) return TG_ERR_UNSUPPORTED;
  const int grid = tg::grid_for(p->N, R);
  const int cap = std::max(1, R * p->max_deg);
  const tg::RefTab<T>& tab = tg::table<T>(p->el);
  tg_status st = tg::set_smem(fused ? (const void*)k_backward_gather<EL, T, true>
                                    : (const void*)k_backward_gather<EL, T, false>, smem);
  if (st != TG_OK) return st;
  if (fused) k_backward_gather<EL, T, true><<<grid, R, smem, s>>>(a, tab, cap);
  else k_backward_gather<EL, T, false><<<grid, R, smem, s>>>(a, tab, cap);
  TG_CK_LAUNCH("k_backward_gather");
  T* gk_const = (a.layout == TG_CONSTANT) ? a.grad_kappa : nullptr;
  if (grad_c || gk_const) {
    FinalOut o{{grad_c, gk_const, nullptr, nullptr}, 2, 0};
    k_backward_final<T><<<1, kFinal, 0, s>>>(a.partials, grid, o);
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
  a.arrivals = nullptr;
  a.sum_out[0] = a.sum_out[1] = nullptr;
  const bool fused = gvals == nullptr;
  T* gc = static_cast<T*>(grad_c);
  switch (p->el) {
    case TG_P1_TRI: return launch<TG_P1_TRI, T>(p, a, fused, gc, s);
    case TG_P2_TRI: return launch<TG_P2_TRI, T>(p, a, fused, gc, s);
    default: return launch<TG_P1_TET, T>(p, a, fused, gc, s);
  }
}

// ------------------------------------------------------------------ load vector
// Reverse mode of F[g(a) nc + k] = |det J| h_ak, with h_ak = sum_b Mhat_ab f_bk
// (PER_NODE), sum_q w_q phi_qa f_eqk (PER_QP) or m1_a f_k (CONSTANT).
// For an upstream gradient gF:
//   dL/df           the transpose of each of those maps, times |det J|;
//   dL/dx_b         = sign(det J) (sum_ak gF_ak h_ak) n_b   for the vertices b
// (only |det J| depends on the coordinates: d|det J| = |det J| tr(J^{-1} dJ)).
template <typename T>
struct LoadBwdArgs {
  const int32_t* __restrict__ inc_ptr;
  const int32_t* __restrict__ inc_e;
  const int32_t* __restrict__ cells;
  const T* __restrict__ coords;
  const T* __restrict__ f;
  int layout;
  const T* __restrict__ gF;
  T* __restrict__ grad_f;
  T* __restrict__ grad_coords;
  int accumulate;
  double* __restrict__ partials;
  int64_t N;
  unsigned long long* status;
  // element-once kernel: arrival counter and the global sums' outputs
  // (dL/dc, constant-kappa gradient; NULL = not requested)
  unsigned int* arrivals;
  T* sum_out[2];
};

template <int EL, typename T, int NC>
__global__ void __launch_bounds__(BB) k_load_backward(const LoadBwdArgs<T> a, const __grid_constant__ tg::RefTab<T> tab,
                                                      int cap) {
  using El = tg::Elem<EL>;
  constexpr int NV = El::nv, D = El::dim, NQ = El::nq;
  __shared__ tg::RefTab<T> ts;
  __shared__ double red[BB / 32][NC];
  extern __shared__ __align__(16) unsigned char dsm[];
  T* contrib = reinterpret_cast<T*>(dsm);  // [D + NC][cap]
  tg::copy_table(ts, tab);
  const int R = blockDim.x;
  const int64_t r0 = (int64_t)blockIdx.x * R;
  const int64_t r1 = r0 + R < a.N ? r0 + R : a.N;
  double pk[NC];
#pragma unroll
  for (int k = 0; k < NC; ++k) pk[k] = 0.0;
  const int J0 = __ldg(a.inc_ptr + r0), J1 = __ldg(a.inc_ptr + r1);
  for (int j = J0 + (int)threadIdx.x; j < J1; j += R) {
    const int ea = __ldg(a.inc_e + j);
    const int64_t e = ea >> 3;
    const int la = ea & 7;
    const int kk = j - J0;
    const int32_t* cl = a.cells + e * NV;
    int v[NV];
#pragma unroll
    for (int b = 0; b < NV; ++b) v[b] = __ldg(cl + b);
    tg::Geom<D, T> g;
    if constexpr (D == 2) tg::tri_geom(a.coords, v[0], v[1], v[2], g);
    else tg::tet_geom(a.coords, v[0], v[1], v[2], v[3], g);
    const T adet = tg::absv(g.det);
    T gxc[D], gfc[NC];
#pragma unroll
    for (int r = 0; r < D; ++r) gxc[r] = T(0);
#pragma unroll
    for (int k = 0; k < NC; ++k) gfc[k] = T(0);
    if (!(adet > tg::det_tiny<T>())) {
      tg::record_error(a.status, TG_ERR_DEGENERATE_ELEMENT, e);
    } else {
      T gv[NV][NC];
#pragma unroll
      for (int b = 0; b < NV; ++b)
#pragma unroll
        for (int k = 0; k < NC; ++k) gv[b][k] = __ldg(a.gF + (int64_t)v[b] * NC + k);
      // dL/df
      if (a.grad_f) {
        if (a.layout == TG_PER_NODE) {
#pragma unroll
          for (int k = 0; k < NC; ++k) {
            T s = T(0);
#pragma unroll
            for (int b = 0; b < NV; ++b) s += ts.M[b][la] * gv[b][k];
            gfc[k] = adet * s;
          }
        } else if (la == 0) {
          if (a.layout == TG_PER_QP) {
#pragma unroll
            for (int q = 0; q < NQ; ++q)
#pragma unroll
              for (int k = 0; k < NC; ++k) {
                T s = T(0);
#pragma unroll
                for (int b = 0; b < NV; ++b) s += ts.phi[q][b] * gv[b][k];
                T* d = a.grad_f + (e * NQ + q) * NC + k;
                const T val = adet * ts.w[q] * s;
                *d = a.accumulate ? *d + val : val;
              }
          } else {
#pragma unroll
            for (int k = 0; k < NC; ++k) {
              T s = T(0);
#pragma unroll
              for (int b = 0; b < NV; ++b) s += ts.m1[b] * gv[b][k];
              pk[k] += (double)(adet * s);
            }
          }
        }
      }
      // dL/dx for the geometric vertices
      if (a.grad_coords && la <= D) {
        T Le = T(0);
#pragma unroll
        for (int k = 0; k < NC; ++k) {
          if (a.layout == TG_PER_NODE) {
            T fb[NV];
#pragma unroll
            for (int b = 0; b < NV; ++b) fb[b] = __ldg(a.f + (int64_t)v[b] * NC + k);
#pragma unroll
            for (int p = 0; p < NV; ++p) {
              T h = T(0);
#pragma unroll
              for (int b = 0; b < NV; ++b) h += ts.M[p][b] * fb[b];
              Le += gv[p][k] * h;
            }
          } else if (a.layout == TG_PER_QP) {
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
              T s = T(0);
#pragma unroll
              for (int p = 0; p < NV; ++p) s += ts.phi[q][p] * gv[p][k];
              Le += ts.w[q] * __ldg(a.f + (e * NQ + q) * NC + k) * s;
            }
          } else {
            T s = T(0);
#pragma unroll
            for (int p = 0; p < NV; ++p) s += ts.m1[p] * gv[p][k];
            Le += __ldg(a.f + k) * s;
          }
        }
        const T sgn = g.det > T(0) ? T(1) : T(-1);
#pragma unroll
        for (int r = 0; r < D; ++r) {
          T col[D + 1];
#pragma unroll
          for (int b = 0; b <= D; ++b) col[b] = g.n[b][r];
          gxc[r] = sgn * Le * tg::sel(la, col);
        }
      }
    }
#pragma unroll
    for (int r = 0; r < D; ++r) contrib[r * cap + kk] = gxc[r];
#pragma unroll
    for (int k = 0; k < NC; ++k) contrib[(D + k) * cap + kk] = gfc[k];
  }
  __syncthreads();
  const int64_t i = r0 + threadIdx.x;
  if (i < r1) {
    const int js = __ldg(a.inc_ptr + i) - J0, je = __ldg(a.inc_ptr + i + 1) - J0;
    if (a.grad_coords) {
#pragma unroll
      for (int r = 0; r < D; ++r) {
        T gx = T(0);
        for (int k = js; k < je; ++k) gx += contrib[r * cap + k];
        T* d = a.grad_coords + i * D + r;
        *d = a.accumulate ? *d + gx : gx;
      }
    }
    if (a.grad_f && a.layout == TG_PER_NODE) {
#pragma unroll
      for (int k = 0; k < NC; ++k) {
        T gf = T(0);
        for (int m = js; m < je; ++m) gf += contrib[(D + k) * cap + m];
        T* d = a.grad_f + i * NC + k;
        *d = a.accumulate ? *d + gf : gf;
      }
    }
  }
  // fixed-order block sums of the CONSTANT-layout partials
#pragma unroll
  for (int k = 0; k < NC; ++k)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) pk[k] += __shfl_down_sync(0xffffffffu, pk[k], o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < NC; ++k) red[wid][k] = pk[k];
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 0; k < kSlots; ++k) {
      double s = 0.0;
      if (k < NC)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w][k];
      a.partials[kSlots * blockIdx.x + k] = s;
    }
  }
}

template <int EL, typename T>
tg_status launch_load_bwd(const tg_pattern* p, const LoadBwdArgs<T>& a, int ncomp, cudaStream_t s) {
  size_t smem = 0;
  const int R = bwd_rows<T>(p, tg::Elem<EL>::dim + ncomp, &smem);
  if (R == 0) return TG_ERR_UNSUPPORTED;
  const int grid = tg::grid_for(p->N, R);
  const int cap = std::max(1, R * p->max_deg);
  const tg::RefTab<T>& tab = tg::table<T>((tg_element)EL);
  tg_status st = tg::set_smem(ncomp == 1 ? (const void*)k_load_backward<EL, T, 1>
                                         : (const void*)k_load_backward<EL, T, 3>, smem);
  if (st != TG_OK) return st;
  if (ncomp == 1) k_load_backward<EL, T, 1><<<grid, R, smem, s>>>(a, tab, cap);
  else k_load_backward<EL, T, 3><<<grid, R, smem, s>>>(a, tab, cap);
  TG_CK_LAUNCH("k_load_backward");
  if (a.grad_f && a.layout == TG_CONSTANT) {
    FinalOut o{{nullptr, nullptr, nullptr, nullptr}, ncomp, a.accumulate};
    for (int k = 0; k < ncomp; ++k) o.out[k] = a.grad_f + k;
    k_backward_final<T><<<1, kFinal, 0, s>>>(a.partials, grid, o);
    TG_CK_LAUNCH("k_backward_final");
  }
  return TG_OK;
}

template <typename T>
tg_status load_backward(const tg_pattern* p, const void* coords, const void* f, tg_layout fl, int ncomp,
                        const void* gF, void* grad_f, void* grad_coords, int accumulate, cudaStream_t s) {
  LoadBwdArgs<T> a;
  a.inc_ptr = p->inc_ptr;
  a.inc_e = p->inc_e;
  a.cells = p->cells;
  a.coords = static_cast<const T*>(coords);
  a.f = static_cast<const T*>(f);
  a.layout = fl;
  a.gF = static_cast<const T*>(gF);
  a.grad_f = static_cast<T*>(grad_f);
  a.grad_coords = static_cast<T*>(grad_coords);
  a.accumulate = accumulate;
  a.partials = p->partials;
  a.N = p->N;
  a.status = p->status;
  switch (p->el) {
    case TG_P1_TRI: return launch_load_bwd<TG_P1_TRI, T>(p, a, ncomp, s);
    case TG_P2_TRI: return launch_load_bwd<TG_P2_TRI, T>(p, a, ncomp, s);
    default: return launch_load_bwd<TG_P1_TET, T>(p, a, ncomp, s);
  }
}

}  // namespace

extern "C" tg_status tg_assemble_backward(const tg_pattern* p, tg_dtype dtype, const void* coords, const void* kappa,
                                          tg_layout kappa_layout, double c, const void* grad_vals, const void* lam,
                                          const void* U, void* grad_kappa, void* grad_coords, void* grad_c,
                                          tg_stream stream) {
  if (!p || (dtype != TG_F32 && dtype != TG_F64)) return TG_ERR_INVALID_ARG;
  if (!tg::scalar_kind(p->el) || !kappa || (p->N > 0 && !coords)) return TG_ERR_INVALID_ARG;
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

extern "C" tg_status tg_assemble_load_backward(const tg_pattern* p, tg_dtype dtype, const void* coords, const void* f,
                                               tg_layout f_layout, int32_t ncomp, const void* grad_F, void* grad_f,
                                               void* grad_coords, int32_t accumulate, tg_stream stream) {
  if (!p || (dtype != TG_F32 && dtype != TG_F64) || !f || !grad_F || (p->N > 0 && !coords)) return TG_ERR_INVALID_ARG;
  if (p->el == TG_Q1_QUAD_VEC2) return TG_ERR_INVALID_ARG;
  if ((ncomp != 1 && ncomp != 3) || !(f_layout == TG_PER_NODE || f_layout == TG_PER_QP || f_layout == TG_CONSTANT))
    return TG_ERR_INVALID_ARG;
  const size_t es = dtype == TG_F32 ? 4 : 8;
  if (((uintptr_t)coords % (p->dim == 2 ? 2 * es : es)) != 0) return TG_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  return dtype == TG_F32 ? load_backward<float>(p, coords, f, f_layout, ncomp, grad_F, grad_f, grad_coords, accumulate, s)
                         : load_backward<double>(p, coords, f, f_layout, ncomp, grad_F, grad_f, grad_coords, accumulate,
                                                 s);
}

