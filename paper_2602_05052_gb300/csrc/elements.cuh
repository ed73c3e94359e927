// Per-element geometry and local-matrix rows (Stage I Map, Algorithm 1) for
// the kernels of libtg.so.  Affine simplices: J, det J and the push-forward
// are constant over the element (SM A.2), so geometry is computed once per
// (element, visit) from the vertex coordinates.
//
// Notation: for P1, n_b = det(J) * grad(phi_b) ("det-scaled gradients"):
// rows of det(J) J^{-1} for b >= 1 (2D: (e2y, -e2x), (-e1y, e1x); 3D: the
// cross products e2 x e3, e3 x e1, e1 x e2 of the edge vectors), and
// n_0 = -(sum of the others).  Then |det J| grad(phi_a).grad(phi_b) =
// n_a.n_b / |det J|, so one reciprocal per element suffices.
#pragma once

#include "tg_internal.cuh"

namespace tg {

template <typename T>
__device__ __forceinline__ typename Vec2<T>::type ldg2(const T* __restrict__ coords, int v) {
  using V2 = typename Vec2<T>::type;
  return __ldg(reinterpret_cast<const V2*>(coords) + v);
}

template <typename T, int N>
__device__ __forceinline__ T sel(int k, const T (&a)[N]) {
  T r = a[0];
#pragma unroll
  for (int m = 1; m < N; ++m) r = (k == m) ? a[m] : r;
  return r;
}

// Geometry of one element.  dim 2: n[b][0..1]; dim 3: n[b][0..2].
template <int DIM, typename T>
struct Geom {
  T n[DIM + 1][DIM];
  T det;
};

template <typename T>
__device__ __forceinline__ void tri_geom_x(const T (&x0)[2], const T (&x1)[2], const T (&x2)[2], Geom<2, T>& g) {
  const T e1x = x1[0] - x0[0], e1y = x1[1] - x0[1];
  const T e2x = x2[0] - x0[0], e2y = x2[1] - x0[1];
  g.n[1][0] = e2y;
  g.n[1][1] = -e2x;
  g.n[2][0] = -e1y;
  g.n[2][1] = e1x;
  g.n[0][0] = -(g.n[1][0] + g.n[2][0]);
  g.n[0][1] = -(g.n[1][1] + g.n[2][1]);
  g.det = e1x * e2y - e1y * e2x;
}

template <typename T>
__device__ __forceinline__ void tri_geom(const T* __restrict__ coords, int v0, int v1, int v2, Geom<2, T>& g) {
  const auto p0 = ldg2(coords, v0);
  const auto p1 = ldg2(coords, v1);
  const auto p2 = ldg2(coords, v2);
  const T x0[2] = {p0.x, p0.y}, x1[2] = {p1.x, p1.y}, x2[2] = {p2.x, p2.y};
  tri_geom_x(x0, x1, x2, g);
}

template <typename T>
__device__ __forceinline__ void cross3(const T (&a)[3], const T (&b)[3], T (&c)[3]) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}

template <typename T>
__device__ __forceinline__ void tet_geom_x(const T (&x0)[3], const T (&x1)[3], const T (&x2)[3], const T (&x3)[3],
                                           Geom<3, T>& g) {
  T e[3][3];
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    e[0][r] = x1[r] - x0[r];
    e[1][r] = x2[r] - x0[r];
    e[2][r] = x3[r] - x0[r];
  }
  cross3(e[1], e[2], g.n[1]);
  cross3(e[2], e[0], g.n[2]);
  cross3(e[0], e[1], g.n[3]);
#pragma unroll
  for (int r = 0; r < 3; ++r) g.n[0][r] = -(g.n[1][r] + g.n[2][r] + g.n[3][r]);
  g.det = e[0][0] * g.n[1][0] + e[0][1] * g.n[1][1] + e[0][2] * g.n[1][2];
}

template <typename T>
__device__ __forceinline__ void tet_geom(const T* __restrict__ coords, int v0, int v1, int v2, int v3,
                                         Geom<3, T>& g) {
  T x[4][3];
  const int v[4] = {v0, v1, v2, v3};
#pragma unroll
  for (int k = 0; k < 4; ++k)
#pragma unroll
    for (int r = 0; r < 3; ++r) x[k][r] = __ldg(coords + 3ll * v[k] + r);
  tet_geom_x(x[0], x[1], x[2], x[3], g);
}

// Determinant only (load vector).
template <typename T>
__device__ __forceinline__ T tri_det(const T* __restrict__ coords, int v0, int v1, int v2) {
  const auto x0 = ldg2(coords, v0);
  const auto x1 = ldg2(coords, v1);
  const auto x2 = ldg2(coords, v2);
  return (x1.x - x0.x) * (x2.y - x0.y) - (x1.y - x0.y) * (x2.x - x0.x);
}

template <typename T>
__device__ __forceinline__ T tet_det(const T* __restrict__ coords, int v0, int v1, int v2, int v3) {
  Geom<3, T> g;
  tet_geom(coords, v0, v1, v2, v3, g);
  return g.det;
}

// Index of (a, b), a <= b, in a packed upper triangle of NV rows.
__host__ __device__ constexpr int sym_idx(int NV, int a, int b) { return a * NV - a * (a - 1) / 2 + (b - a); }

// n_a . n_b: a product, then fused multiply-adds.
template <int DIM, typename T>
__device__ __forceinline__ T dot_n(const T (&na)[DIM], const T (&nb)[DIM]) {
  T x = na[0] * nb[0];
#pragma unroll
  for (int r = 1; r < DIM; ++r) x = fma(na[r], nb[r], x);
  return x;
}

// The dot products d_ab = n_a . n_b of a P1 element's det-scaled gradients
// in FP64, packed upper triangle (sym_idx).  The FP64 pipe bounds FP64
// assembly, so only the DIM (DIM + 1) / 2 products among n_1 .. n_DIM are
// formed; n_0 = -(n_1 + ... + n_DIM) gives the rest:
//   d_0b = -(d_1b + ... + d_DIMb) (b >= 1),  d_00 = -(d_01 + ... + d_0DIM),
// each summed in increasing index.  (FP32 forms every product directly:
// fewer live registers, and the FP32 pipe has room.)
template <int DIM, typename T>
__device__ __forceinline__ void p1_dots(const Geom<DIM, T>& g, T (&d)[(DIM + 1) * (DIM + 2) / 2]) {
  constexpr int NV = DIM + 1;
#pragma unroll
  for (int a = 1; a < NV; ++a)
#pragma unroll
    for (int b = a; b < NV; ++b) d[sym_idx(NV, a, b)] = dot_n<DIM, T>(g.n[a], g.n[b]);
#pragma unroll
  for (int b = 1; b < NV; ++b) {
    T x = d[sym_idx(NV, 1, b)];
#pragma unroll
    for (int c = 2; c < NV; ++c) x += d[c <= b ? sym_idx(NV, c, b) : sym_idx(NV, b, c)];
    d[sym_idx(NV, 0, b)] = -x;
  }
  T x = d[sym_idx(NV, 0, 1)];
#pragma unroll
  for (int b = 2; b < NV; ++b) x += d[sym_idx(NV, 0, b)];
  d[0] = -x;
}

// One entry of the P1 matrix from its dot product:
//   K_ab = s d_ab + mc M_ab,  s = sum_q w_q kappa_q / |det J|,  mc = c |det J|,
// one multiply and one fused multiply-add in a fixed order (K_ab == K_ba).
template <typename T>
__device__ __forceinline__ T p1_entry(T dab, T s, T mc, T Mab) {
  return fma(s, dab, mc * Mab);
}

// Row la of the scalar local matrix of a P1 element (triangle or tet),
// entry for entry the values of p1_elem_sym.  M: the reference mass table;
// FP64 uses its two values M[0][0] (diagonal) and M[0][1] (off the
// diagonal), each scaled by mc once, as the P1 mass matrix has no others.
template <int DIM, typename T>
__device__ __forceinline__ void p1_row(const Geom<DIM, T>& g, int la, T s, T mc, const T (&M)[6][6],
                                       T (&Krow)[DIM + 1]) {
  constexpr int NV = DIM + 1;
  if constexpr (sizeof(T) == 8) {
    T d[NV * (NV + 1) / 2];
    p1_dots<DIM, T>(g, d);
    const T md = mc * M[0][0], mo = mc * M[0][1];
#pragma unroll
    for (int b = 0; b < NV; ++b) {
      T col[NV];
#pragma unroll
      for (int a = 0; a < NV; ++a) col[a] = d[a <= b ? sym_idx(NV, a, b) : sym_idx(NV, b, a)];
      Krow[b] = fma(s, sel(la, col), la == b ? md : mo);
    }
  } else {
    const T (&Mla)[6] = M[la];
    T na[DIM];
#pragma unroll
    for (int r = 0; r < DIM; ++r) {
      T col[NV];
#pragma unroll
      for (int b = 0; b < NV; ++b) col[b] = g.n[b][r];
      na[r] = sel(la, col);
    }
#pragma unroll
    for (int b = 0; b < NV; ++b) Krow[b] = p1_entry<T>(dot_n<DIM, T>(na, g.n[b]), s, mc, Mla[b]);
  }
}
// Row la of the P2 triangle matrix with kappa at the 6 points:
//   K[la][b] = sum_q (w_q kappa_q / |det|) gh_q,la^T C gh_q,b + c |det| M[la][b]
// with C = det^2 J^{-1} J^{-T} = [[n1.n1, n1.n2], [n1.n2, n2.n2]].
// ts serves the reads indexed by the runtime la (a shared-memory copy), tc
// the ones with compile-time indices (the kernel's constant parameter).
template <typename T>
__device__ __forceinline__ void p2_row(const Geom<2, T>& g, int la, const T (&kq)[6], T inv, T mc,
                                       const RefTab<T>& ts, const RefTab<T>& tc, T (&Krow)[6]) {
  const T c00 = g.n[1][0] * g.n[1][0] + g.n[1][1] * g.n[1][1];
  const T c01 = g.n[1][0] * g.n[2][0] + g.n[1][1] * g.n[2][1];
  const T c11 = g.n[2][0] * g.n[2][0] + g.n[2][1] * g.n[2][1];
#pragma unroll
  for (int b = 0; b < 6; ++b) Krow[b] = T(0);
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    const T ga0 = ts.gh[q][la][0], ga1 = ts.gh[q][la][1];
    const T wk = (tc.w[q] * kq[q]) * inv;
    const T w00 = wk * c00, w01 = wk * c01, w11 = wk * c11;
    const T hx = fma(w00, ga0, w01 * ga1);
    const T hy = fma(w01, ga0, w11 * ga1);
#pragma unroll
    for (int b = 0; b < 6; ++b) Krow[b] = fma(hx, tc.gh[q][b][0], fma(hy, tc.gh[q][b][1], Krow[b]));
  }
#pragma unroll
  for (int b = 0; b < 6; ++b) Krow[b] = fma(mc, ts.M[la][b], Krow[b]);
}

__device__ __forceinline__ int pos_of(uint32_t w0, uint32_t w1, int b) {
  return (int)(((b < 4 ? w0 : w1) >> (8 * (b & 3))) & 0xffu);
}

}  // namespace tg
