// Plane-stress bilinear quadrilaterals with the SIMP material law (the SM's
// topology-optimisation benchmark):
//   E(rho) = E_min + rho^p (E_max - E_min),   K(rho) = sum_e E(rho_e) K0_e,
//   dC/drho_e = -p rho_e^(p-1) (E_max - E_min) u_e^T K0_e u_e.
// K0_e (unit Young's modulus) integrates, over the 2 x 2 Gauss points of the
// non-affine map (J, det J and the physical gradients g_a per point),
//   |det J_q| w_q (l g_ai g_bj + m g_aj g_bi + m delta_ij g_a . g_b)
// for DoFs (a, i), (b, j), with the plane-stress constants
// l = nu / (1 - nu^2), m = 1 / (2 (1 + nu)).  u^T K0 u is the same sum of
// the strain energy density l (tr eps)^2 + 2 m eps : eps.
//
// Assembly: one thread per node owns its two DoF rows and adds, for each
// incident element in increasing element order, the element's two rows
// scaled by E(rho_e): deterministic, no atomics.  Sensitivity: one thread
// per element.
#include <cmath>

#include "gather.cuh"

namespace {

// Small CTAs: the benchmark's meshes are small (a few thousand nodes) and
// the FP64 element arithmetic is bound by each SM's FP64 pipe, so the work
// is spread over as many SMs as possible.
constexpr int ST = 32;

template <typename T>
struct SimpArgs {
  const int32_t* __restrict__ cells;
  const int32_t* __restrict__ inc_ptr;
  const int32_t* __restrict__ inc_e;
  const uint32_t* __restrict__ inc_pos;
  const int32_t* __restrict__ row_ptr_dof;
  const T* __restrict__ coords;
  const T* __restrict__ rho;
  T e_min, e_max, penal, lam, mu;
  const T* __restrict__ u;
  T* __restrict__ out;
  int64_t n;  // nodes (assembly) or elements (sensitivity)
  unsigned long long* status;
};

template <typename T>
__device__ __forceinline__ T simp_tiny() {
  return sizeof(T) == 8 ? T(1e-300) : T(1e-30);
}

// Physical gradients g[b][k] of the four corners and w_q |det J_q| at Gauss
// point q; false for a non-positive-measure point.
template <typename T>
__device__ __forceinline__ bool quad_point(const T (&x)[4][2], const tg::RefTab<T>& tab, int q, T (&g)[4][2], T& wd) {
  T J00 = T(0), J01 = T(0), J10 = T(0), J11 = T(0);  // J[i][k] = d x_i / d ref_k
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    J00 = fma(x[b][0], tab.gh[q][b][0], J00);
    J01 = fma(x[b][0], tab.gh[q][b][1], J01);
    J10 = fma(x[b][1], tab.gh[q][b][0], J10);
    J11 = fma(x[b][1], tab.gh[q][b][1], J11);
  }
  const T det = J00 * J11 - J01 * J10;
  const T ad = det < T(0) ? -det : det;
  if (!(ad > simp_tiny<T>())) return false;
  const T inv = tg::recip(det);
  // g = ghat J^{-1}:  J^{-1} = [[J11, -J01], [-J10, J00]] / det
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    const T s = tab.gh[q][b][0], t = tab.gh[q][b][1];
    g[b][0] = (s * J11 - t * J10) * inv;
    g[b][1] = (t * J00 - s * J01) * inv;
  }
  wd = tab.w[q] * ad;
  return true;
}

template <typename T>
__device__ __forceinline__ void load_quad(const SimpArgs<T>& a, int64_t e, int (&v)[4], T (&x)[4][2]) {
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    v[b] = __ldg(a.cells + e * 4 + b);
    const auto p = tg::ldg2(a.coords, v[b]);
    x[b][0] = p.x;
    x[b][1] = p.y;
  }
}

template <typename T>
__device__ __forceinline__ T simp_modulus(const SimpArgs<T>& a, int64_t e) {
  const T r = __ldg(a.rho + e);
  return a.e_min + pow(r, a.penal) * (a.e_max - a.e_min);
}

template <typename T>
__global__ void __launch_bounds__(ST) k_simp_assemble(const SimpArgs<T> a, const __grid_constant__ tg::RefTab<T> tab) {
  const int64_t i = (int64_t)blockIdx.x * ST + threadIdx.x;
  if (i >= a.n) return;
  T* row0 = a.out + a.row_ptr_dof[2 * i];
  T* row1 = a.out + a.row_ptr_dof[2 * i + 1];
  const int len2 = a.row_ptr_dof[2 * i + 1] - a.row_ptr_dof[2 * i];  // 2 x node-row length
  for (int k = 0; k < len2; ++k) {
    row0[k] = T(0);
    row1[k] = T(0);
  }
  for (int j = a.inc_ptr[i]; j < a.inc_ptr[i + 1]; ++j) {
    const int64_t e = a.inc_e[j] >> 3;
    const int la = a.inc_e[j] & 7;
    const uint32_t pw = a.inc_pos[j];
    int v[4];
    T x[4][2];
    load_quad(a, e, v, x);
    T k0[2][4][2];  // rows (la, c), columns (b, jj)
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
      for (int b = 0; b < 4; ++b) k0[c][b][0] = k0[c][b][1] = T(0);
    bool ok = true;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      T g[4][2], wd;
      if (!quad_point(x, tab, q, g, wd)) {
        ok = false;
        break;
      }
      T ga[2];
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        T s = g[0][r];
#pragma unroll
        for (int b = 1; b < 4; ++b)
          if (la == b) s = g[b][r];
        ga[r] = s;
      }
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const T dot = ga[0] * g[b][0] + ga[1] * g[b][1];
#pragma unroll
        for (int c = 0; c < 2; ++c)
#pragma unroll
          for (int jj = 0; jj < 2; ++jj)
            k0[c][b][jj] += wd * (a.lam * ga[c] * g[b][jj] + a.mu * ga[jj] * g[b][c] + (c == jj ? a.mu * dot : T(0)));
      }
    }
    if (!ok) {
      tg::record_error(a.status, TG_ERR_DEGENERATE_ELEMENT, e);
      continue;
    }
    const T E = simp_modulus(a, e);
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int pos = (int)((pw >> (8 * b)) & 255u);
#pragma unroll
      for (int jj = 0; jj < 2; ++jj) {
        row0[2 * pos + jj] += E * k0[0][b][jj];
        row1[2 * pos + jj] += E * k0[1][b][jj];
      }
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(ST) k_simp_sensitivity(const SimpArgs<T> a, const __grid_constant__ tg::RefTab<T> tab) {
  const int64_t e = (int64_t)blockIdx.x * ST + threadIdx.x;
  if (e >= a.n) return;
  int v[4];
  T x[4][2];
  load_quad(a, e, v, x);
  T ue[4][2];
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    ue[b][0] = __ldg(a.u + 2ll * v[b]);
    ue[b][1] = __ldg(a.u + 2ll * v[b] + 1);
  }
  T energy = T(0);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    T g[4][2], wd;
    if (!quad_point(x, tab, q, g, wd)) {
      tg::record_error(a.status, TG_ERR_DEGENERATE_ELEMENT, e);
      a.out[e] = T(0);
      return;
    }
    T du[2][2] = {{T(0), T(0)}, {T(0), T(0)}};  // du[i][k] = d u_i / d x_k
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
      for (int ii = 0; ii < 2; ++ii)
#pragma unroll
        for (int k = 0; k < 2; ++k) du[ii][k] = fma(ue[b][ii], g[b][k], du[ii][k]);
    const T tr = du[0][0] + du[1][1];
    const T e01 = T(0.5) * (du[0][1] + du[1][0]);
    const T epe = du[0][0] * du[0][0] + du[1][1] * du[1][1] + T(2) * e01 * e01;
    energy += wd * (a.lam * tr * tr + T(2) * a.mu * epe);
  }
  const T r = __ldg(a.rho + e);
  a.out[e] = -a.penal * pow(r, a.penal - T(1)) * (a.e_max - a.e_min) * energy;
}

template <typename T>
SimpArgs<T> simp_args(const tg_pattern* p, const void* coords, const void* rho, double e_min, double e_max,
                      double penal, double nu) {
  SimpArgs<T> a;
  a.cells = p->cells;
  a.inc_ptr = p->inc_ptr;
  a.inc_e = p->inc_e;
  a.inc_pos = p->inc_pos;
  a.row_ptr_dof = p->row_ptr_dof;
  a.coords = static_cast<const T*>(coords);
  a.rho = static_cast<const T*>(rho);
  a.e_min = (T)e_min;
  a.e_max = (T)e_max;
  a.penal = (T)penal;
  a.lam = (T)(nu / (1.0 - nu * nu));
  a.mu = (T)(1.0 / (2.0 * (1.0 + nu)));
  a.u = nullptr;
  a.out = nullptr;
  a.n = 0;
  a.status = p->status;
  return a;
}

tg_status check(const tg_pattern* p, tg_dtype dtype, const void* coords, const void* rho, double nu) {
  if (!p || (dtype != TG_F32 && dtype != TG_F64) || p->el != TG_Q1_QUAD_VEC2) return TG_ERR_INVALID_ARG;
  if (p->N > 0 && (!coords || !rho)) return TG_ERR_INVALID_ARG;
  if (!(nu > -1.0 && nu < 0.5)) return TG_ERR_INVALID_ARG;
  const size_t es = dtype == TG_F32 ? 4 : 8;
  if (((uintptr_t)coords % (2 * es)) != 0) return TG_ERR_INVALID_ARG;
  return TG_OK;
}

}  // namespace

extern "C" {

tg_status tg_assemble_simp(const tg_pattern* p, tg_dtype dtype, const void* coords, const void* rho, double e_min,
                           double e_max, double penal, double nu, void* vals_out, tg_stream stream) {
  tg_status st = check(p, dtype, coords, rho, nu);
  if (st != TG_OK) return st;
  if (p->nnz > 0 && !vals_out) return TG_ERR_INVALID_ARG;
  if (p->N == 0) return TG_OK;
  cudaStream_t s = (cudaStream_t)stream;
  const unsigned grid = (unsigned)tg::grid_for(p->N, ST);
  if (dtype == TG_F32) {
    SimpArgs<float> a = simp_args<float>(p, coords, rho, e_min, e_max, penal, nu);
    a.out = static_cast<float*>(vals_out);
    a.n = p->N;
    k_simp_assemble<float><<<grid, ST, 0, s>>>(a, tg::table<float>(TG_Q1_QUAD_VEC2));
  } else {
    SimpArgs<double> a = simp_args<double>(p, coords, rho, e_min, e_max, penal, nu);
    a.out = static_cast<double*>(vals_out);
    a.n = p->N;
    k_simp_assemble<double><<<grid, ST, 0, s>>>(a, tg::table<double>(TG_Q1_QUAD_VEC2));
  }
  TG_CK_LAUNCH("k_simp_assemble");
  return TG_OK;
}

tg_status tg_simp_sensitivity(const tg_pattern* p, tg_dtype dtype, const void* coords, const void* rho, double e_min,
                              double e_max, double penal, double nu, const void* u, void* dc_out, tg_stream stream) {
  tg_status st = check(p, dtype, coords, rho, nu);
  if (st != TG_OK) return st;
  if (p->E > 0 && (!u || !dc_out)) return TG_ERR_INVALID_ARG;
  if (p->E == 0) return TG_OK;
  cudaStream_t s = (cudaStream_t)stream;
  const unsigned grid = (unsigned)tg::grid_for(p->E, ST);
  if (dtype == TG_F32) {
    SimpArgs<float> a = simp_args<float>(p, coords, rho, e_min, e_max, penal, nu);
    a.u = static_cast<const float*>(u);
    a.out = static_cast<float*>(dc_out);
    a.n = p->E;
    k_simp_sensitivity<float><<<grid, ST, 0, s>>>(a, tg::table<float>(TG_Q1_QUAD_VEC2));
  } else {
    SimpArgs<double> a = simp_args<double>(p, coords, rho, e_min, e_max, penal, nu);
    a.u = static_cast<const double*>(u);
    a.out = static_cast<double*>(dc_out);
    a.n = p->E;
    k_simp_sensitivity<double><<<grid, ST, 0, s>>>(a, tg::table<double>(TG_Q1_QUAD_VEC2));
  }
  TG_CK_LAUNCH("k_simp_sensitivity");
  return TG_OK;
}

}  // extern "C"
