// Boundary facets: Neumann and Robin terms routed into the element
// assembly's CSR values and load vector (the mixed-boundary-condition
// benchmark of the SM: a Map over boundary quadrature and a boundary
// routing into the same Sparse-Reduce).
//
// Routing, built once per facet set: the nodes that carry facets (fnode,
// ascending), each with its facet incidences (f, local vertex a) in
// increasing facet order (finc) and, per incidence, the 8-bit positions of
// the facet's vertex columns in the node's CSR row (fpos).
//
// Assembly: one thread per boundary node walks its incidences in facet
// order and adds each facet's row into the node's CSR row and load entry.
// A node's row is written by its thread only, so the additions are free of
// races and happen in a fixed order.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "tg_internal.cuh"

struct tg_facets {
  int device = 0;
  tg_element el = TG_P1_TRI;
  int nf = 2;  // vertices per facet
  int64_t F = 0, M = 0, N = 0;
  const int32_t* row_ptr = nullptr;       // the pattern's (borrowed)
  unsigned long long* status = nullptr;   // the pattern's device status (borrowed)
  int32_t* facets = nullptr;              // [F][nf]
  int32_t* fnode = nullptr;               // [M]
  int32_t* finc_ptr = nullptr;            // [M + 1]
  int32_t* finc = nullptr;                // [F * nf]: f * 4 + a
  uint32_t* fpos = nullptr;               // [F * nf]: 8-bit positions of the facet's vertices in the row
  unsigned long long* build_status = nullptr;
};

namespace {

constexpr int FT = 128;

// Reference-facet quadrature: weights w[q] (sum 1 on the edge, 1/2 on the
// face) and the facet's linear basis at the points, phi[q][a].
template <typename T>
struct FacetTab {
  T w[3];
  T phi[3][3];
};

// Edge: 2-point Gauss rule on [0, 1], t = 1/2 -+ sqrt(3)/6, weights 1/2.
// Face: the 3-point rule of the reference triangle, points (1/6, 1/6),
// (2/3, 1/6), (1/6, 2/3), weights 1/6; phi = (1 - x - y, x, y).
template <typename T>
FacetTab<T> facet_table(int nf) {
  FacetTab<T> t;
  std::memset(&t, 0, sizeof(t));
  if (nf == 2) {
    const double h = std::sqrt(3.0) / 6.0;
    const double ts[2] = {0.5 - h, 0.5 + h};
    for (int q = 0; q < 2; ++q) {
      t.w[q] = (T)0.5;
      t.phi[q][0] = (T)(1.0 - ts[q]);
      t.phi[q][1] = (T)ts[q];
    }
  } else {
    const double xs[3][2] = {{1.0 / 6, 1.0 / 6}, {2.0 / 3, 1.0 / 6}, {1.0 / 6, 2.0 / 3}};
    for (int q = 0; q < 3; ++q) {
      t.w[q] = (T)(1.0 / 6);
      t.phi[q][0] = (T)(1.0 - xs[q][0] - xs[q][1]);
      t.phi[q][1] = (T)xs[q][0];
      t.phi[q][2] = (T)xs[q][1];
    }
  }
  return t;
}

// Positions of every incidence's facet vertices in the owning row; an
// incidence whose vertex pair shares no element records TG_ERR_INVALID_ARG.
__global__ void __launch_bounds__(FT) k_facet_pos(const int32_t* __restrict__ facets, int nf,
                                                  const int32_t* __restrict__ fnode,
                                                  const int32_t* __restrict__ finc_ptr,
                                                  const int32_t* __restrict__ finc,
                                                  const int32_t* __restrict__ row_ptr,
                                                  const int32_t* __restrict__ col_idx, int64_t M,
                                                  uint32_t* __restrict__ fpos, unsigned long long* status) {
  const int64_t m = (int64_t)blockIdx.x * FT + threadIdx.x;
  if (m >= M) return;
  const int i = fnode[m];
  const int r0 = row_ptr[i], r1 = row_ptr[i + 1];
  for (int j = finc_ptr[m]; j < finc_ptr[m + 1]; ++j) {
    const int f = finc[j] >> 2;
    uint32_t w = 0;
    for (int b = 0; b < nf; ++b) {
      const int v = facets[(int64_t)f * nf + b];
      int lo = r0, hi = r1;
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (col_idx[mid] < v) lo = mid + 1;
        else hi = mid;
      }
      if (lo >= r1 || col_idx[lo] != v || lo - r0 > 255) {
        tg::record_error(status, TG_ERR_INVALID_ARG, f);
        w = 0;
        break;
      }
      w |= (uint32_t)(lo - r0) << (8 * b);
    }
    fpos[j] = w;
  }
}

template <typename T>
struct FacetArgs {
  const int32_t* __restrict__ facets;
  const int32_t* __restrict__ fnode;
  const int32_t* __restrict__ finc_ptr;
  const int32_t* __restrict__ finc;
  const uint32_t* __restrict__ fpos;
  const int32_t* __restrict__ row_ptr;
  const T* __restrict__ coords;
  const T* __restrict__ alpha;
  int alpha_layout;
  const T* __restrict__ g;
  int g_layout;
  T* __restrict__ vals;
  T* __restrict__ F;
  int64_t M;
  unsigned long long* status;
};

// |J_f|: the edge length (2D) or twice the face area (3D).
template <int NF, typename T>
__device__ __forceinline__ T facet_measure(const T* __restrict__ X, const int (&v)[NF]) {
  if constexpr (NF == 2) {
    const T dx = X[2ll * v[1]] - X[2ll * v[0]], dy = X[2ll * v[1] + 1] - X[2ll * v[0] + 1];
    return sqrt(dx * dx + dy * dy);
  } else {
    T e1[3], e2[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      e1[r] = X[3ll * v[1] + r] - X[3ll * v[0] + r];
      e2[r] = X[3ll * v[2] + r] - X[3ll * v[0] + r];
    }
    const T cx = e1[1] * e2[2] - e1[2] * e2[1];
    const T cy = e1[2] * e2[0] - e1[0] * e2[2];
    const T cz = e1[0] * e2[1] - e1[1] * e2[0];
    return sqrt(cx * cx + cy * cy + cz * cz);
  }
}

template <typename T>
__device__ __forceinline__ T facet_tiny() {
  return sizeof(T) == 8 ? T(1e-300) : T(1e-37);
}

// Values of a facet coefficient at the NQ points: one per facet, per point,
// a constant, or (PER_NODE) the facet interpolant of nodal values.
template <int NF, typename T>
__device__ __forceinline__ void facet_coef(const T* __restrict__ c, int layout, int64_t f, const int (&v)[NF],
                                           const FacetTab<T>& tab, T (&cq)[NF]) {
  constexpr int NQ = NF;
  if (layout == TG_PER_QP) {
#pragma unroll
    for (int q = 0; q < NQ; ++q) cq[q] = __ldg(c + f * NQ + q);
  } else if (layout == TG_PER_NODE) {
    T cv[NF];
#pragma unroll
    for (int b = 0; b < NF; ++b) cv[b] = __ldg(c + v[b]);
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      T s = T(0);
#pragma unroll
      for (int b = 0; b < NF; ++b) s += tab.phi[q][b] * cv[b];
      cq[q] = s;
    }
  } else {
    const T k = layout == TG_PER_ELEMENT ? __ldg(c + f) : __ldg(c);
#pragma unroll
    for (int q = 0; q < NQ; ++q) cq[q] = k;
  }
}

template <int NF, typename T>
__global__ void __launch_bounds__(FT) k_facets(const FacetArgs<T> a, const __grid_constant__ FacetTab<T> tab) {
  constexpr int NQ = NF;  // 2 points on an edge, 3 on a face
  const int64_t m = (int64_t)blockIdx.x * FT + threadIdx.x;
  if (m >= a.M) return;
  const int i = a.fnode[m];
  T* row = a.vals ? a.vals + a.row_ptr[i] : nullptr;
  for (int j = a.finc_ptr[m]; j < a.finc_ptr[m + 1]; ++j) {
    const int f = a.finc[j] >> 2, la = a.finc[j] & 3;
    int v[NF];
#pragma unroll
    for (int b = 0; b < NF; ++b) v[b] = __ldg(a.facets + (int64_t)f * NF + b);
    const T J = facet_measure<NF, T>(a.coords, v);
    if (!(J > facet_tiny<T>())) {
      tg::record_error(a.status, TG_ERR_DEGENERATE_ELEMENT, f);
      continue;
    }
    T pa[NQ];  // phi_a at the points
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      T s = tab.phi[q][0];
#pragma unroll
      for (int b = 1; b < NF; ++b)
        if (la == b) s = tab.phi[q][b];
      pa[q] = s;
    }
    if (row && a.alpha) {
      T al[NQ];
      facet_coef<NF, T>(a.alpha, a.alpha_layout, f, v, tab, al);
      const uint32_t pw = a.fpos[j];
#pragma unroll
      for (int b = 0; b < NF; ++b) {
        T s = T(0);
#pragma unroll
        for (int q = 0; q < NQ; ++q) s += tab.w[q] * al[q] * pa[q] * tab.phi[q][b];
        T* slot = row + ((pw >> (8 * b)) & 255u);
        *slot = *slot + J * s;
      }
    }
    if (a.F && a.g) {
      T gq[NQ];
      facet_coef<NF, T>(a.g, a.g_layout, f, v, tab, gq);
      T s = T(0);
#pragma unroll
      for (int q = 0; q < NQ; ++q) s += tab.w[q] * gq[q] * pa[q];
      a.F[i] = a.F[i] + J * s;
    }
  }
}

template <typename T>
tg_status assemble(const tg_facets* fc, const void* coords, const void* alpha, tg_layout al, const void* g,
                   tg_layout gl, void* vals, void* F, cudaStream_t s) {
  FacetArgs<T> a;
  a.facets = fc->facets;
  a.fnode = fc->fnode;
  a.finc_ptr = fc->finc_ptr;
  a.finc = fc->finc;
  a.fpos = fc->fpos;
  a.row_ptr = fc->row_ptr;
  a.coords = static_cast<const T*>(coords);
  a.alpha = static_cast<const T*>(alpha);
  a.alpha_layout = al;
  a.g = static_cast<const T*>(g);
  a.g_layout = gl;
  a.vals = static_cast<T*>(vals);
  a.F = static_cast<T*>(F);
  a.M = fc->M;
  a.status = fc->status;
  const FacetTab<T> tab = facet_table<T>(fc->nf);
  const unsigned grid = (unsigned)((fc->M + FT - 1) / FT);
  if (fc->nf == 2) k_facets<2, T><<<grid, FT, 0, s>>>(a, tab);
  else k_facets<3, T><<<grid, FT, 0, s>>>(a, tab);
  TG_CK_LAUNCH("k_facets");
  return TG_OK;
}

void free_facets(tg_facets* fc) {
  void* bufs[] = {fc->facets, fc->fnode, fc->finc_ptr, fc->finc, fc->fpos, fc->build_status};
  for (void* b : bufs)
    if (b) cudaFree(b);
  delete fc;
}

}  // namespace

extern "C" {

tg_status tg_build_facets(const tg_pattern* p, const int32_t* facets, int64_t n_facets, tg_stream stream,
                          tg_facets** out) {
  if (!out) return TG_ERR_INVALID_ARG;
  *out = nullptr;
  if (!p || n_facets < 0 || (n_facets > 0 && !facets)) return TG_ERR_INVALID_ARG;
  if (p->el != TG_P1_TRI && p->el != TG_P1_TET) {
    tg::set_error("tg_build_facets: facets are built for P1 triangles and tetrahedra");
    return TG_ERR_UNSUPPORTED;
  }
  if (n_facets > (int64_t)INT32_MAX / 4) return TG_ERR_INDEX_OVERFLOW;
  cudaStream_t s = (cudaStream_t)stream;
  tg_facets* fc = new tg_facets;
  fc->device = p->device;
  fc->el = p->el;
  fc->nf = p->el == TG_P1_TRI ? 2 : 3;
  fc->F = n_facets;
  fc->N = p->N;
  fc->row_ptr = p->row_ptr;
  fc->status = p->status;
  const int nf = fc->nf;
  struct Guard {
    tg_facets* fc;
    bool ok = false;
    ~Guard() {
      if (!ok) free_facets(fc);
    }
  } guard{fc};
  // host side: validation and the per-node incidence lists (facet order)
  std::vector<int32_t> h((size_t)n_facets * nf);
  if (n_facets > 0) {
    TG_CK(cudaMemcpyAsync(h.data(), facets, h.size() * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    TG_CK(cudaStreamSynchronize(s));
  }
  std::vector<int32_t> deg(p->N, 0);
  for (int64_t f = 0; f < n_facets; ++f) {
    for (int b = 0; b < nf; ++b) {
      const int32_t v = h[f * nf + b];
      if (v < 0 || v >= p->N) {
        tg::set_error("tg_build_facets: facet " + std::to_string(f) + " has a node outside [0, n_nodes)");
        return TG_ERR_INDEX_RANGE;
      }
      for (int c = 0; c < b; ++c)
        if (h[f * nf + c] == v) {
          tg::set_error("tg_build_facets: facet " + std::to_string(f) + " repeats a vertex");
          return TG_ERR_DEGENERATE_ELEMENT;
        }
    }
    for (int b = 0; b < nf; ++b) ++deg[h[f * nf + b]];
  }
  std::vector<int32_t> fnode, fptr(1, 0), slot(p->N, -1);
  for (int64_t i = 0; i < p->N; ++i)
    if (deg[i] > 0) {
      slot[i] = (int32_t)fnode.size();
      fnode.push_back((int32_t)i);
      fptr.push_back(fptr.back() + deg[i]);
    }
  fc->M = (int64_t)fnode.size();
  std::vector<int32_t> finc((size_t)n_facets * nf), cur(fptr.begin(), fptr.end() - 1);
  for (int64_t f = 0; f < n_facets; ++f)
    for (int b = 0; b < nf; ++b) finc[cur[slot[h[f * nf + b]]]++] = (int32_t)(f * 4 + b);
  // device copies and the row positions
  const size_t nI = finc.size();
  TG_CK(cudaMalloc(&fc->build_status, 2 * sizeof(unsigned long long)));
  const unsigned long long init[2] = {0ull, ~0ull};
  TG_CK(cudaMemcpyAsync(fc->build_status, init, sizeof(init), cudaMemcpyHostToDevice, s));
  TG_CK(cudaMalloc(&fc->facets, std::max<size_t>(h.size(), 1) * sizeof(int32_t)));
  TG_CK(cudaMalloc(&fc->fnode, std::max<size_t>(fnode.size(), 1) * sizeof(int32_t)));
  TG_CK(cudaMalloc(&fc->finc_ptr, fptr.size() * sizeof(int32_t)));
  TG_CK(cudaMalloc(&fc->finc, std::max<size_t>(nI, 1) * sizeof(int32_t)));
  TG_CK(cudaMalloc(&fc->fpos, std::max<size_t>(nI, 1) * sizeof(uint32_t)));
  if (!h.empty()) TG_CK(cudaMemcpyAsync(fc->facets, h.data(), h.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s));
  if (!fnode.empty())
    TG_CK(cudaMemcpyAsync(fc->fnode, fnode.data(), fnode.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s));
  TG_CK(cudaMemcpyAsync(fc->finc_ptr, fptr.data(), fptr.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s));
  if (nI) TG_CK(cudaMemcpyAsync(fc->finc, finc.data(), nI * sizeof(int32_t), cudaMemcpyHostToDevice, s));
  if (fc->M > 0) {
    k_facet_pos<<<(unsigned)((fc->M + FT - 1) / FT), FT, 0, s>>>(fc->facets, nf, fc->fnode, fc->finc_ptr, fc->finc,
                                                                 p->row_ptr, p->col_idx, fc->M, fc->fpos,
                                                                 fc->build_status);
    TG_CK_LAUNCH("k_facet_pos");
  }
  unsigned long long st[2];
  TG_CK(cudaMemcpyAsync(st, fc->build_status, sizeof(st), cudaMemcpyDeviceToHost, s));
  TG_CK(cudaStreamSynchronize(s));
  if (st[0] != TG_OK) {
    tg::set_error("tg_build_facets: facet " + std::to_string((long long)st[1]) +
                  " is not a facet of the mesh (a vertex pair shares no element)");
    return (tg_status)st[0];
  }
  guard.ok = true;
  *out = fc;
  return TG_OK;
}

tg_status tg_assemble_facets(const tg_facets* fc, tg_dtype dtype, const void* coords, const void* alpha,
                             tg_layout alpha_layout, const void* g, tg_layout g_layout, void* vals_inout,
                             void* F_inout, tg_stream stream) {
  if (!fc || (dtype != TG_F32 && dtype != TG_F64)) return TG_ERR_INVALID_ARG;
  if (alpha && !(alpha_layout == TG_PER_ELEMENT || alpha_layout == TG_PER_QP || alpha_layout == TG_CONSTANT))
    return TG_ERR_INVALID_ARG;
  if (g && !(g_layout == TG_PER_NODE || g_layout == TG_PER_QP || g_layout == TG_CONSTANT)) return TG_ERR_INVALID_ARG;
  if (alpha && !vals_inout) return TG_ERR_INVALID_ARG;
  if (g && !F_inout) return TG_ERR_INVALID_ARG;
  if (fc->M == 0 || (!alpha && !g)) return TG_OK;
  if (!coords) return TG_ERR_INVALID_ARG;
  const size_t es = dtype == TG_F32 ? 4 : 8;
  if (fc->nf == 2 && ((uintptr_t)coords % (2 * es)) != 0) {
    tg::set_error("coords must be aligned to 2 * sizeof(dtype) for 2D meshes");
    return TG_ERR_INVALID_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  return dtype == TG_F32
             ? assemble<float>(fc, coords, alpha, alpha_layout, g, g_layout, alpha ? vals_inout : nullptr,
                               g ? F_inout : nullptr, s)
             : assemble<double>(fc, coords, alpha, alpha_layout, g, g_layout, alpha ? vals_inout : nullptr,
                                g ? F_inout : nullptr, s);
}

tg_status tg_facets_shape(const tg_facets* fc, int64_t* n_facets, int64_t* n_boundary_nodes) {
  if (!fc) return TG_ERR_INVALID_ARG;
  if (n_facets) *n_facets = fc->F;
  if (n_boundary_nodes) *n_boundary_nodes = fc->M;
  return TG_OK;
}

void tg_facets_destroy(tg_facets* fc) {
  if (!fc) return;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(fc->device);
  free_facets(fc);
  cudaSetDevice(prev);
}

}  // extern "C"
