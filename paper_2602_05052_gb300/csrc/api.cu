// Status handling, quadrature tables and pattern accessors of libtg.so.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>

#include "tg_internal.cuh"

namespace tg {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }

tg_status cuda_fail(cudaError_t err, const char* what, const char* file, int line) {
  char buf[512];
  std::snprintf(buf, sizeof(buf), "%s failed: %s (%s:%d)", what, cudaGetErrorString(err), file, line);
  g_last_error = buf;
  if (err == cudaErrorMemoryAllocation) return TG_ERR_OUT_OF_MEMORY;
  return TG_ERR_CUDA;
}

int sm_count() {
  int dev = 0, n = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  return n > 0 ? n : 1;
}

// Quadrature rules on the reference simplex (weights sum to its measure).
//  * P1 triangle: points (1/6,1/6), (2/3,1/6), (1/6,2/3), weights 1/6.
//  * P2 triangle: the symmetric 6-point degree-4 rule (Dunavant 1985) from
//    its closed form: orbits (1-2a, a, a), a = (8 - sqrt10 +- sqrt(38 - 44
//    sqrt(2/5)))/18, with weights (620 +- sqrt(213125 - 53320 sqrt10))/3720
//    (normalised to 1; halved here).  Orbit with the larger a first; within an
//    orbit the odd barycentric coordinate sits at l0, l1, l2 in turn.
//  * tetrahedron: barycentric (a, b, b, b) permutations, a = (5 + 3 sqrt5)/20,
//    b = (5 - sqrt5)/20, weights 1/24; point q has the large coordinate at l_q.
//  * quadrilateral: the 2 x 2 Gauss-Legendre rule on [0, 1]^2, coordinates
//    1/2 -+ sqrt(3)/6, weights 1/4; s varies fastest.
int quadrature_rule(tg_element el, double* w, double* x) {
  if (el == TG_Q1_QUAD_VEC2) {
    const double h = std::sqrt(3.0) / 6.0, g[2] = {0.5 - h, 0.5 + h};
    for (int q = 0; q < 4; ++q) {
      x[2 * q] = g[q & 1];
      x[2 * q + 1] = g[q >> 1];
      w[q] = 0.25;
    }
    return 4;
  }
  if (el == TG_P1_TRI) {
    const double pts[6] = {1.0 / 6, 1.0 / 6, 2.0 / 3, 1.0 / 6, 1.0 / 6, 2.0 / 3};
    for (int q = 0; q < 3; ++q) w[q] = 1.0 / 6;
    std::memcpy(x, pts, sizeof(pts));
    return 3;
  }
  if (el == TG_P2_TRI) {
    const double r = std::sqrt(38.0 - 44.0 * std::sqrt(2.0 / 5.0));
    const double a = (8.0 - std::sqrt(10.0) + r) / 18.0;
    const double b = (8.0 - std::sqrt(10.0) - r) / 18.0;
    const double s = std::sqrt(213125.0 - 53320.0 * std::sqrt(10.0));
    const double wa = 0.5 * (620.0 + s) / 3720.0;
    const double wb = 0.5 * (620.0 - s) / 3720.0;
    const double pts[12] = {a, a, 1 - 2 * a, a, a, 1 - 2 * a, b, b, 1 - 2 * b, b, b, 1 - 2 * b};
    const double ws[6] = {wa, wa, wa, wb, wb, wb};
    std::memcpy(x, pts, sizeof(pts));
    std::memcpy(w, ws, sizeof(ws));
    return 6;
  }
  const double a = (5.0 + 3.0 * std::sqrt(5.0)) / 20.0, b = (5.0 - std::sqrt(5.0)) / 20.0;
  const double pts[12] = {b, b, b, a, b, b, b, a, b, b, b, a};
  for (int q = 0; q < 4; ++q) w[q] = 1.0 / 24;
  std::memcpy(x, pts, sizeof(pts));
  return 4;
}

// Reference basis on the reference simplex at point x (d coordinates):
// values v[a] and gradients g[a][s].
static void ref_basis(tg_element el, const double* x, double* v, double (*g)[3]) {
  for (int a = 0; a < 6; ++a) {
    v[a] = 0;
    g[a][0] = g[a][1] = g[a][2] = 0;
  }
  if (el == TG_Q1_QUAD_VEC2) {  // bilinear corners (0,0), (1,0), (1,1), (0,1)
    const double s = x[0], t = x[1];
    v[0] = (1 - s) * (1 - t);
    v[1] = s * (1 - t);
    v[2] = s * t;
    v[3] = (1 - s) * t;
    g[0][0] = -(1 - t);
    g[0][1] = -(1 - s);
    g[1][0] = 1 - t;
    g[1][1] = -s;
    g[2][0] = t;
    g[2][1] = s;
    g[3][0] = -t;
    g[3][1] = 1 - s;
    return;
  }
  if (el == TG_P1_TRI || el == TG_P2_TRI) {
    const double l[3] = {1.0 - x[0] - x[1], x[0], x[1]};
    const double dl[3][2] = {{-1, -1}, {1, 0}, {0, 1}};
    if (el == TG_P1_TRI) {
      for (int a = 0; a < 3; ++a) {
        v[a] = l[a];
        g[a][0] = dl[a][0];
        g[a][1] = dl[a][1];
      }
      return;
    }
    for (int a = 0; a < 3; ++a) {  // vertex functions l(2l - 1)
      v[a] = l[a] * (2 * l[a] - 1);
      for (int s = 0; s < 2; ++s) g[a][s] = (4 * l[a] - 1) * dl[a][s];
    }
    const int ed[3][2] = {{0, 1}, {1, 2}, {2, 0}};
    for (int k = 0; k < 3; ++k) {  // edge functions 4 l_i l_j
      const int i = ed[k][0], j = ed[k][1];
      v[3 + k] = 4 * l[i] * l[j];
      for (int s = 0; s < 2; ++s) g[3 + k][s] = 4 * (l[j] * dl[i][s] + l[i] * dl[j][s]);
    }
    return;
  }
  const double l0 = 1.0 - x[0] - x[1] - x[2];
  v[0] = l0;
  v[1] = x[0];
  v[2] = x[1];
  v[3] = x[2];
  for (int s = 0; s < 3; ++s) {
    g[0][s] = -1;
    g[1 + s][s] = 1;
  }
}

template <typename T>
RefTab<T> ref_table(tg_element el) {
  RefTab<T> t;
  std::memset(&t, 0, sizeof(t));
  if (el == TG_P1_TET_VEC3) el = TG_P1_TET;
  double w[6], x[18];
  const int nq = quadrature_rule(el, w, x);
  const int d = dim_of(el), nv = nv_of(el);
  double M[6][6] = {{0}}, m1[6] = {0}, ws = 0;
  for (int q = 0; q < nq; ++q) {
    double v[6], g[6][3];
    ref_basis(el, x + q * d, v, g);
    t.w[q] = (T)w[q];
    ws += w[q];
    for (int a = 0; a < nv; ++a) {
      t.phi[q][a] = (T)v[a];
      for (int s = 0; s < 3; ++s) t.gh[q][a][s] = (T)g[a][s];
      m1[a] += w[q] * v[a];
      for (int b = a; b < nv; ++b) M[a][b] += w[q] * v[a] * v[b];
    }
  }
  for (int a = 0; a < nv; ++a) {
    t.m1[a] = (T)m1[a];
    for (int b = 0; b < nv; ++b) t.M[a][b] = (T)(b >= a ? M[a][b] : M[b][a]);  // exactly symmetric
  }
  t.wsum = (T)ws;
  return t;
}

template RefTab<float> ref_table<float>(tg_element);
template RefTab<double> ref_table<double>(tg_element);

}  // namespace tg

extern "C" {

const char* tg_status_string(tg_status s) {
  switch (s) {
    case TG_OK: return "TG_OK";
    case TG_ERR_INVALID_ARG: return "TG_ERR_INVALID_ARG";
    case TG_ERR_INDEX_RANGE: return "TG_ERR_INDEX_RANGE";
    case TG_ERR_DEGENERATE_ELEMENT: return "TG_ERR_DEGENERATE_ELEMENT";
    case TG_ERR_INDEX_OVERFLOW: return "TG_ERR_INDEX_OVERFLOW";
    case TG_ERR_OUT_OF_MEMORY: return "TG_ERR_OUT_OF_MEMORY";
    case TG_ERR_CUDA: return "TG_ERR_CUDA";
    case TG_ERR_TIMEOUT: return "TG_ERR_TIMEOUT";
    case TG_ERR_UNSUPPORTED: return "TG_ERR_UNSUPPORTED";
  }
  return "TG_ERR_UNKNOWN";
}

const char* tg_last_error_message(void) { return tg::g_last_error.c_str(); }

int32_t tg_quadrature(tg_element el, double* w, double* xhat) {
  if (el < TG_P1_TRI || el > TG_Q1_QUAD_VEC2) return 0;
  if (el == TG_P1_TET_VEC3) el = TG_P1_TET;
  double ww[6], xx[18];
  const int nq = tg::quadrature_rule(el, ww, xx);
  const int d = tg::dim_of(el);
  if (w) std::memcpy(w, ww, sizeof(double) * nq);
  if (xhat) std::memcpy(xhat, xx, sizeof(double) * nq * d);
  return nq;
}

tg_status tg_pattern_info(const tg_pattern* p, int64_t* n_rows, int64_t* nnz, const int32_t** row_ptr,
                          const int32_t** col_idx, const int32_t** elem_slot, int32_t* slot_stride) {
  if (!p) return TG_ERR_INVALID_ARG;
  const int nc = tg::ncomp_of(p->el);
  const bool vec = nc > 1;
  if (n_rows) *n_rows = nc * p->N;
  if (nnz) *nnz = (int64_t)nc * nc * p->nnz;
  if (row_ptr) *row_ptr = vec ? p->row_ptr_dof : p->row_ptr;
  if (col_idx) *col_idx = vec ? p->col_idx_dof : p->col_idx;
  if (elem_slot) *elem_slot = p->elem_slot;
  if (slot_stride) *slot_stride = p->nv * p->nv;
  return TG_OK;
}

tg_status tg_pattern_shape(const tg_pattern* p, tg_element* el, int64_t* n_elems, int64_t* n_nodes,
                           int32_t* max_row_len, int32_t* max_degree) {
  if (!p) return TG_ERR_INVALID_ARG;
  if (el) *el = p->el;
  if (n_elems) *n_elems = p->E;
  if (n_nodes) *n_nodes = p->N;
  if (max_row_len) *max_row_len = p->max_row_len;
  if (max_degree) *max_degree = p->max_deg;
  return TG_OK;
}

tg_status tg_pattern_row_blocks(const tg_pattern* p, int32_t* rows_per_block, int64_t* n_blocks) {
  if (!p) return TG_ERR_INVALID_ARG;
  const bool on = p->bel != nullptr;
  if (rows_per_block) *rows_per_block = on ? p->blk_rows : 0;
  if (n_blocks) *n_blocks = on ? p->n_blk : 0;
  return TG_OK;
}

tg_status tg_pattern_layouts(const tg_pattern* p, uint32_t* flags) {
  if (!p || !flags) return TG_ERR_INVALID_ARG;
  *flags = (p->bel ? TG_LAYOUT_ROW_BLOCKS : 0u) | (p->fan ? TG_LAYOUT_FANS : 0u) |
           (p->elem_pos ? TG_LAYOUT_ELEM_POS : 0u) |
           (p->emask ? TG_LAYOUT_EDGE_MASKS : 0u);
  return TG_OK;
}

tg_status tg_get_device_status(const tg_pattern* p, int64_t* first_bad_elem) {
  if (!p) return TG_ERR_INVALID_ARG;
  TG_CK(cudaSetDevice(p->device));
  TG_CK(cudaDeviceSynchronize());
  unsigned long long h[2];
  TG_CK(cudaMemcpy(h, p->status, sizeof(h), cudaMemcpyDeviceToHost));
  const unsigned long long reset[2] = {0ull, ~0ull};
  TG_CK(cudaMemcpy(p->status, reset, sizeof(reset), cudaMemcpyHostToDevice));
  // a CTA that gave up on a timed-out wait never arrived: restart the
  // arrival counter of the last-CTA sums
  if (h[0] == TG_ERR_TIMEOUT && p->arrivals) TG_CK(cudaMemset(p->arrivals, 0, 16));
  if (first_bad_elem) *first_bad_elem = (h[1] == ~0ull) ? -1 : (int64_t)h[1];
  return (tg_status)h[0];
}

void tg_pattern_destroy(tg_pattern* p) {
  if (!p) return;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(p->device);
  void* bufs[] = {p->cells,    p->inc_ptr,  p->inc_e,   p->inc_pos, p->row_ptr, p->col_idx, p->elem_slot,
                  p->row_ptr_dof, p->col_idx_dof, p->status, p->partials, p->bel, p->boff, p->bvbase, p->bel_cnt,
                  p->brec, p->elem_pos, p->arrivals,
                  p->iperm, p->urp, p->iinc, p->irp, p->elem_scratch, p->fan, p->fan_off, p->emask};
  for (void* b : bufs)
    if (b) cudaFree(b);
  cudaSetDevice(prev);
  delete p;
}

}  // extern "C"
