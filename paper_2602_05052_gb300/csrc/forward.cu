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

#include "async.cuh"
#include "gather.cuh"

namespace {

constexpr int BS = 128;  // rows per CTA (scalar kernels)
constexpr int EB = 64;   // rows per CTA (elasticity: 9 * row length accumulators per thread)

using tg::FwdArgs;
using tg::tab_bytes;
using tg::copy_table;
using tg::absv;
using tg::load_kq;
using tg::scalar_row;

// One CTA per block of R consecutive rows (staged gather, gather.cuh).
// Shared memory: the reference tables, then the stage buffer.
template <int EL, typename T>
__global__ void __launch_bounds__(BS) k_bilinear_gather(const FwdArgs<T> a, const __grid_constant__ tg::RefTab<T> tab,
                                                        int cap) {
  extern __shared__ __align__(16) unsigned char smem[];
  auto& ts = *reinterpret_cast<tg::RefTab<T>*>(smem);
  copy_table(ts, tab);
  const int64_t r0 = (int64_t)blockIdx.x * blockDim.x;
  const int64_t r1 = r0 + blockDim.x < a.n ? r0 + blockDim.x : a.n;
  tg::assemble_rows<EL, T>(a, ts, smem + tab_bytes<T>(), cap, r0, r1);
}

// P1 fast path (incidence records) as a persistent, software-pipelined
// kernel.  Each CTA walks row blocks b = blockIdx.x, + gridDim.x, ...; the
// contiguous streams of a block (its slices of inc_ptr, row_ptr and the
// records) are brought into one of two shared-memory stages by 1D bulk
// copies that thread 0 issues one block ahead, completing on the stage's
// mbarrier, while the whole CTA processes the previous block.  Only the
// gathers of coordinates and coefficients remain on the critical path.
//
// Stage s: ip [IPN] | rp [IPN] | rec [NV][RECN], IPN = R + 8, RECN = cap + 8
// (bulk copies move whole 16-byte groups, so ranges are widened to
// multiples of 4 words; the pattern arrays carry 16 bytes of tail padding).
template <int D, typename T>
__global__ void __launch_bounds__(BS, (D == 2 && sizeof(T) == 4) ? 5 : 1) k_bilinear_p1(
    const FwdArgs<T> a, const __grid_constant__ tg::RefTab<T> tab, int cap, int64_t nblocks) {
  constexpr int NV = D + 1, NQ = D == 2 ? 3 : 4;
  constexpr int UB = (D == 2 && sizeof(T) == 4) ? 3 : 2;
  extern __shared__ __align__(16) unsigned char smem[];
  auto& ts = *reinterpret_cast<tg::RefTab<T>*>(smem);
  const int R = blockDim.x;
  const int IPN = R + 8, RECN = cap + 8;
  unsigned char* p = smem + tab_bytes<T>();
  uint64_t* bar = reinterpret_cast<uint64_t*>(p);
  p += 16;
  int* meta = reinterpret_cast<int*>(p);  // [2][8]: r0, r1, J0, J1, a0, j0a
  p += 64;
  int* st_ip[2];
  int* st_rp[2];
  uint32_t* st_rec[2];
  for (int s = 0; s < 2; ++s) {
    st_ip[s] = reinterpret_cast<int*>(p);
    p += IPN * 4;
    st_rp[s] = reinterpret_cast<int*>(p);
    p += IPN * 4;
    st_rec[s] = reinterpret_cast<uint32_t*>(p);
    p += (size_t)NV * RECN * 4;
  }
  T* contrib = reinterpret_cast<T*>(p);
  uint32_t* posw = reinterpret_cast<uint32_t*>(contrib + (size_t)NV * cap);
  uint8_t* owner = reinterpret_cast<uint8_t*>(posw + cap);
  T* acc = reinterpret_cast<T*>(p + tg::staged_head<T, NV, 1>(cap));
  if (threadIdx.x == 0) {
    tg::mbar_init(&bar[0], 1);
    tg::mbar_init(&bar[1], 1);
    tg::fence_mbar_init();
  }
  copy_table(ts, tab);  // includes a CTA barrier

  const int64_t G = gridDim.x;
  const int64_t stride = a.rec_stride;
  // issue the copies of block blk into stage s (thread 0)
  auto issue = [&](int s, int64_t blk, int J0, int J1) {
    const int r0 = (int)(blk * R), r1 = (int)(blk * R + R < a.n ? blk * R + R : a.n);
    const int a0 = r0 & ~3, nip = (r1 + 1 - a0 + 3) & ~3;
    const int j0a = J0 & ~3, nrec = (J1 - j0a + 3) & ~3;
    int* m = meta + 8 * s;
    m[0] = r0;
    m[1] = r1;
    m[2] = J0;
    m[3] = J1;
    m[4] = a0;
    m[5] = j0a;
    const uint32_t bytes = 2u * nip * 4 + (J1 > J0 ? (uint32_t)NV * nrec * 4 : 0u);
    tg::fence_proxy_async();
    tg::mbar_arrive_expect_tx(&bar[s], bytes);
    tg::bulk_copy_g2s(st_ip[s], a.inc_ptr + a0, nip * 4, &bar[s]);
    tg::bulk_copy_g2s(st_rp[s], a.row_ptr + a0, nip * 4, &bar[s]);
    if (J1 > J0)
      for (int k = 0; k < NV; ++k) tg::bulk_copy_g2s(st_rec[s] + k * RECN, a.rec + k * stride + j0a, nrec * 4, &bar[s]);
  };
  auto block_J = [&](int64_t blk, int& J0, int& J1) {
    J0 = __ldg(a.inc_ptr + blk * R);
    J1 = __ldg(a.inc_ptr + (blk * R + R < a.n ? blk * R + R : a.n));
  };

  int64_t b = blockIdx.x;
  int nJ0 = 0, nJ1 = 0;
  if (threadIdx.x == 0 && b < nblocks) {
    int J0, J1;
    block_J(b, J0, J1);
    issue(0, b, J0, J1);
    if (b + G < nblocks) block_J(b + G, nJ0, nJ1);
  }
  for (int k = 0; b < nblocks; ++k, b += G) {
    const int s = k & 1;
    if (threadIdx.x == 0 && b + G < nblocks) {
      issue(s ^ 1, b + G, nJ0, nJ1);
      if (b + 2 * G < nblocks) block_J(b + 2 * G, nJ0, nJ1);
    }
    if (!tg::mbar_wait(&bar[s], (k >> 1) & 1)) {
      tg::record_error(a.status, TG_ERR_TIMEOUT, 0);
      return;
    }
    const int* m = meta + 8 * s;
    const int r0 = m[0], r1 = m[1], J0 = m[2], J1 = m[3], a0 = m[4], j0a = m[5];
    const int* ip = st_ip[s] - a0;  // ip[i] = inc_ptr[i] for i in [r0, r1]
    const int* rp = st_rp[s] - a0;
    const uint32_t* rc = st_rec[s] - j0a;
    // phase 0: incidence -> row map
    const int i = r0 + (int)threadIdx.x;
    int js = 0, je = 0;
    if (i < r1) {
      js = ip[i] - J0;
      je = ip[i + 1] - J0;
      for (int q = js; q < je; ++q) owner[q] = (uint8_t)threadIdx.x;
    }
    __syncthreads();
    // phase 1: element rows of every incidence of the block
    for (int base = J0 + (int)threadIdx.x; base < J1; base += UB * R) {
      uint32_t ra[UB], rv[UB][D];
      int own[UB];
#pragma unroll
      for (int u = 0; u < UB; ++u) {
        const int j = base + u * R;
        const bool ok = j < J1;
        ra[u] = ok ? rc[j] : 0u;
#pragma unroll
        for (int q = 0; q < D; ++q) rv[u][q] = ok ? rc[(q + 1) * RECN + j] : 0u;
        own[u] = r0 + (ok ? owner[j - J0] : 0);
      }
      T x[UB][NV][D];
      T kq[UB][NQ];
#pragma unroll
      for (int u = 0; u < UB; ++u) tg::p1_gather<D, T>(a, ra[u], rv[u], own[u], x[u], kq[u]);
#pragma unroll
      for (int u = 0; u < UB; ++u) {
        const int j = base + u * R;
        if (j >= J1) continue;
        T Krow[NV];
        if (!tg::p1_local_row<D, T>(x[u], kq[u], a.c, ts, Krow)) {
          tg::record_error(a.status, TG_ERR_DEGENERATE_ELEMENT, ra[u] & 0xffffffu);
#pragma unroll
          for (int q = 0; q < NV; ++q) Krow[q] = T(0);
        }
        posw[j - J0] = tg::p1_positions<D>(ra[u], rv[u]);
#pragma unroll
        for (int q = 0; q < NV; ++q) contrib[q * cap + (j - J0)] = Krow[q];
      }
    }
    __syncthreads();
    // phase 2: rows summed in increasing element order into the CSR-local copy
    const int rbase = rp[r0];
    if (i < r1) {
      T* row = acc + (rp[i] - rbase);
      const int len = rp[i + 1] - rp[i];
      for (int q = 0; q < len; ++q) row[q] = T(0);
      for (int q = js; q < je; ++q) {
        const uint32_t w0 = posw[q];
#pragma unroll
        for (int c = 0; c < NV; ++c) row[tg::pos_of(w0, 0u, c)] += contrib[c * cap + q];
      }
    }
    __syncthreads();
    const int nz = rp[r1] - rbase;
    T* out = a.out + rbase;
    for (int q = threadIdx.x; q < nz; q += R) out[q] = acc[q];
    __syncthreads();  // stage s and the work buffers are free again
  }
}

template <int D, typename T>
size_t p1_pipe_smem(int R, int cap, int max_row) {
  constexpr int NV = D + 1;
  return tab_bytes<T>() + 16 + 64 + 2 * ((size_t)(R + 8) * 8 + (size_t)NV * (cap + 8) * 4) +
         tg::staged_bytes<T, NV, 1>(R, cap, max_row);
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
    if (!scalar_row<EL, T>(a, ts, e, la, Krow)) {
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

// Vector P1 elasticity, one thread per node: the node's three DoF rows are
// consecutive in the DoF CSR and together hold 9 * len entries in the order
// [component i][column node p][component j], accumulated in shared memory.
//   block (a, b) = (1/|det|) ( L n_a n_b^T + M n_b n_a^T + M (n_a.n_b) I ),
//   L = sum_q w_q lam_q, M = sum_q w_q mu_q.
template <typename T>
__global__ void __launch_bounds__(EB) k_elastic_gather(const FwdArgs<T> a, const __grid_constant__ tg::RefTab<T> tab) {
  extern __shared__ __align__(16) unsigned char smem[];
  auto& ts = *reinterpret_cast<tg::RefTab<T>*>(smem);
  T* acc = reinterpret_cast<T*>(smem + tab_bytes<T>()) + threadIdx.x;
  copy_table(ts, tab);
  const int64_t i = (int64_t)blockIdx.x * EB + threadIdx.x;
  if (i >= a.n) return;
  const int r0 = __ldg(a.row_ptr + i), len = __ldg(a.row_ptr + i + 1) - r0;
  for (int p = 0; p < 9 * len; ++p) acc[p * EB] = T(0);
  const int j0 = __ldg(a.inc_ptr + i), j1 = __ldg(a.inc_ptr + i + 1);
  for (int j = j0; j < j1; ++j) {
    const int ea = __ldg(a.inc_e + j);
    const int64_t e = ea >> 3;
    const int la = ea & 7;
    const uint32_t w0 = __ldg(a.inc_pos + j);
    const int32_t* cl = a.cells + e * 4;
    tg::Geom<3, T> g;
    tg::tet_geom(a.coords, __ldg(cl), __ldg(cl + 1), __ldg(cl + 2), __ldg(cl + 3), g);
    const T adet = absv(g.det);
    if (!(adet > tg::det_tiny<T>())) {
      tg::record_error(a.status, TG_ERR_DEGENERATE_ELEMENT, e);
      continue;
    }
    const T inv = T(1) / adet;
    const T L = tg::weighted_coef<T, 4>(a.coef, a.layout, e, ts.w, ts.wsum) * inv;
    const T M = tg::weighted_coef<T, 4>(a.coef2, a.layout, e, ts.w, ts.wsum) * inv;
    T na[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const T col[4] = {g.n[0][r], g.n[1][r], g.n[2][r], g.n[3][r]};
      na[r] = tg::sel(la, col);
    }
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int pos = tg::pos_of(w0, 0u, b);
      const T d = na[0] * g.n[b][0] + na[1] * g.n[b][1] + na[2] * g.n[b][2];
#pragma unroll
      for (int ii = 0; ii < 3; ++ii)
#pragma unroll
        for (int jj = 0; jj < 3; ++jj) {
          T v = L * na[ii] * g.n[b][jj] + M * g.n[b][ii] * na[jj];
          if (ii == jj) v += M * d;
          acc[((ii * len + pos) * 3 + jj) * EB] += v;
        }
    }
  }
  T* out = a.out + 9ll * r0;
  for (int p = 0; p < 9 * len; ++p) out[p] = acc[p * EB];
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
  a.rec = p->rec;
  a.rec_stride = (p->E * p->nv + 3) & ~3ll;
  return a;
}

bool aligned(const void* ptr, size_t a) { return ((uintptr_t)ptr % a) == 0; }

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
  if constexpr (EL == TG_P1_TRI || EL == TG_P1_TET) {
    if (p->rec) {
      constexpr int D = El::dim;
      // rows per block: the largest R in {128, 64, 32} whose two stages and
      // work buffers fit in 100 KB (at least two CTAs per SM)
      int Rp = 128;
      while (Rp > 32 && p1_pipe_smem<D, T>(Rp, Rp * std::max(1, p->max_deg), p->max_row_len) > 100 * 1024) Rp /= 2;
      const int capp = Rp * std::max(1, p->max_deg);
      const size_t smp = p1_pipe_smem<D, T>(Rp, capp, p->max_row_len);
      auto kern = k_bilinear_p1<D, T>;
      tg_status st = set_smem((const void*)kern, smp);
      if (st != TG_OK) return st;
      int per_sm = 0;
      TG_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, Rp, smp));
      const int64_t nblocks = (p->N + Rp - 1) / Rp;
      const int grid = (int)std::min<int64_t>(nblocks, (int64_t)std::max(per_sm, 1) * tg::sm_count());
      kern<<<grid, Rp, smp, s>>>(a, tab, capp, nblocks);
      TG_CK_LAUNCH("k_bilinear_p1");
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

template <typename T>
tg_status elastic(const tg_pattern* p, const void* coords, const void* lam, const void* mu, tg_layout l, void* vals,
                  cudaStream_t s) {
  FwdArgs<T> a = base_args<T>(p, coords);
  a.coef = static_cast<const T*>(lam);
  a.coef2 = static_cast<const T*>(mu);
  a.layout = l;
  a.out = static_cast<T*>(vals);
  const size_t smem = tab_bytes<T>() + (size_t)EB * 9 * p->max_row_len * sizeof(T);
  tg_status st = set_smem((const void*)k_elastic_gather<T>, smem);
  if (st != TG_OK) return st;
  k_elastic_gather<T><<<tg::grid_for(p->N, EB), EB, smem, s>>>(a, table<T>(TG_P1_TET));
  TG_CK_LAUNCH("k_elastic_gather");
  return TG_OK;
}

bool layout_ok(tg_layout l, bool allow_node) {
  return l == TG_PER_ELEMENT || l == TG_PER_QP || l == TG_CONSTANT || (allow_node && l == TG_PER_NODE);
}

tg_status bilinear_entry(const tg_pattern* p, tg_dtype dtype, const void* coords, const void* kappa, tg_layout kl,
                         double c, void* vals, tg_stream stream, bool atomic) {
  tg_status st = check_common(p, dtype, coords);
  if (st != TG_OK) return st;
  if (p->el == TG_P1_TET_VEC3 || !layout_ok(kl, false) || !kappa || (p->nnz > 0 && !vals)) return TG_ERR_INVALID_ARG;
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

tg_status tg_assemble_elasticity(const tg_pattern* p, tg_dtype dtype, const void* coords, const void* lam,
                                 const void* mu, tg_layout layout, void* vals_out, tg_stream stream) {
  tg_status st = check_common(p, dtype, coords);
  if (st != TG_OK) return st;
  if (p->el != TG_P1_TET_VEC3 || !layout_ok(layout, false) || !lam || !mu || (p->nnz > 0 && !vals_out))
    return TG_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  return dtype == TG_F32 ? elastic<float>(p, coords, lam, mu, layout, vals_out, s)
                         : elastic<double>(p, coords, lam, mu, layout, vals_out, s);
}

tg_status tg_assemble_load(const tg_pattern* p, tg_dtype dtype, const void* coords, const void* f, tg_layout f_layout,
                           int32_t ncomp, void* F_out, tg_stream stream) {
  tg_status st = check_common(p, dtype, coords);
  if (st != TG_OK) return st;
  if ((ncomp != 1 && ncomp != 3) || !f || !F_out || !(f_layout == TG_PER_NODE || f_layout == TG_PER_QP ||
                                                       f_layout == TG_CONSTANT))
    return TG_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  return dtype == TG_F32 ? load<float>(p, coords, f, f_layout, ncomp, F_out, s)
                         : load<double>(p, coords, f, f_layout, ncomp, F_out, s);
}

}  // extern "C"
