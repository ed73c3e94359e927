// Pattern construction: the "routing" of Algorithm 2, precomputed from the
// mesh topology alone (Stage II of the method).
//
// Steps, all on the device:
//   1. validate the cells and count the incidences of every node;
//   2. exclusive scan -> inc_ptr; scatter (element, local index) pairs and
//      sort every node's list by element index (fixed Reduce order);
//   3. per node: the sorted, de-duplicated set of nodes of its incident
//      elements is its CSR row (structural zeros kept); scan -> row_ptr;
//   4. per incidence: 8-bit positions of the element's nodes inside the
//      owning row (inc_pos) and the element-to-slot map (elem_slot);
//   5. P1: row blocks with their distinct elements and packed incidence
//      records (the element-once kernels);
//   6. vector elasticity: expansion of the node CSR to the DoF CSR
//      (DoF = 3 * node + component, 3x3 blocks).
#include <cstdio>
#include <vector>

#include "tg_internal.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kScanThreads = 512;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

__global__ void k_count(const int32_t* __restrict__ cells, int64_t E, int nv, int64_t N, int32_t* __restrict__ deg,
                        unsigned long long* status) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < E; e += stride) {
    int v[6];
    bool bad = false;
    for (int a = 0; a < nv; ++a) {
      v[a] = cells[e * nv + a];
      if (v[a] < 0 || (int64_t)v[a] >= N) bad = true;
    }
    if (bad) {
      tg::record_error(status, TG_ERR_INDEX_RANGE, e);
      continue;
    }
    for (int a = 0; a < nv; ++a)
      for (int b = a + 1; b < nv; ++b)
        if (v[a] == v[b]) bad = true;
    if (bad) {
      tg::record_error(status, TG_ERR_DEGENERATE_ELEMENT, e);
      continue;
    }
    for (int a = 0; a < nv; ++a) atomicAdd(deg + v[a], 1);
  }
}

// Exclusive scan of one tile of kScanTile values; the tile total goes to
// tile_sums[blockIdx.x].
template <typename Tin>
__global__ void __launch_bounds__(kScanThreads) k_scan_tile(const Tin* __restrict__ in, int64_t* __restrict__ out,
                                                            int64_t* __restrict__ tile_sums, int64_t n) {
  __shared__ int64_t warp_sums[kScanThreads / 32];
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  int64_t v[kScanItems];
  int64_t s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    v[k] = (base + k < n) ? (int64_t)in[base + k] : 0;
    s += v[k];
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int64_t x = s;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_sums[wid] = x;
  __syncthreads();
  if (wid == 0) {
    int64_t w = lane < kScanThreads / 32 ? warp_sums[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < kScanThreads / 32) warp_sums[lane] = w;
  }
  __syncthreads();
  int64_t run = x - s + (wid > 0 ? warp_sums[wid - 1] : 0);
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    if (base + k < n) out[base + k] = run;
    run += v[k];
  }
  if (threadIdx.x == kScanThreads - 1) tile_sums[blockIdx.x] = run;
}

__global__ void k_scan_add(int64_t* __restrict__ out, const int64_t* __restrict__ tile_off, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] += tile_off[i / kScanTile];
}

__global__ void k_narrow(const int64_t* __restrict__ in, int32_t* __restrict__ out, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = (int32_t)in[i];
}

__global__ void k_fill(const int32_t* __restrict__ cells, int64_t E, int nv, int32_t* __restrict__ cursor,
                       int32_t* __restrict__ inc_e) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < E; e += stride)
    for (int a = 0; a < nv; ++a) {
      const int v = cells[e * nv + a];
      const int slot = atomicAdd(cursor + v, 1);
      inc_e[slot] = (int32_t)(e * 8 + a);
    }
}

// Sort each node's incidence list by element index (insertion sort; lists
// are short).  Fixes the order in which every Reduce sums.
__global__ void k_sort_incidence(const int32_t* __restrict__ inc_ptr, int32_t* __restrict__ inc_e, int64_t N) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int j0 = inc_ptr[i], j1 = inc_ptr[i + 1];
  for (int j = j0 + 1; j < j1; ++j) {
    const int x = inc_e[j];
    int k = j - 1;
    while (k >= j0 && inc_e[k] > x) {
      inc_e[k + 1] = inc_e[k];
      --k;
    }
    inc_e[k + 1] = x;
  }
}

// Insert v into the sorted unique list cols[0..len); false when full.
__device__ __forceinline__ bool insert_unique(int* cols, int& len, int v) {
  int k = len - 1;
  while (k >= 0 && cols[k] > v) --k;
  if (k >= 0 && cols[k] == v) return true;
  if (len >= TG_MAX_ROW) return false;
  for (int m = len - 1; m > k; --m) cols[m + 1] = cols[m];
  cols[k + 1] = v;
  ++len;
  return true;
}

__device__ __forceinline__ int lower_bound(const int* cols, int len, int v) {
  int lo = 0, hi = len;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (cols[mid] < v) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// FILL = false: row lengths, largest row and degree.  FILL = true: columns,
// per-incidence positions and the element-to-slot map.
template <bool FILL>
__global__ void __launch_bounds__(128) k_rows(const int32_t* __restrict__ cells, const int32_t* __restrict__ inc_ptr,
                                              const int32_t* __restrict__ inc_e, int64_t N, int nv, int npw, int nc,
                                              int32_t* __restrict__ row_len, int* __restrict__ maxes,
                                              const int32_t* __restrict__ row_ptr, int32_t* __restrict__ col_idx,
                                              uint32_t* __restrict__ inc_pos, int32_t* __restrict__ elem_slot,
                                              unsigned long long* status) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  int cols[TG_MAX_ROW];
  int len = 0;
  bool ok = true;
  const int j0 = inc_ptr[i], j1 = inc_ptr[i + 1];
  for (int j = j0; j < j1 && ok; ++j) {
    const int e = inc_e[j] >> 3;
    for (int b = 0; b < nv && ok; ++b) ok = insert_unique(cols, len, cells[(int64_t)e * nv + b]);
  }
  if (!FILL) {
    if (!ok) tg::record_error(status, TG_ERR_UNSUPPORTED, j0 < j1 ? (inc_e[j0] >> 3) : 0);
    row_len[i] = len;
    atomicMax(maxes + 0, len);
    atomicMax(maxes + 1, j1 - j0);
    return;
  }
  const int r0 = row_ptr[i];
  for (int p = 0; p < len; ++p) col_idx[r0 + p] = cols[p];
  for (int j = j0; j < j1; ++j) {
    const int e = inc_e[j] >> 3, a = inc_e[j] & 7;
    uint32_t w0 = 0, w1 = 0;
    for (int b = 0; b < nv; ++b) {
      const uint32_t pos = (uint32_t)lower_bound(cols, len, cells[(int64_t)e * nv + b]);
      if (b < 4) w0 |= pos << (8 * b);
      else w1 |= pos << (8 * (b - 4));
      const int64_t slot = (int64_t)nc * nc * r0 + (int64_t)nc * pos;
      elem_slot[((int64_t)e * nv + a) * nv + b] = (int32_t)slot;
    }
    inc_pos[(int64_t)j * npw] = w0;
    if (npw == 2) inc_pos[(int64_t)j * npw + 1] = w1;
  }
}

// DoF-level CSR of a vector kind with nc DoFs per node (DoF = nc node +
// component): node row n becomes nc DoF rows of nc len entries, block
// (n, m) at columns nc m .. nc m + nc - 1.
__global__ void k_expand(const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col_idx, int64_t N, int nc,
                         int32_t* __restrict__ row_ptr_dof, int32_t* __restrict__ col_idx_dof) {
  const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  const int r0 = row_ptr[n], len = row_ptr[n + 1] - r0;
  for (int i = 0; i < nc; ++i) {
    row_ptr_dof[nc * n + i] = nc * nc * r0 + nc * i * len;
    for (int p = 0; p < len; ++p)
      for (int j = 0; j < nc; ++j)
        col_idx_dof[(int64_t)nc * nc * r0 + (int64_t)(i * len + p) * nc + j] = nc * col_idx[r0 + p] + j;
  }
  if (n == N - 1) row_ptr_dof[nc * N] = nc * nc * row_ptr[N];
}

// ------------------------------------------------------------------ row blocks
// The element-once kernels walk the rows in an internal order: nodes sorted
// by their smallest incident element (a space-filling-curve element order
// makes consecutive rows a compact patch), cut into blocks of R rows, each
// block in ascending node id.
//
// key[u]: smallest element incident to node u (E for an isolated node).
__global__ void k_row_key(const int32_t* __restrict__ inc_ptr, const int32_t* __restrict__ inc_e, int64_t N,
                          int64_t E, int32_t* __restrict__ key, int32_t* __restrict__ iso) {
  const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= N) return;
  const int j0 = inc_ptr[u], j1 = inc_ptr[u + 1];
  key[u] = j1 > j0 ? (inc_e[j0] >> 3) : (int32_t)E;
  iso[u] = j1 > j0 ? 0 : 1;
}

// Bucket sizes: the vertices of element e whose key is e.
__global__ void k_key_count(const int32_t* __restrict__ cells, int nv, int64_t E, const int32_t* __restrict__ key,
                            int32_t* __restrict__ cnt) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= E) return;
  int c = 0;
  for (int a = 0; a < nv; ++a) c += key[cells[e * nv + a]] == (int32_t)e;
  cnt[e] = c;
}

// Bucket e lists the vertices keyed to e in ascending id.
__global__ void k_key_place(const int32_t* __restrict__ cells, int nv, int64_t E, const int32_t* __restrict__ key,
                            const int64_t* __restrict__ off, int32_t* __restrict__ order) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= E) return;
  int vs[6], n = 0;
  for (int a = 0; a < nv; ++a) {
    const int v = cells[e * nv + a];
    if (key[v] == (int32_t)e) {
      int k = n++;
      while (k > 0 && vs[k - 1] > v) {
        vs[k] = vs[k - 1];
        --k;
      }
      vs[k] = v;
    }
  }
  for (int k = 0; k < n; ++k) order[off[e] + k] = vs[k];
}

// Isolated nodes last, ascending.
__global__ void k_iso_place(const int32_t* __restrict__ iso, const int64_t* __restrict__ rank, int64_t N, int64_t base,
                            int32_t* __restrict__ order) {
  const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (u < N && iso[u]) order[base + rank[u]] = (int32_t)u;
}

// Ascending node ids inside every block of R (<= 128) internal rows; the
// inverse permutation.
__global__ void __launch_bounds__(128) k_blk_sort(const int32_t* __restrict__ order, int64_t N, int R,
                                                  int32_t* __restrict__ iperm, int32_t* __restrict__ ipos) {
  __shared__ int sk[128];
  const int64_t r0 = (int64_t)blockIdx.x * R;
  const int n = (int)(r0 + R < N ? R : N - r0);
  for (int k = threadIdx.x; k < 128; k += blockDim.x) sk[k] = k < n ? order[r0 + k] : INT32_MAX;
  __syncthreads();
  for (int k = 2; k <= 128; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < 128; i += blockDim.x) {
        const int ixj = i ^ j;
        if (ixj > i) {
          const int x = sk[i], y = sk[ixj];
          if ((x > y) == ((i & k) == 0)) {
            sk[i] = y;
            sk[ixj] = x;
          }
        }
      }
      __syncthreads();
    }
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    iperm[r0 + k] = sk[k];
    ipos[sk[k]] = (int32_t)(r0 + k);
  }
}

// Per internal row: incidence count, CSR row length and CSR row start.
__global__ void k_irow(const int32_t* __restrict__ iperm, const int32_t* __restrict__ inc_ptr,
                       const int32_t* __restrict__ row_ptr, int64_t N, int32_t* __restrict__ deg_i,
                       int32_t* __restrict__ len_i, int32_t* __restrict__ urp) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int u = iperm[i];
  deg_i[i] = inc_ptr[u + 1] - inc_ptr[u];
  len_i[i] = row_ptr[u + 1] - row_ptr[u];
  urp[i] = row_ptr[u];
}

// Per block of R internal rows: its incidence count and its CSR value count.
__global__ void k_blk_stats(const int32_t* __restrict__ iinc, const int32_t* __restrict__ irp, int64_t N, int R,
                            int64_t nblk, int* __restrict__ maxes) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nblk) return;
  const int64_t r0 = b * R, r1 = r0 + R < N ? r0 + R : N;
  atomicMax(maxes + 0, iinc[r1] - iinc[r0]);
  atomicMax(maxes + 1, irp[r1] - irp[r0]);
}

// One CTA per row block: sort the elements of the block's incidences, keep
// the distinct ones (written at uq_out[J0 ...], count in bel_cnt), and pack
// every incidence's record (brec, internal incidence order).  P = power of
// two >= the block's incidences.
__global__ void __launch_bounds__(256) k_blocks(const int32_t* __restrict__ iperm, const int32_t* __restrict__ iinc,
                                                const int32_t* __restrict__ inc_ptr, const int32_t* __restrict__ inc_e,
                                                const uint32_t* __restrict__ inc_pos, int nv, int64_t N, int R, int P,
                                                int32_t* __restrict__ uq_out, int32_t* __restrict__ bel_cnt,
                                                uint32_t* __restrict__ brec, int* __restrict__ max_elems) {
  extern __shared__ int sk[];
  int* key = sk;      // [P]
  int* uq = sk + P;   // [P]
  __shared__ int s_nbe;
  const int64_t b = blockIdx.x;
  const int64_t r0 = b * R, r1 = r0 + R < N ? r0 + R : N;
  const int J0 = iinc[r0], J1 = iinc[r1], n = J1 - J0;
  for (int k = n + (int)threadIdx.x; k < P; k += blockDim.x) key[k] = INT32_MAX;
  for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
    const int u = iperm[i], src = inc_ptr[u], dst = iinc[i] - J0, deg = iinc[i + 1] - iinc[i];
    for (int m = 0; m < deg; ++m) key[dst + m] = inc_e[src + m] >> 3;
  }
  __syncthreads();
  // bitonic sort, ascending
  for (int k = 2; k <= P; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < P; i += blockDim.x) {
        const int ixj = i ^ j;
        if (ixj > i) {
          const int x = key[i], y = key[ixj];
          if ((x > y) == ((i & k) == 0)) {
            key[i] = y;
            key[ixj] = x;
          }
        }
      }
      __syncthreads();
    }
  if (threadIdx.x == 0) {
    int m = 0;
    for (int k = 0; k < n; ++k)
      if (k == 0 || key[k] != key[k - 1]) uq[m++] = key[k];
    s_nbe = m;
    bel_cnt[b] = m;
    atomicMax(max_elems, m);
  }
  __syncthreads();
  const int nbe = s_nbe;
  for (int k = threadIdx.x; k < nbe; k += blockDim.x) uq_out[J0 + k] = uq[k];
  for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
    const int u = iperm[i], src = inc_ptr[u], dst = iinc[i], deg = iinc[i + 1] - iinc[i];
    for (int m = 0; m < deg; ++m) {
      const int e = inc_e[src + m] >> 3, a = inc_e[src + m] & 7;
      int lo = 0, hi = nbe;
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (uq[mid] < e) lo = mid + 1;
        else hi = mid;
      }
      // field c of a record: the position of vertex (a + c) mod nv (field 0
      // the diagonal), the column order of the Map's rotated output rows
      if (nv <= 4) {
        const uint32_t w = inc_pos[src + m];  // 8-bit positions, each < 16 here
        uint32_t r = 0;
        for (int c = 0; c < nv; ++c) r |= ((w >> (8 * ((a + c) % nv))) & 15u) << (4 * c);
        brec[dst + m] = r | ((uint32_t)a << (4 * nv)) | ((uint32_t)lo << (4 * nv + 2));
      } else {  // P2: two inc_pos words of 8-bit positions, each < 32 here
        const uint32_t w0 = inc_pos[2 * (src + m)], w1 = inc_pos[2 * (src + m) + 1];
        uint32_t r = 0;
        for (int c = 0; c < nv; ++c) {
          const int b = (a + c) % nv;
          r |= (((b < 4 ? w0 >> (8 * b) : w1 >> (8 * (b - 4)))) & 31u) << (5 * c);
        }
        brec[2 * (dst + m)] = r;
        brec[2 * (dst + m) + 1] = (uint32_t)a | ((uint32_t)lo << 3);
      }
    }
  }
}

// Element lists of the blocks, at word boff[b] of bel, for a block with
// nbe = bel_cnt[b] elements, bs = (nbe + 3) & ~3 and bs16 = (nbe + 7) & ~7:
//   words [0, bs):  the elements, ascending (bit 31: owner block, the block
//                   holding the element's vertex of smallest internal row);
//   then nv rows of bs16 16-bit offsets: vertex c of element k is
//                   bvbase[b] + row c [k], bvbase[b] the smallest vertex id
//                   of the block's elements.
// One CTA per block; a block whose vertex ids span 2^16 or more sets *wide.
__global__ void __launch_bounds__(128) k_bel(const int32_t* __restrict__ cells, int nv,
                                             const int32_t* __restrict__ iinc, const int32_t* __restrict__ ipos,
                                             const int32_t* __restrict__ uq, const int32_t* __restrict__ bel_cnt,
                                             const int64_t* __restrict__ boff, int64_t N, int R, int64_t nblk,
                                             uint32_t* __restrict__ bel, int32_t* __restrict__ bvbase,
                                             int* __restrict__ wide) {
  __shared__ int s_min, s_max;
  const int64_t b = blockIdx.y * (int64_t)gridDim.x + blockIdx.x;
  if (b >= nblk) return;
  const int nbe = bel_cnt[b], bs = (nbe + 3) & ~3, bs16 = (nbe + 7) & ~7;
  const int J0 = iinc[b * R];
  if (threadIdx.x == 0) {
    s_min = INT32_MAX;
    s_max = INT32_MIN;
  }
  __syncthreads();
  for (int k = threadIdx.x; k < nbe; k += blockDim.x)
    for (int a = 0; a < nv; ++a) {
      const int v = cells[(int64_t)uq[J0 + k] * nv + a];
      atomicMin(&s_min, v);
      atomicMax(&s_max, v);
    }
  __syncthreads();
  const int vb = nbe > 0 ? s_min : 0;
  if (nbe > 0 && s_max - s_min > 65535) atomicOr(wide, 1);
  if (threadIdx.x == 0) bvbase[b] = vb;
  uint32_t* out = bel + boff[b];
  uint16_t* o16 = reinterpret_cast<uint16_t*>(out + bs);
  for (int k = threadIdx.x; k < bs16; k += blockDim.x) {
    if (k >= nbe) {
      if (k < bs) out[k] = 0u;
      for (int a = 0; a < nv; ++a) o16[a * bs16 + k] = 0;
      continue;
    }
    const int e = uq[J0 + k];
    int pmin = INT32_MAX;
    for (int a = 0; a < nv; ++a) {
      const int v = cells[(int64_t)e * nv + a];
      o16[a * bs16 + k] = (uint16_t)(v - vb);
      pmin = min(pmin, ipos[v]);
    }
    out[k] = (uint32_t)e | ((int64_t)pmin / R == b ? 0x80000000u : 0u);
  }
}

__global__ void k_bel_words(const int32_t* __restrict__ cnt, int64_t nblk, int nv, int32_t* __restrict__ words) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b < nblk) words[b] = ((cnt[b] + 3) & ~3) + nv * (((cnt[b] + 7) & ~7) / 2);
}

// Vector elasticity: per node-level CSR entry (i, j) the mask of node i's
// incident elements (bit m = the m-th in inc_e order) that also hold node
// j, the elements around edge (i, j); 0 on the diagonal.  One thread per row
// (at most 16 entries and 32 incident elements).
__global__ void k_edge_masks(const int32_t* __restrict__ inc_ptr, const int32_t* __restrict__ inc_e,
                             const uint32_t* __restrict__ inc_pos, const int32_t* __restrict__ row_ptr, int64_t N,
                             uint32_t* __restrict__ emask) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  uint32_t mk[16];
  for (int q = 0; q < 16; ++q) mk[q] = 0u;
  const int j0 = inc_ptr[i], deg = inc_ptr[i + 1] - j0, r0 = row_ptr[i], len = row_ptr[i + 1] - r0;
  for (int m = 0; m < deg; ++m) {
    const uint32_t w = inc_pos[j0 + m];
    const int la = inc_e[j0 + m] & 7;
    for (int c = 0; c < 4; ++c)
      if (c != la) mk[(w >> (8 * c)) & 15u] |= 1u << m;
  }
  for (int q = 0; q < len; ++q) emask[r0 + q] = mk[q];
}

// Per element: the position of every vertex's column in every vertex's row.
// (Vector elasticity: the slot map is DoF-level, slot = 9 * row_ptr + 3 * pos.)
__global__ void k_elem_pos(const int32_t* __restrict__ cells, const int32_t* __restrict__ elem_slot,
                           const int32_t* __restrict__ row_ptr, int64_t E, int nv, int pb, bool vec3,
                           uint64_t* __restrict__ out) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= E) return;
  uint64_t w = 0;
  for (int a = 0; a < nv; ++a) {
    const int ra = row_ptr[cells[e * nv + a]];
    for (int b = 0; b < nv; ++b) {
      const int sl = elem_slot[(e * nv + a) * nv + b];
      const int pos = vec3 ? (sl - 9 * ra) / 3 : sl - ra;
      w |= (uint64_t)pos << ((a * nv + b) * pb);
    }
  }
  out[e] = w;
}

// ------------------------------------------------------------------ fans
// P1 triangles: the triangles around a node, walked across the edges they
// share, form its fan (closed around an interior node, open at the boundary).
// Triangle k of the fan lies between the row's neighbours j_k and j_{k+1},
// so every off-diagonal entry of the row is the sum of at most two
// consecutive triangles' entries: the Reduce keeps the row in registers.

constexpr int kFanMax = 15;  // fan steps per row (rows of at most 16 entries)

// Per internal row i: its fan from the row's incidence records (brec, in
// element order): deg, open flag, diagonal position (info), neighbour
// positions in fan order (pos64), and the records of the fan's triangles in
// fan order (rec[i * kFanMax + k]).  The walk starts, for an open fan, at the
// triangle holding the boundary neighbour of smaller position, else at the
// row's first triangle in element order.  A node whose triangles are not one
// fan sets *bad.  Per block: the largest deg (kmax, atomicMax).
__global__ void k_fan_rows(const int32_t* __restrict__ iinc, const int32_t* __restrict__ irp,
                           const uint32_t* __restrict__ brec, int64_t N, int R, uint16_t* __restrict__ info,
                           unsigned long long* __restrict__ pos64, uint16_t* __restrict__ rec,
                           int* __restrict__ kmax, int* __restrict__ bad) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int j0 = iinc[i], deg = iinc[i + 1] - j0, len = irp[i + 1] - irp[i];
  if (deg == 0) {
    info[i] = 0;
    pos64[i] = 0ull;
    return;
  }
  if (deg > kFanMax) {
    atomicOr(bad, 1);
    return;
  }
  // records (nv = 3): positions of vertices a, a + 1, a + 2 in bits
  // [0, 4), [4, 8), [8, 12); a in [12, 14); local element index from 14
  uint32_t r[kFanMax];
  int cnt[16];
  for (int q = 0; q < 16; ++q) cnt[q] = 0;
  int dpos = -1;
  for (int m = 0; m < deg; ++m) {
    r[m] = brec[j0 + m];
    cnt[(r[m] >> 4) & 15u]++;
    cnt[(r[m] >> 8) & 15u]++;
    const int d = (int)(r[m] & 15u);
    if (dpos >= 0 && d != dpos) atomicOr(bad, 1);
    dpos = d;
  }
  int start = 0, prev = (int)((r[0] >> 4) & 15u);
  bool open = false;
  for (int q = 0; q < 16 && !open; ++q) {
    if (cnt[q] > 2) {
      atomicOr(bad, 1);
      return;
    }
    if (cnt[q] == 1) {
      for (int m = 0; m < deg; ++m)
        if ((int)((r[m] >> 4) & 15u) == q || (int)((r[m] >> 8) & 15u) == q) {
          start = m;
          break;
        }
      prev = q;
      open = true;
    }
  }
  for (int q = 0; q < 16; ++q)
    if (cnt[q] > 2) {
      atomicOr(bad, 1);
      return;
    }
  unsigned used = 0;
  unsigned long long pw = 0;
  int m = start, k = 0, next = -1;
  while (true) {
    used |= 1u << m;
    const int p1 = (int)((r[m] >> 4) & 15u), p2 = (int)((r[m] >> 8) & 15u);
    const bool swap = prev == p2;
    next = swap ? p1 : p2;
    const uint32_t le = r[m] >> 14, a = (r[m] >> 12) & 3u;
    if (le >= 2048u) {
      atomicOr(bad, 1);
      return;
    }
    rec[i * kFanMax + k] = (uint16_t)(le | (a << 11) | ((swap ? 1u : 0u) << 13));
    pw |= (unsigned long long)prev << (4 * k);
    ++k;
    int nm = -1;
    for (int q = 0; q < deg; ++q)
      if (!((used >> q) & 1u) && ((int)((r[q] >> 4) & 15u) == next || (int)((r[q] >> 8) & 15u) == next)) {
        nm = q;
        break;
      }
    if (nm < 0) break;
    prev = next;
    m = nm;
  }
  const int nn = open ? deg + 1 : deg;  // neighbours
  if (open) pw |= (unsigned long long)next << (4 * deg);
  if (k != deg || (!open && next != (int)(pw & 15ull)) || nn != len - 1) {
    atomicOr(bad, 1);
    return;
  }
  info[i] = (uint16_t)(deg | (open ? 32 : 0) | (dpos << 6));
  pos64[i] = pw;
  atomicMax(kmax + i / R, deg);
}

// Start and direction of every fan, chosen so that the Reduce's shared-memory
// reads are spread over the banks.  Step k of the Reduce reads, for each row
// of the block, the 16-byte output row of its k-th fan triangle at index le
// of the element list; the eight lanes that a 16-byte access serves together
// (rows 8q .. 8q + 7 of a block) meet in one bank group when their le agree
// modulo 8 (the kernels keep the per-vertex arrays a multiple of 8 rows
// long), and each such collision costs a pass.  A closed fan may start at
// any triangle and run either way, an open one from either end; one thread
// per group of eight rows picks, row after row, the start and direction that
// collide least with the rows placed before.  Only the summation order of
// the diagonal and the load entry depends on the choice.
__global__ void k_fan_rotate(uint16_t* __restrict__ info, unsigned long long* __restrict__ pos64,
                             uint16_t* __restrict__ rec, int64_t N, int R) {
  const int64_t qid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int nq = (R + 7) / 8;
  const int64_t b = qid / nq;
  const int q = (int)(qid % nq);
  const int64_t i0 = b * R + 8 * q;
  if (i0 >= N || 8 * q >= R) return;
  unsigned char used[kFanMax][8];
  for (int k = 0; k < kFanMax; ++k)
    for (int g = 0; g < 8; ++g) used[k][g] = 0;
  for (int t = 0; t < 8 && 8 * q + t < R && i0 + t < N; ++t) {
    const int64_t i = i0 + t;
    const int deg = info[i] & 31;
    if (deg == 0) continue;
    const bool open = (info[i] & 32) != 0;
    uint16_t r0[kFanMax];
    for (int k = 0; k < deg; ++k) r0[k] = rec[i * kFanMax + k];
    const int nrot = open ? 1 : deg;
    int best = 0, best_cost = 1 << 30;
    for (int c = 0; c < 2 * nrot; ++c) {
      const int rot = c % nrot;
      const bool rev = c >= nrot;
      int cost = 0;
      for (int m = 0; m < deg; ++m) {
        const int src = rev ? (open ? deg - 1 - m : (rot - m + deg) % deg) : (rot + m) % deg;
        cost += used[m][r0[src] & 7];
      }
      if (cost < best_cost) {
        best_cost = cost;
        best = c;
      }
    }
    const int rot = best % nrot;
    const bool rev = best >= nrot;
    const unsigned long long pw = pos64[i];
    const int nn = open ? deg + 1 : deg;
    unsigned long long npw = 0;
    for (int m = 0; m < deg; ++m) {
      const int src = rev ? (open ? deg - 1 - m : (rot - m + deg) % deg) : (rot + m) % deg;
      const uint16_t r = rev ? (uint16_t)(r0[src] ^ (1u << 13)) : r0[src];
      rec[i * kFanMax + m] = r;
      used[m][r & 7]++;
    }
    for (int m = 0; m < nn; ++m) {
      // neighbour m of the new order: j_{rot + m} forward; reversed, the
      // next neighbour of triangle rot - m (open: of triangle deg - 1 - m)
      const int src = rev ? (open ? deg - m : (rot - m + 1 + deg) % deg) : (rot + m) % nn;
      npw |= ((pw >> (4 * src)) & 15ull) << (4 * m);
    }
    pos64[i] = npw;
  }
}

__global__ void k_blk_max(const int* __restrict__ v, int64_t n, int* __restrict__ out) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b < n) atomicMax(out, v[b]);
}

// P2 triangles: the same fans at the vertex rows, and the one or two
// triangles of every edge-node row, as 32-bit records (layout in
// tg_internal.cuh).  Vertex row, fan triangle k between neighbours j_k and
// j_{k+1}: the positions of j_k, of the edge node between the row's node and
// j_k, and of the opposite edge node.  Edge row (the node on edge (u, w)),
// triangle k: the positions of its third vertex z and of its edge nodes on
// (w, z) and (z, u), with the swap bit when the triangle's own (u, w) runs
// the other way than the first triangle's.  The records come from the
// rows' incidence records (brec, two words: the six 5-bit positions of
// local nodes (a + c) mod 6, then a and the element's index in the block).
__global__ void k_fan_rows_p2(const int32_t* __restrict__ iinc, const int32_t* __restrict__ irp,
                              const uint32_t* __restrict__ brec, int64_t N, int R, uint32_t* __restrict__ info,
                              uint32_t* __restrict__ rec, int* __restrict__ kmax, int* __restrict__ bad) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int j0 = iinc[i], deg = iinc[i + 1] - j0, len = irp[i + 1] - irp[i];
  if (deg == 0) {
    info[i] = 0;
    return;
  }
  if (deg > kFanMax) {
    atomicOr(bad, 1);
    return;
  }
  uint8_t pos[kFanMax][6];
  int la[kFanMax], le[kFanMax];
  for (int m = 0; m < deg; ++m) {
    const uint32_t x = brec[2 * (j0 + m)], y = brec[2 * (j0 + m) + 1];
    la[m] = (int)(y & 7u);
    le[m] = (int)(y >> 3);
    for (int c = 0; c < 6; ++c) pos[m][(la[m] + c) % 6] = (uint8_t)((x >> (5 * c)) & 31u);
    if (le[m] >= 2048 || (la[m] < 3) != (la[0] < 3)) {
      atomicOr(bad, 1);
      return;
    }
  }
  const int dpos = pos[0][la[0]];
  if (la[0] >= 3) {  // edge node: one or two triangles
    const int a0 = la[0] - 3, u = pos[0][a0], w = pos[0][(a0 + 1) % 3];
    if (deg > 2 || len != 3 + 3 * deg) {
      atomicOr(bad, 1);
      return;
    }
    for (int m = 0; m < deg; ++m) {
      const int a = la[m] - 3, uT = pos[m][a], wT = pos[m][(a + 1) % 3];
      const bool swap = uT != u;
      if (swap ? (uT != w || wT != u) : (wT != w)) {
        atomicOr(bad, 1);
        return;
      }
      rec[i * kFanMax + m] = (uint32_t)le[m] | ((uint32_t)la[m] << 11) | ((swap ? 1u : 0u) << 14) |
                             ((uint32_t)pos[m][(a + 2) % 3] << 15) | ((uint32_t)pos[m][3 + (a + 1) % 3] << 20) |
                             ((uint32_t)pos[m][3 + (a + 2) % 3] << 25);
    }
    info[i] = (uint32_t)deg | 32u | ((uint32_t)dpos << 7) | ((uint32_t)u << 12) | ((uint32_t)w << 17);
    atomicMax(kmax + i / R, deg);
    return;
  }
  // vertex node: walk the fan over the vertex neighbours' positions
  int cnt[32];
  for (int q = 0; q < 32; ++q) cnt[q] = 0;
  for (int m = 0; m < deg; ++m) {
    cnt[pos[m][(la[m] + 1) % 3]]++;
    cnt[pos[m][(la[m] + 2) % 3]]++;
  }
  int start = 0, prev = pos[0][(la[0] + 1) % 3];
  bool open = false;
  for (int q = 0; q < 32; ++q) {
    if (cnt[q] > 2) {
      atomicOr(bad, 1);
      return;
    }
    if (cnt[q] == 1 && !open) {
      for (int m = 0; m < deg; ++m)
        if (pos[m][(la[m] + 1) % 3] == q || pos[m][(la[m] + 2) % 3] == q) {
          start = m;
          break;
        }
      prev = q;
      open = true;
    }
  }
  unsigned used = 0;
  int m = start, k = 0, next = -1, next_e = -1, first = prev;
  while (true) {
    used |= 1u << m;
    const int a = la[m], v1 = pos[m][(a + 1) % 3], v2 = pos[m][(a + 2) % 3];
    const int e1 = pos[m][3 + a], e2 = pos[m][3 + (a + 2) % 3], op = pos[m][3 + (a + 1) % 3];
    const bool swap = prev == v2;
    next = swap ? v1 : v2;
    next_e = swap ? e1 : e2;
    rec[i * kFanMax + k] = (uint32_t)le[m] | ((uint32_t)a << 11) | ((swap ? 1u : 0u) << 14) | ((uint32_t)prev << 15) |
                           ((uint32_t)(swap ? e2 : e1) << 20) | ((uint32_t)op << 25);
    ++k;
    int nm = -1;
    for (int q = 0; q < deg; ++q)
      if (!((used >> q) & 1u) && (pos[q][(la[q] + 1) % 3] == next || pos[q][(la[q] + 2) % 3] == next)) {
        nm = q;
        break;
      }
    if (nm < 0) break;
    prev = next;
    m = nm;
  }
  const int nn = open ? deg + 1 : deg;
  if (k != deg || (!open && next != first) || len != 1 + 2 * nn + deg) {
    atomicOr(bad, 1);
    return;
  }
  info[i] = (uint32_t)deg | (open ? 64u : 0u) | ((uint32_t)dpos << 7) |
            (open ? (((uint32_t)next << 12) | ((uint32_t)next_e << 17)) : 0u);
  atomicMax(kmax + i / R, deg);
}

// Fan starts of the closed vertex fans of a P2 pattern, chosen as in
// k_fan_rotate (rotations only: a record carries its first neighbour's
// positions, which a reversal would change).
__global__ void k_fan_rotate_p2(const uint32_t* __restrict__ info, uint32_t* __restrict__ rec, int64_t N, int R) {
  const int64_t qid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int nq = (R + 7) / 8;
  const int64_t b = qid / nq;
  const int q = (int)(qid % nq);
  const int64_t i0 = b * R + 8 * q;
  if (i0 >= N || 8 * q >= R) return;
  unsigned char used[kFanMax][8];
  for (int k = 0; k < kFanMax; ++k)
    for (int g = 0; g < 8; ++g) used[k][g] = 0;
  for (int t = 0; t < 8 && 8 * q + t < R && i0 + t < N; ++t) {
    const int64_t i = i0 + t;
    const int deg = (int)(info[i] & 31u);
    uint32_t r0[kFanMax];
    for (int k = 0; k < deg; ++k) r0[k] = rec[i * kFanMax + k];
    const bool fixed = (info[i] & (32u | 64u)) != 0u;  // edge rows and open fans keep their order
    const int nrot = fixed || deg == 0 ? 1 : deg;
    int best = 0, best_cost = 1 << 30;
    for (int rot = 0; rot < nrot; ++rot) {
      int cost = 0;
      for (int m = 0; m < deg; ++m) cost += used[m][r0[(rot + m) % deg] & 7u];
      if (cost < best_cost) {
        best_cost = cost;
        best = rot;
      }
    }
    for (int m = 0; m < deg; ++m) {
      const uint32_t r = r0[(best + m) % deg];
      rec[i * kFanMax + m] = r;
      used[m][r & 7u]++;
    }
  }
}

// Scatter the P2 rows' fan data into the blocks' regions: info (32 bits per
// row) then the records [k][t] (32 bits each), both padded to rs rows.
__global__ void k_fan_place_p2(const uint32_t* __restrict__ info, const uint32_t* __restrict__ rec,
                               const int64_t* __restrict__ off, const int* __restrict__ kmax, int64_t N, int R, int rs,
                               int64_t nblk, uint16_t* __restrict__ fan) {
  const int64_t b = blockIdx.x;
  if (b >= nblk) return;
  uint32_t* g = reinterpret_cast<uint32_t*>(fan + off[b]);
  const int kb = kmax[b];
  for (int t = threadIdx.x; t < rs; t += blockDim.x) {
    const int64_t i = b * R + t;
    const bool live = t < R && i < N;
    const uint32_t inf = live ? info[i] : 0u;
    g[t] = inf;
    const int d = (int)(inf & 31u);
    for (int k = 0; k < kb; ++k) g[(1 + k) * rs + t] = k < d ? rec[i * kFanMax + k] : 0u;
  }
}

// Region words of block b: (5 + kmax) * rs.
__global__ void k_fan_words(const int* __restrict__ kmax, int64_t nblk, int rs, int32_t* __restrict__ words) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b < nblk) words[b] = (5 + kmax[b]) * rs;
}

// Scatter the rows' fan data into the blocks' regions (layout in
// tg_internal.cuh); rows past the end of the last block and fan steps past
// a row's deg are zero (a zero record is never read).
__global__ void k_fan_place(const uint16_t* __restrict__ info, const unsigned long long* __restrict__ pos64,
                            const uint16_t* __restrict__ rec, const int64_t* __restrict__ off,
                            const int* __restrict__ kmax, int64_t N, int R, int rs, int64_t nblk,
                            uint16_t* __restrict__ fan) {
  const int64_t b = blockIdx.x;
  if (b >= nblk) return;
  uint16_t* g = fan + off[b];
  const int kb = kmax[b];
  for (int t = threadIdx.x; t < rs; t += blockDim.x) {
    const int64_t i = b * R + t;
    const bool live = t < R && i < N;
    const unsigned long long pw = live ? pos64[i] : 0ull;
    for (int q = 0; q < 4; ++q) g[4 * t + q] = (uint16_t)(pw >> (16 * q));
    g[4 * rs + t] = live ? info[i] : (uint16_t)0;
    const int d = live ? (info[i] & 31) : 0;
    for (int k = 0; k < kb; ++k) g[(5 + k) * rs + t] = k < d ? rec[i * kFanMax + k] : (uint16_t)0;
  }
}

// Device buffers freed on scope exit unless released.
struct Tmp {
  std::vector<void*> bufs;
  ~Tmp() {
    for (void* b : bufs) cudaFree(b);
  }
  template <typename T>
  cudaError_t alloc(T** p, size_t n) {
    cudaError_t e = cudaMalloc((void**)p, n * sizeof(T) + 16);
    if (e == cudaSuccess) bufs.push_back(*p);
    return e;
  }
};

// out[0..n] = exclusive prefix sums of in[0..n), out[n] = total.
template <typename Tin>
tg_status scan_exclusive(const Tin* in, int64_t* out, int64_t n, cudaStream_t s) {
  Tmp tmp;
  const int64_t tiles = n > 0 ? (n + kScanTile - 1) / kScanTile : 0;
  if (tiles == 0) {
    TG_CK(cudaMemsetAsync(out, 0, sizeof(int64_t), s));
    return TG_OK;
  }
  int64_t* sums = nullptr;
  TG_CK(tmp.alloc(&sums, tiles));
  k_scan_tile<Tin><<<(unsigned)tiles, kScanThreads, 0, s>>>(in, out, sums, n);
  TG_CK_LAUNCH("k_scan_tile");
  if (tiles == 1) {
    TG_CK(cudaMemcpyAsync(out + n, sums, sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
    return TG_OK;
  }
  int64_t* offs = nullptr;
  TG_CK(tmp.alloc(&offs, tiles + 1));
  tg_status st = scan_exclusive<int64_t>(sums, offs, tiles, s);
  if (st != TG_OK) return st;
  k_scan_add<<<tg::grid_for(n, kThreads), kThreads, 0, s>>>(out, offs, n);
  TG_CK_LAUNCH("k_scan_add");
  TG_CK(cudaMemcpyAsync(out + n, offs + tiles, sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
  TG_CK(cudaStreamSynchronize(s));  // tmp buffers are freed on return
  return TG_OK;
}

tg_status read_status(const tg_pattern* p, cudaStream_t s, const char* stage) {
  unsigned long long h[2];
  TG_CK(cudaMemcpyAsync(h, p->status, sizeof(h), cudaMemcpyDeviceToHost, s));
  TG_CK(cudaStreamSynchronize(s));
  if (h[0] != 0) {
    char buf[160];
    std::snprintf(buf, sizeof(buf), "%s: %s at element %llu", stage, tg_status_string((tg_status)h[0]), h[1]);
    tg::set_error(buf);
    return (tg_status)h[0];
  }
  return TG_OK;
}


// Rows per block of the element-once kernels.
// Rows per block.  Triangles: 120 rows of a strip of a numbered mesh touch
// about 4 * 120 + 2 distinct elements, one Map round of 4 per thread on 128
// threads.  Tetrahedra touch about 18 distinct elements per row; vector
// elasticity keeps 12 values per element in shared memory, hence 32 rows.
int blk_rows_of(tg_element el) {
  return el == TG_P1_TRI ? 120 : el == TG_P2_TRI ? 128 : 64;
}

// Region words of block b of a P2 pattern: (2 + 2 kmax) * rs (32-bit entries).
__global__ void k_fan_words_p2(const int* __restrict__ kmax, int64_t nblk, int rs, int32_t* __restrict__ words) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b < nblk) words[b] = (2 + 2 * kmax[b]) * rs;
}

tg_status build_fans_p2(tg_pattern* p, cudaStream_t s) {
  const int R = p->blk_rows, rs = (R + 7) & ~7;
  const int64_t N = p->N, nblk = p->n_blk;
  Tmp tmp;
  uint32_t *info = nullptr, *rec = nullptr;
  int *kmax = nullptr, *bad = nullptr;
  int32_t* words = nullptr;
  TG_CK(tmp.alloc(&info, N));
  TG_CK(tmp.alloc(&rec, N * kFanMax));
  TG_CK(tmp.alloc(&kmax, nblk));
  TG_CK(tmp.alloc(&bad, 1));
  TG_CK(tmp.alloc(&words, nblk));
  TG_CK(cudaMemsetAsync(kmax, 0, nblk * sizeof(int), s));
  TG_CK(cudaMemsetAsync(bad, 0, sizeof(int), s));
  k_fan_rows_p2<<<tg::grid_for(N, kThreads), kThreads, 0, s>>>(p->iinc, p->irp, p->brec, N, R, info, rec, kmax, bad);
  TG_CK_LAUNCH("k_fan_rows_p2");
  int hb = 0;
  TG_CK(cudaMemcpyAsync(&hb, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
  TG_CK(cudaStreamSynchronize(s));
  if (hb) return TG_OK;
  k_fan_rotate_p2<<<tg::grid_for(nblk * ((R + 7) / 8), 64), 64, 0, s>>>(info, rec, N, R);
  TG_CK_LAUNCH("k_fan_rotate_p2");
  k_fan_words_p2<<<tg::grid_for(nblk, kThreads), kThreads, 0, s>>>(kmax, nblk, rs, words);
  TG_CK_LAUNCH("k_fan_words_p2");
  TG_CK(cudaMalloc(&p->fan_off, (nblk + 1) * sizeof(int64_t) + 16));
  tg_status st = scan_exclusive<int32_t>(words, p->fan_off, nblk, s);
  if (st != TG_OK) return st;
  int* kmax_all = bad;  // reuse
  TG_CK(cudaMemsetAsync(kmax_all, 0, sizeof(int), s));
  k_blk_max<<<tg::grid_for(nblk, kThreads), kThreads, 0, s>>>(kmax, nblk, kmax_all);
  TG_CK_LAUNCH("k_blk_max");
  int64_t total = 0;
  int hk = 0;
  TG_CK(cudaMemcpyAsync(&total, p->fan_off + nblk, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  TG_CK(cudaMemcpyAsync(&hk, kmax_all, sizeof(int), cudaMemcpyDeviceToHost, s));
  TG_CK(cudaStreamSynchronize(s));
  TG_CK(cudaMalloc(&p->fan, total * sizeof(uint16_t) + 16));
  k_fan_place_p2<<<(unsigned)nblk, 128, 0, s>>>(info, rec, p->fan_off, kmax, N, R, rs, nblk, p->fan);
  TG_CK_LAUNCH("k_fan_place_p2");
  TG_CK(cudaStreamSynchronize(s));  // tmp buffers are freed on return
  p->fan_rs = rs;
  p->fan_kmax = hk;
  p->fan_maxw = (2 + 2 * hk) * rs;
  return TG_OK;
}

// Fans of a P1 triangle pattern with row blocks; leaves p->fan == NULL when
// some node's triangles are not one fan.
tg_status build_fans(tg_pattern* p, cudaStream_t s) {
  const int R = p->blk_rows, rs = (R + 7) & ~7;
  const int64_t N = p->N, nblk = p->n_blk;
  Tmp tmp;
  uint16_t *info = nullptr, *rec = nullptr;
  unsigned long long* pos64 = nullptr;
  int *kmax = nullptr, *bad = nullptr;
  int32_t* words = nullptr;
  int64_t* off = nullptr;
  TG_CK(tmp.alloc(&info, N));
  TG_CK(tmp.alloc(&rec, N * kFanMax));
  TG_CK(tmp.alloc(&pos64, N));
  TG_CK(tmp.alloc(&kmax, nblk));
  TG_CK(tmp.alloc(&bad, 1));
  TG_CK(tmp.alloc(&words, nblk));
  TG_CK(cudaMemsetAsync(kmax, 0, nblk * sizeof(int), s));
  TG_CK(cudaMemsetAsync(bad, 0, sizeof(int), s));
  k_fan_rows<<<tg::grid_for(N, kThreads), kThreads, 0, s>>>(p->iinc, p->irp, p->brec, N, R, info, pos64, rec, kmax,
                                                            bad);
  TG_CK_LAUNCH("k_fan_rows");
  int hb = 0;
  TG_CK(cudaMemcpyAsync(&hb, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
  TG_CK(cudaStreamSynchronize(s));
  if (hb) return TG_OK;
  const int64_t nphase = nblk * ((R + 7) / 8);
  k_fan_rotate<<<tg::grid_for(nphase, 64), 64, 0, s>>>(info, pos64, rec, N, R);
  TG_CK_LAUNCH("k_fan_rotate");
  k_fan_words<<<tg::grid_for(nblk, kThreads), kThreads, 0, s>>>(kmax, nblk, rs, words);
  TG_CK_LAUNCH("k_fan_words");
  TG_CK(cudaMalloc(&p->fan_off, (nblk + 1) * sizeof(int64_t) + 16));
  tg_status st = scan_exclusive<int32_t>(words, p->fan_off, nblk, s);
  if (st != TG_OK) return st;
  int64_t total = 0;
  int* kmax_all = bad;  // reuse
  TG_CK(cudaMemsetAsync(kmax_all, 0, sizeof(int), s));
  k_blk_max<<<tg::grid_for(nblk, kThreads), kThreads, 0, s>>>(kmax, nblk, kmax_all);
  TG_CK_LAUNCH("k_blk_max");
  int hk = 0;
  TG_CK(cudaMemcpyAsync(&total, p->fan_off + nblk, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  TG_CK(cudaMemcpyAsync(&hk, kmax_all, sizeof(int), cudaMemcpyDeviceToHost, s));
  TG_CK(cudaStreamSynchronize(s));
  TG_CK(cudaMalloc(&p->fan, total * sizeof(uint16_t) + 16));
  k_fan_place<<<(unsigned)nblk, 128, 0, s>>>(info, pos64, rec, p->fan_off, kmax, N, R, rs, nblk, p->fan);
  TG_CK_LAUNCH("k_fan_place");
  TG_CK(cudaStreamSynchronize(s));  // tmp buffers are freed on return
  p->fan_rs = rs;
  p->fan_kmax = hk;
  p->fan_maxw = (5 + hk) * rs;
  return TG_OK;
}

// Row blocks (step 5).  Leaves p->bel == NULL when the packed fields do not
// fit (rows longer than 16, too many distinct elements per block): the
// generic kernels are used then.
tg_status build_blocks(tg_pattern* p, cudaStream_t s) {
  const int nv = p->nv, R = blk_rows_of(p->el);
  const int64_t N = p->N, E = p->E, nvE = E * nv, nblk = (N + R - 1) / R;
  // positions: 4 bits in 32-bit records (nv <= 4), 5 bits in 64-bit records
  // (P2: word 0 the six positions, word 1 the local vertex and element)
  const bool wide_rec = nv > 4;
  const int pb = wide_rec ? 5 : 4;
  if (p->max_row_len > (1 << pb)) return TG_OK;
  const int le_bits = wide_rec ? 29 : 32 - nv * pb - 2;
  Tmp tmp;
  // internal row order: nodes by smallest incident element, isolated nodes
  // last, each block of R rows in ascending node id
  int32_t *key = nullptr, *iso = nullptr, *cnt_e = nullptr, *order = nullptr, *ipos = nullptr;
  int64_t *off = nullptr, *iso_rank = nullptr, *tmp64 = nullptr;
  TG_CK(tmp.alloc(&key, N));
  TG_CK(tmp.alloc(&iso, N));
  TG_CK(tmp.alloc(&cnt_e, E));
  TG_CK(tmp.alloc(&order, N));
  TG_CK(tmp.alloc(&ipos, N));
  TG_CK(tmp.alloc(&off, E + 1));
  TG_CK(tmp.alloc(&iso_rank, N + 1));
  TG_CK(tmp.alloc(&tmp64, N + 1));
  k_row_key<<<tg::grid_for(N, kThreads), kThreads, 0, s>>>(p->inc_ptr, p->inc_e, N, E, key, iso);
  k_key_count<<<tg::grid_for(E, kThreads), kThreads, 0, s>>>(p->cells, nv, E, key, cnt_e);
  TG_CK_LAUNCH("k_key_count");
  tg_status st = scan_exclusive<int32_t>(cnt_e, off, E, s);
  if (st != TG_OK) return st;
  k_key_place<<<tg::grid_for(E, kThreads), kThreads, 0, s>>>(p->cells, nv, E, key, off, order);
  TG_CK_LAUNCH("k_key_place");
  if ((st = scan_exclusive<int32_t>(iso, iso_rank, N, s)) != TG_OK) return st;
  int64_t base = 0;
  TG_CK(cudaMemcpyAsync(&base, off + E, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  TG_CK(cudaStreamSynchronize(s));
  k_iso_place<<<tg::grid_for(N, kThreads), kThreads, 0, s>>>(iso, iso_rank, N, base, order);
  TG_CK_LAUNCH("k_iso_place");
  TG_CK(cudaMalloc(&p->iperm, N * sizeof(int32_t) + 16));
  TG_CK(cudaMalloc(&p->urp, N * sizeof(int32_t) + 16));
  TG_CK(cudaMalloc(&p->iinc, (N + 1) * sizeof(int32_t) + 16));
  TG_CK(cudaMalloc(&p->irp, (N + 1) * sizeof(int32_t) + 16));
  k_blk_sort<<<(unsigned)nblk, 128, 0, s>>>(order, N, R, p->iperm, ipos);
  TG_CK_LAUNCH("k_blk_sort");
  int32_t *deg_i = key, *len_i = iso;  // reuse
  k_irow<<<tg::grid_for(N, kThreads), kThreads, 0, s>>>(p->iperm, p->inc_ptr, p->row_ptr, N, deg_i, len_i, p->urp);
  TG_CK_LAUNCH("k_irow");
  if ((st = scan_exclusive<int32_t>(deg_i, tmp64, N, s)) != TG_OK) return st;
  k_narrow<<<tg::grid_for(N + 1, kThreads), kThreads, 0, s>>>(tmp64, p->iinc, N + 1);
  TG_CK_LAUNCH("k_narrow");
  if ((st = scan_exclusive<int32_t>(len_i, tmp64, N, s)) != TG_OK) return st;
  k_narrow<<<tg::grid_for(N + 1, kThreads), kThreads, 0, s>>>(tmp64, p->irp, N + 1);
  TG_CK_LAUNCH("k_narrow");
  int* maxes = nullptr;
  TG_CK(tmp.alloc(&maxes, 3));
  TG_CK(cudaMemsetAsync(maxes, 0, 3 * sizeof(int), s));
  k_blk_stats<<<tg::grid_for(nblk, kThreads), kThreads, 0, s>>>(p->iinc, p->irp, N, R, nblk, maxes);
  TG_CK_LAUNCH("k_blk_stats");
  int h[3];
  TG_CK(cudaMemcpyAsync(h, maxes, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
  TG_CK(cudaStreamSynchronize(s));
  int P = 1;
  while (P < h[0]) P <<= 1;
  if (P > 4096) return TG_OK;  // blocks of very high degree
  int32_t* uq = nullptr;
  int32_t* cnt = nullptr;
  int64_t* boff = nullptr;
  TG_CK(tmp.alloc(&uq, nvE));
  TG_CK(tmp.alloc(&boff, nblk + 1));
  TG_CK(cudaMalloc(&cnt, nblk * sizeof(int32_t) + 16));
  p->bel_cnt = cnt;  // owned by the pattern from here on
  const size_t rec_bytes = nvE * sizeof(uint32_t) * (wide_rec ? 2 : 1) + 16;
  TG_CK(cudaMalloc(&p->brec, rec_bytes));
  TG_CK(cudaMemsetAsync(p->brec, 0, rec_bytes, s));
  k_blocks<<<(unsigned)nblk, 256, 2 * P * sizeof(int), s>>>(p->iperm, p->iinc, p->inc_ptr, p->inc_e, p->inc_pos, nv,
                                                             N, R, P, uq, cnt, p->brec, maxes + 2);
  TG_CK_LAUNCH("k_blocks");
  TG_CK(cudaMemcpyAsync(h + 2, maxes + 2, sizeof(int), cudaMemcpyDeviceToHost, s));
  TG_CK(cudaStreamSynchronize(s));
  if (h[2] > (1 << le_bits)) return TG_OK;  // local element indices do not fit
  // region sizes (nv + 1) * padded count -> word offsets
  int32_t* words = nullptr;
  TG_CK(tmp.alloc(&words, nblk));
  k_bel_words<<<tg::grid_for(nblk, kThreads), kThreads, 0, s>>>(cnt, nblk, nv, words);
  TG_CK_LAUNCH("k_bel_words");
  if ((st = scan_exclusive<int32_t>(words, boff, nblk, s)) != TG_OK) return st;
  int64_t total = 0;
  TG_CK(cudaMemcpyAsync(&total, boff + nblk, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  TG_CK(cudaStreamSynchronize(s));
  TG_CK(cudaMalloc(&p->bel, total * sizeof(uint32_t) + 16));
  TG_CK(cudaMalloc(&p->boff, (nblk + 1) * sizeof(int64_t) + 16));
  TG_CK(cudaMalloc(&p->bvbase, nblk * sizeof(int32_t) + 16));
  TG_CK(cudaMemcpyAsync(p->boff, boff, (nblk + 1) * sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
  int* wide = maxes;  // reuse: maxima already read back
  TG_CK(cudaMemsetAsync(wide, 0, sizeof(int), s));
  const unsigned gx = (unsigned)std::min<int64_t>(nblk, 65535), gy = (unsigned)((nblk + gx - 1) / gx);
  k_bel<<<dim3(gx, gy), 128, 0, s>>>(p->cells, nv, p->iinc, ipos, uq, cnt, p->boff, N, R, nblk, p->bel, p->bvbase,
                                      wide);
  TG_CK_LAUNCH("k_bel");
  int hw = 0;
  TG_CK(cudaMemcpyAsync(&hw, wide, sizeof(int), cudaMemcpyDeviceToHost, s));
  TG_CK(cudaStreamSynchronize(s));
  if (hw) {  // vertex ids of some block span 2^16 or more: no blocks
    cudaFree(p->bel);
    cudaFree(p->boff);
    cudaFree(p->bvbase);
    p->bel = nullptr;
    p->boff = nullptr;
    p->bvbase = nullptr;
    return TG_OK;
  }
  p->blk_rows = R;
  p->blk_pb = pb;
  p->n_blk = nblk;
  p->blk_max_inc = h[0];
  p->blk_max_nz = h[1];
  p->blk_max_elems = h[2];
  if (p->el == TG_P1_TRI && h[2] <= 2048 && (st = build_fans(p, s)) != TG_OK) return st;
  if (p->el == TG_P2_TRI && h[2] <= 2048 && (st = build_fans_p2(p, s)) != TG_OK) return st;
  if (nv * nv * pb <= 64) {
    TG_CK(cudaMalloc(&p->elem_pos, E * sizeof(uint64_t) + 16));
    k_elem_pos<<<tg::grid_for(E, kThreads), kThreads, 0, s>>>(p->cells, p->elem_slot, p->row_ptr, E, nv, pb, false,
                                                              p->elem_pos);
    TG_CK_LAUNCH("k_elem_pos");
  }
  TG_CK(cudaStreamSynchronize(s));  // tmp buffers are freed on return
  return TG_OK;
}

}  // namespace

extern "C" tg_status tg_build_pattern(const int32_t* cells, int64_t n_elems, int64_t n_nodes, tg_element el,
                                      tg_stream stream, tg_pattern** out) {
  if (!out) return TG_ERR_INVALID_ARG;
  *out = nullptr;
  if (el < TG_P1_TRI || el > TG_Q1_QUAD_VEC2 || n_elems < 0 || n_nodes < 1) return TG_ERR_INVALID_ARG;
  if (n_elems > 0 && !cells) return TG_ERR_INVALID_ARG;
  const int nv = tg::nv_of(el);
  if (n_nodes > INT32_MAX || n_elems >= (1ll << 28) || n_elems * nv > INT32_MAX) return TG_ERR_INDEX_OVERFLOW;
  cudaStream_t s = (cudaStream_t)stream;

  tg_pattern* p = new tg_pattern;
  p->el = el;
  p->nv = nv;
  p->dim = tg::dim_of(el);
  p->nq = tg::nq_of(el);
  p->ngeo = el == TG_P2_TRI ? 3 : nv;
  p->npw = nv > 4 ? 2 : 1;
  p->E = n_elems;
  p->N = n_nodes;
  struct Guard {
    tg_pattern*& p;
    bool ok = false;
    ~Guard() {
      if (!ok) tg_pattern_destroy(p);
    }
  } guard{p};
  Tmp tmp;
  const int64_t E = n_elems, N = n_nodes, nvE = n_elems * nv;

  cudaError_t ce = cudaGetDevice(&p->device);
  if (ce != cudaSuccess) return tg::cuda_fail(ce, "cudaGetDevice", __FILE__, __LINE__);
  TG_CK(cudaMalloc(&p->status, 2 * sizeof(unsigned long long)));
  const unsigned long long init[2] = {0ull, ~0ull};
  TG_CK(cudaMemcpyAsync(p->status, init, sizeof(init), cudaMemcpyHostToDevice, s));
  TG_CK(cudaMalloc(&p->cells, nvE * sizeof(int32_t) + 16));
  if (nvE) TG_CK(cudaMemcpyAsync(p->cells, cells, nvE * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));

  // 1. validation and incidence counts
  int32_t* deg = nullptr;
  TG_CK(tmp.alloc(&deg, N));
  TG_CK(cudaMemsetAsync(deg, 0, N * sizeof(int32_t), s));
  const int sms = tg::sm_count();
  const int gE = (int)std::min<int64_t>(std::max<int64_t>(tg::grid_for(E, kThreads), 1), 16ll * sms);
  if (E > 0) {
    k_count<<<gE, kThreads, 0, s>>>(p->cells, E, nv, N, deg, p->status);
    TG_CK_LAUNCH("k_count");
  }
  tg_status st = read_status(p, s, "tg_build_pattern");
  if (st != TG_OK) return st;

  // 2. incidence lists
  int64_t* tmp64 = nullptr;
  TG_CK(tmp.alloc(&tmp64, N + 1));
  if ((st = scan_exclusive<int32_t>(deg, tmp64, N, s)) != TG_OK) return st;
  TG_CK(cudaMalloc(&p->inc_ptr, (N + 1) * sizeof(int32_t) + 16));
  k_narrow<<<tg::grid_for(N + 1, kThreads), kThreads, 0, s>>>(tmp64, p->inc_ptr, N + 1);
  TG_CK_LAUNCH("k_narrow");
  TG_CK(cudaMalloc(&p->inc_e, nvE * sizeof(int32_t) + 16));
  int32_t* cursor = deg;  // reuse: cursor starts at inc_ptr
  TG_CK(cudaMemcpyAsync(cursor, p->inc_ptr, N * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
  if (E > 0) {
    k_fill<<<gE, kThreads, 0, s>>>(p->cells, E, nv, cursor, p->inc_e);
    TG_CK_LAUNCH("k_fill");
  }
  k_sort_incidence<<<tg::grid_for(N, kThreads), kThreads, 0, s>>>(p->inc_ptr, p->inc_e, N);
  TG_CK_LAUNCH("k_sort_incidence");

  // 3. rows
  int32_t* row_len = nullptr;
  int* maxes = nullptr;
  TG_CK(tmp.alloc(&row_len, N));
  TG_CK(tmp.alloc(&maxes, 2));
  TG_CK(cudaMemsetAsync(maxes, 0, 2 * sizeof(int), s));
  const int nc = tg::ncomp_of(el);
  k_rows<false><<<tg::grid_for(N, 128), 128, 0, s>>>(p->cells, p->inc_ptr, p->inc_e, N, nv, p->npw, nc, row_len,
                                                      maxes, nullptr, nullptr, nullptr, nullptr, p->status);
  TG_CK_LAUNCH("k_rows<false>");
  int hmax[2];
  TG_CK(cudaMemcpyAsync(hmax, maxes, sizeof(hmax), cudaMemcpyDeviceToHost, s));
  if ((st = read_status(p, s, "tg_build_pattern (row longer than 255)")) != TG_OK) return st;
  p->max_row_len = hmax[0];
  p->max_deg = hmax[1];
  if ((st = scan_exclusive<int32_t>(row_len, tmp64, N, s)) != TG_OK) return st;
  int64_t nnz = 0;
  TG_CK(cudaMemcpyAsync(&nnz, tmp64 + N, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  TG_CK(cudaStreamSynchronize(s));
  if ((int64_t)nc * nc * nnz > INT32_MAX) {
    tg::set_error("tg_build_pattern: nnz exceeds int32 indices");
    return TG_ERR_INDEX_OVERFLOW;
  }
  p->nnz = nnz;
  TG_CK(cudaMalloc(&p->row_ptr, (N + 1) * sizeof(int32_t) + 16));
  k_narrow<<<tg::grid_for(N + 1, kThreads), kThreads, 0, s>>>(tmp64, p->row_ptr, N + 1);
  TG_CK_LAUNCH("k_narrow");

  // 4. columns, positions, element-to-slot map
  TG_CK(cudaMalloc(&p->col_idx, nnz * sizeof(int32_t) + 16));
  TG_CK(cudaMalloc(&p->inc_pos, nvE * p->npw * sizeof(uint32_t) + 16));
  TG_CK(cudaMalloc(&p->elem_slot, nvE * nv * sizeof(int32_t) + 16));
  k_rows<true><<<tg::grid_for(N, 128), 128, 0, s>>>(p->cells, p->inc_ptr, p->inc_e, N, nv, p->npw, nc, nullptr,
                                                     nullptr, p->row_ptr, p->col_idx, p->inc_pos, p->elem_slot,
                                                     p->status);
  TG_CK_LAUNCH("k_rows<true>");


  // 5. row blocks of the element-once kernels (not for the vector kinds:
  // the plane-stress and elasticity kernels work per node row and per
  // element)
  if (E > 0 && nc == 1) {
    if ((st = build_blocks(p, s)) != TG_OK) return st;
  }

  // 6. DoF-level CSR for elasticity
  // packed positions of the elasticity backward (4-bit fields: rows of at
  // most 16 nodes); it reads the 32-bit slot map otherwise
  if (el == TG_P1_TET_VEC3 && E > 0 && p->max_row_len <= 16 && p->max_deg <= 32) {
    TG_CK(cudaMalloc(&p->emask, nnz * sizeof(uint32_t) + 16));
    k_edge_masks<<<tg::grid_for(N, kThreads), kThreads, 0, s>>>(p->inc_ptr, p->inc_e, p->inc_pos, p->row_ptr, N,
                                                                p->emask);
    TG_CK_LAUNCH("k_edge_masks");
  }
  if (el == TG_P1_TET_VEC3 && E > 0 && p->max_row_len <= 16) {
    TG_CK(cudaMalloc(&p->elem_pos, E * sizeof(uint64_t) + 16));
    k_elem_pos<<<tg::grid_for(E, kThreads), kThreads, 0, s>>>(p->cells, p->elem_slot, p->row_ptr, E, nv, 4, true,
                                                              p->elem_pos);
    TG_CK_LAUNCH("k_elem_pos");
  }
  if (nc > 1) {
    TG_CK(cudaMalloc(&p->row_ptr_dof, (nc * N + 1) * sizeof(int32_t)));
    TG_CK(cudaMalloc(&p->col_idx_dof, (size_t)nc * nc * nnz * sizeof(int32_t) + 16));
    k_expand<<<tg::grid_for(N, kThreads), kThreads, 0, s>>>(p->row_ptr, p->col_idx, N, nc, p->row_ptr_dof,
                                                            p->col_idx_dof);
    TG_CK_LAUNCH("k_expand");
  }

  // per-CTA partials of the backward's global sums (4 values per CTA of at
  // least 32 rows)
  p->n_partials = 4 * ((N + 31) / 32) + 4;
  TG_CK(cudaMalloc(&p->partials, p->n_partials * sizeof(double)));
  TG_CK(cudaMalloc(&p->arrivals, 16));
  TG_CK(cudaMemsetAsync(p->arrivals, 0, 16, s));
  // per-element results of the two-pass kernels: nv * dim values per
  // element (for P1 at least the FP64 forward's K_e and F_e: 9 for
  // triangles, 14 for tetrahedra), 20 for vector elasticity (its forward's
  // geometry records)
  if ((nc == 1 || el == TG_P1_TET_VEC3) && E > 0) {
    const int per = nc != 1 ? 20 : el == TG_P1_TRI ? 9 : el == TG_P1_TET ? 14 : nv * tg::dim_of(el);
    TG_CK(cudaMalloc(&p->elem_scratch, (size_t)E * per * sizeof(double)));
  }
  TG_CK(cudaStreamSynchronize(s));
  if ((st = read_status(p, s, "tg_build_pattern")) != TG_OK) return st;
  guard.ok = true;
  *out = p;
  return TG_OK;
}
