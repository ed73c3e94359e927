// Fan-ordered Reduce of the element-once row blocks (P1 triangles).
//
// Around a mesh node the incident triangles form a fan: walked across the
// edges they share, triangle k lies between the row's neighbours j_k and
// j_{k+1} (a closed fan around an interior node, an open one at the
// boundary).  Every off-diagonal entry (i, j_k) of row i is then the sum of
// the entries of at most two consecutive triangles of the fan, k - 1 and k,
// and the diagonal the sum over all of them.  A thread owning row i walks its
// fan once, keeps the running entries in registers and writes each value as
// soon as both of its terms are known: Algorithm 2's Reduce without any
// shared-memory accumulator.  Sums of two terms do not depend on their order;
// the diagonal and the load entry are summed in fan order, fixed by the
// pattern, so every output is bitwise reproducible.
//
// The blocks are those of blocks.cuh (the same rows, element lists and
// Map); the per-incidence records and CSR row prefix sums are replaced by
// the block's fan region (tg_pattern::fan, layout in tg_internal.cuh), which
// the pipeline stages next to the rows' CSR starts, node ids and element
// list.
#pragma once

#include <cstdint>

#include "blk_bilinear.cuh"

namespace tg {

struct FanArgs {
  const int32_t* __restrict__ urp;    // CSR row start of each internal row
  const int32_t* __restrict__ iperm;  // node of each internal row
  const uint16_t* __restrict__ fan;
  const int64_t* __restrict__ fan_off;
  const uint32_t* __restrict__ bel;
  const int64_t* __restrict__ boff;
  const int32_t* __restrict__ bvbase;
  const int32_t* __restrict__ bel_cnt;
  int64_t N;
  int64_t nblocks;
  int capE;    // distinct elements per block (multiple of 8)
  int capE16;  // capE rounded up to a multiple of 8
  int nv;      // vertices per element (3)
  int R;       // rows per block
  int rs;      // R rounded up to a multiple of 8 (fan region row stride)
  int capF;    // largest fan region, in 16-bit words
};

// Host: FanArgs of a pattern with fans.
inline FanArgs fan_args(const tg_pattern* p) {
  FanArgs g;
  g.urp = p->urp;
  g.iperm = p->iperm;
  g.fan = p->fan;
  g.fan_off = p->fan_off;
  g.bel = p->bel;
  g.boff = p->boff;
  g.bvbase = p->bvbase;
  g.bel_cnt = p->bel_cnt;
  g.N = p->N;
  g.nblocks = p->n_blk;
  // a multiple of 8: the per-vertex row arrays of the Map then start in the
  // same bank group, the one the fans' starts were chosen for
  g.capE = (p->blk_max_elems + 7) & ~7;
  g.capE16 = (p->blk_max_elems + 7) & ~7;
  g.nv = p->nv;
  g.R = p->blk_rows;
  g.rs = p->fan_rs;
  g.capF = p->fan_maxw;
  return g;
}

// Shared-memory bytes of the two stages plus barriers and block metadata.
__host__ __device__ inline size_t fan_stage_bytes(int R, int capF, int capE, int nv) {
  const size_t el_words = (size_t)capE + (size_t)nv * (((capE + 7) & ~7) / 2);
  return 16 + 128 + 2 * ((size_t)(((R + 3) & ~3) + 8) * 8 + (size_t)capF * 2 + el_words * 4);
}

// One row block as seen through its stage (rows indexed locally, t = i - r0).
struct FanView {
  int r0, r1, nbe;
  int bs16;                   // row stride of vo
  int vbase;                  // smallest vertex id of the block's elements
  int rs;                     // fan region row stride
  const int* up;              // up[t]: CSR start of row t's node
  const int* pm;              // pm[t]: node of row t
  const unsigned long long* pos;  // pos[t]: neighbour positions in fan order, 4 bits each
  const uint16_t* info;       // info[t]: deg | open << 5 | diagonal position << 6
  const uint16_t* rec;        // rec[k * rs + t]: fan triangle k of row t
  const uint32_t* info32;     // P2: info32[t], rec32[k * rs + t] (32-bit layout)
  const uint32_t* rec32;
  const uint32_t* be;         // be[k]: element k (with the owner bit)
  const uint16_t* vo;         // vo[c * bs16 + k]: vertex c of element k, minus vbase
  __device__ int vtx(int c, int k) const { return vbase + (int)vo[c * bs16 + k]; }
};

// Fields of a fan record.
__device__ __forceinline__ int fan_le(unsigned r) { return (int)(r & 2047u); }
__device__ __forceinline__ int fan_a(unsigned r) { return (int)((r >> 11) & 3u); }
__device__ __forceinline__ bool fan_swap(unsigned r) { return ((r >> 13) & 1u) != 0u; }

// The view of block blk read straight from the pattern arrays in global
// memory (the batched kernel).
__device__ __forceinline__ FanView fan_view_global(const FanArgs& g, int64_t blk) {
  FanView v;
  const int64_t r0 = blk * g.R;
  v.r0 = (int)r0;
  v.r1 = (int)(r0 + g.R < g.N ? r0 + g.R : g.N);
  v.nbe = g.bel_cnt[blk];
  v.vbase = g.bvbase[blk];
  v.bs16 = (v.nbe + 7) & ~7;
  v.rs = g.rs;
  v.up = g.urp + r0;
  v.pm = g.iperm + r0;
  const uint16_t* f = g.fan + g.fan_off[blk];
  v.pos = reinterpret_cast<const unsigned long long*>(f);
  v.info = f + 4 * g.rs;
  v.rec = f + 5 * g.rs;
  v.info32 = reinterpret_cast<const uint32_t*>(f);
  v.rec32 = v.info32 + g.rs;
  v.be = g.bel + g.boff[blk];
  v.vo = reinterpret_cast<const uint16_t*>(v.be + ((v.nbe + 3) & ~3));
  return v;
}

class FanPipe {
 public:
  // Carves the stages out of shared memory at p (16-byte aligned); returns
  // the first byte after them.  Thread 0 initialises the barriers; the
  // caller's next CTA barrier publishes them.
  __device__ unsigned char* init(unsigned char* p, const FanArgs& g) {
    R_ = g.R;
    RN_ = ((R_ + 3) & ~3) + 8;
    FN_ = g.capF / 2;
    ELN_ = g.capE + g.nv * (g.capE16 / 2);
    SW_ = 2 * RN_ + FN_ + ELN_;  // words per stage (a multiple of 4)
    bar_ = reinterpret_cast<uint64_t*>(p);
    meta_ = reinterpret_cast<int*>(p + 16);
    st_ = reinterpret_cast<int*>(p + 16 + 128);
    if (threadIdx.x == 0) {
      mbar_init(&bar_[0], 1);
      mbar_init(&bar_[1], 1);
      fence_mbar_init();
    }
    return reinterpret_cast<unsigned char*>(st_ + 2 * SW_);
  }

  struct Peek {
    int nbe, vb;
    int64_t bo, f0, f1;
  };
  __device__ static void peek(const FanArgs& g, int64_t blk, Peek& q) {
    q.nbe = __ldg(g.bel_cnt + blk);
    q.bo = __ldg(g.boff + blk);
    q.vb = __ldg(g.bvbase + blk);
    q.f0 = __ldg(g.fan_off + blk);
    q.f1 = __ldg(g.fan_off + blk + 1);
  }

  // Thread 0: copy block blk's streams into stage s: the rows' CSR starts
  // and node ids (widened to whole 16-byte groups; the arrays carry 16 bytes
  // of tail padding), the fan region and the element list (16-byte aligned
  // regions of whole 16-byte groups).
  __device__ void issue(const FanArgs& g, int s, int64_t blk, const Peek& q) {
    const int r0 = (int)(blk * R_), r1 = (int)(blk * R_ + R_ < g.N ? blk * R_ + R_ : g.N);
    const int a0 = r0 & ~3, nup = (r1 - a0 + 3) & ~3;
    const int nf = (int)(q.f1 - q.f0);  // 16-bit words, a multiple of 8
    const int nel = ((q.nbe + 3) & ~3) + g.nv * (((q.nbe + 7) & ~7) / 2);
    int* m = meta_ + 16 * s;
    m[0] = r0;
    m[1] = r1;
    m[2] = r0 - a0;
    m[3] = q.nbe;
    m[4] = q.vb;
    const uint32_t bytes = 4u * (2u * nup + nel) + 2u * nf;
    fence_proxy_async();
    mbar_arrive_expect_tx(&bar_[s], bytes);
    bulk_copy_g2s(up(s), g.urp + a0, nup * 4, &bar_[s]);
    bulk_copy_g2s(pm(s), g.iperm + a0, nup * 4, &bar_[s]);
    if (nf > 0) bulk_copy_g2s(fr(s), g.fan + q.f0, nf * 2, &bar_[s]);
    if (nel > 0) bulk_copy_g2s(el(s), g.bel + q.bo, nel * 4, &bar_[s]);
  }

  // All threads: wait (bounded) for stage s of use k; the outcome is made
  // uniform across the CTA.  On failure thread 0 records TG_ERR_TIMEOUT and
  // waits, again bounded, for the copies it issued, and the CTA must return.
  __device__ bool wait(int s, int k, bool other_issued, unsigned long long* status) {
    const bool ok = mbar_wait(&bar_[s], (k >> 1) & 1);
    if (__syncthreads_or(!ok)) {
      if (threadIdx.x == 0) {
        record_error(status, TG_ERR_TIMEOUT, 0);
        mbar_wait(&bar_[s], (k >> 1) & 1);
        if (other_issued) mbar_wait(&bar_[s ^ 1], ((k + 1) >> 1) & 1);
      }
      return false;
    }
    return true;
  }

  __device__ FanView view(int s, int rs) const {
    const int* m = meta_ + 16 * s;
    FanView v;
    v.r0 = m[0];
    v.r1 = m[1];
    v.nbe = m[3];
    v.vbase = m[4];
    v.bs16 = (v.nbe + 7) & ~7;
    v.rs = rs;
    v.up = up(s) + m[2];
    v.pm = pm(s) + m[2];
    const uint16_t* f = reinterpret_cast<const uint16_t*>(fr(s));
    v.pos = reinterpret_cast<const unsigned long long*>(f);
    v.info = f + 4 * rs;
    v.rec = f + 5 * rs;
    v.info32 = reinterpret_cast<const uint32_t*>(f);
    v.rec32 = v.info32 + rs;
    v.be = el(s);
    v.vo = reinterpret_cast<const uint16_t*>(el(s) + ((v.nbe + 3) & ~3));
    return v;
  }

 private:
  // stage s: up [RN] | pm [RN] | fan region [FN] | el [ELN]
  __device__ int* up(int s) const { return st_ + s * SW_; }
  __device__ int* pm(int s) const { return up(s) + RN_; }
  __device__ int* fr(int s) const { return pm(s) + RN_; }
  __device__ uint32_t* el(int s) const { return reinterpret_cast<uint32_t*>(fr(s) + FN_); }

  int R_, RN_, FN_, ELN_, SW_;
  uint64_t* bar_;
  int* meta_;
  int* st_;
};

// Reduce of the bilinear form (and, with LOAD, the load vector) over the
// fans: thread t owns row t of the block.  KF holds the Map's output rows
// (blk_bilinear.cuh): row a of element le in rotated column order K[a][a],
// K[a][a+1], K[a][a+2] (then F_e[a]).  Fan triangle k contributes K[a][a] to
// the diagonal, its entry of neighbour j_k to that neighbour's value (with
// the previous triangle's) and its entry of j_{k+1} to the next one.
template <typename T, bool LOAD>
__device__ __forceinline__ void fan_reduce_bilinear(const FwdArgs<T>& a, int capE, const FanView& v,
                                                    const void* kf_buf) {
  constexpr int NW = kf_vecs<3, T, LOAD>(), VN = Vec16<T>::n;
  using V = typename Vec16<T>::type;
  const V* KF = reinterpret_cast<const V*>(kf_buf);
  const int t = (int)threadIdx.x;
  if (v.r0 + t >= v.r1) return;
  const unsigned inf = v.info[t];
  const int deg = (int)(inf & 31u);
  T fs = T(0);
  if (deg > 0) {
    const unsigned long long pw = v.pos[t];
    T* out = a.out + v.up[t];
    T diag = T(0), first = T(0), carry = T(0);
    for (int k = 0; k < deg; ++k) {
      const unsigned r = v.rec[k * v.rs + t];
      const V* src = KF + fan_a(r) * NW * capE + fan_le(r);
      V x[NW];
#pragma unroll
      for (int w = 0; w < NW; ++w) x[w] = src[w * capE];
      T kv[NW * VN];
#pragma unroll
      for (int q = 0; q < NW * VN; ++q) kv[q] = Vec16<T>::get(x[q / VN], q % VN);
      diag += kv[0];
      if constexpr (LOAD) fs += kv[3];
      const bool sw = fan_swap(r);
      const T pv = sw ? kv[2] : kv[1];  // entry of neighbour j_k
      const T nx = sw ? kv[1] : kv[2];  // entry of neighbour j_{k+1}
      if (k == 0) first = pv;
      else out[(pw >> (4 * k)) & 15ull] = carry + pv;
      carry = nx;
    }
    if (inf & 32u) {  // open fan: j_0 and j_deg have one triangle each
      out[pw & 15ull] = first;
      out[(pw >> (4 * deg)) & 15ull] = carry;
    } else {
      out[pw & 15ull] = carry + first;
    }
    out[(inf >> 6) & 15u] = diag;
  }
  if constexpr (LOAD) a.F[v.pm[t]] = fs;
}

// Reduce of the P2 bilinear form over the fans (32-bit records).  KF holds
// the Map's output rows in the fan order of blk_bilinear_map: a vertex row
// a as (a, a+1, a+2, edge(a, a+1), edge(a+2, a), opposite edge), an edge row
// as (itself, its endpoints u and w, the third vertex z, edge(w, z),
// edge(z, u)).  Vertex rows: triangle k contributes to the diagonal, to its
// neighbour j_k and the edge node between the row's node and j_k (with the
// previous triangle's entries), to the opposite edge node (alone) and, as
// carries, to j_{k+1} and its edge node.  Edge rows: the one or two
// triangles add the diagonal and the endpoints' entries; the rest is
// theirs alone.
template <typename T>
__device__ __forceinline__ void fan_reduce_p2(const FwdArgs<T>& a, int capE, const FanView& v, const void* kf_buf) {
  constexpr int NW = kf_vecs<6, T, false>(), VN = Vec16<T>::n;
  using V = typename Vec16<T>::type;
  const V* KF = reinterpret_cast<const V*>(kf_buf);
  const int t = (int)threadIdx.x;
  if (v.r0 + t >= v.r1) return;
  const uint32_t inf = v.info32[t];
  const int deg = (int)(inf & 31u);
  if (deg == 0) return;
  T* out = a.out + v.up[t];
  auto put = [&](int q, T x) { out[q] = x; };
  const int x1 = (int)((inf >> 12) & 31u), x2 = (int)((inf >> 17) & 31u);
  T diag = T(0), c1 = T(0), c2 = T(0), f1 = T(0), f2 = T(0);
  int p1 = 0, p2 = 0;
  for (int k = 0; k < deg; ++k) {
    const uint32_t r = v.rec32[k * v.rs + t];
    const V* src = KF + (int)((r >> 11) & 7u) * NW * capE + (int)(r & 2047u);
    V x[NW];
#pragma unroll
    for (int w = 0; w < NW; ++w) x[w] = src[w * capE];
    T kv[NW * VN];
#pragma unroll
    for (int q = 0; q < NW * VN; ++q) kv[q] = Vec16<T>::get(x[q / VN], q % VN);
    const bool sw = ((r >> 14) & 1u) != 0u;
    const int pA = (int)((r >> 15) & 31u), pB = (int)((r >> 20) & 31u), pC = (int)((r >> 25) & 31u);
    diag += kv[0];
    const T s1 = sw ? kv[2] : kv[1], s2 = sw ? kv[1] : kv[2];
    if (inf & 32u) {  // edge node: the endpoints' sums, the rest written directly
      c1 += s1;
      c2 += s2;
      put(pA, kv[3]);
      put(pB, kv[4]);
      put(pC, kv[5]);
    } else {
      const T e1 = sw ? kv[4] : kv[3], e2 = sw ? kv[3] : kv[4];
      if (k == 0) {
        f1 = s1;
        f2 = e1;
        p1 = pA;
        p2 = pB;
      } else {
        put(pA, c1 + s1);
        put(pB, c2 + e1);
      }
      put(pC, kv[5]);
      c1 = s2;
      c2 = e2;
    }
  }
  if (inf & 32u) {
    put(x1, c1);
    put(x2, c2);
  } else if (inf & 64u) {  // open fan: its two ends have one triangle each
    put(p1, f1);
    put(p2, f2);
    put(x1, c1);
    put(x2, c2);
  } else {
    put(p1, c1 + f1);
    put(p2, c2 + f2);
  }
  put((int)((inf >> 7) & 31u), diag);
}

// Reduce of the load vector alone: Fe[a * capE + le] = F_e[a].
template <typename T>
__device__ __forceinline__ void fan_reduce_load(T* __restrict__ F, int capE, const FanView& v, const T* Fe) {
  const int t = (int)threadIdx.x;
  if (v.r0 + t >= v.r1) return;
  const int deg = (int)(v.info[t] & 31u);
  T fs = T(0);
  for (int k = 0; k < deg; ++k) {
    const unsigned r = v.rec[k * v.rs + t];
    fs += Fe[fan_a(r) * capE + fan_le(r)];
  }
  F[v.pm[t]] = fs;
}

}  // namespace tg

// The persistent loop of a fan kernel (as TG_BLK_PIPELINE_BEGIN).  Inside,
// `v` is the current block's view.
#define TG_FAN_PIPELINE_BEGIN(pipe, g, status)                                          \
  const int64_t G_ = gridDim.x;                                                         \
  [[maybe_unused]] const int NT_ = blockDim.x;                                          \
  int64_t b_ = blockIdx.x;                                                              \
  tg::FanPipe::Peek nq_;                                                                \
  if (threadIdx.x == 0 && b_ < (g).nblocks) {                                           \
    tg::FanPipe::Peek q0;                                                               \
    tg::FanPipe::peek(g, b_, q0);                                                       \
    (pipe).issue(g, 0, b_, q0);                                                         \
    if (b_ + G_ < (g).nblocks) tg::FanPipe::peek(g, b_ + G_, nq_);                     \
  }                                                                                     \
  for (int k_ = 0; b_ < (g).nblocks; ++k_, b_ += G_) {                                  \
    const int s_ = k_ & 1;                                                              \
    const bool ahead_ = b_ + G_ < (g).nblocks;                                          \
    if (threadIdx.x == 0 && ahead_) {                                                   \
      (pipe).issue(g, s_ ^ 1, b_ + G_, nq_);                                            \
      if (b_ + 2 * G_ < (g).nblocks) tg::FanPipe::peek(g, b_ + 2 * G_, nq_);            \
    }                                                                                   \
    if (!(pipe).wait(s_, k_, ahead_, status)) return;                                   \
    const tg::FanView v = (pipe).view(s_, (g).rs);

#define TG_FAN_PIPELINE_END }
