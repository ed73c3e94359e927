// Element-once row blocks (P1 triangles and tetrahedra): the pipeline that
// the forward, load and backward kernels share.
//
// A persistent CTA walks the row blocks b = blockIdx.x, + gridDim.x, ...
// Block b owns R consecutive rows of the pattern's internal row order (R <=
// the CTA's threads; a block is a compact patch of the mesh when the
// elements come in a space-filling-curve order).  Its contiguous streams are:
//   - its slices of the internal incidence and CSR-value prefix sums, of the
//     rows' CSR starts and of the rows' node ids;
//   - the records of its incidences (brec);
//   - its list of distinct elements (bel).
// Thread 0 prefetches them into the other of two shared stages with bulk
// copies one block ahead, while the CTA works on the current block:
//   Map    - one thread per distinct element computes that element's local
//            quantities once and leaves them in shared memory;
//   Reduce - one thread per row sums the quantities of its incidences in
//            increasing element order (the fixed order that makes every
//            output bitwise reproducible) and writes its node's outputs.
// An element shared by several blocks is computed once in each of them.
#pragma once

#include <cstdint>

#include "async.cuh"
#include "gather.cuh"

namespace tg {

struct BlkArgs {
  const int32_t* __restrict__ inc_ptr;  // internal incidence prefix sums (iinc)
  const int32_t* __restrict__ row_ptr;  // internal CSR-value prefix sums (irp)
  const int32_t* __restrict__ urp;      // CSR row start of each internal row
  const int32_t* __restrict__ iperm;    // node of each internal row
  const uint32_t* __restrict__ bel;
  const int64_t* __restrict__ boff;
  const int32_t* __restrict__ bvbase;
  const int32_t* __restrict__ bel_cnt;
  const uint32_t* __restrict__ brec;
  int64_t N;
  int64_t nblocks;
  int capE, capJ;  // stage capacities (multiples of 4): distinct elements, incidences
  int capE16;      // capE rounded up to a multiple of 8 (16-bit vertex rows)
  int nv;          // vertices per element
  int R;           // rows per block (at most the CTA's threads)
  int rw;          // 32-bit words per incidence record (1; 2 for P2)
};

// Host: BlkArgs of a pattern with row blocks.
inline BlkArgs blk_args(const tg_pattern* p) {
  BlkArgs g;
  g.inc_ptr = p->iinc;
  g.row_ptr = p->irp;
  g.urp = p->urp;
  g.iperm = p->iperm;
  g.bel = p->bel;
  g.boff = p->boff;
  g.bvbase = p->bvbase;
  g.bel_cnt = p->bel_cnt;
  g.brec = p->brec;
  g.N = p->N;
  g.nblocks = p->n_blk;
  g.capE = (p->blk_max_elems + 3) & ~3;
  g.capJ = (p->blk_max_inc + 3) & ~3;
  g.capE16 = (p->blk_max_elems + 7) & ~7;
  g.nv = p->nv;
  g.R = p->blk_rows;
  g.rw = p->nv > 4 ? 2 : 1;
  return g;
}

// Shared-memory bytes of the two stages plus barriers and block metadata.
__host__ __device__ inline size_t blk_stage_bytes(int R, int capJ, int capE, int nv) {
  const size_t el_words = (size_t)capE + (size_t)nv * (((capE + 7) & ~7) / 2);
  const size_t rw = nv > 4 ? 2 : 1;
  return 16 + 128 + 2 * ((size_t)(R + 8) * 16 + ((size_t)capJ * rw + 8) * 4 + el_words * 4);
}

// Geometry of one row block as seen through its stage.
struct BlkView {
  int r0, r1, J0, J1, nbe;
  int bs16;            // row stride of vo
  int vbase;           // smallest vertex id of the block's elements
  const int* ip;       // ip[i]: internal incidence prefix, i in [r0, r1]
  const int* rp;       // rp[i]: internal CSR-value prefix (rp[i] - rp[r0] = offset in the block)
  const int* up;       // up[i]: CSR start of internal row i's node, i in [r0, r1)
  const int* pm;       // pm[i]: node of internal row i
  const uint32_t* rc;  // rc[j * rw ...] = record j, j in [J0, J1)
  const uint32_t* be;  // be[k]: element k (with the owner bit), k < nbe
  const uint16_t* vo;  // vo[c * bs16 + k]: vertex c of element k, minus vbase
  __device__ int vtx(int c, int k) const { return vbase + (int)vo[c * bs16 + k]; }
};

class BlkPipe {
 public:
  // Carves the stages out of shared memory at p (16-byte aligned); returns
  // the first byte after them.  Thread 0 initialises the barriers; the
  // caller's next CTA barrier publishes them.
  __device__ unsigned char* init(unsigned char* p, const BlkArgs& g) {
    R_ = g.R;
    IPN_ = R_ + 8;
    RECN_ = g.capJ * g.rw + 8;
    ELN_ = g.capE + g.nv * (g.capE16 / 2);
    SW_ = 4 * IPN_ + RECN_ + ELN_;  // words per stage (a multiple of 4)
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

  // Thread 0: incidence range, element count and element-list offset of
  // block blk (plain loads, issued early so that they are in flight while
  // the CTA works).
  struct Peek {
    int J0, J1, nbe, vb;
    int64_t bo;
  };
  __device__ static void peek(const BlkArgs& g, int64_t blk, int R, Peek& q) {
    q.J0 = __ldg(g.inc_ptr + blk * R);
    q.J1 = __ldg(g.inc_ptr + (blk * R + R < g.N ? blk * R + R : g.N));
    q.nbe = __ldg(g.bel_cnt + blk);
    q.bo = __ldg(g.boff + blk);
    q.vb = __ldg(g.bvbase + blk);
  }

  // Thread 0: copy block blk's streams into stage s.  The inc_ptr, row_ptr
  // and brec ranges are widened to whole 16-byte groups (the pattern arrays
  // carry 16 bytes of tail padding); the element list is a 16-byte aligned
  // region of (nbe + 3) & ~3 element words and nv rows of (nbe + 7) & ~7
  // 16-bit vertex offsets.  The stage capacities hold all of them.
  __device__ void issue(const BlkArgs& g, int s, int64_t blk, const Peek& q) {
    const int r0 = (int)(blk * R_), r1 = (int)(blk * R_ + R_ < g.N ? blk * R_ + R_ : g.N);
    const int a0 = r0 & ~3, nip = (r1 + 1 - a0 + 3) & ~3;
    const int j0a = q.J0 & ~(4 / g.rw - 1), nrec = ((q.J1 - j0a) * g.rw + 3) & ~3;
    const int nel = ((q.nbe + 3) & ~3) + g.nv * (((q.nbe + 7) & ~7) / 2);
    int* m = meta_ + 16 * s;
    m[0] = r0;
    m[1] = r1;
    m[2] = q.J0;
    m[3] = q.J1;
    m[4] = a0;
    m[5] = j0a * g.rw;
    m[6] = q.nbe;
    m[7] = q.vb;
    const int nup = (r1 - a0 + 3) & ~3;
    const uint32_t bytes = 4u * (2u * nip + 2u * nup + (q.J1 > q.J0 ? nrec : 0) + nel);
    fence_proxy_async();
    mbar_arrive_expect_tx(&bar_[s], bytes);
    bulk_copy_g2s(ip(s), g.inc_ptr + a0, nip * 4, &bar_[s]);
    bulk_copy_g2s(rp(s), g.row_ptr + a0, nip * 4, &bar_[s]);
    bulk_copy_g2s(up(s), g.urp + a0, nup * 4, &bar_[s]);
    bulk_copy_g2s(pm(s), g.iperm + a0, nup * 4, &bar_[s]);
    if (q.J1 > q.J0) bulk_copy_g2s(rec(s), g.brec + (int64_t)j0a * g.rw, nrec * 4, &bar_[s]);
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

  __device__ BlkView view(int s) const {
    const int* m = meta_ + 16 * s;
    BlkView v;
    v.r0 = m[0];
    v.r1 = m[1];
    v.J0 = m[2];
    v.J1 = m[3];
    v.nbe = m[6];
    v.vbase = m[7];
    v.bs16 = (v.nbe + 7) & ~7;
    v.ip = ip(s) - m[4];
    v.rp = rp(s) - m[4];
    v.up = up(s) - m[4];
    v.pm = pm(s) - m[4];
    v.rc = rec(s) - m[5];
    v.be = el(s);
    v.vo = reinterpret_cast<const uint16_t*>(el(s) + ((v.nbe + 3) & ~3));
    return v;
  }

 private:
  // stage s: ip [IPN] | rp [IPN] | up [IPN] | pm [IPN] | rec [RECN] | el [ELN]
  __device__ int* ip(int s) const { return st_ + s * SW_; }
  __device__ int* rp(int s) const { return ip(s) + IPN_; }
  __device__ int* up(int s) const { return rp(s) + IPN_; }
  __device__ int* pm(int s) const { return up(s) + IPN_; }
  __device__ uint32_t* rec(int s) const { return reinterpret_cast<uint32_t*>(pm(s) + IPN_); }
  __device__ uint32_t* el(int s) const { return rec(s) + RECN_; }

  int R_, IPN_, RECN_, ELN_, SW_;
  uint64_t* bar_;
  int* meta_;
  int* st_;
};

// Fields of an incidence record.  nv <= 4: one word, 4-bit column
// positions, the local vertex a (2 bits), the local index of the element in
// the block's list (the rest).  P2 (nv = 6): word 0 the six 5-bit positions,
// word 1 a (3 bits) and the local element index.
template <int NV>
struct BlkRec {
  uint32_t w;
  __device__ int le() const { return (int)(w >> (4 * NV + 2)); }
  __device__ int a() const { return (int)(w >> (4 * NV)) & 3; }
  __device__ int pos(int b) const { return (int)(w >> (4 * b)) & 15; }
};

template <>
struct BlkRec<6> {
  uint32_t x, y;
  __device__ int le() const { return (int)(y >> 3); }
  __device__ int a() const { return (int)(y & 7u); }
  __device__ int pos(int b) const { return (int)(x >> (5 * b)) & 31; }
};

// Record j of a block view.
template <int NV>
__device__ __forceinline__ BlkRec<NV> blk_rec(const uint32_t* rc, int j) {
  if constexpr (NV == 6) {
    const uint2 w = *reinterpret_cast<const uint2*>(rc + 2 * j);
    return BlkRec<6>{w.x, w.y};
  } else {
    return BlkRec<NV>{rc[j]};
  }
}

// The element of a bel entry (without the owner bit).
__device__ __forceinline__ int64_t bel_elem(uint32_t w) { return (int64_t)(w & 0x7fffffffu); }
__device__ __forceinline__ bool bel_owner(uint32_t w) { return (w >> 31) != 0u; }

}  // namespace tg

// The persistent loop of an element-once kernel.  Inside, `v` is the
// current block's view, R_ the rows per block and NT_ the CTA's threads;
// thread 0 has already issued block b + G into the other stage and peeked
// at b + 2G.  A timed-out wait makes the whole CTA return.
#define TG_BLK_PIPELINE_BEGIN(pipe, g, status)                                          \
  const int64_t G_ = gridDim.x;                                                         \
  const int R_ = (g).R;                                                                 \
  [[maybe_unused]] const int NT_ = blockDim.x;                                          \
  int64_t b_ = blockIdx.x;                                                              \
  tg::BlkPipe::Peek nq_;                                                                \
  if (threadIdx.x == 0 && b_ < (g).nblocks) {                                           \
    tg::BlkPipe::Peek q0;                                                               \
    tg::BlkPipe::peek(g, b_, R_, q0);                                                   \
    (pipe).issue(g, 0, b_, q0);                                                         \
    if (b_ + G_ < (g).nblocks) tg::BlkPipe::peek(g, b_ + G_, R_, nq_);                 \
  }                                                                                     \
  for (int k_ = 0; b_ < (g).nblocks; ++k_, b_ += G_) {                                  \
    const int s_ = k_ & 1;                                                              \
    const bool ahead_ = b_ + G_ < (g).nblocks;                                          \
    if (threadIdx.x == 0 && ahead_) {                                                   \
      (pipe).issue(g, s_ ^ 1, b_ + G_, nq_);                                            \
      if (b_ + 2 * G_ < (g).nblocks) tg::BlkPipe::peek(g, b_ + 2 * G_, R_, nq_);        \
    }                                                                                   \
    if (!(pipe).wait(s_, k_, ahead_, status)) return;                                   \
    const tg::BlkView v = (pipe).view(s_);

#define TG_BLK_PIPELINE_END }
