// Batched assembly: many independent instances (meshes of uneven size, each
// with its own coefficient field) in ONE launch of a persistent kernel.
//
// The work is a flat list of items (instance, first row, last row) built on
// the host when the batch is created or its schedule changes; every CTA of a
// persistent grid (SMs x resident CTAs) walks the list with a static stride,
// so the schedule is deterministic and each row is computed by exactly the
// same device routine as the single-instance kernel (gather.cuh): the result
// of every instance is bit-identical to tg_assemble_bilinear on it.
// Per-call pointers (coordinates, coefficients, outputs, c) travel in the
// kernel parameters (up to kMaxInst instances per launch), so a call is a
// single kernel launch with no host->device copy: safe to capture in a graph.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "fan.cuh"

namespace {

constexpr int kMaxInst = 256;

struct InstDesc {
  const int32_t* row_ptr;
  const int32_t* inc_ptr;
  const int32_t* inc_e;
  const uint32_t* inc_pos;
  const int32_t* cells;
  int64_t N;
  unsigned long long* status;
};

template <typename T>
struct BatchCall {
  int inst0;
  int layout;
  const T* coords[kMaxInst];
  const T* kappa[kMaxInst];
  T* vals[kMaxInst];
  T c[kMaxInst];
};

template <int EL, typename T, int BSZ>
__global__ void __launch_bounds__(BSZ) k_batch(const InstDesc* __restrict__ desc, const int4* __restrict__ items,
                                               int64_t n_items, const __grid_constant__ BatchCall<T> call,
                                               const __grid_constant__ tg::RefTab<T> tab, int cap) {
  extern __shared__ __align__(16) unsigned char smem[];
  auto& ts = *reinterpret_cast<tg::RefTab<T>*>(smem);
  unsigned char* buf = smem + tg::tab_bytes<T>();
  tg::copy_table(ts, tab);
  for (int64_t it = blockIdx.x; it < n_items; it += gridDim.x) {
    const int4 w = items[it];
    const InstDesc d = desc[w.x];
    const int k = w.x - call.inst0;
    tg::FwdArgs<T> a;
    a.row_ptr = d.row_ptr;
    a.inc_ptr = d.inc_ptr;
    a.inc_e = d.inc_e;
    a.inc_pos = d.inc_pos;
    a.cells = d.cells;
    a.elem_slot = nullptr;
    a.coords = call.coords[k];
    a.coef = call.kappa[k];
    a.coef2 = nullptr;
    a.layout = call.layout;
    a.c = call.c[k];
    a.out = call.vals[k];
    a.n = d.N;
    a.status = d.status;
    for (int64_t r = w.y; r < w.z; r += BSZ) tg::assemble_block<EL, T>(a, ts, tab, buf, cap, r, r + BSZ < w.z ? r + BSZ : w.z);
  }
}

// Block mode (every instance has element-once row blocks): one work item per
// (instance, row block), the same Map and Reduce as the single-instance
// kernel (blk_bilinear.cuh) on block views that read the pattern arrays in
// global memory.  Results are bitwise those of tg_assemble_bilinear.
struct InstBlk {
  const int32_t* iinc;
  const int32_t* irp;
  const int32_t* urp;
  const int32_t* iperm;
  const uint32_t* bel;
  const int64_t* boff;
  const int32_t* bvbase;
  const int32_t* bel_cnt;
  const uint32_t* brec;
  const uint16_t* fan;  // fan regions (P1 triangles; NULL: the row-owner Reduce)
  const int64_t* fan_off;
  int fan_rs;
  int64_t N;
  int R;
  unsigned long long* status;
};

template <int EL, typename T, int UB>
__global__ void __launch_bounds__(128) k_batch_blk(const InstBlk* __restrict__ desc, const int2* __restrict__ items,
                                                   int64_t n_items, const __grid_constant__ BatchCall<T> call,
                                                   const __grid_constant__ tg::RefTab<T> tab, int capE, int acc_n,
                                                   int fan_words) {
  constexpr int NV = tg::Elem<EL>::nv;
  extern __shared__ __align__(16) unsigned char smem[];
  T* acc = reinterpret_cast<T*>(smem + (size_t)NV * tg::kf_vecs<NV, T, false>() * capE * 16);
  // a copy of the item's fan region (fan_words 16-bit words at most)
  uint4* frs = reinterpret_cast<uint4*>(smem + (((size_t)NV * tg::kf_vecs<NV, T, false>() * capE * 16 +
                                                  (size_t)acc_n * sizeof(T) + 15) & ~size_t(15)));
  for (int q = threadIdx.x; q < acc_n; q += blockDim.x) acc[q] = T(0);
  __syncthreads();
  for (int64_t it = blockIdx.x; it < n_items; it += gridDim.x) {
    const int2 w = items[it];
    const InstBlk d = desc[w.x];
    const int k = w.x - call.inst0;
    tg::FwdArgs<T> a;
    a.row_ptr = nullptr;
    a.inc_ptr = nullptr;
    a.inc_e = nullptr;
    a.inc_pos = nullptr;
    a.cells = nullptr;
    a.elem_slot = nullptr;
    a.coords = call.coords[k];
    a.coef = call.kappa[k];
    a.coef2 = nullptr;
    a.layout = call.layout;
    a.c = call.c[k];
    a.out = call.vals[k];
    a.n = d.N;
    a.status = d.status;
    a.f = nullptr;
    a.f_layout = 0;
    a.F = nullptr;
    if constexpr (EL == TG_P1_TRI || EL == TG_P2_TRI) {
      if (d.fan != nullptr) {  // the fan-ordered Reduce, as tg_assemble_bilinear takes it
        tg::FanArgs g;
        g.urp = d.urp;
        g.iperm = d.iperm;
        g.fan = d.fan;
        g.fan_off = d.fan_off;
        g.bel = d.bel;
        g.boff = d.boff;
        g.bvbase = d.bvbase;
        g.bel_cnt = d.bel_cnt;
        g.N = d.N;
        g.R = d.R;
        g.rs = d.fan_rs;
        tg::FanView fv = tg::fan_view_global(g, w.y);
        {  // the region into shared memory (read by the Reduce after the Map's barrier)
          const int64_t f0 = d.fan_off[w.y], nq = (d.fan_off[w.y + 1] - f0) / 8;
          const uint4* src = reinterpret_cast<const uint4*>(d.fan + f0);
          for (int q = threadIdx.x; q < nq; q += blockDim.x) frs[q] = __ldg(src + q);
          const uint16_t* f = reinterpret_cast<const uint16_t*>(frs);
          fv.pos = reinterpret_cast<const unsigned long long*>(f);
          fv.info = f + 4 * g.rs;
          fv.rec = f + 5 * g.rs;
          fv.info32 = reinterpret_cast<const uint32_t*>(f);
          fv.rec32 = fv.info32 + g.rs;
        }
        tg::blk_bilinear_map<EL, T, UB, false, EL == TG_P2_TRI>(a, tab, capE, fv, smem);
        __syncthreads();
        if constexpr (EL == TG_P2_TRI) tg::fan_reduce_p2<T>(a, capE, fv, smem);
        else tg::fan_reduce_bilinear<T, false>(a, capE, fv, smem);
        __syncthreads();
        continue;
      }
    }
    tg::BlkView v;
    const int64_t r0 = (int64_t)w.y * d.R;
    v.r0 = (int)r0;
    v.r1 = (int)(r0 + d.R < d.N ? r0 + d.R : d.N);
    v.J0 = d.iinc[v.r0];
    v.J1 = d.iinc[v.r1];
    v.nbe = d.bel_cnt[w.y];
    v.vbase = d.bvbase[w.y];
    v.bs16 = (v.nbe + 7) & ~7;
    v.ip = d.iinc;
    v.rp = d.irp;
    v.up = d.urp;
    v.pm = d.iperm;
    v.rc = d.brec;
    v.be = d.bel + d.boff[w.y];
    v.vo = reinterpret_cast<const uint16_t*>(v.be + ((v.nbe + 3) & ~3));
    tg::blk_bilinear_block<EL, T, UB, false>(a, tab, capE, v, smem, acc);
  }
}

// Fan mode (every instance has fans): one 80-byte record per (instance, row
// block) item, built when the batch is created, with everything the item's
// Map and Reduce need to start: its instance, block rows, element list and
// fan region.  A CTA copies the record of its next item into shared memory
// while it works on the current one, and the item's fan region while its Map
// runs (asynchronous 16-byte copies), so an item starts without a chain of
// dependent global loads.  Same Map, Reduce and item order as k_batch_blk:
// the results are bitwise those of tg_assemble_bilinear.
struct ItemRec {
  const uint32_t* be;   // the block's element list (bel + boff[b])
  const uint4* fan;     // its fan region
  const int32_t* up;    // CSR row starts of its rows (urp + r0)
  const int32_t* pm;    // node of each of its rows (iperm + r0)
  unsigned long long* status;
  int inst, nbe, vbase, nfq;  // nfq: fan region size in 16-byte groups
  int r0, r1, rs;
  int pad[3];
};
static_assert(sizeof(ItemRec) == 80, "ItemRec is five 16-byte groups");

template <int EL, typename T, int UB>
__global__ void __launch_bounds__(128) k_batch_fan(const ItemRec* __restrict__ recs, int64_t n_items,
                                                   const __grid_constant__ BatchCall<T> call,
                                                   const __grid_constant__ tg::RefTab<T> tab, int capE, int fan_words) {
  constexpr int NV = tg::Elem<EL>::nv;
  extern __shared__ __align__(16) unsigned char smem[];
  const size_t kf_bytes = (size_t)NV * tg::kf_vecs<NV, T, false>() * capE * 16;
  uint4* frs = reinterpret_cast<uint4*>(smem + kf_bytes);
  ItemRec* slot = reinterpret_cast<ItemRec*>(smem + kf_bytes + (((size_t)fan_words * 2 + 15) & ~size_t(15)));
  const int tid = (int)threadIdx.x;
  const int64_t G = gridDim.x;
  if (tid < 5 && blockIdx.x < n_items)
    tg::cp_async16(reinterpret_cast<uint4*>(slot) + tid, reinterpret_cast<const uint4*>(recs + blockIdx.x) + tid);
  tg::cp_async_commit();
  tg::cp_async_wait_all();
  __syncthreads();
  int kk = 0;
  for (int64_t it = blockIdx.x; it < n_items; it += G, ++kk) {
    const ItemRec r = slot[kk & 1];
    if (tid < 5 && it + G < n_items)  // the next item's record
      tg::cp_async16(reinterpret_cast<uint4*>(slot + ((kk + 1) & 1)) + tid,
                     reinterpret_cast<const uint4*>(recs + it + G) + tid);
    for (int q = tid; q < r.nfq; q += blockDim.x) tg::cp_async16(frs + q, r.fan + q);  // read by the Reduce
    tg::cp_async_commit();
    const int k = r.inst - call.inst0;
    tg::FwdArgs<T> a;
    a.row_ptr = nullptr;
    a.inc_ptr = nullptr;
    a.inc_e = nullptr;
    a.inc_pos = nullptr;
    a.cells = nullptr;
    a.elem_slot = nullptr;
    a.coords = call.coords[k];
    a.coef = call.kappa[k];
    a.coef2 = nullptr;
    a.layout = call.layout;
    a.c = call.c[k];
    a.out = call.vals[k];
    a.n = 0;
    a.status = r.status;
    a.f = nullptr;
    a.f_layout = 0;
    a.F = nullptr;
    tg::FanView fv;
    fv.r0 = r.r0;
    fv.r1 = r.r1;
    fv.nbe = r.nbe;
    fv.vbase = r.vbase;
    fv.bs16 = (r.nbe + 7) & ~7;
    fv.rs = r.rs;
    fv.up = r.up;
    fv.pm = r.pm;
    const uint16_t* f = reinterpret_cast<const uint16_t*>(frs);
    fv.pos = reinterpret_cast<const unsigned long long*>(f);
    fv.info = f + 4 * r.rs;
    fv.rec = f + 5 * r.rs;
    fv.info32 = reinterpret_cast<const uint32_t*>(f);
    fv.rec32 = fv.info32 + r.rs;
    fv.be = r.be;
    fv.vo = reinterpret_cast<const uint16_t*>(r.be + ((r.nbe + 3) & ~3));
    tg::blk_bilinear_map<EL, T, UB, false, EL == TG_P2_TRI>(a, tab, capE, fv, smem);
    tg::cp_async_wait_all();
    __syncthreads();  // the Map's rows, the fan region and the next record are in place
    if constexpr (EL == TG_P2_TRI) tg::fan_reduce_p2<T>(a, capE, fv, smem);
    else tg::fan_reduce_bilinear<T, false>(a, capE, fv, smem);
    __syncthreads();
  }
}

struct Sched {
  int threads, rows_per_item, ctas_per_sm;
};

std::mutex g_cache_mu;
std::map<std::string, Sched> g_cache;  // autotuned schedules of this process

}  // namespace

struct tg_batch {
  int device = 0;
  tg_element el = TG_P1_TRI;
  int n_inst = 0;
  int max_row_len = 0;
  int max_deg = 0;
  int64_t total_rows = 0;
  std::vector<const tg_pattern*> pats;
  InstDesc* d_desc = nullptr;
  int4* d_items = nullptr;
  std::vector<int64_t> chunk_items;  // item range of each chunk of kMaxInst instances
  Sched sched{128, 512, 0};
  // block mode (all instances have row blocks)
  bool blk = false;
  InstBlk* d_blk = nullptr;
  int2* d_blk_items = nullptr;
  std::vector<int64_t> blk_chunk_items;
  int capE = 0, max_elems = 0;
  int fan_words = 0;  // largest fan region of the instances (16-bit words)
  // fan mode (triangle instances that all have fans): the item records
  ItemRec* d_recs = nullptr;
};

namespace {

tg_status build_items(tg_batch* b) {
  std::vector<int4> items;
  b->chunk_items.assign(1, 0);
  for (int i = 0; i < b->n_inst; ++i) {
    const int64_t N = b->pats[i]->N;
    for (int64_t r = 0; r < N; r += b->sched.rows_per_item)
      items.push_back(make_int4(i, (int)r, (int)std::min<int64_t>(N, r + b->sched.rows_per_item), 0));
    if ((i + 1) % kMaxInst == 0 || i + 1 == b->n_inst) b->chunk_items.push_back((int64_t)items.size());
  }
  if (b->d_items) cudaFree(b->d_items);
  b->d_items = nullptr;
  TG_CK(cudaMalloc(&b->d_items, std::max<size_t>(items.size(), 1) * sizeof(int4)));
  if (!items.empty()) TG_CK(cudaMemcpy(b->d_items, items.data(), items.size() * sizeof(int4), cudaMemcpyHostToDevice));
  return TG_OK;
}

template <int EL, typename T, int BSZ>
tg_status launch_t(tg_batch* b, const void* const* coords, const void* const* kappa, tg_layout kl, const double* c,
                   void* const* vals, cudaStream_t s) {
  auto kern = k_batch<EL, T, BSZ>;
  using El = tg::Elem<EL>;
  const int cap = std::max(1, BSZ * b->max_deg);
  const size_t smem = tg::tab_bytes<T>() + tg::staged_bytes<T, El::nv, El::npw>(BSZ, cap, b->max_row_len);
  tg_status st = tg::set_smem((const void*)kern, smem);
  if (st != TG_OK) return st;
  int per_sm = b->sched.ctas_per_sm;
  if (per_sm <= 0) {
    TG_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, BSZ, smem));
    per_sm = std::max(per_sm, 1);
  }
  const tg::RefTab<T>& tab = tg::table<T>(b->el);
  const size_t nchunks = b->chunk_items.size() - 1;
  for (size_t ch = 0; ch < nchunks; ++ch) {
    BatchCall<T> call;
    std::memset(&call, 0, sizeof(call));
    call.inst0 = (int)(ch * kMaxInst);
    call.layout = kl;
    const int n = std::min(kMaxInst, b->n_inst - call.inst0);
    for (int k = 0; k < n; ++k) {
      call.coords[k] = static_cast<const T*>(coords[call.inst0 + k]);
      call.kappa[k] = static_cast<const T*>(kappa[call.inst0 + k]);
      call.vals[k] = static_cast<T*>(vals[call.inst0 + k]);
      call.c[k] = (T)c[call.inst0 + k];
    }
    const int64_t i0 = b->chunk_items[ch], n_items = b->chunk_items[ch + 1] - i0;
    if (n_items == 0) continue;
    const int grid = (int)std::min<int64_t>(n_items, (int64_t)per_sm * tg::sm_count());
    kern<<<grid, BSZ, smem, s>>>(b->d_desc, b->d_items + i0, n_items, call, tab, cap);
    TG_CK_LAUNCH("k_batch");
  }
  return TG_OK;
}

template <typename T, int BSZ>
tg_status launch_el(tg_batch* b, const void* const* coords, const void* const* kappa, tg_layout kl, const double* c,
                    void* const* vals, cudaStream_t s) {
  switch (b->el) {
    case TG_P1_TRI: return launch_t<TG_P1_TRI, T, BSZ>(b, coords, kappa, kl, c, vals, s);
    case TG_P2_TRI: return launch_t<TG_P2_TRI, T, BSZ>(b, coords, kappa, kl, c, vals, s);
    default: return launch_t<TG_P1_TET, T, BSZ>(b, coords, kappa, kl, c, vals, s);
  }
}

template <int EL, typename T, int UB>
tg_status launch_blk_t(tg_batch* b, const void* const* coords, const void* const* kappa, tg_layout kl, const double* c,
                       void* const* vals, cudaStream_t s) {
  constexpr int NV = tg::Elem<EL>::nv;
  auto kern = k_batch_blk<EL, T, UB>;
  const void* kf = (const void*)kern;
  size_t smem = ((tg::blk_bilinear_work_bytes<NV, T, false>(b->capE, b->max_row_len, 128) + 15) & ~size_t(15)) +
                (size_t)b->fan_words * 2;
  if constexpr (EL == TG_P1_TRI || EL == TG_P2_TRI) {
    if (b->d_recs) {
      kf = (const void*)k_batch_fan<EL, T, UB>;
      smem = (size_t)NV * tg::kf_vecs<NV, T, false>() * b->capE * 16 + (((size_t)b->fan_words * 2 + 15) & ~size_t(15)) +
             2 * sizeof(ItemRec);
    }
  }
  tg_status st = tg::set_smem(kf, smem);
  if (st != TG_OK) return st;
  int per_sm = b->sched.ctas_per_sm;
  if (per_sm <= 0) {
    TG_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kf, 128, smem));
    per_sm = std::max(per_sm, 1);
  }
  const tg::RefTab<T>& tab = tg::table<T>(b->el);
  const size_t nchunks = b->blk_chunk_items.size() - 1;
  for (size_t ch = 0; ch < nchunks; ++ch) {
    BatchCall<T> call;
    std::memset(&call, 0, sizeof(call));
    call.inst0 = (int)(ch * kMaxInst);
    call.layout = kl;
    const int n = std::min(kMaxInst, b->n_inst - call.inst0);
    for (int k = 0; k < n; ++k) {
      call.coords[k] = static_cast<const T*>(coords[call.inst0 + k]);
      call.kappa[k] = static_cast<const T*>(kappa[call.inst0 + k]);
      call.vals[k] = static_cast<T*>(vals[call.inst0 + k]);
      call.c[k] = (T)c[call.inst0 + k];
    }
    const int64_t i0 = b->blk_chunk_items[ch], n_items = b->blk_chunk_items[ch + 1] - i0;
    if (n_items == 0) continue;
    const int grid = (int)std::min<int64_t>(n_items, (int64_t)per_sm * tg::sm_count());
    if (b->d_recs) {
      if constexpr (EL == TG_P1_TRI || EL == TG_P2_TRI) {
        k_batch_fan<EL, T, UB><<<grid, 128, smem, s>>>(b->d_recs + i0, n_items, call, tab, b->capE, b->fan_words);
        TG_CK_LAUNCH("k_batch_fan");
      }
      continue;
    }
    kern<<<grid, 128, smem, s>>>(b->d_blk, b->d_blk_items + i0, n_items, call, tab, b->capE, b->max_row_len * 128,
                                 b->fan_words);
    TG_CK_LAUNCH("k_batch_blk");
  }
  return TG_OK;
}

// UB as the single-instance kernel picks it for the largest block
template <typename T>
tg_status launch_blk(tg_batch* b, const void* const* coords, const void* const* kappa, tg_layout kl, const double* c,
                     void* const* vals, cudaStream_t s) {
  const int need = (b->max_elems + 127) / 128;
  switch (b->el) {
    case TG_P2_TRI:
      return need <= 1 ? launch_blk_t<TG_P2_TRI, T, 1>(b, coords, kappa, kl, c, vals, s)
                       : launch_blk_t<TG_P2_TRI, T, 2>(b, coords, kappa, kl, c, vals, s);
    case TG_P1_TRI:
      if constexpr (sizeof(T) == 8) {
        return need <= 2 ? launch_blk_t<TG_P1_TRI, T, 2>(b, coords, kappa, kl, c, vals, s)
                         : launch_blk_t<TG_P1_TRI, T, 3>(b, coords, kappa, kl, c, vals, s);
      } else {
        return need <= 3 ? launch_blk_t<TG_P1_TRI, T, 3>(b, coords, kappa, kl, c, vals, s)
                         : launch_blk_t<TG_P1_TRI, T, 6>(b, coords, kappa, kl, c, vals, s);
      }
    default:
      if constexpr (sizeof(T) == 8) {
        return need <= 2 ? launch_blk_t<TG_P1_TET, T, 2>(b, coords, kappa, kl, c, vals, s)
                         : launch_blk_t<TG_P1_TET, T, 3>(b, coords, kappa, kl, c, vals, s);
      } else {
        return need <= 4 ? launch_blk_t<TG_P1_TET, T, 4>(b, coords, kappa, kl, c, vals, s)
                         : launch_blk_t<TG_P1_TET, T, 6>(b, coords, kappa, kl, c, vals, s);
      }
  }
}

template <typename T>
tg_status launch(tg_batch* b, const void* const* coords, const void* const* kappa, tg_layout kl, const double* c,
                 void* const* vals, cudaStream_t s) {
  if (b->blk) return launch_blk<T>(b, coords, kappa, kl, c, vals, s);
  switch (b->sched.threads) {
    case 64: return launch_el<T, 64>(b, coords, kappa, kl, c, vals, s);
    case 256: return launch_el<T, 256>(b, coords, kappa, kl, c, vals, s);
    default: return launch_el<T, 128>(b, coords, kappa, kl, c, vals, s);
  }
}

tg_status check_call(const tg_batch* b, tg_dtype dtype, const void* const* coords, const void* const* kappa,
                     tg_layout kl, const double* c, void* const* vals) {
  if (!b || (dtype != TG_F32 && dtype != TG_F64) || !coords || !kappa || !c || !vals) return TG_ERR_INVALID_ARG;
  if (!(kl == TG_PER_QP || kl == TG_PER_ELEMENT || kl == TG_CONSTANT)) return TG_ERR_INVALID_ARG;
  const size_t es = dtype == TG_F32 ? 4 : 8;
  for (int i = 0; i < b->n_inst; ++i) {
    if (!coords[i] || !kappa[i] || (!vals[i] && b->pats[i]->nnz > 0)) return TG_ERR_INVALID_ARG;
    if (((uintptr_t)coords[i] % (b->el == TG_P1_TET ? es : 2 * es)) != 0) return TG_ERR_INVALID_ARG;
  }
  return TG_OK;
}

// Block mode when every instance has element-once row blocks that fit the
// shared-memory budget: descriptors and the (instance, block) item list.
tg_status setup_blocks(tg_batch* b) {
  const int nv = tg::nv_of(b->el);
  int capE = 0, max_elems = 0;
  for (const tg_pattern* p : b->pats) {
    if (p->E > 0 && !p->bel) return TG_OK;  // stays in row-range mode
    capE = std::max(capE, (p->blk_max_elems + 7) & ~7);  // a multiple of 8, as the fans' bank-group choice assumes
    max_elems = std::max(max_elems, p->blk_max_elems);
  }
  // the FP64 budget bounds both dtypes
  const size_t need = nv == 3 ? tg::blk_bilinear_work_bytes<3, double, false>(capE, b->max_row_len, 128)
                    : nv == 4 ? tg::blk_bilinear_work_bytes<4, double, false>(capE, b->max_row_len, 128)
                              : tg::blk_bilinear_work_bytes<6, double, false>(capE, b->max_row_len, 128);
  if (need > 113 * 1024) return TG_OK;
  std::vector<InstBlk> h(b->n_inst);
  std::vector<int2> items;
  b->blk_chunk_items.assign(1, 0);
  for (int i = 0; i < b->n_inst; ++i) {
    const tg_pattern* p = b->pats[i];
    h[i] = InstBlk{p->iinc, p->irp, p->urp, p->iperm, p->bel, p->boff, p->bvbase, p->bel_cnt, p->brec,
                   p->fan, p->fan_off, p->fan_rs, p->N, p->blk_rows, p->status};
    if (p->E > 0)
      for (int64_t k = 0; k < p->n_blk; ++k) items.push_back(make_int2(i, (int)k));
    if ((i + 1) % kMaxInst == 0 || i + 1 == b->n_inst) b->blk_chunk_items.push_back((int64_t)items.size());
  }
  TG_CK(cudaMalloc(&b->d_blk, b->n_inst * sizeof(InstBlk)));
  TG_CK(cudaMemcpy(b->d_blk, h.data(), b->n_inst * sizeof(InstBlk), cudaMemcpyHostToDevice));
  TG_CK(cudaMalloc(&b->d_blk_items, std::max<size_t>(items.size(), 1) * sizeof(int2)));
  if (!items.empty())
    TG_CK(cudaMemcpy(b->d_blk_items, items.data(), items.size() * sizeof(int2), cudaMemcpyHostToDevice));
  b->capE = capE;
  b->max_elems = max_elems;
  for (const tg_pattern* p : b->pats) b->fan_words = std::max(b->fan_words, p->fan ? p->fan_maxw : 0);
  b->blk = true;
  // fan mode: every instance with elements has fans (triangles)
  bool fans = b->el == TG_P1_TRI || b->el == TG_P2_TRI;
  for (const tg_pattern* p : b->pats) fans = fans && (p->E == 0 || p->fan);
  if (!fans || items.empty()) return TG_OK;
  std::vector<ItemRec> recs;
  recs.reserve(items.size());
  for (int i = 0; i < b->n_inst; ++i) {
    const tg_pattern* p = b->pats[i];
    if (p->E == 0) continue;
    const int64_t nb = p->n_blk;
    std::vector<int64_t> boff(nb), foff(nb + 1);
    std::vector<int32_t> cnt(nb), vbase(nb);
    TG_CK(cudaMemcpy(boff.data(), p->boff, nb * sizeof(int64_t), cudaMemcpyDeviceToHost));
    TG_CK(cudaMemcpy(foff.data(), p->fan_off, (nb + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost));
    TG_CK(cudaMemcpy(cnt.data(), p->bel_cnt, nb * sizeof(int32_t), cudaMemcpyDeviceToHost));
    TG_CK(cudaMemcpy(vbase.data(), p->bvbase, nb * sizeof(int32_t), cudaMemcpyDeviceToHost));
    for (int64_t k = 0; k < nb; ++k) {
      const int64_t r0 = k * p->blk_rows, r1 = std::min<int64_t>(p->N, r0 + p->blk_rows);
      ItemRec r{};
      r.be = p->bel + boff[k];
      r.fan = reinterpret_cast<const uint4*>(p->fan + foff[k]);
      r.up = p->urp + r0;
      r.pm = p->iperm + r0;
      r.status = p->status;
      r.inst = i;
      r.nbe = cnt[k];
      r.vbase = vbase[k];
      r.nfq = (int)((foff[k + 1] - foff[k]) / 8);
      r.r0 = (int)r0;
      r.r1 = (int)r1;
      r.rs = p->fan_rs;
      recs.push_back(r);
    }
  }
  if (recs.size() != items.size()) return TG_OK;  // not expected; the block mode serves then
  TG_CK(cudaMalloc(&b->d_recs, recs.size() * sizeof(ItemRec)));
  TG_CK(cudaMemcpy(b->d_recs, recs.data(), recs.size() * sizeof(ItemRec), cudaMemcpyHostToDevice));
  return TG_OK;
}

std::string cache_key(const tg_batch* b, tg_dtype dtype) {
  cudaDeviceProp prop;
  cudaGetDeviceProperties(&prop, b->device);
  int bucket = 0;
  for (int64_t r = b->total_rows; r > 1; r >>= 1) ++bucket;
  return std::string(prop.name) + "|el" + std::to_string((int)b->el) + "|dt" + std::to_string((int)dtype) +
         "|rows2^" + std::to_string(bucket) + "|inst" + std::to_string(b->n_inst) + "|blk" + (b->blk ? "1" : "0");
}

}  // namespace

extern "C" {

tg_status tg_batch_create(const tg_pattern* const* pats, int32_t n_inst, tg_batch** out) {
  if (!out || !pats || n_inst < 1) return TG_ERR_INVALID_ARG;
  *out = nullptr;
  const tg_element el = pats[0] ? pats[0]->el : TG_P1_TRI;
  if (!tg::scalar_kind(el)) return TG_ERR_INVALID_ARG;
  tg_batch* b = new tg_batch;
  b->el = el;
  b->n_inst = n_inst;
  std::vector<InstDesc> h(n_inst);
  for (int i = 0; i < n_inst; ++i) {
    const tg_pattern* p = pats[i];
    if (!p || p->el != el || p->N > INT32_MAX) {
      delete b;
      return TG_ERR_INVALID_ARG;
    }
    b->pats.push_back(p);
    b->max_row_len = std::max(b->max_row_len, p->max_row_len);
    b->max_deg = std::max(b->max_deg, p->max_deg);
    b->total_rows += p->N;
    h[i] = InstDesc{p->row_ptr, p->inc_ptr, p->inc_e, p->inc_pos, p->cells, p->N, p->status};
  }
  cudaError_t e = cudaGetDevice(&b->device);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_desc, n_inst * sizeof(InstDesc));
  if (e == cudaSuccess) e = cudaMemcpy(b->d_desc, h.data(), n_inst * sizeof(InstDesc), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    tg_batch_destroy(b);
    return tg::cuda_fail(e, "tg_batch_create", __FILE__, __LINE__);
  }
  tg_status st = build_items(b);
  if (st == TG_OK) st = setup_blocks(b);
  if (st != TG_OK) {
    tg_batch_destroy(b);
    return st;
  }
  *out = b;
  return TG_OK;
}

tg_status tg_batch_set_schedule(tg_batch* b, int32_t threads, int32_t rows_per_item, int32_t ctas_per_sm) {
  if (!b || !(threads == 64 || threads == 128 || threads == 256) || rows_per_item < threads ||
      rows_per_item % threads != 0 || ctas_per_sm < 0)
    return TG_ERR_INVALID_ARG;
  b->sched = Sched{threads, rows_per_item, ctas_per_sm};
  return build_items(b);
}

tg_status tg_batch_get_schedule(const tg_batch* b, int32_t* threads, int32_t* rows_per_item, int32_t* ctas_per_sm) {
  if (!b) return TG_ERR_INVALID_ARG;
  if (threads) *threads = b->sched.threads;
  if (rows_per_item) *rows_per_item = b->sched.rows_per_item;
  if (ctas_per_sm) *ctas_per_sm = b->sched.ctas_per_sm;
  return TG_OK;
}

tg_status tg_batch_assemble(tg_batch* b, tg_dtype dtype, const void* const* coords, const void* const* kappa,
                            tg_layout kappa_layout, const double* c, void* const* vals_out, tg_stream stream) {
  tg_status st = check_call(b, dtype, coords, kappa, kappa_layout, c, vals_out);
  if (st != TG_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  return dtype == TG_F32 ? launch<float>(b, coords, kappa, kappa_layout, c, vals_out, s)
                         : launch<double>(b, coords, kappa, kappa_layout, c, vals_out, s);
}

tg_status tg_batch_autotune(tg_batch* b, tg_dtype dtype, const void* const* coords, const void* const* kappa,
                            tg_layout kappa_layout, const double* c, void* const* vals_out, int32_t reps,
                            float* best_ms, tg_stream stream) {
  tg_status st = check_call(b, dtype, coords, kappa, kappa_layout, c, vals_out);
  if (st != TG_OK) return st;
  if (reps < 1) return TG_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const std::string key = cache_key(b, dtype);
  {
    std::lock_guard<std::mutex> lk(g_cache_mu);
    auto it = g_cache.find(key);
    if (it != g_cache.end() && !best_ms) {
      b->sched = it->second;
      return build_items(b);
    }
  }
  std::vector<Sched> cands;
  if (b->blk) {  // block mode: only the resident CTAs per SM apply
    for (int cps : {0, 2, 3, 4, 6}) cands.push_back(Sched{128, 128, cps});
  } else {
    for (int t : {64, 128, 256})
      for (int m : {1, 2, 4, 8, 16})
        for (int cps : {0, 2})
          cands.push_back(Sched{t, t * m, cps});
  }
  cudaEvent_t e0, e1;
  TG_CK(cudaEventCreate(&e0));
  TG_CK(cudaEventCreate(&e1));
  Sched best = b->sched;
  float best_t = 1e30f;
  for (const Sched& sc : cands) {
    b->sched = sc;
    if ((st = build_items(b)) != TG_OK) break;
    auto run = [&]() {
      return dtype == TG_F32 ? launch<float>(b, coords, kappa, kappa_layout, c, vals_out, s)
                             : launch<double>(b, coords, kappa, kappa_layout, c, vals_out, s);
    };
    if ((st = run()) != TG_OK) break;  // warm-up
    TG_CK(cudaEventRecord(e0, s));
    for (int r = 0; r < reps && st == TG_OK; ++r) st = run();
    TG_CK(cudaEventRecord(e1, s));
    TG_CK(cudaEventSynchronize(e1));
    if (st != TG_OK) break;
    float ms = 0;
    TG_CK(cudaEventElapsedTime(&ms, e0, e1));
    ms /= reps;
    if (ms < best_t) {
      best_t = ms;
      best = sc;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  b->sched = best;
  tg_status st2 = build_items(b);
  if (st != TG_OK) return st;
  if (st2 != TG_OK) return st2;
  {
    std::lock_guard<std::mutex> lk(g_cache_mu);
    g_cache[key] = best;
  }
  if (best_ms) *best_ms = best_t;
  return TG_OK;
}

void tg_batch_destroy(tg_batch* b) {
  if (!b) return;
  if (b->d_desc) cudaFree(b->d_desc);
  if (b->d_items) cudaFree(b->d_items);
  if (b->d_blk) cudaFree(b->d_blk);
  if (b->d_blk_items) cudaFree(b->d_blk_items);
  if (b->d_recs) cudaFree(b->d_recs);
  delete b;
}

}  // extern "C"
