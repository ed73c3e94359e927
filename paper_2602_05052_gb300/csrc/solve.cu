// Support kernels: CSR matrix-vector product, deterministic dot products and
// the conjugate-gradient solve of the Dirichlet-condensed system (the
// iterative solve that follows assembly, SM B.1 solver configuration, and the
// adjoint solve K^T lam = -dGamma/dU of Eq. (adj)); plus the FMA-rate probe
// used to report the arithmetic roof.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <mutex>
#include <string>
#include <type_traits>
#include <vector>

#include "async.cuh"
#include "tg_internal.cuh"

namespace {

constexpr int ST = 256;

// Four lanes per row, fixed-order shuffle sum.  Rows with mask[row] != 0
// (Dirichlet) produce 0.
template <typename T>
__global__ void __launch_bounds__(ST) k_spmv(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                             const T* __restrict__ v, const T* __restrict__ x, T* __restrict__ y,
                                             int64_t n, const uint8_t* __restrict__ mask) {
  const int64_t t = (int64_t)blockIdx.x * ST + threadIdx.x;
  const int64_t row = t >> 2;
  const int lane = threadIdx.x & 3;
  const unsigned grp = 0xfu << (threadIdx.x & 28);
  if (row >= n) return;  // the four lanes of a row leave together
  T s = T(0);
  const int k1 = __ldg(rp + row + 1);
  for (int k = __ldg(rp + row) + lane; k < k1; k += 4) s += __ldg(v + k) * __ldg(x + __ldg(ci + k));
  s += __shfl_xor_sync(grp, s, 1, 4);
  s += __shfl_xor_sync(grp, s, 2, 4);
  if (lane == 0) y[row] = (mask && mask[row]) ? T(0) : s;
}

// Partial dot products (double accumulation) over a fixed grid; the final
// kernel sums the partials in a fixed order.
template <typename T>
__global__ void __launch_bounds__(ST) k_dot_partial(const T* __restrict__ a, const T* __restrict__ b, int64_t n,
                                                    double* __restrict__ partials) {
  __shared__ double red[ST];
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * ST + threadIdx.x; i < n; i += (int64_t)gridDim.x * ST)
    s += (double)a[i] * (double)b[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = ST / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) partials[blockIdx.x] = red[0];
}

__global__ void __launch_bounds__(ST) k_dot_final(const double* __restrict__ partials, int nb, double* __restrict__ out) {
  __shared__ double red[ST];
  double s = 0.0;
  for (int k = threadIdx.x; k < nb; k += ST) s += partials[k];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = ST / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
}

// x = 0 on the rows the condensed system drops, before the initial residual
// F - K x is formed: an initial guess's values there must not enter it.
template <typename T>
__global__ void k_cg_zero_masked(T* __restrict__ x, const uint8_t* __restrict__ mask, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * ST + threadIdx.x;
  if (i < n && mask[i]) x[i] = T(0);
}

// r = mask ? 0 : F - Kx ;  b = mask ? 0 : F ;  x = mask ? 0 : x ;  p = r
template <typename T>
__global__ void k_cg_init(const T* __restrict__ F, const T* __restrict__ Kx, const uint8_t* __restrict__ mask,
                          T* __restrict__ x, T* __restrict__ r, T* __restrict__ p, T* __restrict__ b, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * ST + threadIdx.x;
  if (i >= n) return;
  const bool d = mask && mask[i];
  const T ri = d ? T(0) : F[i] - Kx[i];
  r[i] = ri;
  p[i] = ri;
  b[i] = d ? T(0) : F[i];
  if (d) x[i] = T(0);
}

// sc = {rr, pAp, rr_new}: x += alpha p, r -= alpha Ap, alpha = rr / pAp
template <typename T>
__global__ void k_cg_xr(T* __restrict__ x, T* __restrict__ r, const T* __restrict__ p, const T* __restrict__ Ap,
                        const double* __restrict__ sc, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * ST + threadIdx.x;
  if (i >= n) return;
  const T alpha = (T)(sc[0] / sc[1]);
  x[i] += alpha * p[i];
  r[i] -= alpha * Ap[i];
}

// p = r + beta p, beta = rr_new / rr
template <typename T>
__global__ void k_cg_p(T* __restrict__ p, const T* __restrict__ r, const double* __restrict__ sc, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * ST + threadIdx.x;
  if (i >= n) return;
  const T beta = (T)(sc[2] / sc[0]);
  p[i] = r[i] + beta * p[i];
}

__global__ void k_cg_shift(double* sc) { sc[0] = sc[2]; }

// ---------------------------------------------------------------- one-launch CG
// A barrier across the CTAs of a cooperative launch (all resident) on a
// 64-bit arrival counter that is 0 when the launch starts: barrier number k
// completes when the counter reaches k * gridDim.x (release on arrival,
// acquire on the poll).  Bounded: after `limit` polls (the CG takes 2^22) a
// CTA sets *err and gives up; the others give up at their next barrier.
constexpr unsigned int kGridPolls = 1u << 22;
// FP64 systems with at least this many matrix entries take the one-launch
// CG's three-barrier form: the second read and the FP64 FMA per entry cost
// more than the third barrier there (48^3 tetrahedral system, 1.76M
// entries: 27 instead of 34 us per iteration).
constexpr int64_t kCgP3MinEntries = int64_t(1) << 19;
__device__ __forceinline__ bool grid_sync(unsigned long long* count, unsigned long long& target, int* err,
                                          unsigned int limit = kGridPolls) {
  __syncthreads();
  int bad = 0;
  if (threadIdx.x == 0) {
    target += gridDim.x;
    asm volatile("red.release.gpu.global.add.u64 [%0], 1;" ::"l"(count) : "memory");
    for (unsigned int t = 0;; ++t) {
      unsigned long long v;
      asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(count) : "memory");
      if (v >= target) break;
      if (t >= limit) {
        bad = 1;
        atomicExch(err, 1);
        break;
      }
    }
  }
  return __syncthreads_or(bad) == 0;
}

// The tree sum of k_dot_partial and k_dot_final over the CTA's 256 values
// (level w adds value t + w to value t, w = 128, 64, ..., 1), every thread
// getting the result.  One warp evaluates it: each lane adds its four pairs
// of level 128 and carries them through levels 64 and 32 in registers, and
// shuffles take levels 16 to 1.  The pairs and their order are the tree's,
// so the sum carries its bits, with two CTA barriers instead of ten (the
// FP64 additions are slow on this GPU; the barrier per level cost more).
__device__ __forceinline__ double cta_tree_sum(double v, double* red) {
  static_assert(ST == 256, "the tree below has eight levels");
  red[threadIdx.x] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    const int l = threadIdx.x;
    const double a0 = red[l] + red[l + 128], a1 = red[l + 32] + red[l + 160];
    const double a2 = red[l + 64] + red[l + 192], a3 = red[l + 96] + red[l + 224];
    double c = (a0 + a2) + (a1 + a3);
#pragma unroll
    for (int w = 16; w > 0; w >>= 1) c += __shfl_down_sync(0xffffffffu, c, w);
    if (l == 0) red[ST] = c;
  }
  __syncthreads();
  return red[ST];
}

// The CG iterations of cg() in one cooperative launch.  The dot products of
// the launch-per-kernel loop reduce over nb partial blocks, thread t of
// block b summing the entries i = b*ST + t + q*nb*ST (q = 0, 1, ...).  Here
// that thread owns exactly those rows, for q < KM: it keeps their x, r, p
// and row bounds in registers and forms their (A p)_i itself, with the four
// strided partial sums of k_spmv's four lanes added in the lanes' shuffle
// order, (s0 + s1) + (s2 + s3).  The launch has min(nb, ceil(n/ST)) CTAs
// (the partials of blocks past the last row are 0).  So A p, p.Ap, the x and
// r updates and r.r need no exchange, and two grid barriers per iteration
// remain: after the p.Ap partials and after the r.r partials.  The direction
// update p = r + beta p is folded into the next product: a column the
// product reads forms r + beta p_old from the previous iterate (the
// expression of k_cg_p, so the same bits), and each thread publishes its
// rows of p_new in the other buffer (p_old / p_new alternate; the first
// iteration uses p = r as k_cg_init left it) and its rows of r.  Per
// iteration the sums, their order and the updates are those of the separate
// kernels, so the iterates are bitwise those of the launch-per-kernel loop.
// Convergence is checked, as there, after every eighth iteration and at
// maxit.  pa / pb: the partial arrays of the two dot products (a CTA never
// overwrites partials another CTA still reads).  Values other CTAs wrote
// during the launch are read through L2 (__ldcg).  On a barrier timeout
// *err is set and every CTA leaves (x is then not written).
// P3 (FP64 systems with many entries): forming r + beta p_old per entry read
// costs a second L2 read and an FP64 FMA per matrix entry, more than a third
// grid barrier; each thread then updates its rows of p in p0 first, a
// barrier follows, and the product reads p itself (the same values, so the
// same bits).
template <typename T, int KM, bool P3>
__global__ void __launch_bounds__(ST) k_cg_loop(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                                const T* __restrict__ vals, const uint8_t* __restrict__ mask, T* x,
                                                T* r, T* p0, T* p1, int64_t n, int nb, double* sc, double* pa,
                                                double* pb, unsigned long long* count, double fnorm, double rtol,
                                                int maxit, int* it_out, int* err) {
  __shared__ double red[ST + 1];
  const int64_t G = (int64_t)nb * ST, g0 = (int64_t)blockIdx.x * ST + threadIdx.x;
  unsigned long long target = 0;
  if (blockIdx.x == 0)
    for (int k = (int)gridDim.x + threadIdx.x; k < nb; k += ST) pa[k] = pb[k] = 0.0;
  bool own[KM], dm[KM];
  int kb[KM], ke[KM];
  T xi[KM], ri[KM], pi[KM], api[KM];
#pragma unroll
  for (int q = 0; q < KM; ++q) {
    const int64_t i = g0 + q * G;
    own[q] = i < n;
    kb[q] = own[q] ? __ldg(rp + i) : 0;
    ke[q] = own[q] ? __ldg(rp + i + 1) : 0;
    dm[q] = own[q] && mask && mask[i];
    xi[q] = own[q] ? x[i] : T(0);
    ri[q] = own[q] ? r[i] : T(0);
    pi[q] = own[q] ? p0[i] : T(0);
    api[q] = T(0);
  }
  double rr = sc[0];
  T beta = T(0);
  bool first = true;
  const T* pold = p0;
  T* pnew = p1;
  int it = 0;
  while (it < maxit) {
    if constexpr (P3) {
      if (!first) {
#pragma unroll
        for (int q = 0; q < KM; ++q) {
          if (!own[q]) continue;
          pi[q] = ri[q] + beta * pi[q];
          p0[g0 + q * G] = pi[q];
        }
        if (!grid_sync(count, target, err)) return;
      }
    }
    double s = 0.0;
#pragma unroll
    for (int q = 0; q < KM; ++q) {
      if (!own[q]) continue;
      T s0 = T(0), s1 = T(0), s2 = T(0), s3 = T(0);
      // p_new at column c: r + beta p_old (p_old itself in the first
      // iteration); eight entries' loads in flight at once, partial sum
      // k mod 4 taking entries in increasing order
      for (int k = kb[q]; k < ke[q]; k += 8) {
        T v[8], pcol[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const bool in = k + j < ke[q];
          const int c = in ? __ldg(ci + k + j) : 0;
          v[j] = in ? __ldg(vals + k + j) : T(0);
          const T po = in ? __ldcg(pold + c) : T(0);
          pcol[j] = (P3 || first) ? po : (in ? __ldcg(r + c) : T(0)) + beta * po;
        }
        s0 += v[0] * pcol[0];
        if (k + 1 < ke[q]) s1 += v[1] * pcol[1];
        if (k + 2 < ke[q]) s2 += v[2] * pcol[2];
        if (k + 3 < ke[q]) s3 += v[3] * pcol[3];
        if (k + 4 < ke[q]) s0 += v[4] * pcol[4];
        if (k + 5 < ke[q]) s1 += v[5] * pcol[5];
        if (k + 6 < ke[q]) s2 += v[6] * pcol[6];
        if (k + 7 < ke[q]) s3 += v[7] * pcol[7];
      }
      api[q] = dm[q] ? T(0) : (s0 + s1) + (s2 + s3);
      if constexpr (!P3) {
        const T pn = first ? pi[q] : ri[q] + beta * pi[q];
        pi[q] = pn;
        pnew[g0 + q * G] = pn;
      }
      s += (double)pi[q] * (double)api[q];
    }
    s = cta_tree_sum(s, red);
    if (threadIdx.x == 0) pa[blockIdx.x] = s;
    if (!grid_sync(count, target, err)) return;
    double f = 0.0;
    for (int k = threadIdx.x; k < nb; k += ST) f += __ldcg(pa + k);
    const double pAp = cta_tree_sum(f, red);
    const T alpha = (T)(rr / pAp);
    double s2 = 0.0;
#pragma unroll
    for (int q = 0; q < KM; ++q) {
      if (!own[q]) continue;
      xi[q] += alpha * pi[q];
      ri[q] -= alpha * api[q];
      r[g0 + q * G] = ri[q];
      s2 += (double)ri[q] * (double)ri[q];
    }
    s2 = cta_tree_sum(s2, red);
    if (threadIdx.x == 0) pb[blockIdx.x] = s2;
    if (!grid_sync(count, target, err)) return;
    double f2 = 0.0;
    for (int k = threadIdx.x; k < nb; k += ST) f2 += __ldcg(pb + k);
    const double rr_new = cta_tree_sum(f2, red);
    beta = (T)(rr_new / rr);
    rr = rr_new;
    first = false;
    if constexpr (!P3) {
      T* t = const_cast<T*>(pold);
      pold = pnew;
      pnew = t;
    }
    ++it;
    if (((it & 7) == 0 || it == maxit) && !(std::sqrt(rr) / fnorm > rtol)) break;
  }
#pragma unroll
  for (int q = 0; q < KM; ++q)
    if (own[q]) x[g0 + q * G] = xi[q];
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    sc[0] = rr;
    *it_out = it;
  }
}

// Launches the one-launch CG with KM row chunks per thread; *launched stays
// false when its CTAs cannot all be resident at once (by the occupancy query,
// or when the launch itself reports too few SMs).
template <typename T, int KM, bool P3>
tg_status cg_loop_launch(const int32_t* rp, const int32_t* ci, const T* vals, const uint8_t* mask, T* x, T* r, T* p0,
                         T* p1, int64_t n, int nb, double* sc, double* pa, double* pb, unsigned int* loop,
                         double fnorm, double rtol, int maxit, cudaStream_t s, bool* launched) {
  *launched = false;
  int per_sm = 0;
  TG_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_cg_loop<T, KM, P3>, ST, 0));
  const int ncta = (int)std::min<int64_t>((int64_t)nb, (n + ST - 1) / ST);
  if ((int64_t)per_sm * tg::sm_count() < ncta) return TG_OK;
  unsigned long long* count = reinterpret_cast<unsigned long long*>(loop);
  int* it_out = reinterpret_cast<int*>(loop + 2);
  int* err = reinterpret_cast<int*>(loop + 3);
  void* args[] = {(void*)&rp,  (void*)&ci,    (void*)&vals,  (void*)&mask, (void*)&x,     (void*)&r,
                  (void*)&p0,  (void*)&p1,    (void*)&n,     (void*)&nb,   (void*)&sc,    (void*)&pa,
                  (void*)&pb,  (void*)&count, (void*)&fnorm, (void*)&rtol, (void*)&maxit, (void*)&it_out,
                  (void*)&err};
  const cudaError_t e =
      cudaLaunchCooperativeKernel((const void*)k_cg_loop<T, KM, P3>, dim3(ncta), dim3(ST), args, 0, s);
  if (e == cudaErrorCooperativeLaunchTooLarge) {
    (void)cudaGetLastError();  // fewer SMs than the occupancy query saw: the graph-captured loop serves
    return TG_OK;
  }
  TG_CK(e);
  *launched = true;
  return TG_OK;
}

struct Dev {
  std::vector<void*> bufs;
  ~Dev() {
    for (void* b : bufs) cudaFree(b);
  }
  cudaError_t alloc(void** p, size_t bytes) {
    cudaError_t e = cudaMalloc(p, bytes);
    if (e == cudaSuccess) bufs.push_back(*p);
    return e;
  }
};

template <typename T>
tg_status dot(const T* a, const T* b, int64_t n, double* partials, int nb, double* out, cudaStream_t s) {
  k_dot_partial<T><<<nb, ST, 0, s>>>(a, b, n, partials);
  k_dot_final<<<1, ST, 0, s>>>(partials, nb, out);
  TG_CK_LAUNCH("k_dot");
  return TG_OK;
}

// Work vectors of one CG solve (n entries each) and its scalars.
template <typename T>
struct CgWork {
  T *r, *pp, *Ap, *b;
  double* sc;        // [4]: rr, pAp, rr_new, ||F_I||^2
  double* partials;  // [nb] (the one-launch loop: [2 nb])
  int nb;
  // the one-launch loop (NULL: launch per kernel): four zeroed words, the
  // 64-bit barrier arrival count, the iteration count and the error flag
  unsigned int* loop = nullptr;
};

// Eight CG iterations captured once as a CUDA graph: the small systems of
// the solve are launch-bound, and one graph launch replaces 64 kernel
// launches.  The graph runs the same kernels in the same order, so the
// iterates are bitwise those of the plain loop.
struct CgGraph {
  cudaStream_t cs = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  ~CgGraph() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (cs) cudaStreamDestroy(cs);
  }
};

template <typename T>
tg_status cg(const tg_pattern* p, const void* vals_, const void* F_, const uint8_t* mask, void* x_, double rtol,
             int maxit, int* iters, double* relres, const CgWork<T>& w, cudaStream_t s, bool use_graph) {
  const int nc = tg::ncomp_of(p->el);
  const bool vec = nc > 1;
  const int64_t n = nc * p->N;
  const int32_t* rp = vec ? p->row_ptr_dof : p->row_ptr;
  const int32_t* ci = vec ? p->col_idx_dof : p->col_idx;
  const T* vals = static_cast<const T*>(vals_);
  const T* F = static_cast<const T*>(F_);
  T* x = static_cast<T*>(x_);
  T *r = w.r, *pp = w.pp, *Ap = w.Ap, *b = w.b;
  double *sc = w.sc, *partials = w.partials;
  const int nb = w.nb;
  if (n == 0) {  // no rows: nothing to solve (and no launch of zero CTAs)
    if (iters) *iters = 0;
    if (relres) *relres = 0.0;
    return TG_OK;
  }
  const int gv = tg::grid_for(n, ST), gs = tg::grid_for(4 * n, ST);
  if (mask) k_cg_zero_masked<T><<<gv, ST, 0, s>>>(x, mask, n);
  k_spmv<T><<<gs, ST, 0, s>>>(rp, ci, vals, x, Ap, n, mask);
  k_cg_init<T><<<gv, ST, 0, s>>>(F, Ap, mask, x, r, pp, b, n);
  TG_CK_LAUNCH("cg init");
  tg_status st;
  if ((st = dot<T>(b, b, n, partials, nb, sc + 3, s)) != TG_OK) return st;
  if ((st = dot<T>(r, r, n, partials, nb, sc + 0, s)) != TG_OK) return st;
  double h[4];
  TG_CK(cudaMemcpyAsync(h, sc, sizeof(h), cudaMemcpyDeviceToHost, s));
  TG_CK(cudaStreamSynchronize(s));
  const double fnorm = std::sqrt(h[3]);
  if (!(fnorm > 0)) {
    // F_I = 0: the solution of K_II x_I = 0 is x = 0, whatever the initial guess
    TG_CK(cudaMemsetAsync(x, 0, (size_t)n * sizeof(T), s));
    TG_CK(cudaStreamSynchronize(s));
    if (iters) *iters = 0;
    if (relres) *relres = 0.0;
    return TG_OK;
  }
  double rel = std::sqrt(h[0]) / fnorm;
  auto iteration = [&](cudaStream_t q) -> tg_status {
    k_spmv<T><<<gs, ST, 0, q>>>(rp, ci, vals, pp, Ap, n, mask);
    tg_status e;
    if ((e = dot<T>(pp, Ap, n, partials, nb, sc + 1, q)) != TG_OK) return e;
    k_cg_xr<T><<<gv, ST, 0, q>>>(x, r, pp, Ap, sc, n);
    if ((e = dot<T>(r, r, n, partials, nb, sc + 2, q)) != TG_OK) return e;
    k_cg_p<T><<<gv, ST, 0, q>>>(pp, r, sc, n);
    k_cg_shift<<<1, 1, 0, q>>>(sc);
    TG_CK_LAUNCH("cg iteration");
    return TG_OK;
  };
  int it = 0;
  if (w.loop && rel > rtol && maxit > 0) {
    // one cooperative launch for all iterations: up to four row chunks per
    // thread, and all CTAs resident at once
    const int64_t chunks = (n + (int64_t)nb * ST - 1) / ((int64_t)nb * ST);
    bool launched = false;
    double* pb = partials + nb;
    T* p1 = b;  // F_I is no longer needed: the second direction buffer
    // FP64 systems of at least kCgP3MinEntries matrix entries: the variant
    // with a third barrier (the FP64 FMA per entry read costs more)
    bool p3 = false;
    if constexpr (sizeof(T) == 8) p3 = (int64_t)nc * nc * p->nnz >= kCgP3MinEntries;
    auto launch = [&](auto km, auto p3c) {
      return cg_loop_launch<T, decltype(km)::value, decltype(p3c)::value>(
          rp, ci, vals, mask, x, r, pp, p1, n, nb, sc, partials, pb, w.loop, fnorm, rtol, maxit, s, &launched);
    };
    using K1 = std::integral_constant<int, 1>;
    using K2 = std::integral_constant<int, 2>;
    using K4 = std::integral_constant<int, 4>;
    using P2 = std::false_type;
    using P3 = std::integral_constant<bool, sizeof(T) == 8>;  // no FP32 instance of the P3 form
    if (chunks <= 1) st = p3 ? launch(K1{}, P3{}) : launch(K1{}, P2{});
    else if (chunks <= 2) st = p3 ? launch(K2{}, P3{}) : launch(K2{}, P2{});
    else if (chunks <= 4) st = p3 ? launch(K4{}, P3{}) : launch(K4{}, P2{});
    if (st != TG_OK) return st;
    if (launched) {
      int hw[2] = {0, 0};
      TG_CK(cudaMemcpyAsync(h, sc, sizeof(double), cudaMemcpyDeviceToHost, s));
      TG_CK(cudaMemcpyAsync(hw, w.loop + 2, sizeof(hw), cudaMemcpyDeviceToHost, s));
      TG_CK(cudaStreamSynchronize(s));
      if (hw[1]) {
        tg::set_error("tg_cg_solve: a grid barrier of the one-launch CG timed out");
        return TG_ERR_TIMEOUT;
      }
      if (iters) *iters = hw[0];
      if (relres) *relres = std::sqrt(h[0]) / fnorm;
      return TG_OK;
    }
  }
  CgGraph g;
  if (use_graph && rel > rtol && maxit >= 8) {
    TG_CK(cudaStreamCreateWithFlags(&g.cs, cudaStreamNonBlocking));
    TG_CK(cudaStreamBeginCapture(g.cs, cudaStreamCaptureModeThreadLocal));
    tg_status e = TG_OK;
    for (int k = 0; k < 8 && e == TG_OK; ++k) e = iteration(g.cs);
    cudaGraph_t graph = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(g.cs, &graph);
    g.graph = graph;
    if (e != TG_OK) return e;
    TG_CK(ce);
    TG_CK(cudaGraphInstantiate(&g.exec, g.graph, 0));
  }
  while (rel > rtol && it < maxit) {
    if (g.exec && it + 8 <= maxit) {
      TG_CK(cudaGraphLaunch(g.exec, s));
      it += 8;
    } else {
      if ((st = iteration(s)) != TG_OK) return st;
      ++it;
    }
    if ((it & 7) == 0 || it == maxit) {
      TG_CK(cudaMemcpyAsync(h, sc, sizeof(double), cudaMemcpyDeviceToHost, s));
      TG_CK(cudaStreamSynchronize(s));
      rel = std::sqrt(h[0]) / fnorm;
    }
  }
  TG_CK(cudaMemcpyAsync(h, sc, sizeof(double), cudaMemcpyDeviceToHost, s));
  TG_CK(cudaStreamSynchronize(s));
  if (iters) *iters = it;
  if (relres) *relres = std::sqrt(h[0]) / fnorm;
  return TG_OK;
}

// Partial dot products per reduction: twice the SM count, capped so that both
// forms of the solve (the no-alloc one keeps its partials in a 4 KB head)
// reduce over the same grid and give the same bits on any GPU.
constexpr size_t kNoAllocHead = 4096;
constexpr int kMaxPartials = (int)(kNoAllocHead / sizeof(double)) - 4;
inline int cg_partials() { return std::min(2 * tg::sm_count(), kMaxPartials); }

// Allocating form: the work vectors live for one call.
template <typename T>
tg_status cg_alloc(const tg_pattern* p, const void* vals, const void* F, const uint8_t* mask, void* x, double rtol,
                   int maxit, int* iters, double* relres, cudaStream_t s) {
  const int64_t n = tg::ncomp_of(p->el) * p->N;
  Dev d;
  CgWork<T> w;
  w.nb = cg_partials();
  // one allocation: scalars, barrier words and partials, then the four work
  // vectors, each rounded up to 256 bytes
  const size_t head = 16384, vb = ((size_t)n * sizeof(T) + 255) / 256 * 256;
  static_assert(4 * sizeof(double) + 4 * sizeof(unsigned int) + 2 * kMaxPartials * sizeof(double) <= 16384,
                "CG head");
  unsigned char* base = nullptr;
  TG_CK(d.alloc((void**)&base, head + 4 * vb));
  w.sc = reinterpret_cast<double*>(base);
  w.loop = reinterpret_cast<unsigned int*>(base + 4 * sizeof(double));
  w.partials = reinterpret_cast<double*>(base + 64);
  w.r = reinterpret_cast<T*>(base + head);
  w.pp = reinterpret_cast<T*>(base + head + vb);
  w.Ap = reinterpret_cast<T*>(base + head + 2 * vb);
  w.b = reinterpret_cast<T*>(base + head + 3 * vb);
  TG_CK(cudaMemsetAsync(w.loop, 0, 4 * sizeof(unsigned int), s));
  return cg<T>(p, vals, F, mask, x, rtol, maxit, iters, relres, w, s, true);
}

// ---------------------------------------------------------------- no-alloc form
// Scratch of tg_cg_solve_noalloc: a fixed device array in this module, so the
// call never allocates.  Layout: [0, 4 KB) scalars (4 doubles) and partial
// dot products (up to kNoAllocMaxPartials doubles), then the four work
// vectors, each rounded up to 256 bytes.
constexpr size_t kNoAllocBytes = TG_CG_NOALLOC_SCRATCH_BYTES;
static __device__ __align__(256) unsigned char g_cg_scratch[kNoAllocBytes];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
struct ScratchEntry {
  void* addr = nullptr;
  unsigned long long ctx = 0;  // identity of the context the address belongs to
};
ScratchEntry g_scratch[kMaxDevices];

// Unique identity of the current CUDA context (cuCtxGetCurrent + cuCtxGetId,
// reached through the runtime's driver entry points, so nothing links the
// driver library), or 0 when it cannot be read.  A context created after
// cudaDeviceReset has a new identity, and this module a new address in it.
unsigned long long current_ctx_id() {
  using GetCurrentFn = int (*)(void**);
  using GetIdFn = int (*)(void*, unsigned long long*);
  static GetCurrentFn get_cur = nullptr;
  static GetIdFn get_id = nullptr;
  static bool looked_up = false;
  if (!looked_up) {
    looked_up = true;
    void* f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, nullptr) == cudaSuccess)
      get_cur = reinterpret_cast<GetCurrentFn>(f);
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, nullptr) == cudaSuccess)
      get_id = reinterpret_cast<GetIdFn>(f);
  }
  void* ctx = nullptr;
  unsigned long long id = 0;
  if (!get_cur || !get_id || get_cur(&ctx) != 0 || !ctx || get_id(ctx, &id) != 0) return 0;
  return id;
}

// Device address of g_cg_scratch on the current device.  It is looked up
// once per device and context (the first call on a device, and the first
// after a cudaDeviceReset; every call when the context identity cannot be
// read); the lookup may load this module, so it must not happen inside a
// stream capture.
tg_status noalloc_scratch(unsigned char** out) {
  int dev = 0;
  TG_CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) {
    tg::set_error("device ordinal beyond the no-alloc scratch table");
    return TG_ERR_UNSUPPORTED;
  }
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  const unsigned long long ctx = current_ctx_id();
  ScratchEntry& ent = g_scratch[dev];
  if (ent.addr == nullptr || ctx == 0 || ent.ctx != ctx) {
    void* a = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&a, g_cg_scratch);
    if (e != cudaSuccess) return tg::cuda_fail(e, "cudaGetSymbolAddress(g_cg_scratch)", __FILE__, __LINE__);
    if (a == nullptr) {
      tg::set_error("cudaGetSymbolAddress(g_cg_scratch) returned a null address");
      return TG_ERR_CUDA;
    }
    ent.addr = a;
    ent.ctx = current_ctx_id();  // the lookup made the device's context current
  }
  *out = static_cast<unsigned char*>(ent.addr);
  return TG_OK;
}

inline size_t round256(size_t b) { return (b + 255) & ~size_t(255); }

template <typename T>
tg_status cg_noalloc(const tg_pattern* p, const void* vals, const void* F, const uint8_t* mask, void* x,
                     double rtol, int maxit, int* iters, double* relres, cudaStream_t s) {
  const int64_t n = tg::ncomp_of(p->el) * p->N;
  const size_t vb = round256((size_t)n * sizeof(T));
  if (kNoAllocHead + 4 * vb > kNoAllocBytes) {
    tg::set_error("tg_cg_solve_noalloc: " + std::to_string(n) + " rows need " +
                  std::to_string(kNoAllocHead + 4 * vb) + " bytes of scratch; the static scratch holds " +
                  std::to_string(kNoAllocBytes));
    return TG_ERR_UNSUPPORTED;
  }
  unsigned char* base = nullptr;
  tg_status st = noalloc_scratch(&base);
  if (st != TG_OK) return st;
  CgWork<T> w;
  w.sc = reinterpret_cast<double*>(base);
  w.partials = w.sc + 4;
  w.nb = cg_partials();
  w.r = reinterpret_cast<T*>(base + kNoAllocHead);
  w.pp = reinterpret_cast<T*>(base + kNoAllocHead + vb);
  w.Ap = reinterpret_cast<T*>(base + kNoAllocHead + 2 * vb);
  w.b = reinterpret_cast<T*>(base + kNoAllocHead + 3 * vb);
  // The scalars start at zero so that nothing of an earlier call can be read
  // back; the vectors and partials are fully written before they are read.
  TG_CK(cudaMemsetAsync(w.sc, 0, 4 * sizeof(double), s));
  // no graph here: instantiating one may allocate
  return cg<T>(p, vals, F, mask, x, rtol, maxit, iters, relres, w, s, false);
}

// out[s] = alpha * lam[row(s)] * U[col(s)]: the adjoint outer product
// dGamma/dK = lam U^T of Eq. (adj) restricted to the CSR pattern.
template <typename T>
__global__ void __launch_bounds__(ST) k_csr_outer(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                                  const T* __restrict__ lam, const T* __restrict__ U, T alpha,
                                                  T* __restrict__ out, int64_t n) {
  const int64_t row = (int64_t)blockIdx.x * (ST / 8) + (threadIdx.x >> 3);
  if (row >= n) return;
  const T l = alpha * lam[row];
  const int k1 = __ldg(rp + row + 1);
  for (int k = __ldg(rp + row) + (threadIdx.x & 7); k < k1; k += 8) out[k] = l * __ldg(U + __ldg(ci + k));
}

// out[i] = alpha x[i], zero on the rows the condensed system drops.
template <typename T>
__global__ void __launch_bounds__(ST) k_scale_masked(const T* __restrict__ x, const uint8_t* __restrict__ mask,
                                                     T alpha, T* __restrict__ out, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * ST + threadIdx.x; i < n; i += (int64_t)gridDim.x * ST)
    out[i] = (mask && mask[i]) ? T(0) : alpha * x[i];
}

template <typename T>
__global__ void __launch_bounds__(256) k_fma_rate(T* __restrict__ out, int iters, T a, T b) {
  T x[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) x[k] = T(threadIdx.x + k) * T(1e-3);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = fma(x[k], a, b);
  }
  T s = T(0);
#pragma unroll
  for (int k = 0; k < 8; ++k) s += x[k];
  out[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" {

tg_status tg_spmv(const tg_pattern* p, tg_dtype dtype, const void* vals, const void* x, void* y, tg_stream stream) {
  if (!p || (dtype != TG_F32 && dtype != TG_F64)) return TG_ERR_INVALID_ARG;
  const int nc = tg::ncomp_of(p->el);
  const bool vec = nc > 1;
  const int64_t n = nc * p->N;
  if (n == 0) return TG_OK;
  if ((nc * nc * p->nnz > 0 && !vals) || !x || !y) return TG_ERR_INVALID_ARG;
  const int32_t* rp = vec ? p->row_ptr_dof : p->row_ptr;
  const int32_t* ci = vec ? p->col_idx_dof : p->col_idx;
  cudaStream_t s = (cudaStream_t)stream;
  const int g = tg::grid_for(4 * n, ST);
  if (dtype == TG_F32)
    k_spmv<float><<<g, ST, 0, s>>>(rp, ci, (const float*)vals, (const float*)x, (float*)y, n, nullptr);
  else
    k_spmv<double><<<g, ST, 0, s>>>(rp, ci, (const double*)vals, (const double*)x, (double*)y, n, nullptr);
  TG_CK_LAUNCH("k_spmv");
  return TG_OK;
}

tg_status tg_cg_solve(const tg_pattern* p, tg_dtype dtype, const void* vals, const void* F, const uint8_t* dirichlet,
                      void* x, double rtol, int32_t maxit, int32_t* iters, double* relres, tg_stream stream) {
  if (!p || (dtype != TG_F32 && dtype != TG_F64) || !vals || !F || !x || maxit < 0 || !(rtol >= 0))
    return TG_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  int it = 0;
  double rr = 0;
  tg_status st = dtype == TG_F32 ? cg_alloc<float>(p, vals, F, dirichlet, x, rtol, maxit, &it, &rr, s)
                                 : cg_alloc<double>(p, vals, F, dirichlet, x, rtol, maxit, &it, &rr, s);
  if (iters) *iters = it;
  if (relres) *relres = rr;
  return st;
}

tg_status tg_cg_solve_noalloc(const tg_pattern* p, tg_dtype dtype, const void* vals, const void* F,
                              const uint8_t* dirichlet, void* x, double rtol, int32_t maxit, int32_t* iters,
                              double* relres, tg_stream stream) {
  if (!p || (dtype != TG_F32 && dtype != TG_F64) || !vals || !F || !x || maxit < 0 || !(rtol >= 0))
    return TG_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  int it = 0;
  double rr = 0;
  tg_status st = dtype == TG_F32 ? cg_noalloc<float>(p, vals, F, dirichlet, x, rtol, maxit, &it, &rr, s)
                                 : cg_noalloc<double>(p, vals, F, dirichlet, x, rtol, maxit, &it, &rr, s);
  if (iters) *iters = it;
  if (relres) *relres = rr;
  return st;
}

tg_status tg_csr_outer(const tg_pattern* p, tg_dtype dtype, const void* lam, const void* U, double alpha, void* out,
                       tg_stream stream) {
  if (!p || (dtype != TG_F32 && dtype != TG_F64)) return TG_ERR_INVALID_ARG;
  const int nc = tg::ncomp_of(p->el);
  const bool vec = nc > 1;
  const int64_t n = nc * p->N;
  if (nc * nc * p->nnz == 0) return TG_OK;  // no slot to write
  if (!lam || !U || !out) return TG_ERR_INVALID_ARG;
  const int32_t* rp = vec ? p->row_ptr_dof : p->row_ptr;
  const int32_t* ci = vec ? p->col_idx_dof : p->col_idx;
  cudaStream_t s = (cudaStream_t)stream;
  const int g = tg::grid_for(n, ST / 8);
  if (dtype == TG_F32)
    k_csr_outer<float><<<g, ST, 0, s>>>(rp, ci, (const float*)lam, (const float*)U, (float)alpha, (float*)out, n);
  else
    k_csr_outer<double><<<g, ST, 0, s>>>(rp, ci, (const double*)lam, (const double*)U, alpha, (double*)out, n);
  TG_CK_LAUNCH("k_csr_outer");
  return TG_OK;
}

tg_status tg_scale_masked(tg_dtype dtype, const void* x, const uint8_t* dirichlet, double alpha, void* out,
                          int64_t n, tg_stream stream) {
  if ((dtype != TG_F32 && dtype != TG_F64) || n < 0 || (n > 0 && (!x || !out))) return TG_ERR_INVALID_ARG;
  if (n == 0) return TG_OK;
  cudaStream_t s = (cudaStream_t)stream;
  const int g = (int)std::min<int64_t>(tg::grid_for(n, ST), 8 * tg::sm_count());
  if (dtype == TG_F32)
    k_scale_masked<float><<<g, ST, 0, s>>>((const float*)x, dirichlet, (float)alpha, (float*)out, n);
  else
    k_scale_masked<double><<<g, ST, 0, s>>>((const double*)x, dirichlet, alpha, (double*)out, n);
  TG_CK_LAUNCH("k_scale_masked");
  return TG_OK;
}

}  // extern "C"

namespace {

// The bounded wait of the pipelined kernels on a shared-memory barrier that
// nothing completes (no arrival, no copy): the wait gives up after max_tries
// polls and records TG_ERR_TIMEOUT in the status word, as the kernels do.
__global__ void k_diag_wait_timeout(unsigned long long* status, uint32_t max_tries) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    tg::mbar_init(&bar, 1);
    tg::fence_mbar_init();
  }
  __syncthreads();
  const bool ok = tg::mbar_wait(&bar, 0, max_tries);
  if (__syncthreads_or(!ok) && threadIdx.x == 0) tg::record_error(status, TG_ERR_TIMEOUT, 0);
}

// A grid barrier that never completes: CTA 1 leaves without arriving, CTA 0
// waits at most `limit` polls and gives up (err = 1).
__global__ void k_diag_grid_barrier(unsigned long long* count, int* err, unsigned int limit) {
  if (blockIdx.x != 0) return;
  unsigned long long target = 0;
  grid_sync(count, target, err, limit);
}

// y[i] = the FP64 reciprocal the P1 forward takes of |det J|.
__global__ void k_diag_recip(const double* __restrict__ x, double* __restrict__ y, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = tg::recip_fast(x[i]);
}

}  // namespace

extern "C" {

tg_status tg_diag_recip(const double* x, double* y, int64_t n, tg_stream stream) {
  if (n < 0 || (n > 0 && (!x || !y))) return TG_ERR_INVALID_ARG;
  if (n == 0) return TG_OK;
  k_diag_recip<<<(unsigned)std::min<int64_t>((n + 255) / 256, 4096), 256, 0, (cudaStream_t)stream>>>(x, y, n);
  TG_CK_LAUNCH("k_diag_recip");
  return TG_OK;
}

tg_status tg_diag_wait_timeout(const tg_pattern* p, int32_t max_tries, tg_stream stream) {
  if (!p || max_tries < 1 || max_tries > (1 << 22)) return TG_ERR_INVALID_ARG;
  k_diag_wait_timeout<<<1, 32, 0, (cudaStream_t)stream>>>(p->status, (uint32_t)max_tries);
  TG_CK_LAUNCH("k_diag_wait_timeout");
  return TG_OK;
}

tg_status tg_diag_grid_barrier_timeout(int32_t max_polls, tg_stream stream) {
  if (max_polls < 1 || max_polls > (int32_t)kGridPolls) return TG_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  Dev d;
  unsigned char* w = nullptr;
  TG_CK(d.alloc((void**)&w, 16));
  TG_CK(cudaMemsetAsync(w, 0, 16, s));
  unsigned long long* count = reinterpret_cast<unsigned long long*>(w);
  int* err = reinterpret_cast<int*>(w + 8);
  unsigned int limit = (unsigned int)max_polls;
  void* args[] = {(void*)&count, (void*)&err, (void*)&limit};
  TG_CK(cudaLaunchCooperativeKernel((const void*)k_diag_grid_barrier, dim3(2), dim3(ST), args, 0, s));
  int he = 0;
  TG_CK(cudaMemcpyAsync(&he, err, sizeof(int), cudaMemcpyDeviceToHost, s));
  TG_CK(cudaStreamSynchronize(s));
  if (he) {
    tg::set_error("tg_diag_grid_barrier_timeout: the grid barrier gave up, as intended");
    return TG_ERR_TIMEOUT;
  }
  return TG_OK;
}

tg_status tg_diag_fma_rate(tg_dtype dtype, double* flops, tg_stream stream) {
  if (!flops || (dtype != TG_F32 && dtype != TG_F64)) return TG_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const int blocks = 8 * tg::sm_count(), threads = 256;
  const int iters = dtype == TG_F64 ? 2048 : 65536;
  void* out = nullptr;
  TG_CK(cudaMalloc(&out, (size_t)blocks * threads * 8));
  cudaEvent_t e0, e1;
  TG_CK(cudaEventCreate(&e0));
  TG_CK(cudaEventCreate(&e1));
  float best = 1e30f;
  for (int rep = 0; rep < 4; ++rep) {
    TG_CK(cudaEventRecord(e0, s));
    if (dtype == TG_F64) k_fma_rate<double><<<blocks, threads, 0, s>>>((double*)out, iters, 0.999999, 1e-6);
    else k_fma_rate<float><<<blocks, threads, 0, s>>>((float*)out, iters, 0.999999f, 1e-6f);
    TG_CK(cudaEventRecord(e1, s));
    TG_CK(cudaEventSynchronize(e1));
    float ms = 0;
    TG_CK(cudaEventElapsedTime(&ms, e0, e1));
    if (rep > 0 && ms < best) best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  *flops = 2.0 * 8.0 * iters * (double)blocks * threads / (best * 1e-3);
  return TG_OK;
}

}  // extern "C"
