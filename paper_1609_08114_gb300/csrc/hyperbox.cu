// hyperbox.cu -- support functions of hyperboxes in closed form.
//
// Section 6, Eq. 8: max over l <= x <= u of c . x equals sum_i c_i h_i with
// h_i = l_i when c_i < 0 and h_i = u_i otherwise.  The paper runs one LP per
// 32-thread block with a single active thread.  Here the work is a pure HBM
// stream, so every lane owns one LP: each warp stages the contiguous rows of
// its 32 LPs (c, and l, u unless the box is shared) into shared memory with
// coalesced 16-byte loads, then each lane sums its own row from shared memory
// in index order from +0.0, rounding every product and every sum separately
// (no FMA contraction) so the result is reproducible bit for bit.
#include <map>
#include <mutex>
#include <tuple>

#include "lpb_internal.cuh"

namespace lpb {
namespace {

constexpr int kWarps = 8;
constexpr int kChunk = 32;   // staged row length: whole rows up to 32, column chunks beyond

__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }

// c < 0 (false for -0.0 and NaN).  For doubles the test runs on the integer
// bits: the FP64 unit of this GPU is the bottleneck of the FP64 sum already.
__device__ __forceinline__ bool negative(float c) { return c < 0.f; }
__device__ __forceinline__ bool negative(double c) {
  const unsigned long long u = static_cast<unsigned long long>(__double_as_longlong(c));
  const unsigned long long mag = u & 0x7fffffffffffffffull;
  return (u >> 63) && mag != 0ull && mag <= 0x7ff0000000000000ull;
}

// Warp-cooperative copy of `len` elements; 16-byte vectors when both ends are
// 16-byte aligned, scalar elements for the rest.
template <typename T>
__device__ __forceinline__ void warp_copy_in(T *dst, const T *src, int len, int lane) {
  const bool vec = ((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst)) & 15) == 0;
  int done = 0;
  if (vec) {
    constexpr int per = 16 / sizeof(T);
    const int nv = len / per;
    const int4 *s4 = reinterpret_cast<const int4 *>(src);
    int4 *d4 = reinterpret_cast<int4 *>(dst);
    for (int v = lane; v < nv; v += 32) d4[v] = __ldcs(s4 + v);
    done = nv * per;
  }
  for (int i = done + lane; i < len; i += 32) dst[i] = __ldcs(src + i);
}

template <typename T>
__device__ __forceinline__ void warp_copy_out(T *dst, const T *src, int len, int lane) {
  const bool vec = ((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst)) & 15) == 0;
  int done = 0;
  if (vec) {
    constexpr int per = 16 / sizeof(T);
    const int nv = len / per;
    const int4 *s4 = reinterpret_cast<const int4 *>(src);
    int4 *d4 = reinterpret_cast<int4 *>(dst);
    for (int v = lane; v < nv; v += 32) __stcs(d4 + v, s4[v]);
    done = nv * per;
  }
  for (int i = done + lane; i < len; i += 32) __stcs(dst + i, src[i]);
}

template <typename T, bool kShared>
__global__ void __launch_bounds__(kWarps * 32) hyperbox_kernel(HyperboxParams P) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int n = P.n;
  const size_t box_elems = kShared ? ((2 * size_t(n) * sizeof(T) + 15) & ~size_t(15)) / sizeof(T) : 0;
  T *sbox = reinterpret_cast<T *>(smem);
  const int rs = n > kChunk ? kChunk + 1 : n;
  const size_t per_warp = size_t(kShared ? 1 : 3) * 32 * rs;
  T *wc = sbox + box_elems + size_t(wid) * per_warp;
  T *wl = wc + 32 * size_t(rs);
  T *wu = wl + 32 * size_t(rs);
  const T *gc = static_cast<const T *>(P.c);
  const T *gl = static_cast<const T *>(P.l);
  const T *gu = static_cast<const T *>(P.u);
  if (kShared) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) { sbox[i] = gl[i]; sbox[n + i] = gu[i]; }
    __syncthreads();
  }
  const int64_t nwarps = (P.count + 31) / 32;
  if (n > kChunk) {
    // Long rows: stage 32 columns of the warp's 32 rows at a time; the running
    // sum carries over so the order stays i = 0, 1, ..., n-1.
    for (int64_t w = int64_t(blockIdx.x) * kWarps + wid; w < nwarps; w += int64_t(gridDim.x) * kWarps) {
      const int64_t lp0 = w * 32;
      const int cnt = int(P.count - lp0 < 32 ? P.count - lp0 : 32);
      T acc = T(0);
      for (int i0 = 0; i0 < n; i0 += kChunk) {
        const int ch = min(kChunk, n - i0);
        for (int r = 0; r < cnt; ++r) {
          const int64_t g = (lp0 + r) * n + i0;
          if (lane < ch) {
            wc[r * rs + lane] = __ldcs(gc + g + lane);
            if (!kShared) {
              wl[r * rs + lane] = __ldcs(gl + g + lane);
              wu[r * rs + lane] = __ldcs(gu + g + lane);
            }
          }
        }
        __syncwarp();
        if (lane < cnt) {
          for (int i = 0; i < ch; ++i) {
            const T ci = wc[lane * rs + i];
            const T h = negative(ci) ? (kShared ? sbox[i0 + i] : wl[lane * rs + i])
                                    : (kShared ? sbox[n + i0 + i] : wu[lane * rs + i]);
            acc = add_rn(acc, mul_rn(ci, h));
            wc[lane * rs + i] = h;
          }
        }
        __syncwarp();
        if (P.x)
          for (int r = 0; r < cnt; ++r)
            if (lane < ch) __stcs(static_cast<T *>(P.x) + (lp0 + r) * n + i0 + lane, wc[r * rs + lane]);
        __syncwarp();
      }
      if (lane < cnt) static_cast<T *>(P.obj)[lp0 + lane] = acc;
    }
    return;
  }
  for (int64_t w = int64_t(blockIdx.x) * kWarps + wid; w < nwarps; w += int64_t(gridDim.x) * kWarps) {
    const int64_t lp0 = w * 32;
    const int cnt = int(P.count - lp0 < 32 ? P.count - lp0 : 32);
    const int len = cnt * n;
    warp_copy_in(wc, gc + lp0 * n, len, lane);
    if (!kShared) {
      warp_copy_in(wl, gl + lp0 * n, len, lane);
      warp_copy_in(wu, gu + lp0 * n, len, lane);
    }
    __syncwarp();
    if (lane < cnt) {
      T acc = T(0);
      T *row_c = wc + size_t(lane) * n;
      const T *row_l = kShared ? sbox : wl + size_t(lane) * n;
      const T *row_u = kShared ? sbox + n : wu + size_t(lane) * n;
      for (int i = 0; i < n; ++i) {
        const T ci = row_c[i];
        const T h = negative(ci) ? row_l[i] : row_u[i];
        acc = add_rn(acc, mul_rn(ci, h));
        if (P.x) row_c[i] = h;          // the maximiser replaces c in place
      }
      static_cast<T *>(P.obj)[lp0 + lane] = acc;
    }
    __syncwarp();
    if (P.x) {
      warp_copy_out(static_cast<T *>(P.x) + lp0 * n, wc, len, lane);
      __syncwarp();
    }
  }
}

// ---- TMA-streamed variant ------------------------------------------------
//
// CTA of `lps` threads, one LP per thread per chunk; chunk k of the CTA covers
// LPs (blockIdx.x + k * gridDim.x) * lps ...  Thread 0 issues one bulk copy per
// array per chunk into stage k % kStages and arms the stage's mbarrier with the
// byte count; everyone waits on the barrier (bounded), sums its row from shared
// memory, and the stage is refilled once all threads are past it.

template <typename T, bool kShared, int kStages>
__global__ void hyperbox_tma_kernel(HyperboxParams P, int lps, uint32_t *err) {
  extern __shared__ __align__(128) unsigned char hb_smem[];
  __shared__ __align__(8) uint64_t bars[kStages];
  const int tid = threadIdx.x, n = P.n;
  const size_t row_bytes = size_t(n) * sizeof(T);
  const size_t arr_bytes = size_t(lps) * row_bytes;          // one array of one chunk (multiple of 16)
  const int narr = kShared ? 1 : 3;
  const size_t box_bytes = kShared ? ((2 * row_bytes + 127) & ~size_t(127)) : 0;
  T *sbox = reinterpret_cast<T *>(hb_smem);
  unsigned char *stage0 = hb_smem + box_bytes;
  const size_t stage_bytes = (narr * arr_bytes + 127) & ~size_t(127);
  const int64_t nfull = P.count / lps;                      // chunks loaded by TMA
  const T *gc = static_cast<const T *>(P.c), *gl = static_cast<const T *>(P.l), *gu = static_cast<const T *>(P.u);
  if (kShared)
    for (int i = tid; i < n; i += blockDim.x) { sbox[i] = gl[i]; sbox[n + i] = gu[i]; }
  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) mbar_init(&bars[s], 1);
    fence_mbar_init();
  }
  __syncthreads();
  auto issue = [&](int64_t chunk, int s) {                   // thread 0 only
    unsigned char *dst = stage0 + size_t(s) * stage_bytes;
    const int64_t lp0 = chunk * lps;
    mbar_expect_tx(&bars[s], unsigned(narr * arr_bytes));
    bulk_load(dst, gc + lp0 * n, unsigned(arr_bytes), &bars[s]);
    if (!kShared) {
      bulk_load(dst + arr_bytes, gl + lp0 * n, unsigned(arr_bytes), &bars[s]);
      bulk_load(dst + 2 * arr_bytes, gu + lp0 * n, unsigned(arr_bytes), &bars[s]);
    }
  };
  // chunks of this CTA: blockIdx.x, blockIdx.x + gridDim.x, ...
  const int64_t mine = nfull > blockIdx.x ? (nfull - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  if (tid == 0)
    for (int s = 0; s < kStages && s < mine; ++s) issue(blockIdx.x + int64_t(s) * gridDim.x, s);
  bool failed = false;
  for (int64_t k = 0; k < mine; ++k) {
    const int s = int(k % kStages);
    const unsigned phase = unsigned((k / kStages) & 1);
    const int64_t chunk = blockIdx.x + k * gridDim.x;
    failed = !mbar_wait_for(&bars[s], phase, kCopyWaitNs);
    if (__syncthreads_or(failed)) {
      if (tid == 0) {
        atomicOr(err, ERR_WAIT_TIMEOUT);
        // Let the copies this CTA issued land before it exits (bounded again, by
        // kDrainWaitNs in all): stage s2 still expects the completion of chunk
        // k2 = k, k+1, ... < mine.  If they do not, the CTA leaves with copies
        // outstanding and says so in the error word.
        const unsigned long long t0 = global_ns();
        for (int64_t k2 = k; k2 < k + kStages && k2 < mine; ++k2) {
          const unsigned long long used = global_ns() - t0;
          if (used > kDrainWaitNs ||
              !mbar_wait_for(&bars[k2 % kStages], unsigned((k2 / kStages) & 1), kDrainWaitNs - used)) {
            atomicOr(err, ERR_COPY_IN_FLIGHT);
            break;
          }
        }
      }
      __syncthreads();
      break;
    }
    T *wc = reinterpret_cast<T *>(stage0 + size_t(s) * stage_bytes);
    const T *wl = reinterpret_cast<const T *>(reinterpret_cast<unsigned char *>(wc) + arr_bytes);
    const T *wu = reinterpret_cast<const T *>(reinterpret_cast<unsigned char *>(wc) + 2 * arr_bytes);
    const int64_t lp = chunk * lps + tid;
    {
      T acc = T(0);
      T *rc = wc + size_t(tid) * n;
      const T *rl = kShared ? sbox : wl + size_t(tid) * n;
      const T *ru = kShared ? sbox + n : wu + size_t(tid) * n;
      for (int i = 0; i < n; ++i) {
        const T ci = rc[i];
        const T h = negative(ci) ? rl[i] : ru[i];
        acc = add_rn(acc, mul_rn(ci, h));
        if (P.x) rc[i] = h;
      }
      static_cast<T *>(P.obj)[lp] = acc;
    }
    __syncthreads();                                          // stage s fully read
    if (tid == 0) {
      if (P.x) {                                              // the maximisers go back by bulk store
        fence_async_smem();
        bulk_store(static_cast<T *>(P.x) + chunk * lps * n, wc, unsigned(arr_bytes));
        bulk_commit();
        bulk_wait_read();
      }
      if (k + kStages < mine) {
        fence_async_smem();
        issue(blockIdx.x + (k + kStages) * gridDim.x, s);
      }
    }
  }
  if (tid == 0 && P.x) bulk_wait_read();
  // The partial last chunk (count % lps LPs) with plain loads, by the last CTA.
  const int64_t tail0 = nfull * lps;
  if (blockIdx.x == gridDim.x - 1 && tail0 < P.count) {
    const int64_t lp = tail0 + tid;
    if (lp < P.count) {
      T acc = T(0);
      for (int i = 0; i < n; ++i) {
        const T ci = gc[lp * n + i];
        const T h = negative(ci) ? (kShared ? sbox[i] : gl[lp * n + i]) : (kShared ? sbox[n + i] : gu[lp * n + i]);
        acc = add_rn(acc, mul_rn(ci, h));
        if (P.x) static_cast<T *>(P.x)[lp * n + i] = h;
      }
      static_cast<T *>(P.obj)[lp] = acc;
    }
  }
}

}  // namespace

// Row length of a staged row: the whole row, or a padded column chunk (the
// odd stride keeps lanes reading their own rows on distinct banks).
static __host__ __device__ inline int staged_row(int n) { return n > kChunk ? kChunk + 1 : n; }

size_t hyperbox_smem_bytes(int n, int elem_bytes, bool shared_box) {
  const size_t box = shared_box ? ((2 * size_t(n) * elem_bytes + 15) & ~size_t(15)) : 0;
  return box + size_t(kWarps) * (shared_box ? 1 : 3) * 32 * size_t(staged_row(n)) * elem_bytes;
}

namespace {

template <typename T, bool S>
cudaError_t launch_t(const HyperboxParams &p, cudaStream_t s) {
  const size_t smem = hyperbox_smem_bytes(p.n, int(sizeof(T)), S);
  cudaError_t e = cudaFuncSetAttribute(hyperbox_kernel<T, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, hyperbox_kernel<T, S>, kWarps * 32, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const int64_t need = (p.count + 32 * kWarps - 1) / (32 * kWarps);
  const int grid = int(need < int64_t(sms) * per_sm ? need : int64_t(sms) * per_sm);
  hyperbox_kernel<T, S><<<grid, kWarps * 32, smem, s>>>(p);
  return cudaGetLastError();
}

}  // namespace

namespace {

// Shared memory of the TMA variant with `lps` LPs per chunk and `stages` stages.
size_t tma_smem(int n, int es, bool shared, int lps, int stages) {
  const size_t row = size_t(n) * es;
  const size_t box = shared ? ((2 * row + 127) & ~size_t(127)) : 0;
  const size_t stage = ((shared ? 1 : 3) * size_t(lps) * row + 127) & ~size_t(127);
  return box + size_t(stages) * stage;
}

constexpr size_t kTmaSmemMax = size_t(200) * 1024;

// Resident CTAs per SM of `fn` at `smem` bytes, cached per (device, kernel,
// CTA size, shared memory): the lookup runs once per shape, not per call.
int cached_occupancy(const void *fn, int threads, size_t smem) {
  static std::mutex mu;
  static std::map<std::tuple<int, const void *, int, size_t>, int> table;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  const auto key = std::make_tuple(dev, fn, threads, smem);
  std::lock_guard<std::mutex> lock(mu);
  const auto it = table.find(key);
  if (it != table.end()) return it->second;
  int per_sm = 0;
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kTmaSmemMax)) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem) != cudaSuccess)
    per_sm = 0;
  table.emplace(key, per_sm);
  return per_sm;
}

template <typename T, bool S>
cudaError_t launch_tma(const HyperboxParams &p, uint32_t *err, cudaStream_t s, bool *launched) {
  *launched = false;
  const void *fns[2] = {reinterpret_cast<const void *>(hyperbox_tma_kernel<T, S, 1>),
                        reinterpret_cast<const void *>(hyperbox_tma_kernel<T, S, 2>)};
  // The row staging needs `stages * (1 or 3) * n` elements of shared memory per
  // thread; the shape with the most resident threads per SM wins (double
  // buffering, then longer chunks, on a tie).
  int best_threads = 0, best_stages = 0, best_lps = 0, best_per_sm = 0;
  for (int stages = 2; stages >= 1; --stages)
    for (int lps = 128; lps >= 32; lps /= 2) {
      const size_t smem = tma_smem(p.n, int(sizeof(T)), S, lps, stages);
      if (smem > kTmaSmemMax) continue;
      const int per_sm = cached_occupancy(fns[stages - 1], lps, smem);
      if (per_sm * lps > best_threads) {
        best_threads = per_sm * lps; best_stages = stages; best_lps = lps; best_per_sm = per_sm;
      }
    }
  if (best_threads == 0) return cudaSuccess;               // caller falls back
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const size_t smem = tma_smem(p.n, int(sizeof(T)), S, best_lps, best_stages);
  const int64_t nfull = p.count / best_lps;
  int64_t grid = int64_t(sms) * best_per_sm;
  if (grid > nfull) grid = nfull;
  if (grid < 1) grid = 1;
  if (best_stages == 2) hyperbox_tma_kernel<T, S, 2><<<int(grid), best_lps, smem, s>>>(p, best_lps, err);
  else hyperbox_tma_kernel<T, S, 1><<<int(grid), best_lps, smem, s>>>(p, best_lps, err);
  *launched = true;
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_hyperbox(const HyperboxParams &p, uint32_t *err, cudaStream_t s) {
  if (p.count == 0) return cudaSuccess;
  // Bulk copies need 16-byte aligned addresses; chunks of 32k rows are whole
  // multiples of 16 bytes.
  const uintptr_t al = reinterpret_cast<uintptr_t>(p.c) | reinterpret_cast<uintptr_t>(p.obj) |
                       (p.shared_box ? 0 : reinterpret_cast<uintptr_t>(p.l) | reinterpret_cast<uintptr_t>(p.u)) |
                       reinterpret_cast<uintptr_t>(p.x);
  if ((al & 15) == 0) {
    bool launched = false;
    cudaError_t e;
    if (p.dtype == LPB_DTYPE_F64)
      e = p.shared_box ? launch_tma<double, true>(p, err, s, &launched) : launch_tma<double, false>(p, err, s, &launched);
    else
      e = p.shared_box ? launch_tma<float, true>(p, err, s, &launched) : launch_tma<float, false>(p, err, s, &launched);
    if (launched || e != cudaSuccess) return e;
  }
  if (p.dtype == LPB_DTYPE_F64)
    return p.shared_box ? launch_t<double, true>(p, s) : launch_t<double, false>(p, s);
  return p.shared_box ? launch_t<float, true>(p, s) : launch_t<float, false>(p, s);
}

}  // namespace lpb
