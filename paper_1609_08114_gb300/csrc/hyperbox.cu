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
#include "lpb_internal.cuh"

namespace lpb {
namespace {

constexpr int kWarps = 8;
constexpr int kChunk = 32;   // staged row length: whole rows up to 32, column chunks beyond

__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }

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
            const T h = (ci < T(0)) ? (kShared ? sbox[i0 + i] : wl[lane * rs + i])
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
        const T h = (ci < T(0)) ? row_l[i] : row_u[i];
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

cudaError_t launch_hyperbox(const HyperboxParams &p, cudaStream_t s) {
  if (p.count == 0) return cudaSuccess;
  if (p.dtype == LPB_DTYPE_F64)
    return p.shared_box ? launch_t<double, true>(p, s) : launch_t<double, false>(p, s);
  return p.shared_box ? launch_t<float, true>(p, s) : launch_t<float, false>(p, s);
}

}  // namespace lpb
