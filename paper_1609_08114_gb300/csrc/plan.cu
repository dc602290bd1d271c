// plan.cu -- size classes and largest-first work lists for mixed-size batches.
//
// Every LP gets a class from fixed size thresholds (the register-tableau
// templates, then the shared-memory / L2-slot tableau kernel for the rest),
// and each class's list is ordered by decreasing estimated cost
// (m + 1)(n + 1), so that each persistent launch starts its largest LPs first
// and the small ones fill the tail.  Three small kernels -- histogram, scan,
// scatter -- keep every count on the device, so a solve needs no host
// synchronisation.  Within one cost bucket the order follows the atomic
// arrival order; results do not depend on it.
#include "lpb_internal.cuh"

namespace lpb {
namespace {

constexpr int kBuckets = 64;

__device__ __forceinline__ int cost_bucket(int m, int n) {
  // buckets of half a unit of log2((m + 1)(n + 1)), largest first
  const float c = log2f(float(max(m, 0) + 1) * float(max(n, 0) + 1));
  int q = int(c * 2.0f);
  q = q < 0 ? 0 : (q >= kBuckets ? kBuckets - 1 : q);
  return kBuckets - 1 - q;
}

__device__ __forceinline__ int class_of(const ClassPlanParams &P, int m, int n) {
  for (int c = 0; c < P.nclass - 1; ++c)
    if (m <= P.max_m[c] && n <= P.max_n[c]) return c;
  return P.nclass - 1;
}

__global__ void classify_hist(ClassPlanParams P) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P.count; i += gridDim.x * blockDim.x) {
    const int c = class_of(P, P.m[i], P.n[i]);
    atomicAdd(&P.hist[c * kBuckets + cost_bucket(P.m[i], P.n[i])], 1);
  }
}

__global__ void classify_scan(ClassPlanParams P) {
  // one warp per class: exclusive scan of its bucket counts
  const int c = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (c >= P.nclass) return;
  int base = 0;
  for (int q0 = 0; q0 < kBuckets; q0 += 32) {
    const int v = P.hist[c * kBuckets + q0 + lane];
    int incl = v;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const int t = __shfl_up_sync(kFull, incl, off);
      if (lane >= off) incl += t;
    }
    P.hist[c * kBuckets + q0 + lane] = base + incl - v;
    base += __shfl_sync(kFull, incl, 31);
  }
  if (lane == 0) P.class_count[c] = base;
}

__global__ void classify_scatter(ClassPlanParams P) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P.count; i += gridDim.x * blockDim.x) {
    const int c = class_of(P, P.m[i], P.n[i]);
    const int pos = atomicAdd(&P.hist[c * kBuckets + cost_bucket(P.m[i], P.n[i])], 1);
    if (pos < P.count) P.lists[int64_t(c) * P.count + pos] = i;
  }
}

}  // namespace

size_t classify_hist_bytes(int nclass) { return size_t(nclass) * kBuckets * sizeof(int32_t); }

cudaError_t launch_classify(const ClassPlanParams &p, int sms, cudaStream_t s) {
  if (p.nclass < 1 || p.nclass > kMaxClasses) return cudaErrorInvalidValue;
  cudaError_t e = cudaMemsetAsync(p.hist, 0, classify_hist_bytes(p.nclass), s);
  if (e != cudaSuccess) return e;
  const int threads = 256;
  int grid = (p.count + threads - 1) / threads;
  if (grid > 4 * sms) grid = 4 * sms;
  if (grid < 1) grid = 1;
  classify_hist<<<grid, threads, 0, s>>>(p);
  classify_scan<<<1, 32 * kMaxClasses, 0, s>>>(p);
  classify_scatter<<<grid, threads, 0, s>>>(p);
  return cudaGetLastError();
}

}  // namespace lpb
