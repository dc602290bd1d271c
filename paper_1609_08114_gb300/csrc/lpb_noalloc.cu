// lpb_noalloc.cu -- lpb_solve_noalloc: the batched solve with its scratch in a
// fixed device array that the library itself owns.
//
// Who needs this: callers that cannot allocate device memory on their own --
// for example plug-ins hosted by a framework that hands out all device memory
// from its own pool and does not let guests call cudaMalloc, or a tight
// control loop where cudaMalloc / cudaFree are off limits because they may
// synchronise the whole device.  Such a caller still owns the inputs and the
// outputs; only the solver's scratch (work lists, per-CTA tableau slots, the
// basis buffer when the caller passes none, the work counters) moves into the
// array below.
//
// Costs and limits:
//  * the array is kNoAllocBytes (32 MiB) of device memory, held by every GPU
//    on which this library's module is loaded, until the process exits;
//  * one array per device serves every call, so calls that overlap on the GPU
//    (different streams, threads or host processes sharing the context) race
//    on it and corrupt each other's results -- serialise them;
//  * a batch whose scratch exceeds the array is rejected up front with
//    LPB_ENOMEM, before anything is launched.
#include <mutex>

#include "lpb_internal.cuh"

namespace {

constexpr size_t kNoAllocBytes = size_t(32) << 20;
constexpr size_t kHeaderBytes = 256;   // work counters and the error word

// Host code must not use this name as a device address: it resolves to a
// host-side shadow.  The device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

struct DeviceScratch {
  bool ready = false;
  unsigned char *base = nullptr;   // device address of g_noalloc_scratch on this device
  lpb::DeviceInfo info{};
};

constexpr int kMaxDevices = 64;
DeviceScratch g_scratch[kMaxDevices];
std::mutex g_mutex;

// One-time set-up per device, with that device current: resolve the array's
// device address and read the attributes the pass plan needs.
lpb_err scratch_for_current_device(DeviceScratch **out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return LPB_ECUDA;
  if (dev < 0 || dev >= kMaxDevices) return LPB_EUNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_mutex);
  DeviceScratch &s = g_scratch[dev];
  if (!s.ready) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) return LPB_ECUDA;
    int sms = 0, optin = 0, l2 = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev) != cudaSuccess)
      return LPB_ECUDA;
    s.base = static_cast<unsigned char *>(p);
    s.info = lpb::DeviceInfo{sms, size_t(optin), size_t(l2)};
    s.ready = true;
  }
  *out = &s;
  return LPB_OK;
}

}  // namespace

extern "C" lpb_err lpb_solve_noalloc(const lpb_batch *b, const lpb_options *o, const lpb_result *r,
                                     void *stream) {
  if (!b || !o || !r) return LPB_EINVAL;
  if (b->count < 0) return LPB_EINVAL;
  if (b->count == 0) return LPB_OK;
  if (!b->m || !b->n || !b->a_off || !b->b_off || !b->c_off || !b->A || !b->b || !b->c) return LPB_EINVAL;
  if (!r->status || !r->obj || !r->x) return LPB_EINVAL;
  DeviceScratch *s = nullptr;
  lpb_err e = scratch_for_current_device(&s);
  if (e != LPB_OK) return e;
  size_t need = 0;
  e = lpb::solve_workspace_bytes(s->info, b, o, r->basis != nullptr, &need);
  if (e != LPB_OK) return e;
  if (need > kNoAllocBytes - kHeaderBytes) return LPB_ENOMEM;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int32_t *ctr = reinterpret_cast<int32_t *>(s->base);
  uint32_t *err = reinterpret_cast<uint32_t *>(s->base + lpb::kCounters * sizeof(int32_t));
  // The array keeps whatever the previous call left: the error word starts
  // this call at zero (run_solve zeroes the counters itself).
  if (cudaMemsetAsync(err, 0, sizeof(uint32_t), st) != cudaSuccess) return LPB_ECUDA;
  return lpb::run_solve(s->info, ctr, err, b, o, r, s->base + kHeaderBytes, kNoAllocBytes - kHeaderBytes, st,
                        nullptr, nullptr);
}

// The device error word of lpb_solve_noalloc lives in the same fixed array, so
// its callers read it here rather than through a handle: wait for `stream`,
// copy the word into the caller's host variable, clear it.  No allocation.
extern "C" lpb_err lpb_noalloc_sync_error(void *stream, uint32_t *word) {
  DeviceScratch *s = nullptr;
  const lpb_err e = scratch_for_current_device(&s);
  if (e != LPB_OK) return e;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  uint32_t *err = reinterpret_cast<uint32_t *>(s->base + lpb::kCounters * sizeof(int32_t));
  uint32_t v = 0;
  if (cudaMemcpyAsync(&v, err, sizeof(v), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaMemsetAsync(err, 0, sizeof(uint32_t), st) != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess)
    return LPB_ECUDA;
  if (word) *word = v;
  return v ? LPB_EDEVICE : LPB_OK;
}
