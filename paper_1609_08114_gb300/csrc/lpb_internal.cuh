// lpb_internal.cuh -- device-side types and helpers shared by the liblpb kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <climits>
#include <cmath>

#include "lpb.h"

namespace lpb {

constexpr unsigned kFull = 0xffffffffu;
// Reduction keys pack (variable index << kIdxBits) | (row or column).  Rows and
// columns stay below 2^13, variables below 3 * 2^13, so keys fit in 29 bits.
constexpr int kIdxBits = 13;
constexpr int kIdxMask = (1 << kIdxBits) - 1;
constexpr int kMaxDim = 4096;           // largest m or n accepted by this build

// Bits of the handle's device error word.
enum : uint32_t {
  ERR_LIST_OVERFLOW = 1u,   // a work list received more entries than it can hold
  ERR_SLOT_OVERFLOW = 2u,   // an LP did not fit the tableau slot of its launch
  ERR_BAD_LAUNCH = 4u,      // a kernel was launched with an inconsistent configuration
  ERR_WAIT_TIMEOUT = 8u,    // a bounded wait on an asynchronous copy gave up
  ERR_COPY_IN_FLIGHT = 16u, // a CTA left while copies into its shared memory were still
                            // outstanding (only after ERR_WAIT_TIMEOUT and a second deadline):
                            // the shared memory of CTAs that run on that SM after it may be
                            // overwritten, so no result of that launch can be trusted
};

enum Mode : int { MODE_FP64 = 0, MODE_FP32_REFINE = 1, MODE_FP32 = 2 };
constexpr int STATUS_PENDING = -1;      // internal: the LP waits for a later pass

struct BatchDev {
  int count, max_m, max_n, dtype;
  const int32_t *m, *n;
  const int64_t *a_off, *b_off, *c_off;
  const void *A, *b, *c;
};

struct ResultDev {
  int32_t *status, *iters;
  double *obj, *x, *y;
  int32_t *basis;
  const int64_t *y_off;   // where y and basis of LP k start; null: at b_off[k] (packed like b)
};

// A list of LP indices with a device-resident length.  `items == nullptr`
// means the identity list 0..B.count-1.
struct WorkList {
  const int32_t *items;
  const int32_t *count;
};

// Input element `i` of an array of dtype `dt`, widened to double.
__device__ __forceinline__ double ld_in(const void *p, int64_t i, int dt) {
  return dt == LPB_DTYPE_F64 ? __ldg(static_cast<const double *>(p) + i)
                             : static_cast<double>(__ldg(static_cast<const float *>(p) + i));
}

// Round a double to the nearest float (ties to even) with integer operations:
// on this GPU the FP64 unit, which also performs double->float conversions,
// runs at a small fraction of the FP32 rate.  Normal results take the integer
// path (the top 23 of the 52 mantissa bits, rounded on the 29 dropped bits);
// zero keeps its sign; subnormal, overflowing and non-finite values, which the
// solver does not expect, use the hardware conversion.
__device__ __forceinline__ float d2f_rn(double d) {
  const unsigned long long u = static_cast<unsigned long long>(__double_as_longlong(d));
  const unsigned hi = unsigned(u >> 32), lo = unsigned(u);
  const unsigned sign = hi & 0x80000000u, ahi = hi & 0x7fffffffu;
  const unsigned e = ahi >> 20;
  if (e >= 897u && e <= 1150u) {          // biased exponents of the normal floats
    unsigned f = ((ahi - (896u << 20)) << 3) | (lo >> 29);
    const unsigned rem = lo & 0x1fffffffu;
    f += (rem > 0x10000000u) || (rem == 0x10000000u && (f & 1u));
    return __uint_as_float(sign | f);
  }
  if ((ahi | lo) == 0u) return __uint_as_float(sign);
  return __double2float_rn(d);
}

// Float -> double, exact, in integer operations for normal floats and zeros
// (the hardware conversion runs on the slow FP64 unit); subnormal, infinite
// and NaN inputs take the hardware conversion.
__device__ __forceinline__ double f2d_exact(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned e = (u >> 23) & 0xffu;
  if (e != 0u && e != 0xffu) {
    const unsigned hi = (u & 0x80000000u) | ((e + (1023u - 127u)) << 20) | ((u >> 3) & 0xfffffu);
    const unsigned lo = u << 29;
    return __hiloint2double(int(hi), int(lo));
  }
  if ((u & 0x7fffffffu) == 0u) return __hiloint2double(int(u & 0x80000000u), 0);
  return double(f);
}

// a >= b for finite doubles, compared as integers (sign-magnitude order) so
// that no FP64 instruction is spent; false when a is not finite.
__device__ __forceinline__ unsigned long long d2ord(double d) {
  const unsigned long long u = static_cast<unsigned long long>(__double_as_longlong(d));
  return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
}
__device__ __forceinline__ double neg_bits(double d) {   // -d by the sign bit
  return __longlong_as_double(__double_as_longlong(d) ^ static_cast<long long>(0x8000000000000000ull));
}
__device__ __forceinline__ double abs_bits(double d) {   // |d| by the sign bit
  return __longlong_as_double(__double_as_longlong(d) & 0x7fffffffffffffffll);
}

// Finite test on the exponent bits (no FP64 instruction).
__device__ __forceinline__ bool finite_bits(double d) {
  return (unsigned(static_cast<unsigned long long>(__double_as_longlong(d)) >> 32) & 0x7ff00000u) != 0x7ff00000u;
}

__device__ __forceinline__ bool dge(double a, double b) { return finite_bits(a) && d2ord(a) >= d2ord(b); }

// Input element `i` as the tableau's type T.
template <typename T>
__device__ __forceinline__ T ld_as(const void *p, int64_t i, int dt);
template <>
__device__ __forceinline__ float ld_as<float>(const void *p, int64_t i, int dt) {
  return dt == LPB_DTYPE_F64 ? d2f_rn(__ldg(static_cast<const double *>(p) + i))
                             : __ldg(static_cast<const float *>(p) + i);
}
template <>
__device__ __forceinline__ double ld_as<double>(const void *p, int64_t i, int dt) {
  return ld_in(p, i, dt);
}

// Key of variable `var` at pivot `it` of LP `lp` under the random pivot rule:
// the upper 32 bits of the first SplitMix64 output (Steele, Lea and Flood,
// OOPSLA 2014) from the state seed ^ (lp << 40) ^ (it << 20) ^ var.
__device__ __forceinline__ unsigned rpc_key(unsigned long long seed, long long lp, int it, int var) {
  unsigned long long z = (seed ^ (static_cast<unsigned long long>(lp) << 40) ^
                          (static_cast<unsigned long long>(it) << 20) ^ static_cast<unsigned long long>(var)) +
                         0x9e3779b97f4a7c15ull;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return unsigned((z ^ (z >> 31)) >> 32);
}

// (value, key) order: smaller value first, then smaller key.
template <typename T>
__device__ __forceinline__ void keep_better(T &v, int &k, T ov, int ok) {
  if (ov < v || (ov == v && ok < k)) { v = ov; k = ok; }
}

template <typename T>
__device__ __forceinline__ void warp_argmin(T &v, int &k) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const T ov = __shfl_xor_sync(kFull, v, off);
    const int ok = __shfl_xor_sync(kFull, k, off);
    keep_better(v, k, ov, ok);
  }
}

// Order-preserving image of a float in the unsigned integers (negative values
// have their bits inverted, non-negative ones get the sign bit set), so that
// the warp reduction instruction can take the minimum.
__device__ __forceinline__ unsigned f2ord(float f) {
  const unsigned u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float ord2f(unsigned o) {
  return __uint_as_float((o & 0x80000000u) ? (o & 0x7fffffffu) : ~o);
}

// (value, key) arg-min of a warp with two warp-reduction instructions: the
// least value, then the least key among the lanes holding it.  Keys are >= 0.
__device__ __forceinline__ void warp_argmin_f32(float &v, int &k) {
  const unsigned o = f2ord(v);
  const unsigned mo = __reduce_min_sync(kFull, o);
  const unsigned kk = (o == mo) ? unsigned(k) : 0xffffffffu;
  k = int(__reduce_min_sync(kFull, kk));
  v = ord2f(mo);
}
template <>
__device__ __forceinline__ void warp_argmin<float>(float &v, int &k) { warp_argmin_f32(v, k); }

// Maximum of a 64-bit unsigned value over the warp (every lane takes part)
// with two warp-reduction instructions: the largest high word, then the
// largest low word among the lanes holding it.  Non-negative doubles order
// like their bit patterns, so this is also the maximum of such doubles.  A
// warp then makes one shared-memory atomic instead of one per thread (same-
// address 64-bit atomics serialise).
__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long v) {
  const unsigned hi = __reduce_max_sync(kFull, unsigned(v >> 32));
  const unsigned lo = __reduce_max_sync(kFull, unsigned(v >> 32) == hi ? unsigned(v) : 0u);
  return (static_cast<unsigned long long>(hi) << 32) | lo;
}

// Every thread of the block receives the block-wide minimum.  `bv`/`bk` hold
// one slot per warp; a call site must not reuse them before the block has
// passed another __syncthreads().
template <typename T>
__device__ __forceinline__ void block_argmin(T &v, int &k, T *bv, int *bk) {
  warp_argmin(v, k);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (lane == 0) { bv[w] = v; bk[w] = k; }
  __syncthreads();
  // Lanes past the last warp repeat slot 0, which cannot change the minimum.
  v = bv[lane < nw ? lane : 0];
  k = bk[lane < nw ? lane : 0];
  warp_argmin(v, k);
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(kFull, v, off);
  return v;
}

// Bulk prefetch of [p, p + bytes) into L2, shrunk to whole 16-byte units
// inside the range; a hint with no completion to wait for.
__device__ __forceinline__ void prefetch_l2(const void *p, size_t bytes) {
  const uintptr_t lo = (reinterpret_cast<uintptr_t>(p) + 15) & ~uintptr_t(15);
  const uintptr_t hi = (reinterpret_cast<uintptr_t>(p) + bytes) & ~uintptr_t(15);
  if (hi > lo && hi - lo < (uintptr_t(1) << 31))
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(lo), "r"(unsigned(hi - lo)) : "memory");
}

// FP64 -> FP32 round to nearest even on the integer bits, without branches.
// Magnitudes below the smallest normal float become a signed zero; magnitudes
// that round beyond the float range, infinities and NaNs set `bad`.
__device__ __forceinline__ float d2f_tile(double d, int &bad) {
  const unsigned long long u = static_cast<unsigned long long>(__double_as_longlong(d));
  const unsigned hi = unsigned(u >> 32), lo = unsigned(u);
  const unsigned ahi = hi & 0x7fffffffu;
  unsigned f = ((ahi - (896u << 20)) << 3) | (lo >> 29);
  const unsigned rem = lo & 0x1fffffffu;
  f += unsigned(rem > 0x10000000u) | (unsigned(rem == 0x10000000u) & f);
  const bool normal = ahi >= (897u << 20);
  bad |= int(ahi >= (1151u << 20)) | int(normal & (f >= 0x7f800000u));
  return __uint_as_float((hi & 0x80000000u) | (normal ? f : 0u));
}

// FP64 -> FP32 by truncation on the integer bits (relative error below 2^-23,
// the FP32 tableau's own precision; the refinement works with the exact A):
// magnitudes below the smallest normal float become a signed zero.  `amax`
// keeps the largest high word of |d| seen, so that one test afterwards
// catches values beyond the float range, infinities and NaNs.
__device__ __forceinline__ float d2f_trunc(double d, unsigned &amax) {
  const unsigned long long u = static_cast<unsigned long long>(__double_as_longlong(d));
  const unsigned hi = unsigned(u >> 32), lo = unsigned(u);
  const unsigned ahi = hi & 0x7fffffffu;
  amax = max(amax, ahi);
  const unsigned f = __funnelshift_l(lo, ahi - (896u << 20), 3);   // ((ahi - bias) << 3) | (lo >> 29)
  return __uint_as_float((hi & 0x80000000u) | (ahi >= (897u << 20) ? f : 0u));
}

// A double's high word as a float, truncated to 20 mantissa bits (relative
// error below 2^-20), in integer operations: magnitudes below the float range
// give 0, above it infinity.  Used where FP32 accuracy is ample (products with
// the small refinement corrections).
__device__ __forceinline__ float hi2f(unsigned hi) {
  const unsigned ahi = hi & 0x7fffffffu;
  const unsigned f = ahi < (897u << 20) ? 0u : (ahi >= (1151u << 20) ? 0x7f800000u : ((ahi - (896u << 20)) << 3));
  return __uint_as_float((hi & 0x80000000u) | f);
}

// Approximate reciprocal (one special-function-unit instruction, about 1 ulp).
__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// ---- bulk asynchronous copies (TMA engine) and transaction mbarriers ------
//
// A bulk copy needs 16-byte aligned source and destination and a size that is
// a multiple of 16 bytes.  Waits on an mbarrier are bounded in time, by the
// GPU's global nanosecond timer: a copy of a few hundred KB lands in
// microseconds, so kCopyWaitNs (20 ms, room for the SM being time-sliced with
// other contexts) marks a copy as failed (callers record ERR_WAIT_TIMEOUT and
// hand the work elsewhere); before the CTA leaves, it waits up to kDrainWaitNs
// (1 s) more for the copies it issued, and records ERR_COPY_IN_FLIGHT if even
// that runs out.

constexpr unsigned long long kCopyWaitNs = 20ull * 1000 * 1000;
constexpr unsigned long long kDrainWaitNs = 1000ull * 1000 * 1000;

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
// One arrival that also announces `bytes` of copies completing on the barrier.
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)),
               "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned phase) {
  unsigned ok;
  asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
               : "=r"(ok) : "r"(smem_u32(bar)), "r"(phase) : "memory");
  return ok != 0;
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Wait for `phase` of `bar` to complete; false once `ns` nanoseconds have
// passed without it.
__device__ __forceinline__ bool mbar_wait_for(uint64_t *bar, unsigned phase, unsigned long long ns) {
  const unsigned long long t0 = global_ns();
  for (;;) {
    if (mbar_try_wait(bar, phase)) return true;
    if (global_ns() - t0 > ns) return false;
  }
}
__device__ __forceinline__ void bulk_load(void *dst, const void *src, unsigned bytes, uint64_t *bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n"
               ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void bulk_store(void *dst, const void *src, unsigned bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;\n" ::"l"(dst), "r"(smem_u32(src)),
               "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;\n" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory"); }

// Append `lp` to a work list of capacity `cap`; flags an overflow instead of
// writing out of bounds.
__device__ __forceinline__ void list_push(int32_t *items, int32_t *count, int cap, int lp,
                                          uint32_t *err) {
  const int at = atomicAdd(count, 1);
  if (at < cap) items[at] = lp;
  else atomicOr(err, ERR_LIST_OVERFLOW);
}

// ---- launch parameters ----------------------------------------------------

struct TableauParams {
  BatchDev B;
  ResultDev R;
  WorkList in;                 // LPs this launch solves
  int32_t *queue;              // work counter, zeroed before the launch
  int32_t *defer_items, *defer_count;     // LPs needing more artificial columns than kcap
  int32_t *resolve_items, *resolve_count; // LPs failing FP32 verification
  int list_cap;                // capacity of the defer / resolve lists
  int32_t *bbuf;               // basis output (and warm-start input): packed like b when
  int bpacked;                 //   bpacked, else max_m entries per LP
  int warm;                    // start from the basis in bbuf (FP64 re-solve)
  void *slots;                 // per-CTA slots for the tableau rows beyond shared memory
  size_t slot_bytes;
  size_t tab_smem;             // bytes of tableau rows in shared memory (tableau kernel)
  int lim_m, lim_n;            // size bounds of this launch (register kernel: its class)
  int kcap;                    // artificial columns this launch can hold
  int mode;                    // Mode
  int max_iter;                // 0: 50 (m + n)
  double eps_p, eps_d, feas_tol;
  uint32_t *err;
  int rule;                    // lpb_pivot_rule
  unsigned long long seed;     // LPB_PIVOT_RPC seed
  long long lp_base;           // batch index of LP 0 of this launch (LPB_PIVOT_RPC keys)
  int shared;                  // every LP shares A and b (lpb_solve_shared): warm starts
};

struct BackwardParams {
  BatchDev B;
  const int32_t *status, *basis;   // forward result: basis packed like b (required)
  const double *x, *y;
  const double *g_obj, *g_x;       // upstream gradients (either may be null)
  double *g_c, *g_b, *g_A;
  void *slots;                     // per-CTA FP64 elimination slots for large systems
  size_t slot_bytes;
  int32_t *queue;
  uint32_t *err;
};

// Size classes of a mixed batch (plan.cu).  Class c < nclass - 1 takes the LPs
// with m <= max_m[c] and n <= max_n[c] not taken by an earlier class; the last
// class takes the rest.  lists holds nclass lists of `count` slots each.
constexpr int kMaxClasses = 8;
struct ClassPlanParams {
  int count, nclass;
  const int32_t *m, *n;
  int max_m[kMaxClasses], max_n[kMaxClasses];
  int32_t *hist;          // nclass * 64 cost-bucket counters (scratch)
  int32_t *lists;         // class c's LPs at lists[c * count ...], largest cost first
  int32_t *class_count;   // nclass list lengths
};

struct HyperboxParams {
  int64_t count;
  int n, dtype, shared_box;
  const void *c, *l, *u;
  void *obj, *x;
};

// Launchers (simplex_tableau.cu, hyperbox.cu).
// Shared-memory bytes of the tableau kernel's buffers (everything but rows),
// and the bytes of one tableau row, for LPs up to max_m x max_n with up to
// kcap negated rows.  A launch holds `tab_smem` bytes of rows in shared
// memory after those buffers and the rest of each tableau in a slot of
// `slot_bytes` per CTA.
size_t tableau_fixed_bytes(int elem_bytes, int max_m, int max_n, int kcap, bool refine);
size_t tableau_row_bytes(int elem_bytes, int max_n, int kcap);
cudaError_t tableau_max_ctas_per_sm(int elem_bytes, int threads, size_t smem, int *ctas);
cudaError_t launch_tableau(const TableauParams &p, bool fp64, int grid, int threads, size_t smem, cudaStream_t s);
// Register-resident FP32 kernel (simplex_reg.cu): configuration index for
// (max_m, max_n) or -1, its occupancy, and its launch.  It defers to the
// defer list every LP it does not take (Phase I, sizes, non-finite data).
size_t classify_hist_bytes(int nclass);
cudaError_t launch_classify(const ClassPlanParams &p, int sms, cudaStream_t s);
int reg_pick(int max_m, int max_n, int want_warps, bool se = false);
bool reg_has_se(int cfg);
int reg_count();
void reg_limits(int cfg, int *max_m, int *max_n, int *warps);
cudaError_t reg_occupancy(int cfg, int max_m, int max_n, int dtype, int rule, int *ctas, int *threads, size_t *smem);
cudaError_t launch_reg(const TableauParams &p, int cfg, int grid, size_t smem, cudaStream_t s);
// Several tiny LPs per warp (simplex_pack.cu): lanes per LP for LPs up to
// max_m x max_n (8 or 16; 0 when they do not fit), occupancy and launch.
int pack_lanes(int max_m, int max_n);
cudaError_t pack_occupancy(int lanes, int *ctas, int *threads);
cudaError_t launch_pack(const TableauParams &p, int lanes, int grid, cudaStream_t s);
// One warp per LP, the tableau in shared memory (simplex_warp.cu): whether LPs
// up to max_m x max_n fit (m, n <= 127), warps per CTA, shared memory and
// CTAs per SM, and the launch.
bool warp_fits(int max_m, int max_n);
cudaError_t warp_occupancy(int max_m, int max_n, int *ctas, int *threads, size_t *smem);
cudaError_t launch_warp(const TableauParams &p, int grid, int threads, size_t smem, cudaStream_t s);
size_t hyperbox_smem_bytes(int n, int elem_bytes, bool shared_box);
cudaError_t launch_hyperbox(const HyperboxParams &p, uint32_t *err, cudaStream_t s);
// Backward kernel (backward.cu).
size_t backward_smem_bytes(int max_m, int max_n);
size_t backward_slot_bytes(int max_m, int max_n);
cudaError_t backward_grid(int sms, size_t smem, int *grid);
cudaError_t launch_backward(const BackwardParams &p, int grid, size_t smem, cudaStream_t s);

// ---- a whole solve (lpb_api.cu) -------------------------------------------

struct DeviceInfo {
  int sms;
  size_t smem_optin, l2_bytes;
};

constexpr int kCounters = 8;   // device int32 work queues and list lengths of one solve

// Workspace bytes of a solve (`basis_given`: the caller passes a basis array).
lpb_err solve_workspace_bytes(const DeviceInfo &d, const lpb_batch *b, const lpb_options *o,
                              bool basis_given, size_t *bytes);
// Zero `ctr` (kCounters device ints) and launch every pass of a solve on `s`,
// with scratch from `ws`.  prof_ev (3 pairs) / prof_ran (3 flags) may be null.
// lp_base: batch index of the batch's LP 0 (a chunk of a larger batch), which
// the random pivot rule's keys use.  y_off (device, nullable): where y and the
// basis of LP k go in the result (default: b_off[k]).  shared: every LP reads
// the same A and b, so the register kernel may start an LP from the basis of
// the one it solved before.
lpb_err run_solve(const DeviceInfo &d, int32_t *ctr, uint32_t *err, const lpb_batch *b,
                  const lpb_options *o, const lpb_result *r, void *ws, size_t ws_bytes, cudaStream_t s,
                  cudaEvent_t *prof_ev, bool *prof_ran, int *kernels = nullptr, long long lp_base = 0,
                  const int64_t *y_off = nullptr, int shared = 0);

}  // namespace lpb
