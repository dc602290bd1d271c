// simplex_reg.cu -- register-resident FP32 tableau for LPs whose slack basis is
// feasible (all b_i >= 0), with the FP64 refinement and verification fused in.
//
// Section 3.1 Steps 1-3 on one LP per CTA of W warps (Section 4.1: a block of
// threads per LP; W = 1 gives one warp per tiny LP).  Type-1 LPs of the
// paper's sizes take only ~13 pivots at m = n = 100, so a solve is dominated
// by moving the LP on chip and by the latency of each pivot, not by the
// rank-1 arithmetic.  Design:
//
//   * The LP's input A, b and c (FP64 or FP32, as given) arrive in shared
//     memory by bulk copies on one transaction barrier (or by asynchronous
//     copies when not 16-byte aligned) and A stays there for the whole solve;
//     the FP64 refinement reads it back from there.  The next LP is claimed
//     in stages while this one is solved, and its copies are issued as soon
//     as this LP's certificate has read A, b and c for the last time.
//   * The compact FP32 tableau lives in registers: lane l of every warp owns
//     rows l, l+32, ..., l+32(R-1); warp w owns columns w, w+W, ..., w+W(C-1).
//     The objective row sits at the fixed row 32R-1 (lane 31, register row
//     R-1) and the right-hand side at the fixed column WC-1 (warp W-1, register
//     column C-1); rows and columns between the LP's edge and those slots are
//     zero and stay zero under pivoting, so they need no masks.
//   * Step 1: each warp judges its own columns (lane c takes column w + W c)
//     by the largest-coefficient, random or steepest-edge rule.
//   * Step 2: each warp runs the min-ratio test on its own candidate column
//     (its lanes hold the rows: a warp reduction), and after the one block
//     barrier of the pivot every warp takes the best of the W candidates.
//   * Step 3: each warp takes the pivot row from its owner lane by shuffles
//     and the pivot column from the winning warp's shared-memory slot; the
//     update is R x C FMAs per lane.
//   * Arg-min reductions use the warp reduction instruction on an
//     order-preserving integer image of the float (value first, then key).
//
// FP64 input is rounded to FP32 in integer arithmetic (d2f_tile, d2f_trunc):
// the FP64 unit of this GPU, which also converts double to float, is a small
// fraction of the FP32 rate.
//
// After an FP32 optimum the basis inverse is in the registers (the columns of
// the non-basic slacks).  Iterative refinement with FP64 residuals gives x_B
// and y; an FP64 KKT certificate (x >= 0, A x <= b, y >= 0, A^T y >= c,
// c^T x = b^T y) decides between writing the result and, after up to two more
// refinement rounds, queueing the LP for the FP64 re-solve.  LPs with some
// b_i < 0 (Phase I), or larger than the template, or with non-finite data go
// to the shared-memory kernel.
#include <type_traits>

#include "lpb_internal.cuh"

namespace lpb {
namespace {

template <int K>
using ic = std::integral_constant<int, K>;

// Calls f(ic<k>) for a block-uniform k in [LO, HI) by binary search (a few
// uniform branches instead of a select over every register).
template <int LO, int HI, typename F>
__device__ __forceinline__ void dispatch(int k, F &&f) {
  if constexpr (HI - LO == 1) {
    f(ic<LO>{});
  } else {
    constexpr int MID = (LO + HI) / 2;
    if (k < MID) dispatch<LO, MID>(k, f);
    else dispatch<MID, HI>(k, f);
  }
}

// Asynchronous global -> shared copies (cp.async); cp_async_wait_all waits
// for every copy this thread issued.
__device__ __forceinline__ void cp_async8(void *dst, const void *src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(static_cast<unsigned>(__cvta_generic_to_shared(dst))),
               "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async4(void *dst, const void *src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(static_cast<unsigned>(__cvta_generic_to_shared(dst))),
               "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

constexpr int kBad = 1 << 30;   // a key larger than any real key
// Shared-constraint batches: consecutive objectives claimed at a time, and
// warm starts between two cold builds of the tableau (FP32 round-off grows
// with the pivots a tableau has been through).
constexpr int kShareChunk = 16;
constexpr int kWarmMax = 32;

// Prefetch A, b and c of an LP into L2 when it fits the launch.
__device__ __forceinline__ void prefetch_lp(const TableauParams &P, int m, int n, long long aoff, long long boff,
                                            long long coff) {
  if (m < 1 || n < 1 || m > P.lim_m || n > P.lim_n || m > P.B.max_m || n > P.B.max_n) return;
  const size_t es = P.B.dtype == LPB_DTYPE_F64 ? 8 : 4;
  prefetch_l2(static_cast<const unsigned char *>(P.B.A) + size_t(aoff) * es, size_t(m) * size_t(n) * es);
  prefetch_l2(static_cast<const unsigned char *>(P.B.b) + size_t(boff) * es, size_t(m) * es);
  prefetch_l2(static_cast<const unsigned char *>(P.B.c) + size_t(coff) * es, size_t(n) * es);
}

// Step 1-2 result of one warp for one pivot: its best entering column and
// that column's min-ratio row.
struct WarpChoice {
  float v;       // reduced cost (0 under Bland's rule), +inf if none
  int key;       // (entering variable << kIdxBits) | column, kBad if none
  float theta;   // min ratio
  int lkey;      // (leaving variable << kIdxBits) | row, kBad if unbounded
};

// Element i of an input vector staged in shared memory with its input dtype.
__device__ __forceinline__ double vin(const double *v, int i, int dt) {
  return dt == LPB_DTYPE_F64 ? v[i] : double(reinterpret_cast<const float *>(v)[i]);
}

// A claimed work item and its LP's sizes and offsets, as the claimer thread
// gathers them by asynchronous copies while the LP before it is solved.
struct RegDesc {
  long long aoff, boff, coff;
  int item, lp, m, n;
};

template <int R, int C, int W>
struct RegShared {
  static constexpr int ROWS = 32 * R, COLS = W * C;
  float colbuf[2][W][ROWS];                  // each warp's candidate column, by pivot parity
  WarpChoice choice[2][W];                   // by pivot parity
  alignas(16) double bin[ROWS];              // the LP's b and c as given (FP64 or FP32)
  alignas(16) double cin[COLS];
  float rhs[ROWS];
  int basic[ROWS];
  int nonb[COLS];
  alignas(16) float objv[W][(C + 3) & ~3];   // objective row, per warp
  RegDesc desc[2];                           // this LP's and the next one's, by LP parity
  int cstage;                                // how far the next LP's descriptor has come
  int pre;                                   // the next LP's A, b and c are already requested
  int nsb, nns;
  int warm_ok;                               // shared constraints: start from the previous basis
  unsigned long long wbmax[W], wcmax[W];     // |b|max and |c|max bits, per warp
  uint64_t abar;                             // completion of the bulk copies of A
  double xb[ROWS], rr[ROWS], yv[ROWS], sax[ROWS], dj[COLS];
  float part[W][ROWS];
  float rhof[ROWS], rrf[ROWS], dxf[ROWS], dyf[ROWS];
  int posx[COLS];
  int sb[ROWS], jb[ROWS], sp[ROWS];
  int ns[COLS], kr[COLS];
  double red[2][W];
  double tpd[2];                             // the certificate's primal and dual tolerances
};

template <int R, int C, int W>
__host__ __device__ constexpr size_t reg_fixed_bytes() { return (sizeof(RegShared<R, C, W>) + 15) & ~size_t(15); }

// Row stride (in elements) of the resident copy of A.  Rows start on 16-byte
// boundaries (bulk copies), and the stride in 16-byte units is odd, so the
// lanes of a warp reading one column touch as few banks twice as that allows.
__host__ __device__ inline int a_stride(int max_n, int es) {
  const int per = 16 / es;                                // elements per 16 bytes
  int s = (max_n + per - 1) / per;
  if ((s & 1) == 0) ++s;
  return s * per;
}

// Smallest power of two >= k (1 <= k <= 32).
__host__ __device__ constexpr int pow2_at_least(int k) { return k <= 1 ? 1 : 2 * pow2_at_least((k + 1) / 2); }

// Sums v[c] over the 32 lanes of a warp for every c < P (P a power of two):
// log2(P) halving exchanges, in which each lane keeps half of its columns and
// adds the partner's copy of them, then plain butterflies.  On return lane l
// holds the total of column l / (32 / P): P - 1 + log2(32 / P) shuffles in
// place of 5 P.
template <int P>
__device__ __forceinline__ float reduce_scatter(float (&v)[P], int lane) {
#pragma unroll
  for (int h = P / 2, off = 16; h >= 1; h /= 2, off /= 2) {
    const bool upper = (lane & off) != 0;
#pragma unroll
    for (int k = 0; k < h; ++k) {
      const float send = upper ? v[k] : v[k + h];
      const float keep = upper ? v[k + h] : v[k];
      v[k] = keep + __shfl_xor_sync(kFull, send, off);
    }
  }
  float s = v[0];
#pragma unroll
  for (int off = 16 / P; off >= 1; off /= 2) s += __shfl_xor_sync(kFull, s, off);
  return s;
}

// Input element i of a staged vector rounded to FP32 without branches (see
// d2f_tile); non-finite or out-of-range values set `bad`.
__device__ __forceinline__ float vin_tile(const double *v, int i, int dt, int &bad) {
  if (dt == LPB_DTYPE_F64) return d2f_tile(v[i], bad);
  const float f = reinterpret_cast<const float *>(v)[i];
  bad |= !isfinite(f);
  return f;
}

template <typename T>
__device__ __forceinline__ double a_at(const unsigned char *sa, int dt, int idx) {
  return dt == LPB_DTYPE_F64 ? reinterpret_cast<const double *>(sa)[idx]
                             : double(reinterpret_cast<const float *>(sa)[idx]);
}

// Minimum resident CTAs per SM: more for the small tableaux, fewer for the
// 4-warp CTAs with 128 rows, whose tableau alone takes C * 4 registers.
template <int R, int C, int W>
constexpr int reg_min_blocks() {
  return W == 1 ? 16 : R * C <= 8 ? (W <= 4 ? 4 : 3) : (R == 4 && W <= 4) ? 2 : (W <= 4 ? 3 : 2);
}

// Steepest-edge weight gamma_c = 1 + sum_i t_ic^2 of this warp's column
// wid + W lane, for lanes c < C, over the constraint rows (every row but the
// objective row, lane 31's row R-1; padding rows are zero).  Columns go four
// at a time through a reduce-scatter, so few registers are live.
template <int R, int C>
__device__ __forceinline__ float se_gamma(const float (&T)[R][C], int lane) {
  const float keep_last = lane == 31 ? 0.f : 1.f;
  float g = 0.f;
#pragma unroll
  for (int c0 = 0; c0 < C; c0 += 4) {
    float v[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      float s = 0.f;
      if (c0 + k < C) {
#pragma unroll
        for (int r = 0; r < R - 1; ++r) s = fmaf(T[r][c0 + k], T[r][c0 + k], s);
        const float t = T[R - 1][c0 + k] * keep_last;
        s = fmaf(t, t, s);
      }
      v[k] = s;
    }
    const float tot = reduce_scatter<4>(v, lane);            // lane l: column c0 + l / 8
    const float mine = __shfl_sync(kFull, tot, ((lane - c0) & 3) * 8);
    if (lane >= c0 && lane < c0 + 4) g = mine;
  }
  return 1.f + g;
}

// SE: steepest-edge pricing in Step 1 (a separate instantiation, so that the
// other rules' kernels carry none of its registers or instructions).
template <int R, int C, int W, bool SE>
__global__ void __launch_bounds__(W * 32, reg_min_blocks<R, C, W>()) reg_kernel(TableauParams P) {
  using SH = RegShared<R, C, W>;
  constexpr int ROWS = SH::ROWS, COLS = SH::COLS;
  constexpr int NT = W * 32;
  extern __shared__ __align__(16) unsigned char reg_smem[];
  SH &sh = *reinterpret_cast<SH *>(reg_smem);
  unsigned char *sA = reg_smem + reg_fixed_bytes<R, C, W>();   // resident input A
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const float eps_p = float(P.eps_p), eps_d = float(P.eps_d);
  const int dt = P.B.dtype;
  const int es = dt == LPB_DTYPE_F64 ? 8 : 4;
  const int sld_pad = a_stride(P.lim_n, es);
  const int nitems = P.in.count ? min(*P.in.count, P.list_cap) : P.B.count;
  float T[R][C];

  if (tid == 0) {
    mbar_init(&sh.abar, 1);
    fence_mbar_init();
    sh.pre = 0;
  }
  unsigned aphase = 0;        // parity of the next completion of sh.abar
  // Lane 0 of the last warp claims work items one LP ahead.  Each global round
  // trip of the claim waits a phase of the current LP before it is used: the
  // queue atomic when an LP starts; the item's LP index (stage 1) after the
  // tableau is built; its sizes and offsets (stage 2) after the pivots; an L2
  // prefetch of its data (stage 3) during the refinement.  Stages 1 and 2 copy
  // into the descriptor slot of the next LP asynchronously; an LP that ends
  // early has its remaining stages done when the next one starts.
  const int claimer = NT - 32;
  // A shared-constraint batch (one A and b, many objectives) is claimed in
  // chunks of consecutive objectives, so that a CTA starts each objective from
  // the optimal basis of the one before (the tableau stays in registers).
  auto claim = [&](int cur) -> int {
    if (P.shared) {
      if (cur >= 0 && (cur + 1) % kShareChunk != 0 && cur + 1 < nitems) return cur + 1;
      return atomicAdd(P.queue, 1) * kShareChunk;
    }
    return atomicAdd(P.queue, 1);
  };
  // Sizes this launch's template and limits hold (else the LP is deferred).
  auto fits_lp = [&](int m, int n) {
    return m >= 1 && n >= 1 && m <= ROWS - 1 && n <= COLS - 1 && m <= P.B.max_m && n <= P.B.max_n &&
           m <= P.lim_m && n <= P.lim_n;
  };
  int next = 0;
  int slot = 0;                 // descriptor slot of the current LP (same in every thread)
  auto stage1 = [&]() {         // claimer: item and LP index of the claimed item
    RegDesc &d = sh.desc[slot ^ 1];
    d.item = next;
    if (next < nitems) {
      if (P.in.items) cp_async4(&d.lp, P.in.items + next);
      else d.lp = next;
    }
    sh.cstage = 1;
  };
  auto stage2 = [&]() {         // claimer: sizes and offsets
    cp_async_wait_all();
    RegDesc &d = sh.desc[slot ^ 1];
    if (d.item < nitems) {
      const int l = d.lp;
      cp_async4(&d.m, P.B.m + l);
      cp_async4(&d.n, P.B.n + l);
      cp_async8(&d.aoff, P.B.a_off + l);
      cp_async8(&d.boff, P.B.b_off + l);
      cp_async8(&d.coff, P.B.c_off + l);
    }
    sh.cstage = 2;
  };
  auto stage3 = [&]() {         // claimer: L2 prefetch of the next LP's data
    cp_async_wait_all();
    const RegDesc &d = sh.desc[slot ^ 1];
    if (d.item < nitems && !P.shared) prefetch_lp(P, d.m, d.n, d.aoff, d.boff, d.coff);
    sh.cstage = 3;
  };
  if (tid == claimer) {
    next = claim(-1);
    slot = 1;                   // the first LP's descriptor goes to slot 0
    stage1();
    stage2();
    cp_async_wait_all();
    slot = 0;
  }
  slot = 0;
  // The basis of the last tableau: every lane keeps, for its rows lane + 32 r,
  // the basic variable and the right-hand side (the same FP32 values warp W-1
  // holds in its last column); lane c < C keeps the variable of the warp's
  // column wid + W c.  valid_tab: the registers hold a basis tableau of this
  // batch's A and b; warm_run: objectives solved since the last cold start.
  int bvar[R];
  float rhsr[R];
  int nvar = kBad >> kIdxBits;
  int valid_tab = 0, warm_run = 0;
  int sld_res = sld_pad;                       // row stride of the resident A
  for (int first = 1;; first = 0) {
    if (tid == claimer && !first) {   // stages the last LP did not reach; its slot becomes current
      const int st = sh.cstage;
      if (st < 1) stage1();
      if (st < 2) stage2();
      if (st < 3) stage3();
      cp_async_wait_all();
    }
    if (!first) slot ^= 1;
    if (tid == 0) sh.warm_ok = P.shared && valid_tab && warm_run < kWarmMax;
    __syncthreads();
    const RegDesc &D = sh.desc[slot];
    const int item = D.item;
    if (item >= nitems) break;
    const bool pre = sh.pre != 0;          // reset by thread 0 after the next barrier
    const bool warm = sh.warm_ok != 0;     // keep the basis; load and price only the new objective
    warm_run = warm ? warm_run + 1 : 0;
    valid_tab = 0;
    const int lp = D.lp;
    const int m = D.m, n = D.n;
    const int64_t aoff = D.aoff, boff = D.boff, coff = D.coff;
    // ---- admission: sizes that fit the template, b >= 0, finite b and c ----
    const bool fits = fits_lp(m, n);
    const unsigned char *Ag = static_cast<const unsigned char *>(P.B.A) + aoff * es;
    // A is contiguous in global memory: when its start and size are whole
    // 16-byte units it comes in one bulk copy and keeps its row length in
    // shared memory (one copy instruction instead of one per row, at the price
    // of more bank conflicts in the column reads); else rows whose start and
    // length are whole 16-byte units go by one bulk copy each into rows of a
    // padded stride, and the rest by 4- or 8-byte asynchronous copies.
    const bool dense = fits && !warm && ((reinterpret_cast<uintptr_t>(Ag) | uintptr_t(m) * uintptr_t(n) * es) & 15) == 0;
    const bool bulk = fits && !warm && !dense && ((reinterpret_cast<uintptr_t>(Ag) | uintptr_t(n) * es) & 15) == 0;
    if (!warm) sld_res = dense ? n : sld_pad;   // a warm start reuses the resident A in its layout
    const int sld = sld_res;
    // b and c go by bulk copy on the same barrier as A when their starts and
    // lengths are whole 16-byte units, so that one wait covers all three.
    const unsigned char *bgp = static_cast<const unsigned char *>(P.B.b) + boff * es;
    const unsigned char *cgp = static_cast<const unsigned char *>(P.B.c) + coff * es;
    const bool bulk_bc = fits && !warm && ((reinterpret_cast<uintptr_t>(bgp) | reinterpret_cast<uintptr_t>(cgp) |
                                            uintptr_t(m) * es | uintptr_t(n) * es) & 15) == 0;
    const bool bulk_c = fits && warm && ((reinterpret_cast<uintptr_t>(cgp) | uintptr_t(n) * es) & 15) == 0;
    if (fits && !pre) {
      if (!bulk_bc && !bulk_c) {      // b (not on a warm start, it is resident) and c by small copies
        if (dt == LPB_DTYPE_F64) {
          const double *bg = reinterpret_cast<const double *>(bgp), *cg = reinterpret_cast<const double *>(cgp);
          for (int i = tid; i < (warm ? 0 : m); i += NT) cp_async8(sh.bin + i, bg + i);
          for (int j = tid; j < n; j += NT) cp_async8(sh.cin + j, cg + j);
        } else {
          const float *bg = reinterpret_cast<const float *>(bgp), *cg = reinterpret_cast<const float *>(cgp);
          for (int i = tid; i < (warm ? 0 : m); i += NT) cp_async4(reinterpret_cast<float *>(sh.bin) + i, bg + i);
          for (int j = tid; j < n; j += NT) cp_async4(reinterpret_cast<float *>(sh.cin) + j, cg + j);
        }
      }
      if (dense || bulk || bulk_bc || bulk_c) {
        if (wid == 0) {
          if (lane == 0) {
            mbar_expect_tx(&sh.abar, (dense || bulk ? unsigned(m) * unsigned(n) * unsigned(es) : 0u) +
                                         (bulk_bc ? unsigned(m + n) * unsigned(es) : 0u) +
                                         (bulk_c ? unsigned(n) * unsigned(es) : 0u));
            if (bulk_bc) {
              bulk_load(sh.bin, bgp, unsigned(m) * es, &sh.abar);
              bulk_load(sh.cin, cgp, unsigned(n) * es, &sh.abar);
            }
            if (bulk_c) bulk_load(sh.cin, cgp, unsigned(n) * es, &sh.abar);
            if (dense) bulk_load(sA, Ag, unsigned(m) * unsigned(n) * es, &sh.abar);
          }
          __syncwarp();
          if (bulk)
            for (int i = lane; i < m; i += 32)
              bulk_load(sA + size_t(i) * sld * es, Ag + size_t(i) * n * es, unsigned(n) * es, &sh.abar);
        }
      }
      if (!bulk && !dense && !warm) {
        if (dt == LPB_DTYPE_F64) {
          const double *A = reinterpret_cast<const double *>(Ag);
          double *sa = reinterpret_cast<double *>(sA);
          for (int i = wid; i < m; i += W)
            for (int j = lane; j < n; j += 32) cp_async8(sa + i * sld + j, A + int64_t(i) * n + j);
        } else {
          const float *A = reinterpret_cast<const float *>(Ag);
          float *sa = reinterpret_cast<float *>(sA);
          for (int i = wid; i < m; i += W)
            for (int j = lane; j < n; j += 32) cp_async4(sa + i * sld + j, A + int64_t(i) * n + j);
        }
      }
    }
    if (tid == claimer) {
      next = claim(item);
      sh.cstage = 0;
    }
    int neg = 0;
    cp_async_wait_all();
    int timed_out = 0;
    if (dense || bulk || bulk_bc || bulk_c) {
      timed_out = !mbar_wait_for(&sh.abar, aphase, kCopyWaitNs);
      aphase ^= 1u;
    }
    const int any_timeout = __syncthreads_or(timed_out);
    if (tid == 0) sh.pre = 0;
    if (any_timeout) {
      // The copy engine did not deliver the data in time: hand this LP and the one
      // claimed after it to the generic kernel, wait up to kDrainWaitNs more for
      // the copies to land, and stop this CTA.  Only if that wait runs out too
      // does the CTA leave with copies into its shared memory outstanding; it
      // then records ERR_COPY_IN_FLIGHT, which voids the launch's results.
      if (tid == 0) {
        atomicOr(P.err, ERR_WAIT_TIMEOUT);
        P.R.status[lp] = STATUS_PENDING;
        list_push(P.defer_items, P.defer_count, P.list_cap, lp, P.err);
        if (!mbar_wait_for(&sh.abar, aphase ^ 1u, kDrainWaitNs)) atomicOr(P.err, ERR_COPY_IN_FLIGHT);
      }
      if (tid == claimer && next < nitems) {
        const int lp2 = P.in.items ? P.in.items[next] : next;
        P.R.status[lp2] = STATUS_PENDING;
        list_push(P.defer_items, P.defer_count, P.list_cap, lp2, P.err);
      }
      __syncthreads();
      break;
    }
    if (fits) {
      // On the bits of the doubles (integer operations; FP64 ones have long
      // latency here): |v| orders like its bit pattern.  b_i < 0 or NaN and
      // non-finite c_j send the LP elsewhere.
      constexpr unsigned long long kMag = 0x7fffffffffffffffull, kInf = 0x7ff0000000000000ull;
      unsigned long long bm = 0ull, cm = 0ull;
      for (int i = tid; i < (warm ? 0 : m); i += NT) {
        const unsigned long long u = static_cast<unsigned long long>(__double_as_longlong(vin(sh.bin, i, dt)));
        const unsigned long long a = u & kMag;
        neg |= int((u >> 63) != 0ull && a != 0ull) | int(a > kInf);
        bm = a > bm ? a : bm;
      }
      for (int j = tid; j < n; j += NT) {
        const unsigned long long a =
            static_cast<unsigned long long>(__double_as_longlong(vin(sh.cin, j, dt))) & kMag;
        neg |= int(a >= kInf);
        cm = a > cm ? a : cm;
      }
      bm = warp_max_u64(bm <= kInf ? bm : 0ull);      // NaN magnitudes take no part
      cm = warp_max_u64(cm < kInf ? cm : 0ull);
      if (lane == 0) {                               // a warm start keeps b and its |b|max
        if (!warm) sh.wbmax[wid] = bm;
        sh.wcmax[wid] = cm;
      }
    }
    // ---- the tableau: A rounded to FP32, b in column COLS-1, -c in row ROWS-1 ----
    // (built before the block learns the checks above: one vote covers both,
    // and an LP with some b_i < 0 or non-finite data is simply not used)
    int bad = neg;
    if (fits && !warm) {
    if (dt == LPB_DTYPE_F64) {
      const double *sa = reinterpret_cast<const double *>(sA);
      unsigned amax = 0u;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int i = lane + 32 * r;
#pragma unroll
        for (int c = 0; c < C; ++c) {
          const int j = wid + W * c;
          T[r][c] = (i < m && j < n) ? d2f_trunc(sa[i * sld + j], amax) : 0.f;
        }
      }
      bad |= int(amax >= (1151u << 20));     // |a| >= 2^128, Inf or NaN
    } else {
      const float *sa = reinterpret_cast<const float *>(sA);
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int i = lane + 32 * r;
#pragma unroll
        for (int c = 0; c < C; ++c) {
          const int j = wid + W * c;
          const float v = (i < m && j < n) ? sa[i * sld + j] : 0.f;
          bad |= !isfinite(v);
          T[r][c] = v;
        }
      }
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int i = lane + 32 * r;
      rhsr[r] = i < m ? vin_tile(sh.bin, i, dt, bad) : 0.f;
      bvar[r] = i < m ? n + i : kBad >> kIdxBits;
    }
    nvar = (wid + W * lane < n && lane < C) ? wid + W * lane : kBad >> kIdxBits;
    if (wid == W - 1) {
#pragma unroll
      for (int r = 0; r < R; ++r) T[r][C - 1] = rhsr[r];
    }
    if (lane == 31) {
#pragma unroll
      for (int c = 0; c < C; ++c) {
        const int j = wid + W * c;
        if (j < n) T[R - 1][c] = -vin_tile(sh.cin, j, dt, bad);
      }
    }
    } else if (fits) {
      // Warm start: the basis of the previous objective.  Its objective row for
      // this c is r_j = sum_i c_B(i) t_ij - c_j on the non-basic columns and
      // z = sum_i c_B(i) rhs_i on the right-hand side (c of slacks is 0).
      constexpr int CP = pow2_at_least(C);
      float cb[R];
#pragma unroll
      for (int r = 0; r < R; ++r) cb[r] = bvar[r] < n ? vin_tile(sh.cin, bvar[r], dt, bad) : 0.f;
      float col[CP];
#pragma unroll
      for (int c = 0; c < CP; ++c) {
        float acc = 0.f;
        if (c < C) {
#pragma unroll
          for (int r = 0; r < R; ++r) acc = fmaf(cb[r], T[r][c], acc);
        }
        col[c] = acc;
      }
      const float tot = reduce_scatter<CP>(col, lane);   // lane l: column l / (32 / CP)
      float *objw = sh.objv[wid];
      if (lane % (32 / CP) == 0 && lane / (32 / CP) < C) objw[lane / (32 / CP)] = tot;
      __syncwarp();
      if (lane < C) {
        const bool rhs_col = wid == W - 1 && lane == C - 1;
        const float cj = !rhs_col && nvar < n ? vin_tile(sh.cin, nvar, dt, bad) : 0.f;
        objw[lane] -= cj;
      }
      __syncwarp();
      if (lane == 31) {
#pragma unroll
        for (int c = 0; c < C; ++c) T[R - 1][c] = objw[c];
      }
      __syncwarp();
    }
    bad = __syncthreads_or(bad);
    if (!fits || bad) {      // the shared-memory kernel handles it (Phase I, sizes, bad data)
      if (tid == 0) {
        P.R.status[lp] = STATUS_PENDING;
        list_push(P.defer_items, P.defer_count, P.list_cap, lp, P.err);
      }
      __syncthreads();
      continue;
    }

    valid_tab = 1;

    if (tid == claimer) stage1();
    // ---- Steps 1-3, one block barrier per pivot ----
    // Each warp takes its own best entering column (Step 1 over its columns)
    // and runs the min-ratio test on it (Step 2); after the barrier every warp
    // picks the best of the W choices, and the pivot column comes from the
    // winning warp's slot.  Slots are double-buffered by pivot parity: a warp
    // can be at most one barrier ahead of the others.
    const int max_iter = P.max_iter > 0 ? P.max_iter : 50 * (m + n);
    int iters = 0, status = LPB_OPTIMAL, degenerate_run = 0;
    bool bland = false;
    float *objw = sh.objv[wid];
    for (int par = 0;; par ^= 1) {
      // Step 1 in this warp: lane 31 publishes the objective row with 16-byte
      // stores; lane c judges column wid + W c.
      if (lane == 31) {
#pragma unroll
        for (int c = 0; c < C; c += 4) {
          float4 q;
          q.x = T[R - 1][c];
          q.y = c + 1 < C ? T[R - 1][c + 1] : 0.f;
          q.z = c + 2 < C ? T[R - 1][c + 2] : 0.f;
          q.w = c + 3 < C ? T[R - 1][c + 3] : 0.f;
          *reinterpret_cast<float4 *>(objw + c) = q;
        }
      }
      __syncwarp();
      // No candidate: the largest value of the order-preserving image, above
      // every random-rule key (whose bit patterns may exceed that of +inf).
      float cv = __int_as_float(0x7fffffff);
      int ck = kBad;
      float gam = 1.f;
      if constexpr (SE) {
        if (!bland) gam = se_gamma<R, C>(T, lane);
      }
      {
        const int j = wid + W * lane;
        if (lane < C && j < COLS - 1) {                // the last column is the right-hand side
          const float rj = objw[lane];
          if (rj < -eps_d) {
            // The random rule ranks by the upper 31 bits of the variable's key,
            // stored as the bits of a non-negative float: the arg-min compares
            // the order-preserving integer image, never the float value.
            if constexpr (SE) cv = bland ? 0.f : -__fdiv_rn(rj * rj, gam);     // the largest r_j^2 / gamma_j
            else cv = bland ? 0.f : P.rule == LPB_PIVOT_RPC ? __uint_as_float(rpc_key(P.seed, P.lp_base + lp, iters, nvar) >> 1) : rj;
            ck = (nvar << kIdxBits) | j;
          }
        }
      }
      warp_argmin_f32(cv, ck);
      // Step 2 on this warp's candidate.
      float tv = __int_as_float(0x7f800000);
      int tk = kBad;
      if (ck != kBad) {
        const int ce = (ck & kIdxMask) / W;
        float col[R];
        dispatch<0, C>(ce, [&](auto K) {
#pragma unroll
          for (int r = 0; r < R; ++r) col[r] = T[r][K.value];
        });
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const int i = lane + 32 * r;
          if (col[r] > eps_p) keep_better(tv, tk, rhsr[r] * rcp_approx(col[r]), (bvar[r] << kIdxBits) | i);
        }
        warp_argmin_f32(tv, tk);
#pragma unroll
        for (int r = 0; r < R; ++r) sh.colbuf[par][wid][lane + 32 * r] = col[r];
      }
      if (lane == 0) sh.choice[par][wid] = WarpChoice{cv, ck, tv, tk};
      __syncthreads();
      // The pivot: the best (value, key) over the warps' choices.
      float ev = __int_as_float(0x7fffffff);
      int ek = kBad;
      if (lane < W) {
        ev = sh.choice[par][lane].v;
        ek = sh.choice[par][lane].key;
      }
      warp_argmin_f32(ev, ek);
      if (ek == kBad) { status = LPB_OPTIMAL; break; }
      const int e = ek & kIdxMask;
      const int we = e % W, ce = e / W;
      const WarpChoice &wc = sh.choice[par][we];
      const int lk = wc.lkey;
      const float theta = wc.theta;
      if (lk == kBad) { status = LPB_UNBOUNDED; break; }
      if (iters >= max_iter) { status = LPB_ITER_LIMIT; break; }
      const int l = lk & kIdxMask, leave_var = lk >> kIdxBits;
      const int lr = l >> 5, ll = l & 31;
      const float *pcol = sh.colbuf[par][we];
      const float rp = __frcp_rn(pcol[l]);
      float cf[R];           // pivot column; 0 on the pivot row, which is only scaled
      float gf[R];           // pivot column / p
#pragma unroll
      for (int r = 0; r < R; ++r) {
        cf[r] = (lane + 32 * r == l) ? 0.f : pcol[lane + 32 * r];
        gf[r] = cf[r] * rp;
      }
      // Step 3: every lane takes the pivot row from lane ll by shuffles:
      // T -= (pivot column / p) (x) (pivot row); the owner lane scales its
      // row by 1/p.
      dispatch<0, R>(lr, [&](auto LR) {
#pragma unroll
        for (int c = 0; c < C; ++c) {
          const float pr = __shfl_sync(kFull, T[LR.value][c], ll);
#pragma unroll
          for (int r = 0; r < R; ++r) T[r][c] = fmaf(-gf[r], pr, T[r][c]);
        }
        const float prh = __shfl_sync(kFull, rhsr[LR.value], ll);
#pragma unroll
        for (int r = 0; r < R; ++r) rhsr[r] = fmaf(-gf[r], prh, rhsr[r]);
        if (lane == ll) {
#pragma unroll
          for (int c = 0; c < C; ++c) T[LR.value][c] *= rp;
          rhsr[LR.value] *= rp;
          bvar[LR.value] = ek >> kIdxBits;
        }
      });
      if (wid == we) {        // new column e: -t_ie / p, and 1/p at the pivot
        dispatch<0, C>(ce, [&](auto K) {
#pragma unroll
          for (int r = 0; r < R; ++r) T[r][K.value] = (lane + 32 * r == l) ? rp : -cf[r] * rp;
        });
        if (lane == ce) nvar = leave_var;
      }
      ++iters;
      if (theta <= eps_p) {
        if (++degenerate_run >= m + n) bland = true;
      } else {
        degenerate_run = 0;
        bland = false;
      }
    }
    valid_tab = status == LPB_OPTIMAL || status == LPB_UNBOUNDED;   // a basis tableau to start from
    // The final basis and right-hand side back to shared memory (every warp
    // holds the same copy of the rows; warp 0 writes them).
    if (wid == 0) {
#pragma unroll
      for (int r = 0; r < R; ++r) {
        sh.basic[lane + 32 * r] = bvar[r];
        sh.rhs[lane + 32 * r] = rhsr[r];
      }
    }
    if (lane < C) sh.nonb[wid + W * lane] = nvar;
    if (tid == claimer) stage2();
    __syncthreads();

    const int64_t yoff = P.R.y_off ? P.R.y_off[lp] : boff;    // outputs packed like b, or at y_off
    int32_t *bp = P.bbuf ? P.bbuf + (P.bpacked ? yoff : int64_t(lp) * P.B.max_m) : nullptr;
    if (status != LPB_OPTIMAL || P.mode != MODE_FP32_REFINE) {
      if (status == LPB_OPTIMAL) {   // plain FP32: results straight from the tableau
        for (int j = tid; j < n; j += NT) P.R.x[coff + j] = 0.0;
        if (P.R.y) for (int i = tid; i < m; i += NT) P.R.y[yoff + i] = 0.0;
        __syncthreads();
        for (int i = tid; i < m; i += NT)
          if (sh.basic[i] < n) P.R.x[coff + sh.basic[i]] = double(sh.rhs[i]);
        if (lane == 31 && P.R.y) {
#pragma unroll
          for (int c = 0; c < C; ++c) {
            if (wid == W - 1 && c == C - 1) continue;    // the right-hand side
            const int v = sh.nonb[wid + W * c];
            if (v >= n && v < n + m) P.R.y[yoff + (v - n)] = double(T[R - 1][c]);
          }
        }
        if (wid == W - 1 && lane == 31) {
          P.R.status[lp] = LPB_OPTIMAL;
          P.R.obj[lp] = double(T[R - 1][C - 1]);
          if (P.R.iters) P.R.iters[lp] = iters;
        }
      } else if (P.mode == MODE_FP32_REFINE) {   // unbounded / iteration cap: confirm in FP64
        if (tid == 0) {
          P.R.status[lp] = STATUS_PENDING;
          if (P.R.iters) P.R.iters[lp] = iters;
          list_push(P.resolve_items, P.resolve_count, P.list_cap, lp, P.err);
        }
      } else {                                   // plain FP32: final as found
        for (int j = tid; j < n; j += NT) P.R.x[coff + j] = 0.0;
        if (P.R.y) for (int i = tid; i < m; i += NT) P.R.y[yoff + i] = 0.0;
        if (tid == 0) {
          P.R.status[lp] = status;
          if (P.R.iters) P.R.iters[lp] = iters;
          P.R.obj[lp] = status == LPB_UNBOUNDED ? INFINITY : NAN;
        }
      }
      if (bp) for (int i = tid; i < m; i += NT) bp[i] = sh.basic[i];
      __syncthreads();
      continue;
    }

    // ---- FP64 refinement and certificate, with A read from shared memory ----
    // Lists: the q-th basic structural sits in row sb[q] and column jb[q] of
    // A; the p-th non-basic slack sits in tableau column ns[p] and row kr[p]
    // of A.  Warp 0 builds the row lists, warp 1 the column lists (a one-warp
    // CTA builds both).
    constexpr int kColWarp = W > 1 ? 1 : 0;
    if (wid == 0) {
      int base = 0;
      for (int i0 = 0; i0 < m; i0 += 32) {
        const int i = i0 + lane;
        const int v = i < m ? sh.basic[i] : n;
        const bool pr = i < m && v < n;
        const unsigned mk = __ballot_sync(kFull, pr);
        if (pr) {
          const int q = base + __popc(mk & ((1u << lane) - 1u));
          sh.sb[q] = i;
          sh.jb[q] = v;
        }
        base += __popc(mk);
      }
      if (lane == 0) sh.nsb = base;
    }
    if (wid == kColWarp) {
      int base = 0;
      for (int j0 = 0; j0 < COLS - 1; j0 += 32) {
        const int j = j0 + lane;
        const int v = j < COLS - 1 ? sh.nonb[j] : 0;
        const bool pr = j < COLS - 1 && v >= n && v < n + m;
        const unsigned mk = __ballot_sync(kFull, pr);
        if (pr) {
          const int q = base + __popc(mk & ((1u << lane) - 1u));
          sh.ns[q] = j;
          sh.kr[q] = v - n;
        }
        base += __popc(mk);
      }
      if (lane == 0) sh.nns = base;
    }
    for (int i = tid; i < ROWS; i += NT) {
      sh.sp[i] = -1;
      sh.yv[i] = 0.0;
      sh.rhof[i] = 0.f;
      sh.dyf[i] = 0.f;
      sh.xb[i] = i < m ? double(sh.rhs[i]) : 0.0;
    }
    for (int j = tid; j < COLS; j += NT) sh.posx[j] = -1;
    if (tid == 0) {        // FP64 work is scarce here: one thread, not every warp
      unsigned long long bm = 0ull, cm = 0ull;
      for (int w = 0; w < W; ++w) {
        bm = max(bm, sh.wbmax[w]);
        cm = max(cm, sh.wcmax[w]);
      }
      sh.tpd[0] = P.feas_tol * (1.0 + __longlong_as_double(static_cast<long long>(bm)));
      sh.tpd[1] = P.feas_tol * (1.0 + __longlong_as_double(static_cast<long long>(cm)));
    }
    __syncthreads();
    const int nsb = sh.nsb, nns = sh.nns;
    for (int i = tid; i < m; i += NT) {
      const int v = sh.basic[i];
      if (v >= n) sh.sp[v - n] = i;
      else sh.posx[v] = i;
    }
    // y of the non-basic slacks from the objective row that the last pivot
    // step published (column j sits in warp j mod W, slot j / W): one warp
    // converts them, one FP64 conversion per 32 slacks.
    if (wid == W - 1)
      for (int p2 = lane; p2 < nns; p2 += 32) {
        const int j = sh.ns[p2];
        sh.yv[sh.kr[p2]] = double(sh.objv[j % W][j / W]);
      }
    __syncthreads();
    // FP64 dot products (the FP64 unit is the scarce resource here: these two
    // are the only FP64 loops, m nsb + n nns multiply-adds in all).
    //   row_dot(i):  sum_q A[i, jb[q]] x[sb[q]]       (A_B x_B, row i)
    //   col_dot(j):  sum_p A[kr[p], j] y[kr[p]]       ((A^T y)_j over the non-basic slacks)
    auto row_dot = [&](int i) {
      double s0 = 0.0;
      if (dt == LPB_DTYPE_F64) {
        const double *ar = reinterpret_cast<const double *>(sA) + i * sld;
#pragma unroll 4
        for (int q = 0; q < nsb; ++q) s0 = fma(ar[sh.jb[q]], sh.xb[sh.sb[q]], s0);
      } else {
        const float *ar = reinterpret_cast<const float *>(sA) + i * sld;
#pragma unroll 4
        for (int q = 0; q < nsb; ++q) s0 = fma(double(ar[sh.jb[q]]), sh.xb[sh.sb[q]], s0);
      }
      return s0;
    };
    auto col_dot = [&](int j) {
      double s0 = 0.0;
      if (dt == LPB_DTYPE_F64) {
        const double *ac = reinterpret_cast<const double *>(sA) + j;
#pragma unroll 4
        for (int q = 0; q < nns; ++q) s0 = fma(ac[sh.kr[q] * sld], sh.yv[sh.kr[q]], s0);
      } else {
        const float *ac = reinterpret_cast<const float *>(sA) + j;
#pragma unroll 4
        for (int q = 0; q < nns; ++q) s0 = fma(double(ac[sh.kr[q] * sld]), sh.yv[sh.kr[q]], s0);
      }
      return s0;
    };
    // FP32 products of A with small corrections, and the sum of their
    // magnitudes for the error bound: A is read as hi2f of its high word.
    auto row_delta = [&](int i, float &mag) {
      float s0 = 0.f, e0 = 0.f;
      if (dt == LPB_DTYPE_F64) {
        const unsigned *ar = reinterpret_cast<const unsigned *>(sA) + 2 * i * sld + 1;
#pragma unroll 4
        for (int q = 0; q < nsb; ++q) {
          const float a = hi2f(ar[2 * sh.jb[q]]), d = sh.dxf[sh.sb[q]];
          s0 = fmaf(a, d, s0);
          e0 = fmaf(fabsf(a), fabsf(d), e0);
        }
      } else {
        const float *ar = reinterpret_cast<const float *>(sA) + i * sld;
#pragma unroll 4
        for (int q = 0; q < nsb; ++q) {
          const float a = ar[sh.jb[q]], d = sh.dxf[sh.sb[q]];
          s0 = fmaf(a, d, s0);
          e0 = fmaf(fabsf(a), fabsf(d), e0);
        }
      }
      mag = e0;
      return s0;
    };
    auto col_delta = [&](int j, float &mag) {
      float s0 = 0.f, e0 = 0.f;
      if (dt == LPB_DTYPE_F64) {
        const unsigned *ac = reinterpret_cast<const unsigned *>(sA) + 2 * j + 1;
#pragma unroll 4
        for (int q = 0; q < nns; ++q) {
          const int k = sh.kr[q];
          const float a = hi2f(ac[2 * k * sld]), d = sh.dyf[k];
          s0 = fmaf(a, d, s0);
          e0 = fmaf(fabsf(a), fabsf(d), e0);
        }
      } else {
        const float *ac = reinterpret_cast<const float *>(sA) + j;
#pragma unroll 4
        for (int q = 0; q < nns; ++q) {
          const int k = sh.kr[q];
          const float a = ac[k * sld], d = sh.dyf[k];
          s0 = fmaf(a, d, s0);
          e0 = fmaf(fabsf(a), fabsf(d), e0);
        }
      }
      mag = e0;
      return s0;
    };
    // Refinement rounds: FP64 residuals at the current point, one correction
    // with the FP32 basis inverse, the certificate.  Almost every LP passes
    // after the first round; one that fails gets up to two more rounds before
    // it goes to the FP64 re-solve.
    const double tol = P.feas_tol, tp = sh.tpd[0], td = sh.tpd[1];
    constexpr float kDeltaErr = 1.f / 32768.f;
    int fail = 0;
    for (int round = 0;; ++round) {
      // Residuals in FP64: sax = b - A x and r = sax - x_slack (rows, on the low
      // threads); the reduced costs d = A^T y - c of every column (high
      // threads), whose negatives on the basic structurals are the dual residual.
      for (int i = tid; i < m; i += NT) {
        const double ax = vin(sh.bin, i, dt) - row_dot(i);
        const double r = sh.sp[i] >= 0 ? ax - sh.xb[sh.sp[i]] : ax;
        sh.sax[i] = ax;
        sh.rr[i] = r;
        sh.rrf[i] = float(r);
      }
      for (int j = NT - 1 - tid; j < n; j += NT) {
        const double d = col_dot(j) - vin(sh.cin, j, dt);
        sh.dj[j] = d;
        if (sh.posx[j] >= 0) sh.rhof[sh.posx[j]] = float(-d);
      }
      __syncthreads();
      // Corrections with the FP32 basis inverse held in registers: its column for
      // slack k is the tableau column of k when k is non-basic, else a unit vector.
      {
        constexpr int CP = pow2_at_least(C);
        float coef[C];
  #pragma unroll
        for (int c = 0; c < C; ++c) {
          const int v = sh.nonb[wid + W * c];
          coef[c] = (c < C - 1 || wid < W - 1) && v >= n && v < n + m ? sh.rrf[v - n] : 0.f;
        }
  #pragma unroll
        for (int r = 0; r < R; ++r) {
          float s = 0.f;
  #pragma unroll
          for (int c = 0; c < C; ++c) s = fmaf(T[r][c], coef[c], s);
          sh.part[wid][lane + 32 * r] = s;
        }
        float rf[R];
  #pragma unroll
        for (int r = 0; r < R; ++r) rf[r] = sh.rhof[lane + 32 * r];
        float dy[CP];
  #pragma unroll
        for (int c = 0; c < CP; ++c) {
          float s = 0.f;
          if (c < C) {
  #pragma unroll
            for (int r = 0; r < R; ++r) s = fmaf(T[r][c], rf[r], s);
          }
          dy[c] = s;
        }
        // Column sums across the lanes; lane l ends with column l / (32 / CP),
        // and the first lane of each group applies it to y.
        const float tot = reduce_scatter<CP>(dy, lane);
        const int c = lane / (32 / CP);
        if (lane % (32 / CP) == 0 && c < C && (c < C - 1 || wid < W - 1)) {
          const int v = sh.nonb[wid + W * c];
          if (v >= n && v < n + m) sh.dyf[v - n] = tot;
        }
      }
      __syncthreads();
      for (int t = tid; t < m; t += NT) {
        float s = 0.f;
  #pragma unroll
        for (int w = 0; w < W; ++w) s += sh.part[w][t];
        const int v = sh.basic[t];
        const double dx = v >= n ? double(s) + sh.rr[v - n] : double(s);
        sh.xb[t] += dx;
        sh.dxf[t] = v < n ? s : 0.f;         // the structural part of the correction (double(s) exactly)
      }
      if (wid == W - 1)                      // y += dy on the non-basic slacks, by one warp
        for (int p2 = lane; p2 < nns; p2 += 32) sh.yv[sh.kr[p2]] += double(sh.dyf[sh.kr[p2]]);
      if (tid == claimer && round == 0) stage3();
      __syncthreads();
      // KKT certificate of the pair that is written out (x: the structural part
      // of x_B; y: the slack duals): x >= 0, A x <= b, y >= 0, A^T y >= c and
      // c^T x = b^T y, each to tol scaled by the data.  b - A x and A^T y - c at
      // the corrected point are the FP64 values above plus FP32 products with
      // the corrections, whose rounding (and the 2^-20 truncation of A) is
      // bounded by 2^-15 times the sum of the products' magnitudes.
      fail = 0;
      for (int q = tid; q < nsb; q += NT) fail |= !(sh.xb[sh.sb[q]] >= -tp);
      for (int p2 = tid; p2 < nns; p2 += NT) fail |= !(sh.yv[sh.kr[p2]] >= -td);
      for (int i = tid; i < m; i += NT) {                 // slack b_i - A_i x of every row
        float mag;
        const float dl = row_delta(i, mag);
        fail |= !(sh.sax[i] - double(dl + kDeltaErr * mag) >= -tp);
      }
      for (int j = NT - 1 - tid; j < n; j += NT) {        // reduced cost A_j^T y - c_j of every column
        float mag;
        const float dl = col_delta(j, mag);
        fail |= !(sh.dj[j] + double(dl - kDeltaErr * mag) >= -td);
      }
      // c^T x in warp 0 and b^T y in warp 1 (FP64; a one-warp CTA forms both).
      if (wid == 0) {
        double cx = 0.0;
        for (int q = lane; q < nsb; q += 32) cx = fma(vin(sh.cin, sh.jb[q], dt), sh.xb[sh.sb[q]], cx);
        cx = warp_sum(cx);
        if (lane == 0) sh.red[0][0] = cx;
      }
      if (wid == kColWarp) {
        double by = 0.0;
        for (int p2 = lane; p2 < nns; p2 += 32) by = fma(vin(sh.bin, sh.kr[p2], dt), sh.yv[sh.kr[p2]], by);
        by = warp_sum(by);
        if (lane == 0) sh.red[1][0] = by;
      }
      if (wid < 2) {         // warps 0 and 1 meet; thread 0 checks the duality gap
        if constexpr (W > 1) asm volatile("bar.sync 1, 64;\n" ::: "memory");
        else __syncwarp();
        if (tid == 0) {
          const double cx = sh.red[0][0], by = sh.red[1][0];
          fail |= !(fabs(cx - by) <= tol * (1.0 + fabs(cx)));
        }
      }
      fail = __syncthreads_or(fail);
      if (!fail || round == 2) break;
      __syncthreads();       // sh.red and the check inputs are rewritten by the next round
    }
    // The next LP's A, b and c, when one bulk copy each serves them: every read
    // of this LP's copies is behind the certificate's last barrier, so the
    // copy engine may overwrite them while this LP's results are written and
    // the loop head runs.  (Shared-constraint batches keep A and b resident.)
    // The last warp issues them (it has the fewest results to write): one lane
    // sets the expected bytes, then three lanes issue one copy each.
    if (wid == W - 1 && !P.shared) {
      const RegDesc &N = sh.desc[slot ^ 1];
      if (N.item < nitems && fits_lp(N.m, N.n)) {
        const unsigned m2 = unsigned(N.m), n2 = unsigned(N.n);
        const unsigned char *Ag2 = static_cast<const unsigned char *>(P.B.A) + N.aoff * es;
        const unsigned char *bg2 = static_cast<const unsigned char *>(P.B.b) + N.boff * es;
        const unsigned char *cg2 = static_cast<const unsigned char *>(P.B.c) + N.coff * es;
        const bool dense2 = ((reinterpret_cast<uintptr_t>(Ag2) | uintptr_t(m2) * n2 * unsigned(es)) & 15) == 0;
        const bool bc2 = ((reinterpret_cast<uintptr_t>(bg2) | reinterpret_cast<uintptr_t>(cg2) |
                           uintptr_t(m2) * unsigned(es) | uintptr_t(n2) * unsigned(es)) & 15) == 0;
        if (dense2 && bc2) {          // the same value in every lane
          if (lane == 0) mbar_expect_tx(&sh.abar, m2 * n2 * unsigned(es) + (m2 + n2) * unsigned(es));
          __syncwarp();
          if (lane == 0) bulk_load(sA, Ag2, m2 * n2 * unsigned(es), &sh.abar);
          else if (lane == 1) bulk_load(sh.bin, bg2, m2 * unsigned(es), &sh.abar);
          else if (lane == 2) bulk_load(sh.cin, cg2, n2 * unsigned(es), &sh.abar);
          if (lane == 0) sh.pre = 1;
        }
      }
    }
    if (fail) valid_tab = 0;            // the next objective starts cold
    if (bp) for (int i = tid; i < m; i += NT) bp[i] = sh.basic[i];
    if (!fail) {
      for (int j = tid; j < n; j += NT) P.R.x[coff + j] = sh.posx[j] >= 0 ? sh.xb[sh.posx[j]] : 0.0;
      if (P.R.y) for (int k = tid; k < m; k += NT) P.R.y[yoff + k] = sh.yv[k];
    }
    if (tid == 0) {
      const double cx = sh.red[0][0];
      if (!fail) {
        P.R.status[lp] = LPB_OPTIMAL;
        P.R.obj[lp] = cx;
      } else {
        P.R.status[lp] = STATUS_PENDING;
        list_push(P.resolve_items, P.resolve_count, P.list_cap, lp, P.err);
      }
      if (P.R.iters) P.R.iters[lp] = iters;
    }
    __syncthreads();
  }
}

struct RegConfig {
  int R, C, W;
  const void *fn;
  const void *fn_se;     // the steepest-edge instantiation, or null
  size_t fixed;
};

#define LPB_REG(R, C, W) \
  RegConfig{R, C, W, reinterpret_cast<const void *>(&reg_kernel<R, C, W, false>), nullptr, reg_fixed_bytes<R, C, W>()}
#define LPB_REG_SE(R, C, W)                                                                         \
  RegConfig{R, C, W, reinterpret_cast<const void *>(&reg_kernel<R, C, W, false>),                   \
            reinterpret_cast<const void *>(&reg_kernel<R, C, W, true>), reg_fixed_bytes<R, C, W>()}
// One-warp CTAs (W = 1) serve batches of tiny LPs (m, n <= 31): one warp per
// LP, so that an SM holds many LPs at once and a pivot costs one warp's work.
const RegConfig kRegConfigs[] = {
    LPB_REG(1, 8, 4), LPB_REG(2, 16, 4), LPB_REG(4, 26, 4), LPB_REG(4, 32, 4),
    LPB_REG_SE(1, 4, 8), LPB_REG_SE(2, 8, 8), LPB_REG_SE(4, 13, 8), LPB_REG_SE(4, 16, 8),
    LPB_REG_SE(1, 8, 1), LPB_REG_SE(1, 16, 1), LPB_REG_SE(1, 32, 1),
};
#undef LPB_REG
#undef LPB_REG_SE
constexpr int kNumReg = int(sizeof(kRegConfigs) / sizeof(kRegConfigs[0]));

size_t reg_smem_bytes(int cfg, int max_m, int max_n, int dtype) {
  const int es = dtype == LPB_DTYPE_F64 ? 8 : 4;
  return kRegConfigs[cfg].fixed + size_t(max_m) * size_t(a_stride(max_n, es)) * es;
}

}  // namespace

int reg_count() { return kNumReg; }

// Largest m and n configuration `cfg` holds, and its warps per CTA.
void reg_limits(int cfg, int *max_m, int *max_n, int *warps) {
  const RegConfig &k = kRegConfigs[cfg];
  *max_m = 32 * k.R - 1;
  *max_n = k.W * k.C - 1;
  *warps = k.W;
}

// Whether configuration `cfg` has a steepest-edge instantiation (the 8-warp ones).
bool reg_has_se(int cfg) { return kRegConfigs[cfg].fn_se != nullptr; }

// Smallest configuration whose rows hold max_m + 1 and columns max_n + 1,
// with `want_w` warps when given (8 warps by default) and, when `se`, a
// steepest-edge instantiation; -1 if none fits.
int reg_pick(int max_m, int max_n, int want_w, bool se) {
  if (want_w <= 0) want_w = 8;
  int best = -1, best_cost = 1 << 30;
  for (int i = 0; i < kNumReg; ++i) {
    const RegConfig &k = kRegConfigs[i];
    if (32 * k.R - 1 < max_m || k.W * k.C - 1 < max_n || k.W != want_w || (se && !k.fn_se)) continue;
    const int cost = k.R * k.C * k.W;
    if (cost < best_cost) { best_cost = cost; best = i; }
  }
  return best;
}

cudaError_t reg_occupancy(int cfg, int max_m, int max_n, int dtype, int rule, int *ctas, int *threads,
                          size_t *smem) {
  const RegConfig &k = kRegConfigs[cfg];
  const void *fn = rule == LPB_PIVOT_STEEPEST ? k.fn_se : k.fn;
  if (!fn) return cudaErrorInvalidValue;
  *threads = 32 * k.W;
  *smem = reg_smem_bytes(cfg, max_m, max_n, dtype);
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(*smem));
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas, fn, *threads, *smem);
}

cudaError_t launch_reg(const TableauParams &p, int cfg, int grid, size_t smem, cudaStream_t s) {
  const RegConfig &k = kRegConfigs[cfg];
  const void *fn = p.rule == LPB_PIVOT_STEEPEST ? k.fn_se : k.fn;
  if (!fn) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (e != cudaSuccess) return e;
  void *args[] = {const_cast<TableauParams *>(&p)};
  return cudaLaunchKernel(fn, dim3(grid), dim3(32 * k.W), args, smem, s);
}

}  // namespace lpb
