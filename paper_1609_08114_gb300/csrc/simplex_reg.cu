// simplex_reg.cu -- register-resident FP32 tableau for LPs whose slack basis is
// feasible (all b_i >= 0), with the FP64 refinement and verification fused in.
//
// Section 3.1 Steps 1-3 on one LP per CTA of W warps (Section 4.1: a block of
// threads per LP).  Type-1 LPs of the paper's sizes take only ~13 pivots at
// m = n = 100, so a solve is dominated by moving the LP on chip and by the
// latency of each pivot, not by the rank-1 arithmetic.  Design:
//
//   * The LP's input A (FP64 or FP32, as given) is copied once into shared
//     memory with asynchronous copies (one memory round trip) and stays there
//     for the whole solve; the FP64 refinement reads it back from there.
//   * The compact FP32 tableau lives in registers: lane l of every warp owns
//     rows l, l+32, ..., l+32(R-1); warp w owns columns w, w+W, ..., w+W(C-1).
//     The objective row sits at the fixed row 32R-1 (lane 31, register row
//     R-1) and the right-hand side at the fixed column WC-1 (warp W-1, register
//     column C-1); rows and columns between the LP's edge and those slots are
//     zero and stay zero under pivoting, so they need no masks.
//   * Step 1: each warp judges its own columns (lane c takes column w + W c)
//     and the W candidates meet in shared memory.
//   * Step 2: the pivot column lives in one warp (its lanes hold the rows), so
//     the min-ratio test is a warp reduction with no block barrier.
//   * Step 3: the lane owning the pivot row scales it by 1/pivot in place; each
//     warp takes its part of it by shuffles and the pivot column from shared
//     memory; the update is R x C FMAs per lane.  Two block barriers per pivot.
//   * Arg-min reductions use the warp reduction instruction on an
//     order-preserving integer image of the float (value first, then key).
//
// FP64 input is rounded to FP32 in integer arithmetic (d2f_rn): the FP64 unit
// of this GPU, which also converts double to float, is a small fraction of the
// FP32 rate.
//
// After an FP32 optimum the basis inverse is in the registers (the columns of
// the non-basic slacks).  One step of iterative refinement with FP64 residuals
// gives x_B and y; an FP64 KKT certificate (x >= 0, A x <= b, y >= 0,
// A^T y >= c, c^T x = b^T y) decides between writing the result and queueing
// the LP for the FP64 re-solve.  LPs with some b_i < 0 (Phase I), or larger
// than the template, or with non-finite data go to the shared-memory kernel.
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

template <int R, int C, int W>
struct RegShared {
  static constexpr int ROWS = 32 * R, COLS = W * C;
  float colbuf[ROWS];
  float rhs[ROWS];
  int basic[ROWS];
  int nonb[COLS];
  float candv[W];
  int candk[W];
  alignas(16) float objv[W][(C + 3) & ~3];   // objective row, per warp
  int l, leave_var, status, item;
  float theta;
  int nsb, nns;
  unsigned long long bmax, cmax;
  double xb[ROWS], rr[ROWS], yv[ROWS], rho[ROWS];
  float part[W][ROWS];
  float rhof[ROWS];
  int sb[ROWS], ns[COLS], sp[ROWS];
  double red[2][W];
};

template <int R, int C, int W>
__host__ __device__ constexpr size_t reg_fixed_bytes() { return (sizeof(RegShared<R, C, W>) + 15) & ~size_t(15); }

// Row stride (in elements) of the resident copy of A: odd, so lanes reading
// consecutive rows of one column hit distinct banks.
__host__ __device__ inline int a_stride(int max_n) { return max_n | 1; }

template <typename T>
__device__ __forceinline__ double a_at(const unsigned char *sa, int dt, int idx) {
  return dt == LPB_DTYPE_F64 ? reinterpret_cast<const double *>(sa)[idx]
                             : double(reinterpret_cast<const float *>(sa)[idx]);
}

template <int R, int C, int W>
__global__ void __launch_bounds__(W * 32, (W <= 4 ? 3 : 2)) reg_kernel(TableauParams P) {
  using SH = RegShared<R, C, W>;
  constexpr int ROWS = SH::ROWS, COLS = SH::COLS;
  constexpr int NT = W * 32;
  extern __shared__ __align__(16) unsigned char reg_smem[];
  SH &sh = *reinterpret_cast<SH *>(reg_smem);
  unsigned char *sA = reg_smem + reg_fixed_bytes<R, C, W>();   // resident input A
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const float eps_p = float(P.eps_p), eps_d = float(P.eps_d);
  const int dt = P.B.dtype;
  const int sld = a_stride(P.lim_n);
  const int nitems = P.in.count ? min(*P.in.count, P.list_cap) : P.B.count;
  float T[R][C];

  for (;;) {
    if (tid == 0) sh.item = atomicAdd(P.queue, 1);
    __syncthreads();
    const int item = sh.item;
    if (item >= nitems) break;
    const int lp = P.in.items ? P.in.items[item] : item;
    const int m = P.B.m[lp], n = P.B.n[lp];
    const int64_t aoff = P.B.a_off[lp], boff = P.B.b_off[lp], coff = P.B.c_off[lp];
    // ---- admission: sizes that fit the template, b >= 0, finite b and c ----
    const bool fits = m >= 1 && n >= 1 && m <= ROWS - 1 && n <= COLS - 1 && m <= P.B.max_m && n <= P.B.max_n &&
                      m <= P.lim_m && n <= P.lim_n;
    if (fits) {    // start streaming A now; its copies land while b and c are checked
      if (dt == LPB_DTYPE_F64) {
        const double *A = static_cast<const double *>(P.B.A) + aoff;
        double *s = reinterpret_cast<double *>(sA);
        for (int i = wid; i < m; i += W)
          for (int j = lane; j < n; j += 32) cp_async8(s + i * sld + j, A + int64_t(i) * n + j);
      } else {
        const float *A = static_cast<const float *>(P.B.A) + aoff;
        float *s = reinterpret_cast<float *>(sA);
        for (int i = wid; i < m; i += W)
          for (int j = lane; j < n; j += 32) cp_async4(s + i * sld + j, A + int64_t(i) * n + j);
      }
    }
    int neg = 0;
    if (tid == 0) { sh.bmax = 0ull; sh.cmax = 0ull; }
    __syncthreads();
    if (fits) {
      double bm = 0.0, cm = 0.0;
      for (int i = tid; i < m; i += NT) {
        const double v = ld_in(P.B.b, boff + i, dt);
        neg |= !(v >= 0.0);   // negative or NaN
        bm = fmax(bm, fabs(v));
      }
      for (int j = tid; j < n; j += NT) {
        const double v = ld_in(P.B.c, coff + j, dt);
        neg |= !finite_bits(v);
        cm = fmax(cm, fabs(v));
      }
      if (bm == bm) atomicMax(&sh.bmax, static_cast<unsigned long long>(__double_as_longlong(bm)));
      if (cm == cm) atomicMax(&sh.cmax, static_cast<unsigned long long>(__double_as_longlong(cm)));
    }
    cp_async_wait_all();
    neg = __syncthreads_or(neg);
    if (!fits || neg) {      // the shared-memory kernel handles it (Phase I, sizes, bad data)
      if (tid == 0) {
        P.R.status[lp] = STATUS_PENDING;
        list_push(P.defer_items, P.defer_count, P.list_cap, lp, P.err);
      }
      __syncthreads();
      continue;
    }
    const double bmax = __longlong_as_double(static_cast<long long>(sh.bmax));
    const double cmax = __longlong_as_double(static_cast<long long>(sh.cmax));

    // ---- the tableau: A rounded to FP32, b in column COLS-1, -c in row ROWS-1 ----
    int bad = 0;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int i = lane + 32 * r;
#pragma unroll
      for (int c = 0; c < C; ++c) {
        const int j = wid + W * c;
        float v = 0.f;
        if (i < m && j < n) {
          if (dt == LPB_DTYPE_F64) {
            const double a = reinterpret_cast<const double *>(sA)[i * sld + j];
            bad |= !finite_bits(a);
            v = d2f_rn(a);
          } else {
            v = reinterpret_cast<const float *>(sA)[i * sld + j];
            bad |= !isfinite(v);
          }
        }
        T[r][c] = v;
      }
    }
    bad = __syncthreads_or(bad);
    if (bad) {
      if (tid == 0) {
        P.R.status[lp] = STATUS_PENDING;
        list_push(P.defer_items, P.defer_count, P.list_cap, lp, P.err);
      }
      __syncthreads();
      continue;
    }
    if (wid == W - 1) {
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int i = lane + 32 * r;
        const float v = i < m ? ld_as<float>(P.B.b, boff + i, dt) : 0.f;
        T[r][C - 1] = v;
        sh.rhs[i] = v;
      }
    }
    if (lane == 31) {
#pragma unroll
      for (int c = 0; c < C; ++c) {
        const int j = wid + W * c;
        if (j < n) T[R - 1][c] = -ld_as<float>(P.B.c, coff + j, dt);
      }
    }
    for (int i = tid; i < ROWS; i += NT) sh.basic[i] = i < m ? n + i : kBad >> kIdxBits;
    for (int j = tid; j < COLS; j += NT) sh.nonb[j] = j < n ? j : kBad >> kIdxBits;

    // ---- Steps 1-3 ----
    const int max_iter = P.max_iter > 0 ? P.max_iter : 50 * (m + n);
    int iters = 0, status = LPB_OPTIMAL, degenerate_run = 0;
    bool bland = false;
    // Step 1 candidates: lane 31 publishes the warp's objective-row entries
    // with 16-byte stores; lane c judges column wid + W c.  Column `ecol` (if
    // >= 0) holds variable `evar`, whose nonb[] entry is rewritten meanwhile.
    float *objw = sh.objv[wid];
    auto candidates = [&](int ecol, int evar) {
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
      float v = __int_as_float(0x7f800000);
      int key = kBad;
      const int j = wid + W * lane;
      if (lane < C && j < COLS - 1) {                  // the last column is the right-hand side
        const float rj = objw[lane];
        if (rj < -eps_d) {
          const int var = (j == ecol) ? evar : sh.nonb[j];
          v = bland ? 0.f : rj;
          key = (var << kIdxBits) | j;
        }
      }
      warp_argmin_f32(v, key);
      if (lane == 0) {
        sh.candv[wid] = v;
        sh.candk[wid] = key;
      }
    };
    __syncthreads();
    candidates(-1, 0);
    __syncthreads();
    for (;;) {
      float ev = lane < W ? sh.candv[lane] : __int_as_float(0x7f800000);
      int ek = lane < W ? sh.candk[lane] : kBad;
      warp_argmin_f32(ev, ek);
      if (ek == kBad) { status = LPB_OPTIMAL; break; }
      const int e = ek & kIdxMask;
      const int we = e % W, ce = e / W;
      float col[R];
      if (wid == we) {
        // Step 2 inside the warp that owns column e.
        dispatch<0, C>(ce, [&](auto K) {
#pragma unroll
          for (int r = 0; r < R; ++r) col[r] = T[r][K.value];
        });
        float v = __int_as_float(0x7f800000);
        int key = kBad;
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const int i = lane + 32 * r;
          if (col[r] > eps_p) keep_better(v, key, sh.rhs[i] * __frcp_rn(col[r]), (sh.basic[i] << kIdxBits) | i);
        }
        warp_argmin_f32(v, key);
#pragma unroll
        for (int r = 0; r < R; ++r) sh.colbuf[lane + 32 * r] = col[r];
        if (lane == 0) {
          if (key == kBad) {
            sh.status = LPB_UNBOUNDED;
          } else {
            const int l = key & kIdxMask;
            sh.status = LPB_OPTIMAL;
            sh.l = l;
            sh.theta = v;
            sh.leave_var = sh.basic[l];
          }
        }
      }
      __syncthreads();                                                      // B1
      if (sh.status == LPB_UNBOUNDED) { status = LPB_UNBOUNDED; break; }
      if (iters >= max_iter) { status = LPB_ITER_LIMIT; break; }
      const int l = sh.l;
      const float theta = sh.theta;
      const int lr = l >> 5, ll = l & 31;
      const float p = sh.colbuf[l];
      const float rp = 1.f / p;
      float cf[R];           // pivot column; 0 on the pivot row, which is only scaled
#pragma unroll
      for (int r = 0; r < R; ++r) cf[r] = (lane + 32 * r == l) ? 0.f : sh.colbuf[lane + 32 * r];
      // Step 3: the owner lane scales the pivot row by 1/p in place, then every
      // warp takes its part of it by shuffles: T -= (pivot column) (x) (new pivot row).
      dispatch<0, R>(lr, [&](auto LR) {
        if (lane == ll) {
#pragma unroll
          for (int c = 0; c < C; ++c) T[LR.value][c] *= rp;
        }
#pragma unroll
        for (int c = 0; c < C; ++c) {
          const float pr = __shfl_sync(kFull, T[LR.value][c], ll);
#pragma unroll
          for (int r = 0; r < R; ++r) T[r][c] = fmaf(-cf[r], pr, T[r][c]);
        }
      });
      if (wid == we) {        // new column e: -t_ie / p, and 1/p at the pivot
        dispatch<0, C>(ce, [&](auto K) {
#pragma unroll
          for (int r = 0; r < R; ++r) T[r][K.value] = (lane + 32 * r == l) ? rp : -col[r] * rp;
        });
      }
      if (tid == 0) {
        sh.basic[l] = ek >> kIdxBits;
        sh.nonb[e] = sh.leave_var;
      }
      if (wid == W - 1) {
#pragma unroll
        for (int r = 0; r < R; ++r) sh.rhs[lane + 32 * r] = T[r][C - 1];
      }
      ++iters;
      if (theta <= eps_p) {
        if (++degenerate_run >= m + n) bland = true;
      } else {
        degenerate_run = 0;
        bland = false;
      }
      candidates(e, sh.leave_var);
      __syncthreads();                                                      // B2
    }

    int32_t *bp = P.bbuf ? P.bbuf + (P.bpacked ? boff : int64_t(lp) * P.B.max_m) : nullptr;
    if (status != LPB_OPTIMAL || P.mode != MODE_FP32_REFINE) {
      if (status == LPB_OPTIMAL) {   // plain FP32: results straight from the tableau
        for (int j = tid; j < n; j += NT) P.R.x[coff + j] = 0.0;
        if (P.R.y) for (int i = tid; i < m; i += NT) P.R.y[boff + i] = 0.0;
        __syncthreads();
        for (int i = tid; i < m; i += NT)
          if (sh.basic[i] < n) P.R.x[coff + sh.basic[i]] = double(sh.rhs[i]);
        if (lane == 31 && P.R.y) {
#pragma unroll
          for (int c = 0; c < C; ++c) {
            if (wid == W - 1 && c == C - 1) continue;    // the right-hand side
            const int v = sh.nonb[wid + W * c];
            if (v >= n && v < n + m) P.R.y[boff + (v - n)] = double(T[R - 1][c]);
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
        if (P.R.y) for (int i = tid; i < m; i += NT) P.R.y[boff + i] = 0.0;
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
    if (wid == 0) {      // structural basic rows, non-basic slack columns (in order)
      int base = 0;
      for (int i0 = 0; i0 < m; i0 += 32) {
        const int i = i0 + lane;
        const bool pr = i < m && sh.basic[i] < n;
        const unsigned mk = __ballot_sync(kFull, pr);
        if (pr) sh.sb[base + __popc(mk & ((1u << lane) - 1u))] = i;
        base += __popc(mk);
      }
      if (lane == 0) sh.nsb = base;
      base = 0;
      for (int j0 = 0; j0 < COLS - 1; j0 += 32) {
        const int j = j0 + lane;
        const bool pr = j < COLS - 1 && sh.nonb[j] >= n && sh.nonb[j] < n + m;
        const unsigned mk = __ballot_sync(kFull, pr);
        if (pr) sh.ns[base + __popc(mk & ((1u << lane) - 1u))] = j;
        base += __popc(mk);
      }
      if (lane == 0) sh.nns = base;
    }
    for (int i = tid; i < ROWS; i += NT) {
      sh.sp[i] = -1;
      sh.yv[i] = 0.0;
      sh.rhof[i] = 0.f;
      sh.xb[i] = i < m ? double(sh.rhs[i]) : 0.0;
    }
    __syncthreads();
    const int nsb = sh.nsb, nns = sh.nns;
    for (int i = tid; i < m; i += NT) {
      const int v = sh.basic[i];
      if (v >= n) sh.sp[v - n] = i;
    }
    if (lane == 31) {
#pragma unroll
      for (int c = 0; c < C; ++c) {
        if (wid == W - 1 && c == C - 1) continue;      // the right-hand side
        const int v = sh.nonb[wid + W * c];
        if (v >= n && v < n + m) sh.yv[v - n] = double(T[R - 1][c]);
      }
    }
    __syncthreads();
    // FP64 residuals: r = b - [A I]_B x_B (one row per thread) and
    // rho_t = c_B(t) - (B^T y)_t (structural basic rows, on the other threads).
    for (int i = tid; i < m; i += NT) {
      double r = ld_in(P.B.b, boff + i, dt);
#pragma unroll 4
      for (int q = 0; q < nsb; ++q) {
        const int t = sh.sb[q];
        r = fma(-a_at<double>(sA, dt, i * sld + sh.basic[t]), sh.xb[t], r);
      }
      if (sh.sp[i] >= 0) r -= sh.xb[sh.sp[i]];
      sh.rr[i] = r;
    }
    for (int q = NT - 1 - tid; q < nsb; q += NT) {
      const int t = sh.sb[q], j = sh.basic[t];
      double r = ld_in(P.B.c, coff + j, dt);
#pragma unroll 4
      for (int p2 = 0; p2 < nns; ++p2) {
        const int k = sh.nonb[sh.ns[p2]] - n;
        r = fma(-a_at<double>(sA, dt, k * sld + j), sh.yv[k], r);
      }
      sh.rho[t] = r;
      sh.rhof[t] = float(r);
    }
    __syncthreads();
    // Corrections with the FP32 basis inverse held in registers: its column for
    // slack k is the tableau column of k when k is non-basic, else a unit vector.
    {
      float coef[C];
#pragma unroll
      for (int c = 0; c < C; ++c) {
        const int v = sh.nonb[wid + W * c];
        coef[c] = (c < C - 1 || wid < W - 1) && v >= n && v < n + m ? float(sh.rr[v - n]) : 0.f;
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
#pragma unroll
      for (int c = 0; c < C; ++c) {
        const int v = sh.nonb[wid + W * c];
        if ((c < C - 1 || wid < W - 1) && v >= n && v < n + m) {   // warp-uniform
          float s = 0.f;
#pragma unroll
          for (int r = 0; r < R; ++r) s = fmaf(T[r][c], rf[r], s);
          s = warp_sum(s);
          if (lane == 0) sh.yv[v - n] += double(s);
        }
      }
    }
    __syncthreads();
    for (int t = tid; t < m; t += NT) {
      float s = 0.f;
#pragma unroll
      for (int w = 0; w < W; ++w) s += sh.part[w][t];
      double dx = double(s);
      const int v = sh.basic[t];
      if (v >= n) dx += sh.rr[v - n];
      sh.xb[t] += dx;
    }
    __syncthreads();
    // FP64 KKT certificate of the pair that is written out (x: the structural
    // part of x_B; y: the slack duals): x >= 0, A x <= b, y >= 0, A^T y >= c and
    // c^T x = b^T y, each to tol scaled by the data.  Rows on the low threads,
    // columns on the high ones.
    const double tol = P.feas_tol, tp = tol * (1.0 + bmax), td = tol * (1.0 + cmax);
    int fail = 0;
    double cx = 0.0, by = 0.0;
    for (int q = tid; q < nsb; q += NT) {
      const int t = sh.sb[q];
      fail |= !(sh.xb[t] >= -tp);
      cx = fma(ld_in(P.B.c, coff + sh.basic[t], dt), sh.xb[t], cx);
    }
    for (int p2 = tid; p2 < nns; p2 += NT) {
      const int k = sh.nonb[sh.ns[p2]] - n;
      fail |= !(sh.yv[k] >= -td);
      by = fma(ld_in(P.B.b, boff + k, dt), sh.yv[k], by);
    }
    for (int i = tid; i < m; i += NT) {                 // slack b_i - A_i x of every row
      double s = ld_in(P.B.b, boff + i, dt);
#pragma unroll 4
      for (int q = 0; q < nsb; ++q) s = fma(-a_at<double>(sA, dt, i * sld + sh.basic[sh.sb[q]]), sh.xb[sh.sb[q]], s);
      fail |= !(s >= -tp);
    }
    for (int j = NT - 1 - tid; j < n; j += NT) {        // reduced cost A_j^T y - c_j of every column
      double d = -ld_in(P.B.c, coff + j, dt);
#pragma unroll 4
      for (int p2 = 0; p2 < nns; ++p2) {
        const int k = sh.nonb[sh.ns[p2]] - n;
        d = fma(a_at<double>(sA, dt, k * sld + j), sh.yv[k], d);
      }
      fail |= !(d >= -td);
    }
    cx = warp_sum(cx);
    by = warp_sum(by);
    if (lane == 0) { sh.red[0][wid] = cx; sh.red[1][wid] = by; }
    fail = __syncthreads_or(fail);
    cx = 0.0;
    by = 0.0;
#pragma unroll
    for (int w = 0; w < W; ++w) { cx += sh.red[0][w]; by += sh.red[1][w]; }
    fail |= !(fabs(cx - by) <= tol * (1.0 + fabs(cx)));
    if (bp) for (int i = tid; i < m; i += NT) bp[i] = sh.basic[i];
    if (fail) {
      if (tid == 0) {
        P.R.status[lp] = STATUS_PENDING;
        if (P.R.iters) P.R.iters[lp] = iters;
        list_push(P.resolve_items, P.resolve_count, P.list_cap, lp, P.err);
      }
    } else {
      for (int j = tid; j < n; j += NT) P.R.x[coff + j] = 0.0;
      __syncthreads();
      for (int q = tid; q < nsb; q += NT) P.R.x[coff + sh.basic[sh.sb[q]]] = sh.xb[sh.sb[q]];
      if (P.R.y) for (int k = tid; k < m; k += NT) P.R.y[boff + k] = sh.yv[k];
      if (tid == 0) {
        P.R.status[lp] = LPB_OPTIMAL;
        if (P.R.iters) P.R.iters[lp] = iters;
        P.R.obj[lp] = cx;
      }
    }
    __syncthreads();
  }
}

struct RegConfig {
  int R, C, W;
  const void *fn;
  size_t fixed;
};

#define LPB_REG(R, C, W) \
  RegConfig{R, C, W, reinterpret_cast<const void *>(&reg_kernel<R, C, W>), reg_fixed_bytes<R, C, W>()}
const RegConfig kRegConfigs[] = {
    LPB_REG(1, 8, 4), LPB_REG(2, 16, 4), LPB_REG(4, 26, 4), LPB_REG(4, 32, 4),
    LPB_REG(1, 4, 8), LPB_REG(2, 8, 8), LPB_REG(4, 13, 8), LPB_REG(4, 16, 8),
};
#undef LPB_REG
constexpr int kNumReg = int(sizeof(kRegConfigs) / sizeof(kRegConfigs[0]));

size_t reg_smem_bytes(int cfg, int max_m, int max_n, int dtype) {
  return kRegConfigs[cfg].fixed + size_t(max_m) * size_t(a_stride(max_n)) * (dtype == LPB_DTYPE_F64 ? 8 : 4);
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

// Smallest configuration whose rows hold max_m + 1 and columns max_n + 1,
// with `want_w` warps when given (8 warps by default); -1 if none fits.
int reg_pick(int max_m, int max_n, int want_w) {
  if (want_w <= 0) want_w = 8;
  int best = -1, best_cost = 1 << 30;
  for (int i = 0; i < kNumReg; ++i) {
    const RegConfig &k = kRegConfigs[i];
    if (32 * k.R - 1 < max_m || k.W * k.C - 1 < max_n || k.W != want_w) continue;
    const int cost = k.R * k.C * k.W;
    if (cost < best_cost) { best_cost = cost; best = i; }
  }
  return best;
}

cudaError_t reg_occupancy(int cfg, int max_m, int max_n, int dtype, int *ctas, int *threads,
                          size_t *smem) {
  const RegConfig &k = kRegConfigs[cfg];
  *threads = 32 * k.W;
  *smem = reg_smem_bytes(cfg, max_m, max_n, dtype);
  cudaError_t e = cudaFuncSetAttribute(k.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(*smem));
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas, k.fn, *threads, *smem);
}

cudaError_t launch_reg(const TableauParams &p, int cfg, int grid, size_t smem, cudaStream_t s) {
  const RegConfig &k = kRegConfigs[cfg];
  cudaError_t e = cudaFuncSetAttribute(k.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (e != cudaSuccess) return e;
  void *args[] = {const_cast<TableauParams *>(&p)};
  return cudaLaunchKernel(k.fn, dim3(grid), dim3(32 * k.W), args, smem, s);
}

}  // namespace lpb
