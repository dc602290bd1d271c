// simplex_tableau.cu -- batched dense-tableau simplex, one CTA per LP.
//
// Section 3.1 Steps 1-3 and the two-phase method of Section 3, for every LP
// of a batch (Section 4.1: one thread block per LP).  Design for sm_103a:
//
//  * Tableau: the compact (exchange) form, (m+1) x (n+1) plus one Phase-I row
//    and one column per negated row's slack.  Column j holds non-basic
//    variable nonb[j]; row i holds basic variable basic[i]; the last column is
//    the right-hand side.  The paper's layout (Section 3.1, Fig. 1) keeps the
//    basic columns too; they are identity columns and carry no information, so
//    the compact form does the same pivots on about half the elements.
//  * Storage: shared memory when the tableau fits (SMEM class), else a per-CTA
//    slot of the workspace that stays resident in L2 (GMEM class).  Rows are
//    contiguous with an odd leading dimension so column reads are free of bank
//    conflicts; warps own rows and lanes own columns in the pivot update.
//  * Steps 1 and 2 are (value, key) arg-min reductions: warp shuffles, then one
//    slot per warp in shared memory (replacing the Data/Indices arrays and
//    sequential-addressing tree of Section 4.2).  Ineligible ratios are +inf
//    (the INT_MAX sentinel of Section 4.2).  Ties go to the lowest variable
//    index (Step 1) and the lowest basic-variable index (Step 2).
//  * Step 3 (Section 4.3) is a rank-1 update with the pivot column, pre-scaled
//    by 1/pivot, broadcast from shared memory.
//  * Work: a persistent grid pops LPs from an atomic queue, so LPs with more
//    pivots do not hold up a wave.
//  * FP32 mode with refinement: after an FP32 solve the basis inverse sits in
//    the tableau's slack columns; one step of FP64 iterative refinement of
//    x_B = B^{-1} b and y = B^{-T} c_B with FP64 residuals follows, then an FP64
//    primal/dual feasibility and duality-gap check.  LPs that fail are queued
//    for an FP64 re-solve warm-started from their FP32 basis.
#include "lpb_internal.cuh"

namespace lpb {
namespace {

constexpr int kMaxThreads = 512;

struct Layout {
  size_t tab, colb, rowb, basic, nonb, redv, redk, ins, xb, rr, yv, rho, sb, ns, sp, total;
};

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

__host__ __device__ inline int tab_ld(int n, int k) { return (n + k + 1) | 1; }

__host__ __device__ inline Layout make_layout(int eb, bool gmem, int max_m, int max_n, int kcap,
                                              bool refine) {
  Layout L{};
  const size_t ld = size_t(tab_ld(max_n, kcap));
  const size_t rows = size_t(max_m) + 2;
  size_t o = 0;
  L.tab = o;   o = align16(o + (gmem ? 0 : rows * ld * eb));
  L.colb = o;  o = align16(o + rows * eb);
  L.rowb = o;  o = align16(o + ld * eb);
  L.basic = o; o = align16(o + size_t(max_m) * 4);
  L.nonb = o;  o = align16(o + ld * 4);
  L.redv = o;  o = align16(o + 64 * size_t(eb));
  L.redk = o;  o = align16(o + 64 * 4);
  L.ins = o;   o = align16(o + size_t(max_n) + 2 * size_t(max_m) + 1);
  if (refine) {
    L.xb = o;  o = align16(o + size_t(max_m) * 8);
    L.rr = o;  o = align16(o + size_t(max_m) * 8);
    L.yv = o;  o = align16(o + size_t(max_m) * 8);
    L.rho = o; o = align16(o + size_t(max_m) * 8);
    L.sb = o;  o = align16(o + size_t(max_m) * 4);
    L.ns = o;  o = align16(o + size_t(max_m) * 4);
    L.sp = o;  o = align16(o + size_t(max_m) * 4);
  }
  L.total = o;
  return L;
}

template <typename T> __device__ __forceinline__ T pos_inf();
template <> __device__ __forceinline__ float pos_inf<float>() { return __int_as_float(0x7f800000); }
template <> __device__ __forceinline__ double pos_inf<double>() { return __longlong_as_double(0x7ff0000000000000LL); }

// Per-LP working state shared by the helper routines.
template <typename T>
struct Tab {
  T *t;           // tableau, row-major with leading dimension ld
  T *colb, *rowb;
  int *basic, *nonb;
  T *redv;
  int *redk;
  unsigned char *ins;
  int m, n, k, nc, ld;   // nc = n + k non-RHS columns; column nc is the RHS
  int nm;                // variables >= nm are artificial
  bool gmem;             // the tableau is a workspace slot (L2), not shared memory
};

// Step 3: pivot on (l, e), updating rows 0..rows-1.
template <typename T>
__device__ void pivot(Tab<T> &S, int rows, int l, int e) {
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
  const int ld = S.ld, nc = S.nc;
  const T p = S.t[size_t(l) * ld + e];
  for (int i = tid; i < rows; i += nt) S.colb[i] = S.t[size_t(i) * ld + e] / p;
  for (int j = tid; j <= nc; j += nt) S.rowb[j] = S.t[size_t(l) * ld + j];
  if (tid == 0) {
    const int v = S.basic[l];
    S.basic[l] = S.nonb[e];
    S.nonb[e] = v;
  }
  __syncthreads();
  if (!S.gmem) {           // shared-memory tableau: short latencies, plain loop
    for (int i = wid; i < rows; i += nw) {
      T *row = S.t + size_t(i) * ld;
      if (i == l) {
        for (int j = lane; j <= nc; j += 32) row[j] = (j == e) ? T(1) / p : S.rowb[j] / p;
      } else {
        const T f = S.colb[i];
        for (int j = lane; j <= nc; j += 32) row[j] = (j == e) ? -f : fma(-f, S.rowb[j], row[j]);
      }
    }
    __syncthreads();
    return;
  }
  // Slot tableau in L2: warps own rows, lanes own columns, and each lane loads
  // kU elements of kR rows before it updates them, so a batch costs one round
  // trip instead of one per element.
  constexpr int kR = 2, kU = 4;
  for (int i0 = wid; i0 < rows; i0 += nw * kR) {
    for (int j0 = lane; j0 <= nc; j0 += 32 * kU) {
      T v[kR][kU], rb[kU];
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const int j = j0 + 32 * u;
        rb[u] = j <= nc ? S.rowb[j] : T(0);
#pragma unroll
        for (int q = 0; q < kR; ++q) {
          const int i = i0 + q * nw;
          v[q][u] = (i < rows && j <= nc) ? S.t[size_t(i) * ld + j] : T(0);
        }
      }
#pragma unroll
      for (int q = 0; q < kR; ++q) {
        const int i = i0 + q * nw;
        if (i >= rows) continue;
        T *row = S.t + size_t(i) * ld;
        const T f = S.colb[i];
#pragma unroll
        for (int u = 0; u < kU; ++u) {
          const int j = j0 + 32 * u;
          if (j > nc) continue;
          if (i == l) row[j] = (j == e) ? T(1) / p : rb[u] / p;
          else row[j] = (j == e) ? -f : fma(-f, rb[u], v[q][u]);
        }
      }
    }
  }
  __syncthreads();
}

// Steps 1-3 on objective row `orow` until a halt condition (Section 3.1).
// Phase 1 also ratio-tests rows whose basic variable is artificial; phase 2
// skips them (they are redundant rows left after Phase I).
template <typename T>
__device__ int run_phase(Tab<T> &S, int orow, int rows, int phase, int &iters, int max_iter,
                         T eps_p, T eps_d) {
  const int tid = threadIdx.x, nt = blockDim.x;
  int degenerate_run = 0;
  bool bland = false;
  for (;;) {
    // Step 1: entering column.
    T v = pos_inf<T>();
    int key = INT_MAX;
    const T *orow_p = S.t + size_t(orow) * S.ld;
    for (int j = tid; j < S.nc; j += nt) {
      const int var = S.nonb[j];
      if (var >= S.nm) continue;
      const T r = orow_p[j];
      if (r < -eps_d) keep_better(v, key, bland ? T(0) : r, (var << kIdxBits) | j);
    }
    block_argmin(v, key, S.redv, S.redk);
    if (key == INT_MAX) return LPB_OPTIMAL;
    const int e = key & kIdxMask;
    // Step 2: leaving row by the minimum ratio.
    v = pos_inf<T>();
    key = INT_MAX;
    for (int i = tid; i < S.m; i += nt) {
      const int bv = S.basic[i];
      if (phase == 2 && bv >= S.nm) continue;
      const T a = S.t[size_t(i) * S.ld + e];
      if (a > eps_p) keep_better(v, key, S.t[size_t(i) * S.ld + S.nc] / a, (bv << kIdxBits) | i);
    }
    block_argmin(v, key, S.redv + 32, S.redk + 32);
    if (key == INT_MAX) return phase == 2 ? LPB_UNBOUNDED : LPB_NUMERIC;
    if (iters >= max_iter) return LPB_ITER_LIMIT;
    const int l = key & kIdxMask;
    pivot(S, rows, l, e);
    ++iters;
    if (v <= eps_p) {
      if (++degenerate_run >= S.m + S.n) bland = true;
    } else {
      degenerate_run = 0;
      bland = false;
    }
  }
}

// Largest |t_ij| over enterable columns of row i (ties: lowest column); -1 if
// none exceeds `eps`.
template <typename T>
__device__ int row_argmax_abs(Tab<T> &S, int i, T eps, int set) {
  T v = pos_inf<T>();
  int key = INT_MAX;
  for (int j = threadIdx.x; j < S.nc; j += blockDim.x) {
    if (S.nonb[j] >= S.nm) continue;
    const T a = fabs(S.t[size_t(i) * S.ld + j]);
    if (a > eps) keep_better(v, key, -a, j);
  }
  block_argmin(v, key, S.redv + 32 * set, S.redk + 32 * set);
  return key == INT_MAX ? -1 : key;
}

// Column currently holding non-basic variable `var`; -1 if it is basic.
template <typename T>
__device__ int column_of(Tab<T> &S, int var, int set) {
  int key = INT_MAX;
  T v = pos_inf<T>();
  for (int j = threadIdx.x; j < S.nc; j += blockDim.x)
    if (S.nonb[j] == var) keep_better(v, key, T(0), j);
  block_argmin(v, key, S.redv + 32 * set, S.redk + 32 * set);
  return key == INT_MAX ? -1 : key;
}

// Warp 0 writes the indices i < cnt with pred(i) into out[] in increasing
// order and returns the count (to every thread, after a barrier).
template <typename Pred>
__device__ int compact(int cnt, int *out, int *s_cnt, Pred pred) {
  if ((threadIdx.x >> 5) == 0) {
    const int lane = threadIdx.x & 31;
    int base = 0;
    for (int i0 = 0; i0 < cnt; i0 += 32) {
      const int i = i0 + lane;
      const bool p = i < cnt && pred(i);
      const unsigned mask = __ballot_sync(kFull, p);
      if (p) out[base + __popc(mask & ((1u << lane) - 1u))] = i;
      base += __popc(mask);
    }
    if (lane == 0) *s_cnt = base;
  }
  __syncthreads();
  return *s_cnt;
}

// Build the initial tableau of LP `lp` (slack form, Eq. 4; negated rows with
// an artificial each and the Phase-I row when some b_i < 0).  Returns false
// if the data holds NaN or Inf.
template <typename T>
__device__ bool build_tableau(Tab<T> &S, const BatchDev &B, int lp, int64_t aoff, int64_t boff,
                              int64_t coff) {
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
  const int m = S.m, n = S.n, ld = S.ld, nc = S.nc;
  const int rows = m + (S.k ? 2 : 1);
  for (size_t idx = tid; idx < size_t(rows) * ld; idx += nt) S.t[idx] = T(0);
  for (int j = tid; j < n; j += nt) S.nonb[j] = j;
  if (tid == 0) S.nonb[nc] = -1;
  __syncthreads();
  if (wid == 0) {   // ranks of the negated rows -> their slack columns
    int base = 0;
    for (int i0 = 0; i0 < m; i0 += 32) {
      const int i = i0 + lane;
      const bool neg = i < m && ld_in(B.b, boff + i, B.dtype) < 0.0;
      const unsigned mask = __ballot_sync(kFull, neg);
      if (i < m) {
        S.basic[i] = neg ? (n + m + i) : (n + i);
        if (neg) {
          const int col = n + base + __popc(mask & ((1u << lane) - 1u));
          S.nonb[col] = n + i;
          S.t[size_t(i) * ld + col] = T(-1);
        }
      }
      base += __popc(mask);
    }
  }
  __syncthreads();
  bool bad = false;
  // Rows go to warps, columns to lanes; each lane keeps kU x kU loads in flight
  // before it stores, so a row block costs one memory round trip.
  constexpr int kU = 4;
  for (int i0 = wid; i0 < m; i0 += nw * kU) {
    for (int j0 = lane; j0 < n; j0 += 32 * kU) {
      T v[kU][kU];
#pragma unroll
      for (int u = 0; u < kU; ++u)
#pragma unroll
        for (int w = 0; w < kU; ++w) {
          const int i = i0 + u * nw, j = j0 + 32 * w;
          v[u][w] = (i < m && j < n) ? ld_as<T>(B.A, aoff + int64_t(i) * n + j, B.dtype) : T(0);
        }
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const int i = i0 + u * nw;
        if (i >= m) continue;
        const T s = S.basic[i] >= n + m ? T(-1) : T(1);
        T *row = S.t + size_t(i) * ld;
#pragma unroll
        for (int w = 0; w < kU; ++w) {
          const int j = j0 + 32 * w;
          if (j < n) {
            bad |= !isfinite(v[u][w]);
            row[j] = s * v[u][w];
          }
        }
      }
    }
  }
  for (int i = tid; i < m; i += nt) {
    const T bi = ld_as<T>(B.b, boff + i, B.dtype);
    bad |= !isfinite(bi);
    S.t[size_t(i) * ld + nc] = S.basic[i] >= n + m ? -bi : bi;
  }
  for (int j = tid; j < n; j += nt) {
    const T cj = ld_as<T>(B.c, coff + j, B.dtype);
    bad |= !isfinite(cj);
    S.t[size_t(m) * ld + j] = -cj;
  }
  bad = __syncthreads_or(bad);
  if (S.k) {   // Phase-I row: w = -(sum of artificials) in the non-basic variables
    for (int j = tid; j <= nc; j += nt) {
      T s = T(0);
      for (int i = 0; i < m; ++i)
        if (S.basic[i] >= n + m) s += S.t[size_t(i) * ld + j];
      S.t[size_t(m + 1) * ld + j] = -s;
    }
    __syncthreads();
  }
  return !bad;
}

// Pivot the variables of `warm` (a basis from an earlier pass, packed like b)
// into the basis.  Returns false when a pivot would be (near) singular or the
// resulting basic solution is infeasible; the caller then starts cold.
template <typename T>
__device__ bool warm_start(Tab<T> &S, const int32_t *warm, int &iters, T eps_p) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const int m = S.m, nm = S.nm;
  __shared__ int s_ok;
  for (int v = tid; v < nm + m; v += nt) S.ins[v] = 0;
  if (tid == 0) s_ok = 1;
  __syncthreads();
  for (int i = tid; i < m; i += nt) {
    const int v = warm[i];
    if (v < 0 || v >= nm) s_ok = 0;
    else S.ins[v] = 1;
  }
  __syncthreads();
  if (!s_ok) return false;
  const int rows = m + (S.k ? 2 : 1);
  for (int t = 0; t < m; ++t) {
    __syncthreads();                              // reduction slots are free again
    const int v = warm[t];
    const int e = column_of(S, v, 0);
    if (e < 0) continue;                          // already basic
    // Row with the largest |t_ie| among rows whose basic variable leaves.
    T bvv = pos_inf<T>();
    int key = INT_MAX;
    for (int i = tid; i < m; i += nt) {
      const int bv = S.basic[i];
      if (bv < nm && S.ins[bv]) continue;
      const T a = fabs(S.t[size_t(i) * S.ld + e]);
      if (a > T(1e-9)) keep_better(bvv, key, -a, i);
    }
    block_argmin(bvv, key, S.redv + 32, S.redk + 32);
    if (key == INT_MAX) return false;
    pivot(S, rows, key, e);
    ++iters;
  }
  int bad = 0;
  for (int i = tid; i < m; i += nt) bad |= S.basic[i] >= nm;
  return !__syncthreads_or(bad);
}

// Dual simplex pivots from a basis that is (nearly) dual feasible but has
// negative basic values: the most negative basic value leaves, the entering
// column minimises r_j / -t_lj over t_lj < -eps_p.  Returns true once every
// basic value is >= -eps_p; false if a row has no entering column or the cap
// is reached (the caller then starts cold).
template <typename T>
__device__ bool dual_cleanup(Tab<T> &S, int rows, int &iters, int max_iter, T eps_p) {
  const int tid = threadIdx.x, nt = blockDim.x;
  for (;;) {
    __syncthreads();
    T v = pos_inf<T>();
    int key = INT_MAX;
    for (int i = tid; i < S.m; i += nt) {
      const int bv = S.basic[i];
      if (bv >= S.nm) continue;
      const T rhs = S.t[size_t(i) * S.ld + S.nc];
      if (rhs < -eps_p) keep_better(v, key, rhs, (bv << kIdxBits) | i);
    }
    block_argmin(v, key, S.redv, S.redk);
    if (key == INT_MAX) return true;
    const int l = key & kIdxMask;
    v = pos_inf<T>();
    key = INT_MAX;
    for (int j = tid; j < S.nc; j += nt) {
      const int var = S.nonb[j];
      if (var >= S.nm) continue;
      const T a = S.t[size_t(l) * S.ld + j];
      if (a < -eps_p) keep_better(v, key, S.t[size_t(S.m) * S.ld + j] / -a, (var << kIdxBits) | j);
    }
    block_argmin(v, key, S.redv + 32, S.redk + 32);
    if (key == INT_MAX || iters >= max_iter) return false;
    pivot(S, rows, l, key & kIdxMask);
    ++iters;
  }
}

// Write the FP64 outputs of LP `lp` from the tableau (FP64 and plain FP32 modes).
__device__ __forceinline__ int32_t *basis_at(const TableauParams &P, int lp, int64_t boff) {
  return P.bbuf ? P.bbuf + (P.bpacked ? boff : int64_t(lp) * P.B.max_m) : nullptr;
}

template <typename T>
__device__ void write_from_tableau(Tab<T> &S, const ResultDev &R, int32_t *basis, int lp,
                                   int64_t boff, int64_t coff, int status, int iters) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const int m = S.m, n = S.n;
  for (int j = tid; j < n; j += nt) R.x[coff + j] = 0.0;
  if (R.y) for (int i = tid; i < m; i += nt) R.y[boff + i] = 0.0;
  __syncthreads();
  if (status == LPB_OPTIMAL) {
    for (int i = tid; i < m; i += nt) {
      const int v = S.basic[i];
      if (v < n) R.x[coff + v] = double(S.t[size_t(i) * S.ld + S.nc]);
    }
    if (R.y)
      for (int j = tid; j < S.nc; j += nt) {
        const int v = S.nonb[j];
        if (v >= n && v < n + m) R.y[boff + (v - n)] = double(S.t[size_t(m) * S.ld + j]);
      }
  }
  if (basis)
    for (int i = tid; i < m; i += nt) basis[i] = S.basic[i] < S.nm ? S.basic[i] : -1;
  if (tid == 0) {
    R.status[lp] = status;
    if (R.iters) R.iters[lp] = iters;
    R.obj[lp] = status == LPB_OPTIMAL ? double(S.t[size_t(m) * S.ld + S.nc])
              : status == LPB_INFEASIBLE ? -INFINITY
              : status == LPB_UNBOUNDED ? INFINITY : NAN;
  }
}

// FP64 refinement and verification of an FP32-optimal basis.  Returns true and
// writes the outputs when the refined pair (x, y) passes the checks.
__device__ bool refine_and_verify(Tab<float> &S, const BatchDev &B, const ResultDev &R,
                                  int32_t *basis, const Layout &L, unsigned char *smem, int lp,
                                  int64_t aoff,
                                  int64_t boff, int64_t coff, int iters, double tol, double bmax,
                                  double cmax) {
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, wid = tid >> 5;
  const int m = S.m, n = S.n, ld = S.ld, nc = S.nc;
  double *xb = reinterpret_cast<double *>(smem + L.xb);
  double *rr = reinterpret_cast<double *>(smem + L.rr);
  double *yv = reinterpret_cast<double *>(smem + L.yv);
  double *rho = reinterpret_cast<double *>(smem + L.rho);
  int *sb = reinterpret_cast<int *>(smem + L.sb);   // rows whose basic variable is structural
  int *ns = reinterpret_cast<int *>(smem + L.ns);   // columns holding a non-basic slack
  int *sp = reinterpret_cast<int *>(smem + L.sp);   // row of basic slack k, or -1
  __shared__ int s_cnt0, s_cnt1;
  __shared__ double s_red[2][32];
  const int dt = B.dtype;

  const int nsb = compact(m, sb, &s_cnt0, [&](int i) { return S.basic[i] < n; });
  const int nns = compact(nc, ns, &s_cnt1, [&](int j) { const int v = S.nonb[j]; return v >= n && v < n + m; });
  for (int k = tid; k < m; k += nt) { sp[k] = -1; yv[k] = 0.0; }
  __syncthreads();
  for (int i = tid; i < m; i += nt) {
    const int v = S.basic[i];
    xb[i] = double(S.t[size_t(i) * ld + nc]);
    if (v >= n && v < n + m) sp[v - n] = i;
  }
  for (int q = tid; q < nns; q += nt) yv[S.nonb[ns[q]] - n] = double(S.t[size_t(m) * ld + ns[q]]);
  __syncthreads();
  // Primal residual r = b - [A I]_B x_B in FP64.
  for (int i = tid; i < m; i += nt) {
    double r = ld_in(B.b, boff + i, dt);
    const int64_t ar = aoff + int64_t(i) * n;
#pragma unroll 4
    for (int q = 0; q < nsb; ++q) {
      const int t = sb[q];
      r = fma(-ld_in(B.A, ar + S.basic[t], dt), xb[t], r);
    }
    if (sp[i] >= 0) r -= xb[sp[i]];
    rr[i] = r;
  }
  // Dual residual rho_t = c_B(t) - (B^T y)_t for structural basic rows (slack rows: 0).
  for (int q = tid; q < nsb; q += nt) {
    const int t = sb[q], j = S.basic[t];
    double r = ld_in(B.c, coff + j, dt);
#pragma unroll 4
    for (int p = 0; p < nns; ++p) {
      const int kk = S.nonb[ns[p]] - n;
      r = fma(-ld_in(B.A, aoff + int64_t(kk) * n + j, dt), yv[kk], r);
    }
    rho[t] = r;
  }
  __syncthreads();
  // Corrections with the FP32 basis inverse: its column for slack k is the
  // tableau column of k when k is non-basic, else the unit vector of k's row.
  for (int t = tid; t < m; t += nt) {
    float d = 0.f;
    const float *row = S.t + size_t(t) * ld;
    for (int p = 0; p < nns; ++p) {
      const int col = ns[p];
      d = fmaf(float(rr[S.nonb[col] - n]), row[col], d);
    }
    const int v = S.basic[t];
    double dx = double(d);
    if (v >= n && v < n + m) dx += rr[v - n];
    xb[t] += dx;
  }
  for (int p = tid; p < nns; p += nt) {
    const int col = ns[p];
    float d = 0.f;
    for (int q = 0; q < nsb; ++q) {
      const int t = sb[q];
      d = fmaf(float(rho[t]), S.t[size_t(t) * ld + col], d);
    }
    yv[S.nonb[col] - n] += double(d);
  }
  __syncthreads();
  // FP64 KKT certificate of the pair that is written out (x: the structural
  // part of x_B; y: the slack duals): x >= 0, A x <= b, y >= 0, A^T y >= c and
  // c^T x = b^T y, each to tol scaled by the data.
  double cx = 0.0, by = 0.0;
  int bad = 0;
  const double tp = tol * (1.0 + bmax), td = tol * (1.0 + cmax);
  for (int q = tid; q < nsb; q += nt) {
    bad |= !(xb[sb[q]] >= -tp);
    cx = fma(ld_in(B.c, coff + S.basic[sb[q]], dt), xb[sb[q]], cx);
  }
  for (int p = tid; p < nns; p += nt) {
    const int kk = S.nonb[ns[p]] - n;
    by = fma(ld_in(B.b, boff + kk, dt), yv[kk], by);
    bad |= !(yv[kk] >= -td);
  }
  for (int i = tid; i < m; i += nt) {     // slack b_i - A_i x of every row
    double s = ld_in(B.b, boff + i, dt);
    const int64_t ar = aoff + int64_t(i) * n;
#pragma unroll 4
    for (int q = 0; q < nsb; ++q) s = fma(-ld_in(B.A, ar + S.basic[sb[q]], dt), xb[sb[q]], s);
    bad |= !(s >= -tp);
  }
  for (int j = tid; j < n; j += nt) {     // reduced cost A_j^T y - c_j of every column
    double d = -ld_in(B.c, coff + j, dt);
#pragma unroll 4
    for (int p = 0; p < nns; ++p) {
      const int kk = S.nonb[ns[p]] - n;
      d = fma(ld_in(B.A, aoff + int64_t(kk) * n + j, dt), yv[kk], d);
    }
    bad |= !(d >= -td);
  }
  cx = warp_sum(cx);
  by = warp_sum(by);
  if (lane == 0) { s_red[0][wid] = cx; s_red[1][wid] = by; }
  bad = __syncthreads_or(bad);
  cx = 0.0; by = 0.0;
  for (int w = 0; w < (nt >> 5); ++w) { cx += s_red[0][w]; by += s_red[1][w]; }
  bad |= !(fabs(cx - by) <= tol * (1.0 + fabs(cx)));
  if (bad) return false;
  for (int j = tid; j < n; j += nt) R.x[coff + j] = 0.0;
  __syncthreads();
  for (int q = tid; q < nsb; q += nt) R.x[coff + S.basic[sb[q]]] = xb[sb[q]];
  if (R.y) for (int k = tid; k < m; k += nt) R.y[boff + k] = yv[k];
  if (basis) for (int i = tid; i < m; i += nt) basis[i] = S.basic[i];
  if (tid == 0) {
    R.status[lp] = LPB_OPTIMAL;
    if (R.iters) R.iters[lp] = iters;
    R.obj[lp] = cx;
  }
  return true;
}

template <typename T, bool kGmem>
__global__ void __launch_bounds__(kMaxThreads) tableau_kernel(TableauParams P) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int tid = threadIdx.x, nt = blockDim.x;
  const bool refine = (P.mode == MODE_FP32_REFINE) && sizeof(T) == 4;
  const Layout L = make_layout(int(sizeof(T)), kGmem, P.B.max_m, P.B.max_n, P.kcap, refine);
  Tab<T> S;
  S.t = kGmem ? reinterpret_cast<T *>(static_cast<unsigned char *>(P.slots) + size_t(blockIdx.x) * P.slot_bytes)
              : reinterpret_cast<T *>(smem + L.tab);
  S.colb = reinterpret_cast<T *>(smem + L.colb);
  S.rowb = reinterpret_cast<T *>(smem + L.rowb);
  S.basic = reinterpret_cast<int *>(smem + L.basic);
  S.nonb = reinterpret_cast<int *>(smem + L.nonb);
  S.redv = reinterpret_cast<T *>(smem + L.redv);
  S.redk = reinterpret_cast<int *>(smem + L.redk);
  S.ins = smem + L.ins;
  S.gmem = kGmem;
  __shared__ int s_item, s_k;
  __shared__ unsigned long long s_bmax, s_cmax;
  const T eps_p = T(P.eps_p), eps_d = T(P.eps_d);
  const int nitems = P.in.count ? min(*P.in.count, P.list_cap) : P.B.count;

  for (;;) {
    if (tid == 0) s_item = atomicAdd(P.queue, 1);
    __syncthreads();
    const int item = s_item;
    if (item >= nitems) break;
    const int lp = P.in.items ? P.in.items[item] : item;
    const int m = P.B.m[lp], n = P.B.n[lp];
    if (m < 1 || n < 1 || m > P.B.max_m || n > P.B.max_n) {
      if (tid == 0) {
        P.R.status[lp] = LPB_BAD_SIZE;
        if (P.R.iters) P.R.iters[lp] = 0;
        P.R.obj[lp] = NAN;
      }
      __syncthreads();
      continue;
    }
    const int64_t aoff = P.B.a_off[lp], boff = P.B.b_off[lp], coff = P.B.c_off[lp];
    // Negated rows, |b|max and |c|max.
    if (tid == 0) { s_k = 0; s_bmax = 0ull; s_cmax = 0ull; }
    __syncthreads();
    int kneg = 0;
    double bm = 0.0, cm = 0.0;
    for (int i = tid; i < m; i += nt) {
      const double v = ld_in(P.B.b, boff + i, P.B.dtype);
      kneg += v < 0.0;
      bm = fmax(bm, fabs(v));
    }
    for (int j = tid; j < n; j += nt) cm = fmax(cm, fabs(ld_in(P.B.c, coff + j, P.B.dtype)));
    kneg = warp_sum(kneg);
    if ((tid & 31) == 0) atomicAdd(&s_k, kneg);
    if (bm == bm) atomicMax(&s_bmax, static_cast<unsigned long long>(__double_as_longlong(bm)));
    if (cm == cm) atomicMax(&s_cmax, static_cast<unsigned long long>(__double_as_longlong(cm)));
    __syncthreads();
    S.m = m; S.n = n; S.k = s_k; S.nc = n + S.k; S.ld = tab_ld(n, S.k); S.nm = n + m;
    const double bmax = __longlong_as_double(static_cast<long long>(s_bmax));
    const double cmax = __longlong_as_double(static_cast<long long>(s_cmax));
    if (S.k > P.kcap) {        // needs more artificial columns than this launch holds
      if (tid == 0) {
        P.R.status[lp] = STATUS_PENDING;
        list_push(P.defer_items, P.defer_count, P.list_cap, lp, P.err);
      }
      __syncthreads();
      continue;
    }
    const int max_iter = P.max_iter > 0 ? P.max_iter : 50 * (m + n);
    int iters = 0, status;
    bool ok = build_tableau(S, P.B, lp, aoff, boff, coff);
    if (!ok) {
      status = LPB_NUMERIC;
    } else {
      bool warm = false;
      if (P.warm && basis_at(P, lp, boff)) {
        warm = warm_start(S, basis_at(P, lp, boff), iters, eps_p) &&
               dual_cleanup(S, m + (S.k ? 2 : 1), iters, max_iter, eps_p);
        if (!warm) {         // cold restart
          iters = 0;
          build_tableau(S, P.B, lp, aoff, boff, coff);
        }
      }
      status = LPB_OPTIMAL;
      if (S.k && !warm) {    // Phase I
        // An FP32 tableau carries the Phase-I objective's round-off relative to
        // its starting value (minus the sum of the negated right-hand sides), so
        // its infeasibility test is relative to that; the FP64 certificate and
        // re-solve settle the LPs it lets through.
        const double w0 = -double(S.t[size_t(m + 1) * S.ld + S.nc]);
        const double ftol = sizeof(T) == 4 ? fmax(P.feas_tol * (1.0 + bmax), 1e-5 * (1.0 + w0))
                                           : P.feas_tol * (1.0 + bmax);
        status = run_phase(S, m + 1, m + 2, 1, iters, max_iter, eps_p, eps_d);
        if (status == LPB_OPTIMAL) {
          const double w = double(S.t[size_t(m + 1) * S.ld + S.nc]);
          if (-w > ftol) {
            status = LPB_INFEASIBLE;
          } else {             // drive zero-level artificials out of the basis
            for (int i = 0; i < m; ++i) {
              if (S.basic[i] < S.nm) continue;
              const int e = row_argmax_abs(S, i, eps_p, 0);
              if (e >= 0) { pivot(S, m + 2, i, e); ++iters; }
              __syncthreads();
            }
          }
        }
      }
      if (status == LPB_OPTIMAL) status = run_phase(S, m, m + 1, 2, iters, max_iter, eps_p, eps_d);
    }
    if constexpr (sizeof(T) == 4) if (P.mode == MODE_FP32_REFINE) {
      bool done = false;
      if (status == LPB_OPTIMAL) {
        int dropped = 0;
        for (int i = tid; i < m; i += nt) dropped |= S.basic[i] >= S.nm;
        if (!__syncthreads_or(dropped))
          done = refine_and_verify(S, P.B, P.R, basis_at(P, lp, boff), L, smem, lp, aoff, boff,
                                   coff, iters, P.feas_tol, bmax, cmax);
      }
      if (!done) {
        if (int32_t *bp = basis_at(P, lp, boff))
          for (int i = tid; i < m; i += nt) bp[i] = S.basic[i] < S.nm ? S.basic[i] : -1;
        if (tid == 0) {
          P.R.status[lp] = STATUS_PENDING;
          if (P.R.iters) P.R.iters[lp] = iters;
          list_push(P.resolve_items, P.resolve_count, P.list_cap, lp, P.err);
        }
      }
      __syncthreads();
      continue;
    }
    write_from_tableau(S, P.R, basis_at(P, lp, boff), lp, boff, coff, status, iters);
    __syncthreads();
  }
}

}  // namespace

size_t tableau_smem_bytes(int eb, bool gmem, int max_m, int max_n, int kcap, int threads, bool refine) {
  (void)threads;
  return make_layout(eb, gmem, max_m, max_n, kcap, refine).total;
}

size_t tableau_slot_bytes(int eb, int max_m, int max_n, int kcap) {
  return align16(size_t(max_m + 2) * size_t(tab_ld(max_n, kcap)) * size_t(eb));
}

template <typename T, bool G>
static cudaError_t prep(size_t smem) {
  return cudaFuncSetAttribute(tableau_kernel<T, G>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              int(smem));
}

cudaError_t tableau_max_ctas_per_sm(int eb, bool gmem, int threads, size_t smem, int *ctas) {
  cudaError_t e;
  if (eb == 8) {
    e = gmem ? prep<double, true>(smem) : prep<double, false>(smem);
    if (e != cudaSuccess) return e;
    return gmem ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas, tableau_kernel<double, true>, threads, smem)
                : cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas, tableau_kernel<double, false>, threads, smem);
  }
  e = gmem ? prep<float, true>(smem) : prep<float, false>(smem);
  if (e != cudaSuccess) return e;
  return gmem ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas, tableau_kernel<float, true>, threads, smem)
              : cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas, tableau_kernel<float, false>, threads, smem);
}

cudaError_t launch_tableau(const TableauParams &p, bool fp64, bool gmem, int grid, int threads,
                           size_t smem, cudaStream_t s) {
  if (threads < 32 || threads > kMaxThreads || (threads & 31) || grid < 1) return cudaErrorInvalidValue;
  cudaError_t e;
  if (fp64) {
    e = gmem ? prep<double, true>(smem) : prep<double, false>(smem);
    if (e != cudaSuccess) return e;
    if (gmem) tableau_kernel<double, true><<<grid, threads, smem, s>>>(p);
    else tableau_kernel<double, false><<<grid, threads, smem, s>>>(p);
  } else {
    e = gmem ? prep<float, true>(smem) : prep<float, false>(smem);
    if (e != cudaSuccess) return e;
    if (gmem) tableau_kernel<float, true><<<grid, threads, smem, s>>>(p);
    else tableau_kernel<float, false><<<grid, threads, smem, s>>>(p);
  }
  return cudaGetLastError();
}

}  // namespace lpb
