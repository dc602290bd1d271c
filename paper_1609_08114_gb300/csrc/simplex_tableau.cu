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
//  * Storage: the leading rows live in shared memory, as many as fit; the rest
//    (none for most LPs) in a per-CTA workspace slot that stays in L2.  Rows
//    have an odd leading dimension, so the column reads of Step 2 are free of
//    bank conflicts.
//  * Work split: warp w owns a contiguous block of rows; lanes own columns.
//    One pivot takes two block barriers.  Before the first, every warp runs
//    Step 2 on its own rows (a warp arg-min, one slot per warp) and the
//    reciprocal of its best pivot.  After it, every warp reduces the slots,
//    keeps the pivot row in registers and applies the rank-1 update of Step 3
//    to its rows; the warp owning the pivot row writes the scaled row to a
//    buffer, and the warp owning the objective row runs Step 1 for the next
//    pivot on its freshly updated row.  After the second barrier the owner
//    copies the scaled pivot row into place.  The Data/Indices arrays and the
//    sequential-addressing reduction of Section 4.2 become warp shuffles;
//    ineligible ratios are +inf (the INT_MAX sentinel of Section 4.2).  Ties
//    go to the lowest variable index (Step 1) and the lowest basic-variable
//    index (Step 2).
//  * Work: a persistent grid pops LPs from an atomic queue, so LPs with more
//    pivots do not hold up a wave.
//  * FP32 mode with refinement: after an FP32 solve the basis inverse sits in
//    the tableau's slack columns; one step of FP64 iterative refinement of
//    x_B = B^{-1} b and y = B^{-T} c_B with FP64 residuals follows, then an FP64
//    primal/dual feasibility and duality-gap check.  LPs that fail are queued
//    for an FP64 re-solve warm-started from their FP32 basis.
#include <type_traits>

#include "lpb_internal.cuh"

namespace lpb {
namespace {

constexpr int kMaxThreads = 1024;

struct Layout {
  size_t tab, colb, rowb, gam, basic, nonb, redv, redk, rcp, redf, sel, ins, wl, xb, rr, yv, rho, sb, ns, sp, dj, jq, kq, total;
};

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

// Row length in elements: whole 16-byte vectors, so that the update moves
// rows with vector accesses.  The padding columns stay zero under pivoting.
__host__ __device__ inline int tab_ld(int n, int k, int eb) {
  const int per = 16 / eb;
  return (n + k + 1 + per - 1) / per * per;
}

// Dynamic shared memory: `tab` bytes of tableau rows, then the buffers.
__host__ __device__ inline Layout make_layout(int eb, size_t tab, int max_m, int max_n, int kcap, bool refine) {
  Layout L{};
  const size_t ld = size_t(tab_ld(max_n, kcap, eb));
  const size_t rows = size_t(max_m) + 2;
  size_t o = 0;
  L.tab = o;   o = align16(o + tab);
  L.colb = o;  o = align16(o + rows * eb);
  L.rowb = o;  o = align16(o + ld * eb);
  L.gam = o;   o = align16(o + ld * eb);
  L.basic = o; o = align16(o + size_t(max_m) * 4);
  L.nonb = o;  o = align16(o + ld * 4);
  L.redv = o;  o = align16(o + 64 * size_t(eb));
  L.redk = o;  o = align16(o + 64 * 4);
  L.rcp = o;   o = align16(o + 33 * size_t(eb));
  L.redf = o;  o = align16(o + 32 * 4);
  L.sel = o;   o = align16(o + 4 * 4);
  L.ins = o;   o = align16(o + size_t(max_n) + 2 * size_t(max_m) + 1);
  L.wl = o;    o = align16(o + size_t(max_m) * 4 + 4);
  if (refine) {
    L.xb = o;  o = align16(o + size_t(max_m) * 8);
    L.rr = o;  o = align16(o + size_t(max_m) * 8);
    L.yv = o;  o = align16(o + size_t(max_m) * 8);
    L.rho = o; o = align16(o + size_t(max_m) * 8);
    L.sb = o;  o = align16(o + size_t(max_m) * 4);
    L.ns = o;  o = align16(o + size_t(max_m) * 4);
    L.sp = o;  o = align16(o + size_t(max_m) * 4);
    L.dj = o;  o = align16(o + size_t(max_n) * 8);
    L.jq = o;  o = align16(o + size_t(max_m) * 4);
    L.kq = o;  o = align16(o + size_t(max_m) * 4);
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
  T *ts;          // rows 0..rs-1 in shared memory (leading dimension ld)
  T *tg;          // rows rs.. in the CTA's workspace slot
  int rs;
  T *colb, *rowb;
  T *gam;         // steepest edge: gamma_j of every column
  int *basic, *nonb;
  T *redv;
  int *redk;
  T *rcp;         // per-warp reciprocal of the warp's best pivot (Step 2)
  float *redf;    // per-warp smallest FP32 ratio (FP64 Step 2)
  int *sel;       // Step 1 result for the next pivot: sel[0] = key or INT_MAX
  unsigned char *ins;
  int *wl;        // warm start: columns whose variable enters
  int m, n, k, nc, ld;   // nc = n + k non-RHS columns; column nc is the RHS
  int nm;                // variables >= nm are artificial
  __device__ __forceinline__ T *row(int i) const {
    return i < rs ? ts + size_t(i) * ld : tg + size_t(i - rs) * ld;
  }
  __device__ __forceinline__ T &at(int i, int j) const { return row(i)[j]; }
};

// Rows [r0, r1) owned by the calling warp when `rows` rows are split into
// contiguous blocks, one per warp.
__device__ __forceinline__ void own_rows(int rows, int &r0, int &r1) {
  const int nw = blockDim.x >> 5, w = threadIdx.x >> 5;
  const int per = (rows + nw - 1) / nw;
  r0 = w * per;
  r1 = min(rows, r0 + per);
}

// 16-byte vectors of the tableau's element type.
template <typename T> struct Vec;
template <> struct Vec<float> {
  using type = float4;
  static constexpr int N = 4;
};
template <> struct Vec<double> {
  using type = double2;
  static constexpr int N = 2;
};
// One vector of a row under Step 3: x - f pr; and the scaled pivot row
// pr * rp.  (The pivot column itself is set afterwards, once per row, so the
// update of every other element carries no test for it.)  Vectors pass by
// value (taking a vector's address would move it to local memory).
__device__ __forceinline__ float4 upd_vec(float4 x, float4 pr, float nf) {
  x.x = fmaf(nf, pr.x, x.x);
  x.y = fmaf(nf, pr.y, x.y);
  x.z = fmaf(nf, pr.z, x.z);
  x.w = fmaf(nf, pr.w, x.w);
  return x;
}
__device__ __forceinline__ double2 upd_vec(double2 x, double2 pr, double nf) {
  x.x = fma(nf, pr.x, x.x);
  x.y = fma(nf, pr.y, x.y);
  return x;
}
__device__ __forceinline__ float4 scale_vec(float4 pr, float rp) {
  return make_float4(pr.x * rp, pr.y * rp, pr.z * rp, pr.w * rp);
}
__device__ __forceinline__ double2 scale_vec(double2 pr, double rp) {
  return make_double2(pr.x * rp, pr.y * rp);
}
// acc + x * x, elementwise (steepest-edge weights), and the elements of a vector.
__device__ __forceinline__ float4 sq_acc(float4 acc, float4 x) {
  return make_float4(fmaf(x.x, x.x, acc.x), fmaf(x.y, x.y, acc.y), fmaf(x.z, x.z, acc.z), fmaf(x.w, x.w, acc.w));
}
__device__ __forceinline__ double2 sq_acc(double2 acc, double2 x) {
  return make_double2(fma(x.x, x.x, acc.x), fma(x.y, x.y, acc.y));
}
__device__ __forceinline__ float vec_el(float4 v, int c) { return c == 0 ? v.x : c == 1 ? v.y : c == 2 ? v.z : v.w; }
__device__ __forceinline__ double vec_el(double2 v, int c) { return c == 0 ? v.x : v.y; }
template <typename V> __device__ __forceinline__ V vec_zero();
template <> __device__ __forceinline__ float4 vec_zero<float4>() { return make_float4(0.f, 0.f, 0.f, 0.f); }
template <> __device__ __forceinline__ double2 vec_zero<double2>() { return make_double2(0.0, 0.0); }

// Step 3 on the calling warp's rows: with rp = 1 / t_le, every row i != l
// becomes row_i - (t_ie rp) row_l and its column e -t_ie rp; the warp owning
// row l writes the scaled row (rp at column e) to S.rowb instead of row l, so
// that other warps can still read the old row; pivot_finish() copies it.
// Lanes own 16-byte vectors of columns, kJ per lane per chunk of 32 kJ
// vectors: a lane keeps its vectors of the pivot row in registers while the
// warp's rows stream past, so each row's multiplier and address are read once
// per chunk and the kJ loads of a row are in flight together.  Column e is
// written by a scalar pass after the vector sweep.  SE: the sweep also adds
// the squares of the values it writes in the constraint rows in use (phase 2
// skips rows whose basic variable is artificial) to gamma_j in S.gam (zero on
// entry), with the scaled pivot row's; column e's gamma is left to the caller.
template <typename T, int kJ, bool SE>
__device__ __forceinline__ void pivot_update(const Tab<T> &S_, int rows, int l, int e, T rp, int phase) {
  const Tab<T> S = S_;   // a register copy: stores through tableau pointers cannot alias it
  using V = typename Vec<T>::type;
  constexpr int NV = Vec<T>::N;
  const int lane = threadIdx.x & 31;
  int r0, r1;
  own_rows(rows, r0, r1);
  for (int i = r0 + lane; i < r1; i += 32) S.colb[i] = i == l ? T(0) : S.at(i, e) * rp;
  __syncwarp();
  if (r0 >= r1) return;
  const bool own_l = l >= r0 && l < r1;
  const int nv = (S.nc + NV) / NV;        // vectors holding columns 0..nc
  const V *prow = reinterpret_cast<const V *>(S.row(l));
  V *rowb = reinterpret_cast<V *>(S.rowb);
  for (int j0 = lane; j0 < nv; j0 += 32 * kJ) {
    // Vectors past the row's end stand in as j0 (loaded, never stored).
    int jj[kJ];
    V pr[kJ], acc[kJ];
#pragma unroll
    for (int k = 0; k < kJ; ++k) {
      jj[k] = j0 + 32 * k < nv ? j0 + 32 * k : j0;
      pr[k] = prow[jj[k]];
      acc[k] = vec_zero<V>();
      if (own_l && j0 + 32 * k < nv) {
        const V sr = scale_vec(pr[k], rp);
        rowb[jj[k]] = sr;
        if (SE) acc[k] = sq_acc(acc[k], sr);      // row l is in use after the pivot
      }
    }
    for (int i = r0; i < r1; ++i) {
      if (i == l) continue;
      const T nf = -S.colb[i];
      V *rw = reinterpret_cast<V *>(S.row(i));
      V v[kJ];
#pragma unroll
      for (int k = 0; k < kJ; ++k) v[k] = rw[jj[k]];
      const bool use = SE && i < S.m && !(phase == 2 && S.basic[i] >= S.nm);
#pragma unroll
      for (int k = 0; k < kJ; ++k)
        if (j0 + 32 * k < nv) {
          const V u = upd_vec(v[k], pr[k], nf);
          rw[jj[k]] = u;
          if (use) acc[k] = sq_acc(acc[k], u);
        }
    }
    if (SE) {
#pragma unroll
      for (int k = 0; k < kJ; ++k)
        if (j0 + 32 * k < nv)
#pragma unroll
          for (int c = 0; c < NV; ++c) {
            const int col = (j0 + 32 * k) * NV + c;
            if (col < S.nc) atomicAdd(S.gam + col, vec_el(acc[k], c));
          }
    }
  }
  __syncwarp();                           // the vector stores of this warp's rows are done
  for (int i = r0 + lane; i < r1; i += 32)
    if (i != l) S.at(i, e) = -S.colb[i];
  if (own_l && lane == 0) S.rowb[e] = rp;
}

// After the barrier that follows pivot_update: the owner of row l copies the
// scaled pivot row into place.
template <typename T>
__device__ __forceinline__ void pivot_finish(const Tab<T> &S_, int rows, int l) {
  const Tab<T> S = S_;   // a register copy: stores through tableau pointers cannot alias it
  using V = typename Vec<T>::type;
  constexpr int NV = Vec<T>::N;
  int r0, r1;
  own_rows(rows, r0, r1);
  if (l >= r0 && l < r1) {
    V *prow = reinterpret_cast<V *>(S.row(l));       // whole vectors: the padding is scaled zero
    const V *rb = reinterpret_cast<const V *>(S.rowb);
    const int nv = (S.nc + NV) / NV;
    for (int j = threadIdx.x & 31; j < nv; j += 32) prow[j] = rb[j];
  }
  __syncwarp();
}

template <typename T, bool SE = false>
__device__ __forceinline__ void update_any(const Tab<T> &S_, int rows, int l, int e, T rp, int phase = 2) {
  const Tab<T> S = S_;   // a register copy: stores through tableau pointers cannot alias it
  // Fewer vectors per lane under steepest edge: its accumulators take the registers.
  pivot_update<T, SE ? (sizeof(T) == 4 ? 2 : 1) : (sizeof(T) == 4 ? 3 : 2), SE>(S, rows, l, e, rp, phase);
}

// A whole pivot on (l, e) for the callers outside the Step 1-3 loop (Phase-I
// clean-up, warm start, dual simplex): the tableau must be stable on entry.
template <typename T>
__device__ __forceinline__ void pivot(const Tab<T> &S_, int rows, int l, int e) {
  const Tab<T> S = S_;   // a register copy: stores through tableau pointers cannot alias it
  if (threadIdx.x == 0) {     // one division (FP64 divisions are slow here), published
    S.rcp[32] = T(1) / S.at(l, e);
    const int v = S.basic[l];
    S.basic[l] = S.nonb[e];
    S.nonb[e] = v;
  }
  __syncthreads();
  const T rp = S.rcp[32];
  update_any(S, rows, l, e, rp);
  __syncthreads();
  pivot_finish(S, rows, l);
  __syncthreads();
}

// Steepest-edge weights gamma_j = 1 + sum_i t_ij^2, summed over the
// constraint rows in row order with one fused multiply-add each (phase 2
// skips rows whose basic variable is artificial: redundant rows left after
// Phase I), into S.gam: of every non-artificial column (`all`: the FP32
// kernel, once when a phase starts, after which its pivots keep them), or of
// the columns eligible on objective row `orow` (the FP64 kernel, before every
// pivot: its weights follow the oracle's summation order exactly).  Every
// thread takes columns; the caller places a barrier before (rows final) and
// after.
template <typename T>
__device__ __forceinline__ void se_weights(const Tab<T> &S_, int orow, int phase, T eps_d, bool all) {
  const Tab<T> S = S_;   // a register copy: stores through tableau pointers cannot alias it
  const T *r = S.row(orow);
  for (int j = threadIdx.x; j < S.nc; j += blockDim.x) {
    if (S.nonb[j] >= S.nm || !(all || r[j] < -eps_d)) continue;
    T g = T(1);
    for (int i = 0; i < S.m; ++i) {
      if (phase == 2 && S.basic[i] >= S.nm) continue;
      const T t = S.at(i, j);
      g = fma(t, t, g);
    }
    S.gam[j] = g;
  }
}

// Step 1 over objective row `orow` in one warp (every lane gets the result):
// eligible columns are those with a reduced cost below -eps_d; the most
// negative one enters (LPC), or the one with the smallest random key at pivot
// `it` (RPC), or the one with the largest r_j^2 / gamma_j (steepest edge, the
// weights in S.gam), or the lowest variable index under Bland's rule.  Column
// `ecol` is taken to hold variable `evar` (a pivot whose swap of nonb may not
// be visible yet).  Keys are (variable << kIdxBits) | column.
template <typename T>
__device__ __forceinline__ void step1_warp(const Tab<T> &S_, int orow, bool bland, T eps_d, int ecol, int evar,
                                           T &v, int &key, int rule, unsigned long long seed, long long lp,
                                           int it) {
  const Tab<T> S = S_;   // a register copy: stores through tableau pointers cannot alias it
  const T *r = S.row(orow);
  v = pos_inf<T>();
  key = INT_MAX;
  if (rule == LPB_PIVOT_RPC && !bland) {
    unsigned best = 0xffffffffu;
    for (int j = threadIdx.x & 31; j < S.nc; j += 32) {
      const int var = j == ecol ? evar : S.nonb[j];
      if (var >= S.nm || !(r[j] < -eps_d)) continue;
      const unsigned k = rpc_key(seed, lp, it, var);
      const int kk = (var << kIdxBits) | j;
      if (k < best || (k == best && kk < key)) { best = k; key = kk; }
    }
    const unsigned mk = __reduce_min_sync(kFull, best);
    key = int(__reduce_min_sync(kFull, best == mk ? unsigned(key) : 0xffffffffu));   // INT_MAX if none
    v = T(0);
    return;
  }
  if (rule == LPB_PIVOT_STEEPEST && !bland) {
    // The value is -r_j^2 / gamma_j.  In FP64 the quotients are first formed
    // in FP32 (relative error below 4e-7; FP64 division is slow here) and only
    // columns within 1e-5 of the largest FP32 score get the exact one, which
    // keeps the exact maximum and its ties among them.
    float cut = 0.f;
    if constexpr (sizeof(T) == 8) {
      float b32 = 0.f;
      for (int j = threadIdx.x & 31; j < S.nc; j += 32) {
        const int var = j == ecol ? evar : S.nonb[j];
        if (var >= S.nm || !(r[j] < -eps_d)) continue;
        const float r32 = d2f_rn(r[j]);
        b32 = fmaxf(b32, __fdiv_rn(r32 * r32, d2f_rn(S.gam[j])));
      }
      b32 = __uint_as_float(__reduce_max_sync(kFull, __float_as_uint(b32)));   // >= 0: bits order like values
      cut = isfinite(b32) ? b32 * (1.f - 1e-5f) : 0.f;
    }
    for (int j = threadIdx.x & 31; j < S.nc; j += 32) {
      const int var = j == ecol ? evar : S.nonb[j];
      if (var >= S.nm) continue;
      const T rj = r[j];
      if (!(rj < -eps_d)) continue;
      if constexpr (sizeof(T) == 8) {
        const float r32 = d2f_rn(rj);
        if (__fdiv_rn(r32 * r32, d2f_rn(S.gam[j])) < cut) continue;
      }
      keep_better(v, key, -((rj * rj) / S.gam[j]), (var << kIdxBits) | j);
    }
    warp_argmin(v, key);
    return;
  }
  for (int j = threadIdx.x & 31; j < S.nc; j += 32) {
    const int var = j == ecol ? evar : S.nonb[j];
    if (var >= S.nm) continue;
    const T rj = r[j];
    if (rj < -eps_d) keep_better(v, key, bland ? T(0) : rj, (var << kIdxBits) | j);
  }
  warp_argmin(v, key);
}

// Phase I: an artificial that has left the basis sits in column e, which no
// pivot chooses again.  The last column moves into it, the right-hand side
// moves down one column and its old place is cleared, so that every later
// pivot sweeps one column less.  Every thread takes part (one row each); the
// tableau must be stable on entry.  With `remap`, a Step-1 choice of the last
// column made before the move is redirected to column e.
template <typename T>
__device__ __forceinline__ void drop_column(Tab<T> &S, int rows, int e, bool remap) {
  const int last = S.nc - 1;
  for (int i = threadIdx.x; i < rows; i += blockDim.x) {
    T *r = S.row(i);
    if (e != last) r[e] = r[last];
    r[last] = r[S.nc];
    r[S.nc] = T(0);
  }
  if (threadIdx.x == 0) {
    if (e != last) {
      S.nonb[e] = S.nonb[last];
      S.gam[e] = S.gam[last];
    }
    if (remap) {
      const int k = S.sel[0];
      if (k != INT_MAX && (k & kIdxMask) == last) S.sel[0] = (k & ~kIdxMask) | e;
    }
  }
  S.nc = last;
  __syncthreads();
}

// Steps 1-3 on objective row `orow` until a halt condition (Section 3.1).
// Phase 1 also ratio-tests rows whose basic variable is artificial; phase 2
// skips them (they are redundant rows left after Phase I).  Phase 1 drops the
// columns of artificials that leave the basis; S_.nc returns the new width.
template <typename T, bool FUSE>
__device__ __forceinline__ int run_phase(Tab<T> &S_, int orow, int rows, int phase, int &iters, int max_iter,
                         T eps_p, T eps_d, int rule, unsigned long long seed, long long lp) {
  Tab<T> S = S_;   // a register copy: stores through tableau pointers cannot alias it
  auto done = [&](int status) {
    S_.nc = S.nc;
    return status;
  };
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int r0, r1;
  own_rows(rows, r0, r1);
  const int per = (rows + nw - 1) / nw;
  const bool obj_warp = orow >= r0 && orow < r1;
  // Steepest edge needs every row of the updated tableau for its weights, so
  // its Step 1 follows the pivot's barrier instead of overlapping it.  The
  // FP32 kernel's steepest-edge instantiation (FUSE) forms the weights once
  // here and its pivots' sweeps keep them (every row adds its part of each
  // column's gamma, by shared-memory atomics in no fixed order); the FP64
  // kernel re-sums them in row order before each pivot, so that it follows
  // the oracle's choices.  The other rules' kernels carry none of the fused
  // code.
  const bool se = rule == LPB_PIVOT_STEEPEST;
  constexpr bool kFuse = FUSE;
  int degenerate_run = 0;
  bool bland = false;
  if (se) {
    se_weights(S, orow, phase, eps_d, kFuse);
    __syncthreads();
  }
  if (w == 0) {            // Step 1 of the first pivot
    T v;
    int key;
    step1_warp(S, orow, false, eps_d, -1, 0, v, key, rule, seed, lp, iters);
    if (lane == 0) S.sel[0] = key;
  }
  __syncthreads();
  for (;;) {
    const int ekey = S.sel[0];
    if (ekey == INT_MAX) {
      __syncthreads();       // the last pivot row copy is visible to every warp
      return done(LPB_OPTIMAL);
    }
    const int e = ekey & kIdxMask;
    // Fused steepest edge: the weights are re-summed by this pivot's sweep
    // (Step 1 of this pivot has read them).
    if (kFuse && se)
      for (int j = threadIdx.x; j < S.nc; j += blockDim.x) S.gam[j] = T(0);
    // Step 2 on this warp's rows, and the reciprocal of its best pivot.
    {
      T v = pos_inf<T>();
      int key = INT_MAX;
      const int hi = min(r1, S.m);
      if constexpr (sizeof(T) == 8) {
        // FP64 division runs on the slow FP64 pipe, so the ratios are first
        // formed in FP32 (relative error below 3e-7) and, after one more
        // barrier, only rows within 1e-5 of the smallest FP32 ratio of the
        // whole tableau get the exact FP64 quotient.  The exact minimum and
        // every exact tie are always among them, so the choice is the one the
        // FP64 quotients of all rows would give; only the warps holding such
        // rows divide, and they alone form the reciprocal of their pivot.
        float m32 = __int_as_float(0x7f800000);
        for (int i = r0 + lane; i < hi; i += 32) {
          const int bv = S.basic[i];
          if (phase == 2 && bv >= S.nm) continue;
          const T *ri = S.row(i);
          const T a = ri[e];
          if (a > eps_p) m32 = fminf(m32, __fdiv_rn(d2f_rn(ri[S.nc]), d2f_rn(a)));
        }
        m32 = ord2f(__reduce_min_sync(kFull, f2ord(m32)));
        if (lane == 0) S.redf[w] = m32;
        __syncthreads();
        float g32 = lane < nw ? S.redf[lane] : __int_as_float(0x7f800000);
        g32 = ord2f(__reduce_min_sync(kFull, f2ord(g32)));
        const float cut = g32 + 1e-5f * fabsf(g32);
        if (m32 <= cut) {
          for (int i = r0 + lane; i < hi; i += 32) {
            const int bv = S.basic[i];
            if (phase == 2 && bv >= S.nm) continue;
            const T *ri = S.row(i);
            const T a = ri[e];
            if (a > eps_p && !(__fdiv_rn(d2f_rn(ri[S.nc]), d2f_rn(a)) > cut))
              keep_better(v, key, ri[S.nc] / a, (bv << kIdxBits) | i);
          }
        }
      } else {
        for (int i = r0 + lane; i < hi; i += 32) {
          const int bv = S.basic[i];
          if (phase == 2 && bv >= S.nm) continue;
          const T *ri = S.row(i);
          const T a = ri[e];
          if (a > eps_p) keep_better(v, key, ri[S.nc] / a, (bv << kIdxBits) | i);
        }
      }
      warp_argmin(v, key);
      if (lane == 0) {
        S.redv[32 + w] = v;
        S.redk[32 + w] = key;
        if (key != INT_MAX) S.rcp[w] = T(1) / S.at(key & kIdxMask, e);
      }
    }
    __syncthreads();
    T theta = pos_inf<T>();
    int lkey = INT_MAX;
    if (lane < nw) { theta = S.redv[32 + lane]; lkey = S.redk[32 + lane]; }
    warp_argmin(theta, lkey);
    if (lkey == INT_MAX) return done(phase == 2 ? LPB_UNBOUNDED : LPB_NUMERIC);
    if (iters >= max_iter) return done(LPB_ITER_LIMIT);
    const int l = lkey & kIdxMask, leave = lkey >> kIdxBits;
    const T rp = S.rcp[l / per];
    if (threadIdx.x == 0) {
      S.basic[l] = S.nonb[e];
      S.nonb[e] = leave;
    }
    if constexpr (kFuse) {
      if (se) update_any<T, true>(S, rows, l, e, rp, phase);
      else update_any(S, rows, l, e, rp);
    } else {
      update_any(S, rows, l, e, rp);
    }
    ++iters;
    if (theta <= eps_p) {
      if (++degenerate_run >= S.m + S.n) bland = true;
    } else {
      degenerate_run = 0;
      bland = false;
    }
    if (obj_warp && !se) {   // Step 1 of the next pivot on the updated objective row
      __syncwarp();
      T v;
      int key;
      step1_warp(S, orow, bland, eps_d, e, leave, v, key, rule, seed, lp, iters);
      if (lane == 0) S.sel[0] = key;
    }
    __syncthreads();
    if (kFuse && se && w == 0) {   // gamma of column e, now the leaving variable's: -t_ie / p, and 1/p at row l
      T g = T(0);
      for (int i = lane; i < S.m; i += 32)
        if (i != l && !(phase == 2 && S.basic[i] >= S.nm)) g = fma(S.colb[i], S.colb[i], g);
      g = warp_sum(g);
      if (lane == 0) S.gam[e] = T(1) + g + rp * rp;
      __syncwarp();
    }
    pivot_finish(S, rows, l);
    if (phase == 1 && leave >= S.nm) {   // the artificial's new column is dead
      __syncthreads();                   // the pivot row is in place
      drop_column(S, rows, e, true);
    }
    if (se) {                // Step 1 of the next pivot on the updated objective row and weights
      if (!kFuse) {
        __syncthreads();     // the pivot row is in place
        se_weights(S, orow, phase, eps_d, false);
        __syncthreads();
      }
      if (w == 0) {
        T v;
        int key;
        step1_warp(S, orow, bland, eps_d, -1, 0, v, key, rule, seed, lp, iters);
        if (lane == 0) S.sel[0] = key;
      }
      __syncthreads();
    }
  }
}

// Largest |t_ij| over enterable columns of row i (ties: lowest column); -1 if
// none exceeds `eps`.
template <typename T>
__device__ __forceinline__ int row_argmax_abs(const Tab<T> &S_, int i, T eps, int set) {
  const Tab<T> S = S_;   // a register copy: stores through tableau pointers cannot alias it
  T v = pos_inf<T>();
  int key = INT_MAX;
  for (int j = threadIdx.x; j < S.nc; j += blockDim.x) {
    if (S.nonb[j] >= S.nm) continue;
    const T a = fabs(S.at(i, j));
    if (a > eps) keep_better(v, key, -a, j);
  }
  block_argmin(v, key, S.redv + 32 * set, S.redk + 32 * set);
  return key == INT_MAX ? -1 : key;
}

// Column currently holding non-basic variable `var`; -1 if it is basic.
template <typename T>
__device__ __forceinline__ int column_of(const Tab<T> &S_, int var, int set) {
  const Tab<T> S = S_;   // a register copy: stores through tableau pointers cannot alias it
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
__device__ __forceinline__ int compact(int cnt, int *out, int *s_cnt, Pred pred) {
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
__device__ __forceinline__ bool build_tableau(const Tab<T> &S_, const BatchDev &B_, int lp, int64_t aoff, int64_t boff,
                              int64_t coff) {
  const Tab<T> S = S_;   // a register copy: stores through tableau pointers cannot alias it
  const BatchDev B = B_;
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
  const int m = S.m, n = S.n, ld = S.ld, nc = S.nc;
  const int rows = m + (S.k ? 2 : 1);
  {
    const int rsm = min(rows, S.rs);
    for (size_t idx = tid; idx < size_t(rsm) * ld; idx += nt) S.ts[idx] = T(0);
    for (size_t idx = tid; idx < size_t(rows - rsm) * ld; idx += nt) S.tg[idx] = T(0);
  }
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
          S.at(i, col) = T(-1);
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
        T *row = S.row(i);
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
    S.at(i, nc) = S.basic[i] >= n + m ? -bi : bi;
  }
  for (int j = tid; j < n; j += nt) {
    const T cj = ld_as<T>(B.c, coff + j, B.dtype);
    bad |= !isfinite(cj);
    S.at(m, j) = -cj;
  }
  bad = __syncthreads_or(bad);
  if (S.k) {   // Phase-I row: w = -(sum of artificials) in the non-basic variables
    for (int j = tid; j <= nc; j += nt) {
      T s = T(0);
      for (int i = 0; i < m; ++i)
        if (S.basic[i] >= n + m) s += S.at(i, j);
      S.at(m + 1, j) = -s;
    }
    __syncthreads();
  }
  return !bad;
}

// Pivot the variables of `warm` (a basis from an earlier pass, packed like b)
// into the basis.  Returns false when a pivot would be (near) singular or the
// resulting basic solution is infeasible; the caller then starts cold.
template <typename T>
__device__ __forceinline__ bool warm_start(const Tab<T> &S_, const int32_t *warm, int &iters, T eps_p) {
  const Tab<T> S = S_;   // a register copy: stores through tableau pointers cannot alias it
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
  // Columns now holding a variable of the warm basis, found once: a pivot on
  // column e changes only the variable of column e (to one outside the warm
  // basis), so the list stays valid while its columns are pivoted in order.
  __shared__ int s_nw;
  const int nwl = compact(S.nc, S.wl, &s_nw, [&](int j) { const int v = S.nonb[j]; return v < nm && S.ins[v]; });
  for (int t = 0; t < nwl; ++t) {
    __syncthreads();                              // reduction slots are free again
    const int e = S.wl[t];
    // Row with the largest |t_ie| among rows whose basic variable leaves.
    T bvv = pos_inf<T>();
    int key = INT_MAX;
    for (int i = tid; i < m; i += nt) {
      const int bv = S.basic[i];
      if (bv < nm && S.ins[bv]) continue;
      const T a = fabs(S.at(i, e));
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
__device__ __forceinline__ bool dual_cleanup(const Tab<T> &S_, int rows, int &iters, int max_iter, T eps_p) {
  const Tab<T> S = S_;   // a register copy: stores through tableau pointers cannot alias it
  const int tid = threadIdx.x, nt = blockDim.x;
  for (;;) {
    __syncthreads();
    T v = pos_inf<T>();
    int key = INT_MAX;
    for (int i = tid; i < S.m; i += nt) {
      const int bv = S.basic[i];
      if (bv >= S.nm) continue;
      const T rhs = S.at(i, S.nc);
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
      const T a = S.at(l, j);
      if (a < -eps_p) keep_better(v, key, S.at(S.m, j) / -a, (var << kIdxBits) | j);
    }
    block_argmin(v, key, S.redv + 32, S.redk + 32);
    if (key == INT_MAX || iters >= max_iter) return false;
    pivot(S, rows, l, key & kIdxMask);
    ++iters;
  }
}

// Write the FP64 outputs of LP `lp` from the tableau (FP64 and plain FP32 modes).
__device__ __forceinline__ int32_t *basis_at(const TableauParams &P, int lp, int64_t yoff) {
  return P.bbuf ? P.bbuf + (P.bpacked ? yoff : int64_t(lp) * P.B.max_m) : nullptr;
}

template <typename T>
__device__ __forceinline__ void write_from_tableau(const Tab<T> &S_, const ResultDev &R_, int32_t *basis, int lp,
                                   int64_t yoff, int64_t coff, int status, int iters) {
  const Tab<T> S = S_;   // a register copy: stores through tableau pointers cannot alias it
  const ResultDev R = R_;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int m = S.m, n = S.n;
  for (int j = tid; j < n; j += nt) R.x[coff + j] = 0.0;
  if (R.y) for (int i = tid; i < m; i += nt) R.y[yoff + i] = 0.0;
  __syncthreads();
  if (status == LPB_OPTIMAL) {
    for (int i = tid; i < m; i += nt) {
      const int v = S.basic[i];
      if (v < n) R.x[coff + v] = double(S.at(i, S.nc));
    }
    if (R.y)
      for (int j = tid; j < S.nc; j += nt) {
        const int v = S.nonb[j];
        if (v >= n && v < n + m) R.y[yoff + (v - n)] = double(S.at(m, j));
      }
  }
  if (basis)
    for (int i = tid; i < m; i += nt) basis[i] = S.basic[i] < S.nm ? S.basic[i] : -1;
  if (tid == 0) {
    R.status[lp] = status;
    if (R.iters) R.iters[lp] = iters;
    R.obj[lp] = status == LPB_OPTIMAL ? double(S.at(m, S.nc))
              : status == LPB_INFEASIBLE ? -INFINITY
              : status == LPB_UNBOUNDED ? INFINITY : NAN;
  }
}

// FP64 refinement and verification of an FP32-optimal basis.  Returns true and
// writes the outputs when the refined pair (x, y) passes the checks.
__device__ __forceinline__ bool refine_and_verify(const Tab<float> &S_, const BatchDev &B_, const ResultDev &R_,
                                                  int32_t *basis, const Layout &L, unsigned char *smem, int lp,
                                                  int64_t aoff, int64_t boff, int64_t coff, int64_t yoff, int iters,
                                                  double tol, double bmax, double cmax) {
  const Tab<float> S = S_;   // a register copy: stores through tableau pointers cannot alias it
  const BatchDev B = B_;
  const ResultDev R = R_;
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
  const int m = S.m, n = S.n, nc = S.nc;
  double *xb = reinterpret_cast<double *>(smem + L.xb);    // x_B by row
  double *rr = reinterpret_cast<double *>(smem + L.rr);    // primal residual b - [A I]_B x_B by row
  double *yv = reinterpret_cast<double *>(smem + L.yv);    // y by slack
  double *rho = reinterpret_cast<double *>(smem + L.rho);  // dual residual by row of a basic structural
  double *dj = reinterpret_cast<double *>(smem + L.dj);    // reduced costs A^T y - c by column
  int *sb = reinterpret_cast<int *>(smem + L.sb);   // rows whose basic variable is structural
  int *ns = reinterpret_cast<int *>(smem + L.ns);   // columns holding a non-basic slack
  int *sp = reinterpret_cast<int *>(smem + L.sp);   // row of basic slack k, or -1
  int *jq = reinterpret_cast<int *>(smem + L.jq);   // column of A of the q-th basic structural
  int *kq = reinterpret_cast<int *>(smem + L.kq);   // slack (row of A) of the p-th non-basic slack
  __shared__ int s_cnt0, s_cnt1;
  __shared__ double s_red[2][32];
  __shared__ unsigned long long s_nrm[2];
  const int dt = B.dtype;
  const double tp = tol * (1.0 + bmax), td = tol * (1.0 + cmax);

  const int nsb = compact(m, sb, &s_cnt0, [&](int i) { return S.basic[i] < n; });
  const int nns = compact(nc, ns, &s_cnt1, [&](int j) { const int v = S.nonb[j]; return v >= n && v < n + m; });
  for (int k = tid; k < m; k += nt) { sp[k] = -1; yv[k] = 0.0; }
  __syncthreads();
  for (int i = tid; i < m; i += nt) {
    const int v = S.basic[i];
    xb[i] = double(S.at(i, nc));
    if (v >= n && v < n + m) sp[v - n] = i;
  }
  for (int q = tid; q < nsb; q += nt) jq[q] = S.basic[sb[q]];
  for (int p = tid; p < nns; p += nt) {
    const int k = S.nonb[ns[p]] - n;
    kq[p] = k;
    yv[k] = double(S.at(m, ns[p]));
  }
  // Iterative refinement (at most kSteps corrections) of x_B = B^{-1} b and
  // y = B^{-T} c_B with FP64 residuals and the FP32 basis inverse held in the
  // tableau, until the residuals are 1000 times below the certificate's
  // tolerance.  The residuals of the last pass are the certificate's slacks
  // and reduced costs.
  constexpr int kSteps = 3;
  for (int step = 0;; ++step) {
    if (tid == 0) { s_nrm[0] = 0ull; s_nrm[1] = 0ull; }
    __syncthreads();
    // Primal residual r = b - A_S x_S - x_slack.  Each row's sum over the
    // basic structurals is split over a group of G lanes (G the largest power
    // of two with G m <= threads, at most 32), combined by butterflies in a
    // fixed order.
    double np = 0.0, nd = 0.0;
    {
      int G = 1;
      while (G < 32 && 2 * G * m <= nt) G *= 2;
      const int g = lane & (G - 1), rows_per_pass = nt / G;
      for (int i0 = 0; i0 < m; i0 += rows_per_pass) {
        const int i = i0 + tid / G;
        const bool live = i < m;
        const int64_t ar = aoff + int64_t(live ? i : 0) * n;
        double s0 = 0.0, s1 = 0.0;
        int q = g;
        for (; q + G < nsb; q += 2 * G) {
          s0 = fma(ld_in(B.A, ar + jq[q], dt), xb[sb[q]], s0);
          s1 = fma(ld_in(B.A, ar + jq[q + G], dt), xb[sb[q + G]], s1);
        }
        if (q < nsb) s0 = fma(ld_in(B.A, ar + jq[q], dt), xb[sb[q]], s0);
        double sum = s0 + s1;
        for (int off = 1; off < G; off *= 2) sum += __shfl_xor_sync(kFull, sum, off);
        if (live && g == 0) {
          double r = ld_in(B.b, boff + i, dt) - sum;
          if (sp[i] >= 0) r -= xb[sp[i]];
          rr[i] = r;
          np = fmax(np, fabs(r));
        }
      }
    }
    // Reduced costs d_j = A_j^T y - c_j of every column, one thread per column.
    for (int j = tid; j < n; j += nt) {
      double d = -ld_in(B.c, coff + j, dt);
#pragma unroll 8
      for (int p = 0; p < nns; ++p) {
        const int k = kq[p];
        d = fma(ld_in(B.A, aoff + int64_t(k) * n + j, dt), yv[k], d);
      }
      dj[j] = d;
    }
    {
      const unsigned long long w = warp_max_u64(static_cast<unsigned long long>(__double_as_longlong(np)));
      if (lane == 0 && w > 0ull) atomicMax(&s_nrm[0], w);
    }
    __syncthreads();
    for (int q = tid; q < nsb; q += nt) {      // dual residual c_B - B^T y on the basic structurals
      const double r = -dj[jq[q]];
      rho[sb[q]] = r;
      nd = fmax(nd, fabs(r));
    }
    {
      const unsigned long long w = warp_max_u64(static_cast<unsigned long long>(__double_as_longlong(nd)));
      if (lane == 0 && w > 0ull) atomicMax(&s_nrm[1], w);
    }
    __syncthreads();
    const double rp_ = __longlong_as_double(static_cast<long long>(s_nrm[0]));
    const double rd_ = __longlong_as_double(static_cast<long long>(s_nrm[1]));
    if (step == kSteps || (rp_ <= 1e-3 * tp && rd_ <= 1e-3 * td)) break;   // 1000x below the certificate's bar
    // Corrections with the FP32 basis inverse: its column for slack k is the
    // tableau column of k when k is non-basic, else the unit vector of k's row.
    for (int t = tid; t < m; t += nt) {
      float d = 0.f;
      const float *row = S.row(t);
      for (int p = 0; p < nns; ++p) d = fmaf(float(rr[kq[p]]), row[ns[p]], d);
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
        d = fmaf(float(rho[t]), S.at(t, col), d);
      }
      yv[kq[p]] += double(d);
    }
    __syncthreads();
  }
  // FP64 KKT certificate of the pair that is written out (x: the structural
  // part of x_B; y: the slack duals): x >= 0, A x <= b, y >= 0, A^T y >= c and
  // c^T x = b^T y, each to tol scaled by the data.  The slack of row i is its
  // residual plus its basic slack's value.
  double cx = 0.0, by = 0.0;
  int bad = 0;
  for (int q = tid; q < nsb; q += nt) {
    bad |= !(xb[sb[q]] >= -tp);
    cx = fma(ld_in(B.c, coff + jq[q], dt), xb[sb[q]], cx);
  }
  for (int p = tid; p < nns; p += nt) {
    const int k = kq[p];
    by = fma(ld_in(B.b, boff + k, dt), yv[k], by);
    bad |= !(yv[k] >= -td);
  }
  for (int i = tid; i < m; i += nt) bad |= !(rr[i] + (sp[i] >= 0 ? xb[sp[i]] : 0.0) >= -tp);
  for (int j = tid; j < n; j += nt) bad |= !(dj[j] >= -td);
  cx = warp_sum(cx);
  by = warp_sum(by);
  if (lane == 0) { s_red[0][wid] = cx; s_red[1][wid] = by; }
  bad = __syncthreads_or(bad);
  cx = 0.0; by = 0.0;
  for (int w = 0; w < nw; ++w) { cx += s_red[0][w]; by += s_red[1][w]; }
  bad |= !(fabs(cx - by) <= tol * (1.0 + fabs(cx)));
  if (bad) return false;
  for (int j = tid; j < n; j += nt) R.x[coff + j] = 0.0;
  __syncthreads();
  for (int q = tid; q < nsb; q += nt) R.x[coff + jq[q]] = xb[sb[q]];
  if (R.y) for (int k = tid; k < m; k += nt) R.y[yoff + k] = yv[k];
  if (basis) for (int i = tid; i < m; i += nt) basis[i] = S.basic[i];
  if (tid == 0) {
    R.status[lp] = LPB_OPTIMAL;
    if (R.iters) R.iters[lp] = iters;
    R.obj[lp] = cx;
  }
  return true;
}

// FUSE_SE: the FP32 steepest-edge instantiation (see run_phase).
template <typename T, bool FUSE_SE>
__global__ void __launch_bounds__(kMaxThreads) tableau_kernel(TableauParams P) {
  constexpr bool kFuseSE = FUSE_SE;
  extern __shared__ __align__(16) unsigned char smem[];
  const int tid = threadIdx.x, nt = blockDim.x;
  const bool refine = (P.mode == MODE_FP32_REFINE) && sizeof(T) == 4;
  const Layout L = make_layout(int(sizeof(T)), P.tab_smem, P.B.max_m, P.B.max_n, P.kcap, refine);
  Tab<T> S;
  S.ts = reinterpret_cast<T *>(smem + L.tab);
  S.tg = P.slot_bytes ? reinterpret_cast<T *>(static_cast<unsigned char *>(P.slots) + size_t(blockIdx.x) * P.slot_bytes)
                      : nullptr;
  S.colb = reinterpret_cast<T *>(smem + L.colb);
  S.rowb = reinterpret_cast<T *>(smem + L.rowb);
  S.gam = reinterpret_cast<T *>(smem + L.gam);
  S.basic = reinterpret_cast<int *>(smem + L.basic);
  S.nonb = reinterpret_cast<int *>(smem + L.nonb);
  S.redv = reinterpret_cast<T *>(smem + L.redv);
  S.redk = reinterpret_cast<int *>(smem + L.redk);
  S.rcp = reinterpret_cast<T *>(smem + L.rcp);
  S.redf = reinterpret_cast<float *>(smem + L.redf);
  S.sel = reinterpret_cast<int *>(smem + L.sel);
  S.ins = smem + L.ins;
  S.wl = reinterpret_cast<int *>(smem + L.wl);
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
    const int64_t yoff = P.R.y_off ? P.R.y_off[lp] : boff;    // outputs packed like b, or at y_off
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
    {
      const unsigned long long wb = warp_max_u64(static_cast<unsigned long long>(__double_as_longlong(bm)));
      const unsigned long long wc = warp_max_u64(static_cast<unsigned long long>(__double_as_longlong(cm)));
      if ((tid & 31) == 0) {
        atomicMax(&s_bmax, wb);
        atomicMax(&s_cmax, wc);
      }
    }
    __syncthreads();
    S.m = m; S.n = n; S.k = s_k; S.nc = n + S.k; S.ld = tab_ld(n, S.k, int(sizeof(T))); S.nm = n + m;
    {
      // Leading rows in shared memory as far as they fit, the rest in the slot.
      const int rows = m + (S.k ? 2 : 1);
      const size_t row_bytes = size_t(S.ld) * sizeof(T);
      S.rs = int(min(size_t(rows), P.tab_smem / row_bytes));
      if (size_t(rows - S.rs) * row_bytes > P.slot_bytes && S.k <= P.kcap) {
        if (tid == 0) {
          atomicOr(P.err, ERR_SLOT_OVERFLOW);
          P.R.status[lp] = LPB_NUMERIC;
          if (P.R.iters) P.R.iters[lp] = 0;
          P.R.obj[lp] = NAN;
        }
        __syncthreads();
        continue;
      }
    }
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
      if (P.warm && basis_at(P, lp, yoff)) {
        warm = warm_start(S, basis_at(P, lp, yoff), iters, eps_p) &&
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
        const double w0 = -double(S.at(m + 1, S.nc));
        const double ftol = sizeof(T) == 4 ? fmax(P.feas_tol * (1.0 + bmax), 1e-5 * (1.0 + w0))
                                           : P.feas_tol * (1.0 + bmax);
        // FP32 Phase-I reduced costs carry round-off relative to the Phase-I
        // row, a sum over the negated rows: Step 1's threshold scales with its
        // largest starting entry, so that round-off does not make columns
        // eligible.  (The certificate and the FP64 re-solve keep the results
        // exact.)
        T eps_d1 = eps_d;
        if constexpr (sizeof(T) == 4) {
          const int jm = row_argmax_abs(S, m + 1, T(0), 0);
          if (jm >= 0) eps_d1 = eps_d * fmaxf(1.f, fabsf(S.at(m + 1, jm)));
        }
        status = run_phase<T, kFuseSE>(S, m + 1, m + 2, 1, iters, max_iter, eps_p, eps_d1, P.rule, P.seed, P.lp_base + lp);
        if (status == LPB_OPTIMAL) {
          const double w = double(S.at(m + 1, S.nc));
          if (-w > ftol) {
            status = LPB_INFEASIBLE;
          } else {             // drive zero-level artificials out of the basis
            for (int i = 0; i < m; ++i) {
              if (S.basic[i] < S.nm) continue;
              const int e = row_argmax_abs(S, i, eps_p, 0);
              if (e >= 0) {
                pivot(S, m + 2, i, e);
                ++iters;
                drop_column(S, m + 2, e, false);
              }
              __syncthreads();
            }
          }
        }
      }
      if (status == LPB_OPTIMAL) status = run_phase<T, kFuseSE>(S, m, m + 1, 2, iters, max_iter, eps_p, eps_d, P.rule, P.seed, P.lp_base + lp);
    }
    if constexpr (sizeof(T) == 4) if (P.mode == MODE_FP32_REFINE) {
      bool done = false;
      if (status == LPB_OPTIMAL) {
        int dropped = 0;
        for (int i = tid; i < m; i += nt) dropped |= S.basic[i] >= S.nm;
        if (!__syncthreads_or(dropped))
          done = refine_and_verify(S, P.B, P.R, basis_at(P, lp, yoff), L, smem, lp, aoff, boff,
                                   coff, yoff, iters, P.feas_tol, bmax, cmax);
      }
      if (!done) {
        if (int32_t *bp = basis_at(P, lp, yoff))
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
    write_from_tableau(S, P.R, basis_at(P, lp, yoff), lp, yoff, coff, status, iters);
    __syncthreads();
  }
}

}  // namespace

size_t tableau_fixed_bytes(int eb, int max_m, int max_n, int kcap, bool refine) {
  return make_layout(eb, 0, max_m, max_n, kcap, refine).total;
}

size_t tableau_row_bytes(int eb, int max_n, int kcap) { return size_t(tab_ld(max_n, kcap, eb)) * size_t(eb); }

template <typename T, bool SE>
static cudaError_t prep(size_t smem) {
  return cudaFuncSetAttribute(tableau_kernel<T, SE>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
}

cudaError_t tableau_max_ctas_per_sm(int eb, int threads, size_t smem, int *ctas) {
  if (eb == 8) {
    const cudaError_t e = prep<double, false>(smem);
    return e != cudaSuccess ? e : cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas, tableau_kernel<double, false>, threads, smem);
  }
  const cudaError_t e = prep<float, false>(smem);
  return e != cudaSuccess ? e : cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas, tableau_kernel<float, false>, threads, smem);
}

cudaError_t launch_tableau(const TableauParams &p, bool fp64, int grid, int threads, size_t smem, cudaStream_t s) {
  if (threads < 32 || threads > kMaxThreads || (threads & 31) || grid < 1) return cudaErrorInvalidValue;
  const bool se = !fp64 && p.rule == LPB_PIVOT_STEEPEST;
  const cudaError_t e = fp64 ? prep<double, false>(smem) : se ? prep<float, true>(smem) : prep<float, false>(smem);
  if (e != cudaSuccess) return e;
  if (fp64) tableau_kernel<double, false><<<grid, threads, smem, s>>>(p);
  else if (se) tableau_kernel<float, true><<<grid, threads, smem, s>>>(p);
  else tableau_kernel<float, false><<<grid, threads, smem, s>>>(p);
  return cudaGetLastError();
}

}  // namespace lpb
