// simplex_warp.cu -- one warp per LP, the compact FP32 tableau in shared
// memory, FP64 refinement and certificate fused in (FP64 input, LPs with
// m, n <= 127 whose slack basis is feasible).
//
// Section 3.1 Steps 1-3 on the compact (exchange) tableau, with the paper's
// Section 4.1 "one block per LP" narrowed to one warp per LP: the warps of a
// CTA share nothing but the CTA's shared memory, so a solve has no block
// barrier at all.  At m = n = 100 a tableau is 101 x 108 floats (43.6 KB), so
// an SM holds five LPs at once.  Design:
//
//   * Layout: row i of the tableau (rows 0..m-1 the constraints, row m the
//     objective row, column n the right-hand side) starts at i * S floats.
//     The stride S is a multiple of 4 with S / 4 odd, so that the eight rows a
//     quarter-warp touches in one 16-byte access fall in eight disjoint groups
//     of four banks (no bank conflict in the update).
//   * Steps 1 and 2: lane l takes columns (rows) l, l + 32, ...; arg-min by
//     warp reductions on the order-preserving integer image of the float.
//   * Step 3: lane (r, g) = (lane mod 8, lane / 8) updates rows r + 8t and
//     16-byte column blocks g + 4u (u < U): the pivot row's U blocks stay in
//     registers, the rows stream past with the next row's loads in flight
//     while the current row is written: 2 (m + 1)(n + 1) 4 bytes of shared
//     memory per pivot.  With at most eight warps per SM (the register file)
//     the kernel is bound by latency, not by that bandwidth.
//   * The next LP's A, b and c are prefetched into L2 when this LP's pivots
//     end (issued before the pivots, the lines were often evicted again by
//     the time of the build: 100 x 100 4.46 -> 4.34 ms per 50,000 LPs with
//     the later hint); the tableau is built from them with 16-byte loads, or
//     (large LPs in the wide templates) from rows staged by bulk copies.
//   * Refinement and certificate as in the register kernel (FP64 residuals,
//     one correction with the FP32 basis inverse, KKT certificate), on
//     operands gathered into the dead tableau region: the non-basic slacks'
//     tableau columns and the entries of A that the FP64 products read.
//     Its row (column) loops take two rows (columns) per lane at a time, so
//     two FP64 chains are in flight, in the same summation order per row.
//   * Instruction footprint: eight warps in different phases of one large
//     kernel share an SM's instruction caches, so every loop outside the
//     pivot's hot path is kept rolled (`#pragma unroll 1`): 50,000 LPs of
//     64 x 64 took 2.00 ms with those loops unrolled by the compiler and take
//     1.53 ms rolled.
//
// Sizes beyond the launch's limits, LPs with some b_i < 0 (Phase I) and
// non-finite data go to the shared-memory kernel, as from the register kernel.

#include "lpb_internal.cuh"

namespace lpb {

namespace {

constexpr int kWarpMaxWarps = 8;      // LPs (warps) per CTA at most
constexpr int kWarpMaxDim = 127;      // largest m and n: four rows (columns) per lane
constexpr int kNoKey = 1 << 30;       // a key larger than any real key
constexpr int kRefK = 24;             // basic structurals the on-chip refinement takes at most

// One warp's region of shared memory.
struct WarpLayout {
  int S;          // tableau row stride in floats
  int tab;        // bytes of the tableau region (the tableau, or more: see warp_layout)
  int colb;       // byte offsets of the small arrays
  int rr, dx, bas, nbv, sb, ns;
  int bar;        // the warp's transaction barrier (8 bytes)
  int bytes;      // size of the region (a multiple of 16)
};

__host__ __device__ inline int warp_stride(int max_n) {
  int s = (max_n + 1 + 3) & ~3;
  if ((s & 7) == 0) s += 4;          // S / 4 odd
  return s;
}

// Arrays of one entry per row or column (float or short) hold A8 entries.
// The tableau region holds the tableau and, after the pivots, the
// refinement's operands; when eight regions fit the SM's shared memory with
// room to spare, it grows towards what kRefK basic structurals need.
__host__ __device__ inline WarpLayout warp_layout(int max_m, int max_n) {
  WarpLayout L;
  L.S = warp_stride(max_n);
  const int a8 = ((max_m > max_n ? max_m : max_n) + 1 + 7) & ~7;
  const int arrays = 20 * a8;
  int tab = (max_m + 1) * L.S * 4;   // the tableau (16-byte rows)
  const int want = ((max_m * (kRefK | 1) * 4 + 15) & ~15) + max_m * (kRefK | 1) * 8 + kRefK * max_n * 8 +
                   (max_m + max_n) * 8 + (3 * max_m + max_n + 2 * kRefK) * 8 + 3 * kRefK * 4;
  const int room = ((232448 / kWarpMaxWarps - arrays - 16) & ~15);   // 16: the barrier, aligned
  if (want > tab && room > tab) tab = want < room ? (want + 15) & ~15 : room;
  L.tab = tab;
  int off = tab;
  L.colb = off; off += 4 * a8;       // colb and rr together also serve as a[a8] doubles
  L.rr = off;   off += 4 * a8;
  L.dx = off;   off += 4 * a8;
  L.bas = off;  off += 2 * a8;
  L.nbv = off;  off += 2 * a8;
  L.sb = off;   off += 2 * a8;
  L.ns = off;   off += 2 * a8;
  off = (off + 7) & ~7;
  L.bar = off;  off += 8;
  L.bytes = (off + 15) & ~15;
  return L;
}

// Asynchronous 8-byte copy global -> shared; cp_async_wait_all waits for every
// copy this thread issued.
__device__ __forceinline__ void cp_async8(void *dst, const void *src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

__device__ __forceinline__ float4 ld4(const float *p) { return *reinterpret_cast<const float4 *>(p); }
__device__ __forceinline__ void st4(float *p, float4 v) { *reinterpret_cast<float4 *>(p) = v; }

// v[s] of the lane holding slot s = idx >> 5, from lane idx & 31 (idx is the
// same in every lane).
template <typename V>
__device__ __forceinline__ V pick_slot(const V (&v)[4], int idx) {
  const int s = idx >> 5;
  V r = v[0];
  if (s == 1) r = v[1];
  if (s == 2) r = v[2];
  if (s == 3) r = v[3];
  return __shfl_sync(kFull, r, idx & 31);
}

__device__ __forceinline__ float4 upd4(float4 x, float4 p, float g) {
  x.x = fmaf(-g, p.x, x.x);
  x.y = fmaf(-g, p.y, x.y);
  x.z = fmaf(-g, p.z, x.z);
  x.w = fmaf(-g, p.w, x.w);
  return x;
}

// Step 3's sweep: T[i, :] -= colb[i] * (pivot row) for rows i = rg + 8 t <= m,
// on this lane's blocks cg + 4 u < nbu (pr: the pivot row's blocks).  Slots
// whose eight rows all exist are pipelined two rows at a time; the last,
// partial slot goes alone.
template <int U>
__device__ __forceinline__ void sweep_rows(float *T, int S, const float *colb, int m, int rg, int cg, int nbu,
                                           const float4 (&pr)[U]) {
  bool ok[U];
#pragma unroll
  for (int u = 0; u < U; ++u) ok[u] = cg + 4 * u < nbu;
  const int full = (m + 1) >> 3;            // slots whose eight rows all exist
  const int step = 8 * S;
  float *row = T + rg * S + 4 * cg;
  if (full > 0) {
    float4 a[U], b[U];
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (ok[u]) a[u] = ld4(row + 16 * u);
    float ga = colb[rg], gb = 0.f;
    int t = 0;
    for (; t + 1 < full; t += 2) {
      float *r1 = row + step;
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (ok[u]) b[u] = ld4(r1 + 16 * u);
      gb = colb[rg + 8 * (t + 1)];
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (ok[u]) st4(row + 16 * u, upd4(a[u], pr[u], ga));
      float *r2 = r1 + step;
      if (t + 2 < full) {
#pragma unroll
        for (int u = 0; u < U; ++u)
          if (ok[u]) a[u] = ld4(r2 + 16 * u);
        ga = colb[rg + 8 * (t + 2)];
      }
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (ok[u]) st4(r1 + 16 * u, upd4(b[u], pr[u], gb));
      row = r2;
    }
    if (t < full) {
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (ok[u]) st4(row + 16 * u, upd4(a[u], pr[u], ga));
      row += step;
    }
  }
  if (rg < ((m + 1) & 7)) {                 // the partial slot
    const float g = colb[rg + 8 * full];
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (ok[u]) st4(row + 16 * u, upd4(ld4(row + 16 * u), pr[u], g));
  }
}

// Prefetch A, b and c of an LP into L2 (a hint; nothing waits for it).
__device__ __forceinline__ void warp_prefetch(const TableauParams &P, int m, int n, long long aoff, long long boff,
                                              long long coff) {
  const size_t es = P.B.dtype == LPB_DTYPE_F64 ? 8 : 4;
  prefetch_l2(static_cast<const unsigned char *>(P.B.A) + size_t(aoff) * es, size_t(m) * size_t(n) * es);
  prefetch_l2(static_cast<const unsigned char *>(P.B.b) + size_t(boff) * es, size_t(m) * es);
  prefetch_l2(static_cast<const unsigned char *>(P.B.c) + size_t(coff) * es, size_t(n) * es);
}

// Rows r0..m-1 of the LP's FP64 A (Ag) converted to FP32 by truncation
// (relative error below 2^-23; the refinement works with the exact A) into
// the tableau by plain loads: the elements in order over the 32 lanes, eight
// loads in flight per lane, pairs of doubles with 16-byte loads when the rows
// start on 16-byte boundaries (16-byte aligned A, n even).  `amax` keeps the
// largest high word of |a| (see d2f_trunc).
__device__ __forceinline__ void build_rows_ldg(float *T, int S, const double *Ag, int r0, int m, int n, int lane,
                                               unsigned &amax) {
  const double *A0 = Ag + static_cast<long long>(r0) * n;
  const int tot = (m - r0) * n;
  if ((reinterpret_cast<uintptr_t>(A0) & 15) == 0 && (n & 1) == 0) {
    const double2 *A2 = reinterpret_cast<const double2 *>(A0);
    const int tot2 = tot >> 1;
    int row = r0, col = 2 * lane;
    while (col >= n) { col -= n; ++row; }
    for (int k0 = lane; k0 < tot2; k0 += 32 * 8) {
      double2 v[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int k = k0 + 32 * q;
        if (k < tot2) v[q] = __ldg(A2 + k);
      }
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        if (k0 + 32 * q < tot2) {
          float2 f;
          f.x = d2f_trunc(v[q].x, amax);
          f.y = d2f_trunc(v[q].y, amax);
          *reinterpret_cast<float2 *>(T + row * S + col) = f;
        }
        col += 64;
        while (col >= n) { col -= n; ++row; }
      }
    }
  } else {
    int row = r0, col = lane;
    while (col >= n) { col -= n; ++row; }
    for (int k0 = lane; k0 < tot; k0 += 32 * 8) {
      double v[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int k = k0 + 32 * q;
        if (k < tot) v[q] = __ldg(A0 + k);
      }
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        if (k0 + 32 * q < tot) T[row * S + col] = d2f_trunc(v[q], amax);
        col += 32;
        while (col >= n) { col -= n; ++row; }
      }
    }
  }
}


// Element i of the LP's FP64 b or c rounded to FP32 and its magnitude bits;
// non-finite or out-of-range values set `bad`.
__device__ __forceinline__ float vec_in(const void *v, long long i, int &bad, unsigned long long &mag) {
  const double d = __ldg(static_cast<const double *>(v) + i);
  mag = static_cast<unsigned long long>(__double_as_longlong(d)) & 0x7fffffffffffffffull;
  return d2f_tile(d, bad);
}

// Outcome of the tableau build.
enum : int { BUILD_BAD = 1, BUILD_TIMEOUT = 2 };
constexpr int kBulkBuild = 7000;

// The LP's FP64 A into the tableau's rows 0..m-1 as FP32.  In the templates
// of more than 96 columns (BULK), for an LP of more than kBulkBuild entries
// whose A starts on a 16-byte boundary with rows of whole 16-byte units (n
// even) no shorter than a tableau row, rows arrive in rounds of bulk copies
// (below these, plain loads finish sooner and the bulk path's code only adds
// to the instruction footprint: measured), staged at the top
// of the free part of the tableau region (`tab` bytes): a round stages as many
// rows as fit above the rows already converted (one copy: the rows are
// contiguous), the warp waits on its transaction barrier, then converts them
// in order, two rows at a time, each pair read in full before it is written
// and written below every staged row still unread (a tableau row is no longer
// than an FP64 row).  Rows for which no round of at least four has room go by
// plain loads.  A copy that does not land within kCopyWaitNs gives
// BUILD_TIMEOUT (after ERR_WAIT_TIMEOUT, and ERR_COPY_IN_FLIGHT if it is still
// outstanding kDrainWaitNs later): the warp must then stop using its region.
template <bool BULK>
__device__ __forceinline__ int build_a(const TableauParams &P, unsigned char *region, int tab, int S, int m, int n,
                                       long long aoff, int lane, uint64_t *bar, unsigned &phase) {
  const double *Ag = static_cast<const double *>(P.B.A) + aoff;
  float *T = reinterpret_cast<float *>(region);
  const int SB = S * 4, RB = n * 8;
  unsigned amax = 0u;
  int r0 = 0;
  if (BULK && (reinterpret_cast<uintptr_t>(Ag) & 15) == 0 && (n & 1) == 0 && SB <= RB && m * n > kBulkBuild) {
    const int h = n >> 1;                          // pairs per row
    const float inv_h = 1.f / float(h);
    for (;;) {
      const int rows = min((tab - r0 * SB) / RB, m - r0);
      if (rows <= 0 || (rows < 4 && rows < m - r0)) break;
      const int stage = tab - rows * RB;
      __syncwarp();
      if (lane == 0) {
        fence_async_smem();           // earlier reads and writes of the region before the copy's writes
        mbar_expect_tx(bar, unsigned(rows * RB));
        bulk_load(region + stage, Ag + static_cast<long long>(r0) * n, unsigned(rows * RB), bar);
      }
      const bool ok = mbar_wait_for(bar, phase, kCopyWaitNs);
      phase ^= 1u;
      if (__any_sync(kFull, !ok)) {
        if (lane == 0) {
          atomicOr(P.err, ERR_WAIT_TIMEOUT);
          if (!mbar_wait_for(bar, phase ^ 1u, kDrainWaitNs)) atomicOr(P.err, ERR_COPY_IN_FLIGHT);
        }
        __syncwarp();
        return BUILD_TIMEOUT;
      }
      const double2 *st = reinterpret_cast<const double2 *>(region + stage);
      for (int g = 0; g < rows; g += 2) {
        const int np = min(2, rows - g) * h;       // pairs of this group
        double2 v[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const int pi = lane + 32 * t;
          if (pi < np) v[t] = st[g * h + pi];
        }
        __syncwarp();
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const int pi = lane + 32 * t;
          if (pi < np) {
            const int rr = int((float(pi) + 0.5f) * inv_h);
            float2 f;
            f.x = d2f_trunc(v[t].x, amax);
            f.y = d2f_trunc(v[t].y, amax);
            *reinterpret_cast<float2 *>(T + (r0 + g + rr) * S + 2 * (pi - rr * h)) = f;
          }
        }
      }
      r0 += rows;
      if (r0 >= m) break;
    }
    __syncwarp();
  }
  if (r0 < m) build_rows_ldg(T, S, Ag, r0, m, n, lane, amax);
  return amax >= (1151u << 20) ? BUILD_BAD : 0;     // |a| >= 2^128, Inf or NaN
}

template <int U>
__global__ void __launch_bounds__(kWarpMaxWarps * 32, 1) warp_kernel(TableauParams P, WarpLayout L) {
  extern __shared__ __align__(16) unsigned char warp_smem[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  unsigned char *base = warp_smem + size_t(wid) * size_t(L.bytes);
  float *T = reinterpret_cast<float *>(base);
  float *colb = reinterpret_cast<float *>(base + L.colb);    // pivot-column multipliers; rho
  float *rrs = reinterpret_cast<float *>(base + L.rr);       // FP32 residuals; dy by slack
  float *dxs = reinterpret_cast<float *>(base + L.dx);       // structural corrections by row
  double *xs = reinterpret_cast<double *>(base + L.colb);    // x of basic slacks by slack (over colb, rr)
  short *bas = reinterpret_cast<short *>(base + L.bas);      // basic variable of each row
  short *nbv = reinterpret_cast<short *>(base + L.nbv);      // non-basic variable of each column
  short *sbl = reinterpret_cast<short *>(base + L.sb);       // rows of the basic structurals
  short *nsl = reinterpret_cast<short *>(base + L.ns);       // columns of the non-basic slacks
  const int S = L.S;
  const int rg = lane & 7, cg = lane >> 3;
  const int nitems = P.in.count ? min(*P.in.count, P.list_cap) : P.B.count;
  const float eps_p = float(P.eps_p), eps_d = float(P.eps_d);
  constexpr unsigned long long kInf = 0x7ff0000000000000ull;

  if (blockDim.x > kWarpMaxWarps * 32 || (blockDim.x & 31) || P.B.dtype != LPB_DTYPE_F64) {
    if (threadIdx.x == 0) atomicOr(P.err, ERR_BAD_LAUNCH);
    return;
  }
  uint64_t *bar = reinterpret_cast<uint64_t *>(base + L.bar);
  unsigned bphase = 0;           // parity of the next completion of bar
  if (lane == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  __syncwarp();
  auto fits_lp = [&](int m, int n) {
    return m >= 1 && n >= 1 && m <= P.lim_m && n <= P.lim_n && m <= P.B.max_m && n <= P.B.max_n &&
           m <= kWarpMaxDim && n <= kWarpMaxDim && n + 1 <= 16 * U;
  };
  auto read_desc = [&](int it, int &lp_, int &m_, int &n_, long long &a_, long long &b_, long long &c_) {
    lp_ = P.in.items ? __ldg(P.in.items + it) : it;
    m_ = __ldg(P.B.m + lp_);
    n_ = __ldg(P.B.n + lp_);
    a_ = __ldg(P.B.a_off + lp_);
    b_ = __ldg(P.B.b_off + lp_);
    c_ = __ldg(P.B.c_off + lp_);
  };

  // Work items are claimed one LP ahead: the claim is issued when an LP
  // starts, the claimed LP's descriptor is read while this LP's tableau is
  // built, and its data is prefetched into L2 when this LP's pivots end.
  int item = 0;
  if (lane == 0) item = atomicAdd(P.queue, 1);
  item = __shfl_sync(kFull, item, 0);
  int lp = 0, m = 0, n = 0;
  long long aoff = 0, boff = 0, coff = 0;
  if (item < nitems) read_desc(item, lp, m, n, aoff, boff, coff);
  while (item < nitems) {
    int nitem = 0;
    if (lane == 0) nitem = atomicAdd(P.queue, 1);
    // ---- b and c: checks (their FP32 values wait in registers, rows and
    // columns lane + 32 s, while A is built) ----
    const bool fits = fits_lp(m, n);
    int bad = !fits;
    unsigned long long bm = 0ull, cm = 0ull;
    float bf[4], cf[4];
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      const int i = lane + 32 * s;
      bf[s] = 0.f;
      cf[s] = 0.f;
      if (fits && i < m) {
        unsigned long long a;
        bf[s] = vec_in(P.B.b, boff + i, bad, a);
        bad |= int(__float_as_uint(bf[s]) > 0x80000000u);     // b_i < 0 (Phase I)
        bm = a > bm ? a : bm;
      }
      if (fits && i < n) {
        unsigned long long a;
        cf[s] = vec_in(P.B.c, coff + i, bad, a);
        cm = a > cm ? a : cm;
      }
    }
    nitem = __shfl_sync(kFull, nitem, 0);
    int nlp = 0, nm = 0, nn = 0;
    long long na = 0, nb = 0, nc = 0;
    if (nitem < nitems) read_desc(nitem, nlp, nm, nn, na, nb, nc);
    if (fits) {
      const int br = build_a<(U >= 7)>(P, base, L.tab, S, m, n, aoff, lane, bar, bphase);
      if (br & BUILD_TIMEOUT) {
        // The copy engine did not deliver in time: this LP and the one claimed
        // after it go to the shared-memory kernel, and the warp stops.
        if (lane == 0) {
          P.R.status[lp] = STATUS_PENDING;
          list_push(P.defer_items, P.defer_count, P.list_cap, lp, P.err);
          if (nitem < nitems) {
            P.R.status[nlp] = STATUS_PENDING;
            list_push(P.defer_items, P.defer_count, P.list_cap, nlp, P.err);
          }
        }
        return;
      }
      bad |= br;
      // The right-hand side column, the objective row (-c, and 0 on the
      // right-hand side) and the zero columns n+1 .. 4 ceil((n+1)/4) - 1 that
      // the update sweeps.
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        const int i = lane + 32 * s;
        if (i < m) {
          T[i * S + n] = bf[s];
          bas[i] = short(n + i);
        }
        if (i < n) {
          T[m * S + i] = -cf[s];
          nbv[i] = short(i);
        }
      }
      if (lane == 0) T[m * S + n] = 0.f;
      const int padw = 4 * ((n + 4) >> 2) - (n + 1);
      if (padw > 0)
#pragma unroll 1
        for (int k = lane; k < (m + 1) * padw; k += 32) {
          const int i = k / padw;
          T[i * S + n + 1 + (k - i * padw)] = 0.f;
        }
    }
    bad = __any_sync(kFull, bad);
    if (bad) {             // the shared-memory kernel handles it (Phase I, sizes, bad data)
      if (lane == 0) {
        P.R.status[lp] = STATUS_PENDING;
        list_push(P.defer_items, P.defer_count, P.list_cap, lp, P.err);
      }
      item = nitem; lp = nlp; m = nm; n = nn; aoff = na; boff = nb; coff = nc;
      __syncwarp();
      continue;
    }
    bm = warp_max_u64(bm <= kInf ? bm : 0ull);      // NaN magnitudes take no part
    cm = warp_max_u64(cm < kInf ? cm : 0ull);
    __syncwarp();

    // ---- Steps 1-3 ----
    const int max_iter = P.max_iter > 0 ? P.max_iter : 50 * (m + n);
    const int nbu = (n + 4) >> 2;              // 16-byte blocks holding columns 0..n
    int iters = 0, status = LPB_OPTIMAL, degenerate_run = 0;
    bool bland = false;
    for (;;) {
      // Step 1: column j = lane + 32 s of the objective row.  Candidates are
      // compared on the order-preserving integer image of their value (the
      // random rule's keys are bit patterns that may lie beyond +inf); no
      // candidate is the largest image.
      // The loads that do not depend on the entering column go first: the
      // objective row and the column variables for Step 1, the right-hand
      // side and the row variables for Step 2.
      float rj4[4], rh4[4];
      int nv4[4], bv4[4];
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        const int j = lane + 32 * s;
        rj4[s] = j < n ? T[m * S + j] : 0.f;
        nv4[s] = j < n ? int(nbv[j]) : 0;
        rh4[s] = j < m ? T[j * S + n] : 0.f;
        bv4[s] = j < m ? int(bas[j]) : 0;
      }
      unsigned co = 0xffffffffu;
      int ck = kNoKey;
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        const int j = lane + 32 * s;
        if (j < n) {
          const float rj = rj4[s];
          if (rj < -eps_d) {
            const int v = nv4[s];
            // The random rule ranks by the upper 31 bits of the variable's key,
            // stored as the bits of a non-negative float.
            const float val = bland ? 0.f
                            : P.rule == LPB_PIVOT_RPC ? __uint_as_float(rpc_key(P.seed, P.lp_base + lp, iters, v) >> 1)
                                                      : rj;
            const unsigned o = f2ord(val);
            const int key = (v << kIdxBits) | j;
            if (o < co || (o == co && key < ck)) { co = o; ck = key; }
          }
        }
      }
      float cv = ord2f(co);
      warp_argmin_f32(cv, ck);
      if (ck == kNoKey) { status = LPB_OPTIMAL; break; }
      const int e = ck & kIdxMask;
      // Step 2: the min-ratio test over rows i = lane + 32 s (column e and the
      // right-hand side); a[] keeps column e, with the objective row's entry.
      float tv = __int_as_float(0x7f800000);
      int tk = kNoKey;
      float a[4];
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        const int i = lane + 32 * s;
        a[s] = i <= m ? T[i * S + e] : 0.f;
        if (i < m && a[s] > eps_p) keep_better(tv, tk, rh4[s] * rcp_approx(a[s]), (bv4[s] << kIdxBits) | i);
      }
      warp_argmin_f32(tv, tk);
      if (tk == kNoKey) { status = LPB_UNBOUNDED; break; }
      if (iters >= max_iter) { status = LPB_ITER_LIMIT; break; }
      const int l = tk & kIdxMask, leave_var = tk >> kIdxBits;
      const float rp = __frcp_rn(pick_slot(a, l));
      // Multipliers t_ie / p of every row but the pivot row (0: left alone by
      // the sweep, then scaled).
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        const int i = lane + 32 * s;
        a[s] = i == l ? 0.f : a[s] * rp;
        if (i <= m) colb[i] = a[s];
      }
      float4 pr[U];
      {
        const float *rowl = T + l * S + 4 * cg;
#pragma unroll
        for (int u = 0; u < U; ++u) pr[u] = cg + 4 * u < nbu ? ld4(rowl + 16 * u) : make_float4(0.f, 0.f, 0.f, 0.f);
      }
      __syncwarp();
      // Step 3: rows rg + 8 t stream through two at a time; a row's blocks and
      // multiplier are loaded before the row before it is written.
      sweep_rows<U>(T, S, colb, m, rg, cg, nbu, pr);
      __syncwarp();
      // The pivot row scaled by 1/p from the copy in registers (one lane per
      // column group) with 1/p at column e; column e becomes -t_ie / p.
      if (rg == 0) {
        float *rowl = T + l * S + 4 * cg;
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int c0 = 4 * (cg + 4 * u);
          if (c0 < 4 * nbu) {
            float4 v = pr[u];
            v.x = c0 == e ? rp : v.x * rp;
            v.y = c0 + 1 == e ? rp : v.y * rp;
            v.z = c0 + 2 == e ? rp : v.z * rp;
            v.w = c0 + 3 == e ? rp : v.w * rp;
            st4(rowl + 16 * u, v);
          }
        }
      }
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        const int i = lane + 32 * s;
        if (i <= m && i != l) T[i * S + e] = -a[s];
      }
      if (lane == 0) {
        bas[l] = short(ck >> kIdxBits);
        nbv[e] = short(leave_var);
      }
      __syncwarp();
      ++iters;
      if (tv <= eps_p) {
        if (++degenerate_run >= m + n) bland = true;
      } else {
        degenerate_run = 0;
        bland = false;
      }
    }

    // The next LP's data into L2 now, a refinement's time before its build.
    if (lane == 0 && nitem < nitems && !P.shared && fits_lp(nm, nn)) warp_prefetch(P, nm, nn, na, nb, nc);
    const int64_t yoff = P.R.y_off ? P.R.y_off[lp] : boff;    // outputs packed like b, or at y_off
    int32_t *bp = P.bbuf ? P.bbuf + (P.bpacked ? yoff : int64_t(lp) * P.B.max_m) : nullptr;
    if (bp)
#pragma unroll 1
      for (int i = lane; i < m; i += 32) bp[i] = bas[i];
    if (status != LPB_OPTIMAL || P.mode != MODE_FP32_REFINE) {
      if (status == LPB_OPTIMAL) {           // plain FP32: results straight from the tableau
#pragma unroll
        for (int s = 0; s < 4; ++s) {
          const int j = lane + 32 * s, i = lane + 32 * s;
          if (j < n) {
            const int v = nbv[j];
            if (v < n) P.R.x[coff + v] = 0.0;
            else if (P.R.y) P.R.y[yoff + (v - n)] = f2d_exact(T[m * S + j]);
          }
          if (i < m) {
            const int v = bas[i];
            if (v < n) P.R.x[coff + v] = f2d_exact(T[i * S + n]);
            else if (P.R.y) P.R.y[yoff + (v - n)] = 0.0;
          }
        }
        if (lane == 0) {
          P.R.status[lp] = LPB_OPTIMAL;
          P.R.obj[lp] = f2d_exact(T[m * S + n]);
          if (P.R.iters) P.R.iters[lp] = iters;
        }
      } else if (P.mode == MODE_FP32_REFINE) {   // unbounded / iteration cap: confirm in FP64
        if (lane == 0) {
          P.R.status[lp] = STATUS_PENDING;
          if (P.R.iters) P.R.iters[lp] = iters;
          list_push(P.resolve_items, P.resolve_count, P.list_cap, lp, P.err);
        }
      } else {                                   // plain FP32: final as found
#pragma unroll 1
        for (int j = lane; j < n; j += 32) P.R.x[coff + j] = 0.0;
        if (P.R.y)
#pragma unroll 1
          for (int i = lane; i < m; i += 32) P.R.y[yoff + i] = 0.0;
        if (lane == 0) {
          P.R.status[lp] = status;
          if (P.R.iters) P.R.iters[lp] = iters;
          P.R.obj[lp] = status == LPB_UNBOUNDED ? INFINITY : NAN;
        }
      }
      item = nitem; lp = nlp; m = nm; n = nn; aoff = na; boff = nb; coff = nc;
      __syncwarp();
      continue;
    }

    // ---- FP64 refinement and certificate ----
    // Lists by ballot: sbl[q] is the row of the q-th basic structural, nsl[p]
    // the column of the p-th non-basic slack (as many as basic structurals).
    int k = 0, kn = 0;
#pragma unroll 1
    for (int i0 = 0; i0 < m; i0 += 32) {
      const int i = i0 + lane;
      const bool in = i < m && bas[i] < n;
      const unsigned mk = __ballot_sync(kFull, in);
      if (in) sbl[k + __popc(mk & ((1u << lane) - 1u))] = short(i);
      k += __popc(mk);
    }
#pragma unroll 1
    for (int j0 = 0; j0 < n; j0 += 32) {
      const int j = j0 + lane;
      const bool in = j < n && nbv[j] >= n;
      const unsigned mk = __ballot_sync(kFull, in);
      if (in) nsl[kn + __popc(mk & ((1u << lane) - 1u))] = short(j);
      kn += __popc(mk);
    }
    __syncwarp();
    // The refinement's operands and state on chip: the tableau is dead after
    // the pivots but for its right-hand side, its objective row and the
    // non-basic slacks' columns.  The latter move to the start of the region
    // (compacted, odd stride); the entries of A that the products read follow
    // (A's basic columns, k x m column-major, and the non-basic slacks' rows,
    // k x n, gathered by asynchronous copies in one round trip with b and c),
    // then the FP64 state: x of each row's basic variable, b - A x and the
    // residual by row, the reduced costs by column, y by non-basic slack, and
    // per-q / per-p values that the inner loops read by broadcast.  An LP with
    // more than kRefK basic structurals, or whose operands do not fit, goes to
    // the FP64 re-solve instead.
    const int ks = kn | 1;                    // odd strides: no bank conflicts
    const int off_ac = (m * ks * 4 + 15) & ~15;
    const int off_ar = off_ac + m * ks * 8;
    const int off_bc = off_ar + kn * n * 8;
    const int off_st = off_bc + (m + n) * 8;
    if (kn > kRefK || off_st + (3 * m + n + 2 * kRefK) * 8 + 3 * kRefK * 4 > L.tab) {
      if (lane == 0) {
        P.R.status[lp] = STATUS_PENDING;
        if (P.R.iters) P.R.iters[lp] = iters;
        list_push(P.resolve_items, P.resolve_count, P.list_cap, lp, P.err);
      }
      item = nitem; lp = nlp; m = nm; n = nn; aoff = na; boff = nb; coff = nc;
      __syncwarp();
      continue;
    }
    // x_B and y from the FP32 tableau, before the region is reused.
    float xf[4], yf = 0.f;
#pragma unroll
    for (int s = 0; s < 4; ++s) xf[s] = lane + 32 * s < m ? T[(lane + 32 * s) * S + n] : 0.f;
    if (lane < kn) yf = T[m * S + nsl[lane]];
    float *tcomp = T;                                                    // [m][ks]
    double *ac = reinterpret_cast<double *>(base + off_ac);              // [m][ks]: A[i, j_q]
    double *ar = reinterpret_cast<double *>(base + off_ar);              // [kn][n]
    double *bsm = reinterpret_cast<double *>(base + off_bc);             // b [m], then c [n]
    double *csm = bsm + m;
    double *xrow = reinterpret_cast<double *>(base + off_st);            // x of row t's basic variable
    double *saxs = xrow + m;                                             // b - A x by row
    double *rrd = saxs + m;                                              // residual r by row
    double *djs = rrd + m;                                               // reduced cost by column
    double *yqs = djs + n;                                               // y of the p-th non-basic slack
    double *xq = yqs + kRefK;                                            // x of the q-th basic structural
    float *coef = reinterpret_cast<float *>(xq + kRefK);                 // r of the p-th non-basic slack
    float *dq = coef + kRefK;                                            // dx of the q-th basic structural
    int *krl = reinterpret_cast<int *>(dq + kRefK);                      // row of A of the p-th non-basic slack
    // Compaction in row order, lane p taking column p (with at most 16 columns
    // the half-warps take alternate rows, eight rows a step, else four):
    // compacted rows up to i end before tableau row i + 1 starts (ks < S), so
    // no row is overwritten unread.
    const bool halves = kn <= 16;             // per-column work in both half-warps
    {
      const int p = halves ? (lane & 15) : lane, h = halves ? (lane >> 4) : 0, dr = halves ? 2 : 1;
      const int c = p < kn ? int(nsl[p]) : 0;
#pragma unroll 1
      for (int i0 = 0; i0 < m; i0 += 4 * dr) {
        float v[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          const int i = i0 + h + dr * r;
          v[r] = (p < kn && i < m) ? T[i * S + c] : 0.f;
        }
        __syncwarp();
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          const int i = i0 + h + dr * r;
          if (p < kn && i < m) tcomp[i * ks + p] = v[r];
        }
        __syncwarp();
      }
    }
    {
      const double *Ad = static_cast<const double *>(P.B.A) + aoff;
      // A's basic columns row by row, lane q taking column j_q (with at most 16
      // columns the half-warps take alternate rows): one copy instruction
      // touches only one or two rows' lines.
      {
        const int q = halves ? (lane & 15) : lane, h = halves ? (lane >> 4) : 0, dr = halves ? 2 : 1;
        if (q < k) {
          const double *src = Ad + bas[sbl[q]] + static_cast<long long>(h) * n;
          double *dst = ac + h * ks + q;
#pragma unroll 1
          for (int i = h; i < m; i += dr, src += static_cast<long long>(dr) * n, dst += dr * ks) cp_async8(dst, src);
        }
      }
#pragma unroll 1
      for (int p = 0; p < kn; ++p) {
        const int r = nbv[nsl[p]] - n;
#pragma unroll 1
        for (int j = lane; j < n; j += 32) cp_async8(ar + p * n + j, Ad + static_cast<long long>(r) * n + j);
      }
      const double *bg = static_cast<const double *>(P.B.b) + boff;
      const double *cg64 = static_cast<const double *>(P.B.c) + coff;
#pragma unroll 1
      for (int i = lane; i < m; i += 32) cp_async8(bsm + i, bg + i);
#pragma unroll 1
      for (int j = lane; j < n; j += 32) cp_async8(csm + j, cg64 + j);
    }
#pragma unroll
    for (int s = 0; s < 4; ++s)
      if (lane + 32 * s < m) xrow[lane + 32 * s] = f2d_exact(xf[s]);
    if (lane < kn) {
      yqs[lane] = f2d_exact(yf);
      krl[lane] = nbv[nsl[lane]] - n;
    }
    cp_async_wait_all();
    __syncwarp();
    const double tol = P.feas_tol;
    const double tp = tol * (1.0 + __longlong_as_double(static_cast<long long>(bm)));
    const double td = tol * (1.0 + __longlong_as_double(static_cast<long long>(cm)));
    constexpr float kDeltaErr = 1.f / 32768.f;
    int fail = 0;
    double cx = 0.0;
    for (int round = 0;; ++round) {
      // Row residuals in FP64: b_i - sum_q A[i, j_q] x_q over the basic
      // structurals, and r_i: that minus x of slack i when it is basic.
      // Here and below a lane takes rows (columns) i and i + 32 together; where
      // i + 32 is past the end the second chain repeats row i and is dropped.
      if (lane < k) xq[lane] = xrow[sbl[lane]];
      __syncwarp();
      for (int i = lane; i < m; i += 64) {
        const int i2 = i + 32 < m ? i + 32 : i;
        const double *a1 = ac + i * ks, *a2 = ac + i2 * ks;
        double s1 = 0.0, s2 = 0.0;
#pragma unroll 1
        for (int q = 0; q < k; ++q) {
          const double xv = xq[q];
          s1 = fma(a1[q], xv, s1);
          s2 = fma(a2[q], xv, s2);
        }
        saxs[i] = bsm[i] - s1;
        xs[i] = 0.0;
        if (i2 != i) {
          saxs[i2] = bsm[i2] - s2;
          xs[i2] = 0.0;
        }
      }
      __syncwarp();
#pragma unroll 1
      for (int t = lane; t < m; t += 32)
        if (bas[t] >= n) xs[bas[t] - n] = xrow[t];
      __syncwarp();
#pragma unroll 1
      for (int i = lane; i < m; i += 32) rrd[i] = saxs[i] - xs[i];
      __syncwarp();                           // xs (over colb and rr) is rewritten below
#pragma unroll 1
      for (int i = lane; i < m; i += 32) rrs[i] = d2f_rn(rrd[i]);
      // Reduced costs in FP64: d_j = sum_p A[k_p, j] y_p - c_j.
      for (int j = lane; j < n; j += 64) {
        const int j2 = j + 32 < n ? j + 32 : j;
        double s1 = 0.0, s2 = 0.0;
#pragma unroll 1
        for (int p = 0; p < kn; ++p) {
          const double yv = yqs[p];
          s1 = fma(ar[p * n + j], yv, s1);
          s2 = fma(ar[p * n + j2], yv, s2);
        }
        const double d = s1 - csm[j];
        djs[j] = d;
        dxs[j] = d2f_rn(neg_bits(d));         // -d_j by column, for rho below
        if (j2 != j) {
          const double d2 = s2 - csm[j2];
          djs[j2] = d2;
          dxs[j2] = d2f_rn(neg_bits(d2));
        }
      }
      __syncwarp();
      // rho_t = -d of the basic structural of row t (0 for a basic slack); the
      // residuals of the non-basic slacks, by p.
#pragma unroll 1
      for (int t = lane; t < m; t += 32) colb[t] = bas[t] < n ? dxs[bas[t]] : 0.f;
      if (lane < kn) coef[lane] = rrs[krl[lane]];
      __syncwarp();
      // Corrections with the FP32 basis inverse, whose column for slack k is the
      // tableau column of k when k is non-basic, else a unit vector:
      //   dx_t = sum_p T[t, c_p] r_{k_p} (+ r of the slack itself in a basic slack's row).
      for (int t = lane; t < m; t += 64) {
        const int t2 = t + 32 < m ? t + 32 : t;
        float s1 = 0.f, s2 = 0.f;
#pragma unroll 1
        for (int p = 0; p < kn; ++p) {
          const float cv = coef[p];
          s1 = fmaf(tcomp[t * ks + p], cv, s1);
          s2 = fmaf(tcomp[t2 * ks + p], cv, s2);
        }
        const int v = bas[t];
        const double d = f2d_exact(s1);
        xrow[t] += v >= n ? d + rrd[v - n] : d;
        dxs[t] = v < n ? s1 : 0.f;             // the structural part of the correction
        if (t2 != t) {
          const int v2 = bas[t2];
          const double d2 = f2d_exact(s2);
          xrow[t2] += v2 >= n ? d2 + rrd[v2 - n] : d2;
          dxs[t2] = v2 < n ? s2 : 0.f;
        }
      }
      // dy_p = sum_t T[t, c_p] rho_t for the non-basic slacks (kn <= 32); with
      // at most 16 the half-warps sum alternate rows and add their totals.
      {
        const int p = halves ? (lane & 15) : lane, h = halves ? (lane >> 4) : 0, dr = halves ? 2 : 1;
        float a0 = 0.f, a1 = 0.f;
        if (p < kn) {
          int t = h;
#pragma unroll 1
          for (; t + dr < m; t += 2 * dr) {
            a0 = fmaf(tcomp[t * ks + p], colb[t], a0);
            a1 = fmaf(tcomp[(t + dr) * ks + p], colb[t + dr], a1);
          }
          if (t < m) a0 = fmaf(tcomp[t * ks + p], colb[t], a0);
        }
        float dy = a0 + a1;
        if (halves) dy += __shfl_xor_sync(kFull, dy, 16);
        if (lane < kn) {
          yqs[lane] += f2d_exact(dy);
          coef[lane] = dy;                     // dy of the p-th non-basic slack, for the certificate
        }
      }
      __syncwarp();
      if (lane < k) dq[lane] = dxs[sbl[lane]];
      __syncwarp();
      // KKT certificate of the pair that is written out (x: the structural part
      // of x_B; y: the slack duals): x >= 0, A x <= b, y >= 0, A^T y >= c and
      // c^T x = b^T y, each to tol scaled by the data.  b - A x and A^T y - c at
      // the corrected point are the FP64 values above plus FP32 products with
      // the corrections, whose rounding (and the 2^-20 truncation of A) is
      // bounded by 2^-15 times the sum of the products' magnitudes.
      fail = 0;
      double cxp = 0.0, byp = 0.0;
      for (int i = lane; i < m; i += 64) {      // x >= 0, and the slack b_i - A_i x of every row
        const int i2 = i + 32 < m ? i + 32 : i;
        const unsigned *h1 = reinterpret_cast<const unsigned *>(ac + i * ks) + 1;
        const unsigned *h2 = reinterpret_cast<const unsigned *>(ac + i2 * ks) + 1;
        float dl = 0.f, mg = 0.f, dl2 = 0.f, mg2 = 0.f;
#pragma unroll 1
        for (int q = 0; q < k; ++q) {
          const float d = dq[q], ad = fabsf(d);
          const float a = hi2f(h1[2 * q]), a2 = hi2f(h2[2 * q]);
          dl = fmaf(a, d, dl);
          mg = fmaf(fabsf(a), ad, mg);
          dl2 = fmaf(a2, d, dl2);
          mg2 = fmaf(fabsf(a2), ad, mg2);
        }
        const int v = bas[i];
        if (v < n) {
          fail |= !dge(xrow[i], neg_bits(tp));
          cxp = fma(csm[v], xrow[i], cxp);
        }
        fail |= !dge(saxs[i] - f2d_exact(dl + kDeltaErr * mg), neg_bits(tp));
        if (i2 != i) {
          const int v2 = bas[i2];
          if (v2 < n) {
            fail |= !dge(xrow[i2], neg_bits(tp));
            cxp = fma(csm[v2], xrow[i2], cxp);
          }
          fail |= !dge(saxs[i2] - f2d_exact(dl2 + kDeltaErr * mg2), neg_bits(tp));
        }
      }
      if (lane < kn) {                          // y >= 0
        fail |= !dge(yqs[lane], neg_bits(td));
        byp = fma(bsm[krl[lane]], yqs[lane], byp);
      }
      for (int j = lane; j < n; j += 64) {      // reduced cost A_j^T y - c_j of every column
        const int j2 = j + 32 < n ? j + 32 : j;
        float dl = 0.f, mg = 0.f, dl2 = 0.f, mg2 = 0.f;
#pragma unroll 1
        for (int p = 0; p < kn; ++p) {
          const unsigned *h = reinterpret_cast<const unsigned *>(ar + p * n) + 1;
          const float d = coef[p], ad = fabsf(d);
          const float a = hi2f(h[2 * j]), a2 = hi2f(h[2 * j2]);
          dl = fmaf(a, d, dl);
          mg = fmaf(fabsf(a), ad, mg);
          dl2 = fmaf(a2, d, dl2);
          mg2 = fmaf(fabsf(a2), ad, mg2);
        }
        fail |= !dge(djs[j] + f2d_exact(dl - kDeltaErr * mg), neg_bits(td));
        if (j2 != j) fail |= !dge(djs[j2] + f2d_exact(dl2 - kDeltaErr * mg2), neg_bits(td));
      }
      cx = warp_sum(cxp);
      const double by = warp_sum(byp);
      fail |= !(fabs(cx - by) <= tol * (1.0 + fabs(cx)));
      fail = __any_sync(kFull, fail);
      if (!fail || round == 2) break;
      __syncwarp();          // the scratch arrays are rewritten by the next round
    }
    if (!fail) {
#pragma unroll 1
      for (int j = lane; j < n; j += 32)
        if (nbv[j] < n) P.R.x[coff + nbv[j]] = 0.0;
#pragma unroll 1
      for (int t = lane; t < m; t += 32) {
        const int v = bas[t];
        if (v < n) P.R.x[coff + v] = xrow[t];
        else if (P.R.y) P.R.y[yoff + (v - n)] = 0.0;
      }
      if (P.R.y && lane < kn) P.R.y[yoff + krl[lane]] = yqs[lane];
    }
    if (lane == 0) {
      if (!fail) {
        P.R.status[lp] = LPB_OPTIMAL;
        P.R.obj[lp] = cx;
      } else {
        P.R.status[lp] = STATUS_PENDING;
        list_push(P.resolve_items, P.resolve_count, P.list_cap, lp, P.err);
      }
      if (P.R.iters) P.R.iters[lp] = iters;
    }
    item = nitem; lp = nlp; m = nm; n = nn; aoff = na; boff = nb; coff = nc;
    __syncwarp();
  }
}

template <int U>
const void *warp_fn() {
  return reinterpret_cast<const void *>(&warp_kernel<U>);
}

// Column blocks per lane for LPs up to max_n columns (n + 1 <= 16 U).
int warp_u(int max_n) {
  int u = ((max_n + 1 + 3) / 4 + 3) / 4;
  return u < 2 ? 2 : u;
}

const void *warp_kernel_for(int u) {
  switch (u) {
    case 2: return warp_fn<2>();
    case 3: return warp_fn<3>();
    case 4: return warp_fn<4>();
    case 5: return warp_fn<5>();
    case 6: return warp_fn<6>();
    case 7: return warp_fn<7>();
    case 8: return warp_fn<8>();
    default: return nullptr;
  }
}

}  // namespace

bool warp_fits(int max_m, int max_n) {
  return max_m >= 1 && max_n >= 1 && max_m <= kWarpMaxDim && max_n <= kWarpMaxDim;
}

// Warps (LPs) per CTA and shared memory of the warp kernel for LPs up to
// max_m x max_n: as many warps as the SM's shared memory holds regions, at most
// eight; CTAs per SM from the occupancy calculator.
cudaError_t warp_occupancy(int max_m, int max_n, int *ctas, int *threads, size_t *smem) {
  *ctas = 0;
  if (!warp_fits(max_m, max_n)) return cudaErrorInvalidValue;
  const WarpLayout L = warp_layout(max_m, max_n);
  int nw = int(size_t(232448) / size_t(L.bytes));
  if (nw > kWarpMaxWarps) nw = kWarpMaxWarps;
  if (nw < 1) return cudaSuccess;
  *threads = 32 * nw;
  *smem = size_t(nw) * size_t(L.bytes);
  const void *fn = warp_kernel_for(warp_u(max_n));
  if (!fn) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(*smem));
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas, fn, *threads, *smem);
}

cudaError_t launch_warp(const TableauParams &p, int grid, int threads, size_t smem, cudaStream_t s) {
  if (!warp_fits(p.lim_m, p.lim_n)) return cudaErrorInvalidValue;
  const WarpLayout L = warp_layout(p.lim_m, p.lim_n);
  if (size_t(threads / 32) * size_t(L.bytes) > smem) return cudaErrorInvalidValue;
  const void *fn = warp_kernel_for(warp_u(p.lim_n));
  if (!fn) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (e != cudaSuccess) return e;
  WarpLayout lay = L;
  void *args[] = {const_cast<TableauParams *>(&p), &lay};
  return cudaLaunchKernel(fn, dim3(grid), dim3(threads), args, smem, s);
}

}  // namespace lpb
