// simplex_pack.cu -- several tiny LPs per warp: the FP32 register tableau of
// an LP with m, n <= S - 1 lives in a segment of S lanes (S = 8: four LPs per
// warp; S = 16: two; S = 32: one), with the FP64 refinement and certificate
// fused in.
//
// Section 3.1 Steps 1-3 in the compact (exchange) tableau of each LP.  Lane
// i < S - 1 of a segment holds constraint row i, lane S - 1 the objective row
// (r = -c at the start); register column c < S - 1 is non-basic variable
// column c and column S - 1 the right-hand side.  Rows and columns beyond the
// LP's m and n are zero and stay zero under pivoting.  Every reduction is a
// butterfly of shuffles over xor offsets below S, so it stays inside the
// segment; the segments of a warp pivot in lockstep until the last of them is
// done (a finished segment's lanes idle).  One FP64 warp instruction of the
// refinement then serves 32 / S LPs, which is what bounds tiny LPs on this
// GPU (its FP64 unit runs at a small fraction of the FP32 rate).
//
// Rules: Step 1 takes the most negative reduced cost (ties: lowest variable
// index), the random-key rule, or Bland's lowest eligible index after m + n
// degenerate pivots; Step 2 the least ratio over t_ie > eps_p (ties: lowest
// basic-variable index).  LPs with some b_i < 0 (Phase I) or non-finite data
// are deferred to the shared-memory kernel; unbounded and capped LPs in
// FP32+refine mode, and optima that fail the FP64 certificate after three
// corrections, go to the FP64 re-solve.
#include "lpb_internal.cuh"

namespace lpb {
namespace {

constexpr int kPackWarps = 4;          // warps per CTA; each warp works on its own
constexpr int kNone = 1 << 30;         // a key larger than any real key
constexpr int kPackRounds = 3;         // refinement corrections before an LP is re-solved in FP64

// Per-warp scratch in shared memory (G = 32 / S segments).
template <int S>
struct PackWarp {
  static constexpr int G = 32 / S;
  alignas(16) float objv[G][S];        // the objective row, published for Step 1
  int nvs[G][S];                       // variable of each non-basic column
  int sbj[G][S];                       // the basic structural variables (their column of A)
  int nsk[G][S];                       // the rows whose slack is non-basic (binding rows)
  int nsc[G][S];                       // ... and the tableau column of that slack
  double xv[G][2 * S];                 // value of every variable: structural j at j, slack k at S + k
  double yv[G][S];                     // duals of the rows
  double rr[G][S];                     // FP64 primal residuals b - A x - s
  float rf[G][S];                      // the same in FP32
  float tf[G][S][S + 1];               // the final FP32 tableau, row sl of segment seg at tf[seg][sl]
  float rh[G][S];                      // FP32 dual residual rho_i of each row
};

// Butterfly arg-min over the S lanes of a segment: (value, key) order with the
// value compared through its order-preserving integer image.
template <int S>
__device__ __forceinline__ void seg_argmin(float &v, int &k) {
  unsigned o = f2ord(v);
#pragma unroll
  for (int off = S / 2; off > 0; off >>= 1) {
    const unsigned oo = __shfl_xor_sync(kFull, o, off);
    const int ok = __shfl_xor_sync(kFull, k, off);
    if (oo < o || (oo == o && ok < k)) { o = oo; k = ok; }
  }
  v = ord2f(o);
}

template <int S>
__device__ __forceinline__ double seg_sum(double v) {
#pragma unroll
  for (int off = S / 2; off > 0; off >>= 1) v += __shfl_xor_sync(kFull, v, off);
  return v;
}

template <int S>
__device__ __forceinline__ unsigned seg_max(unsigned v) {
#pragma unroll
  for (int off = S / 2; off > 0; off >>= 1) v = max(v, __shfl_xor_sync(kFull, v, off));
  return v;
}

// Register T[c] for a segment-uniform column c (a select chain: no local memory).
template <int S>
__device__ __forceinline__ float pick(const float (&T)[S], int c) {
  float v = T[0];
#pragma unroll
  for (int k = 1; k < S; ++k) v = (c == k) ? T[k] : v;
  return v;
}

// Magnitude bits of a double's high word (|d| orders like these for finite d).
__device__ __forceinline__ unsigned hi_mag(double d) {
  return unsigned(static_cast<unsigned long long>(__double_as_longlong(d)) >> 32) & 0x7fffffffu;
}

template <int S>
__global__ void __launch_bounds__(kPackWarps * 32) pack_kernel(TableauParams P) {
  constexpr int G = 32 / S;
  __shared__ PackWarp<S> shw[kPackWarps];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  PackWarp<S> &sh = shw[wid];
  const int seg = lane / S, sl = lane % S, base = seg * S;
  const unsigned segmask = (S == 32 ? kFull : ((1u << S) - 1u)) << base;
  const float eps_p = float(P.eps_p), eps_d = float(P.eps_d);
  const int dt = P.B.dtype;
  const int nitems = P.in.count ? min(*P.in.count, P.list_cap) : P.B.count;
  const bool refine = P.mode == MODE_FP32_REFINE;

  // Every loop below is bounded by construction (the work queue, the pivot
  // cap, the refinement rounds); each also carries an explicit guard that
  // records ERR_BAD_LAUNCH and leaves should that reasoning ever fail.
  const int group_cap = nitems / G + 2;
  for (int guard = 0;; ++guard) {
    if (guard > group_cap) {
      if (lane == 0) atomicOr(P.err, ERR_BAD_LAUNCH);
      break;
    }
    int grp = 0;
    if (lane == 0) grp = atomicAdd(P.queue, 1);
    grp = __shfl_sync(kFull, grp, 0);
    if (grp * G >= nitems) break;
    // ---- this segment's LP ----
    const int item = grp * G + seg;
    int lp = -1, m = 0, n = 0;
    int64_t aoff = 0, boff = 0, coff = 0;
    if (item < nitems) {
      lp = P.in.items ? P.in.items[item] : item;
      m = P.B.m[lp];
      n = P.B.n[lp];
      aoff = P.B.a_off[lp];
      boff = P.B.b_off[lp];
      coff = P.B.c_off[lp];
    }
    const bool fits = lp >= 0 && m >= 1 && n >= 1 && m <= S - 1 && n <= S - 1 && m <= P.B.max_m &&
                      n <= P.B.max_n && m <= P.lim_m && n <= P.lim_n;
    // ---- the tableau: A rounded to FP32, b in column S-1, -c in row S-1 ----
    float T[S];
#pragma unroll
    for (int c = 0; c < S; ++c) T[c] = 0.f;
    double bk = 0.0, cj = 0.0;          // b of row sl, c of column sl (as given, in FP64)
    int bad = 0;
    unsigned bmax = 0u, cmax = 0u;
    if (fits) {
      if (sl < m) {
#pragma unroll
        for (int c = 0; c < S - 1; ++c) {
          if (c < n) {
            const double a = ld_in(P.B.A, aoff + int64_t(sl) * n + c, dt);
            bad |= !finite_bits(a);
            T[c] = d2f_rn(a);
          }
        }
        bk = ld_in(P.B.b, boff + sl, dt);
        bad |= !finite_bits(bk) || !dge(bk, -0.0);      // b_i < 0: Phase I elsewhere
        T[S - 1] = d2f_rn(bk);
        bmax = hi_mag(bk);
      }
      if (sl < n) {
        cj = ld_in(P.B.c, coff + sl, dt);
        bad |= !finite_bits(cj);
        cmax = hi_mag(cj);
      }
    }
    // The objective row: lane S-1 takes -c from the lanes holding c.
#pragma unroll
    for (int c = 0; c < S - 1; ++c) {
      const float v = -d2f_rn(__shfl_sync(kFull, cj, base + c));
      if (sl == S - 1 && c < n) T[c] = v;
    }
    // Every lane takes part in each warp-wide vote and shuffle (never behind a
    // short-circuit or a lane-dependent branch): lanes of empty segments too.
    const unsigned bad_lanes = __ballot_sync(kFull, bad);
    const bool defer = fits && (bad_lanes & segmask) != 0u;
    bmax = seg_max<S>(bmax);
    cmax = seg_max<S>(cmax);
    bool act = fits && !defer;                    // this segment is pivoting
    if (defer && sl == 0) {
      P.R.status[lp] = STATUS_PENDING;
      list_push(P.defer_items, P.defer_count, P.list_cap, lp, P.err);
    }
    int bvar = (act && sl < m) ? n + sl : kNone >> kIdxBits;   // basic variable of row sl
    int nv = (act && sl < n) ? sl : kNone >> kIdxBits;        // variable of non-basic column sl
    const int max_iter = P.max_iter > 0 ? P.max_iter : 50 * (m + n);
    int iters = 0, status = LPB_OPTIMAL, degenerate_run = 0;
    bool bland = false;

    // ---- Steps 1-3, all segments in lockstep ----
    const int pivot_cap = (P.max_iter > 0 ? P.max_iter : 100 * S) + 2;
    for (int guard = 0; __any_sync(kFull, act); ++guard) {
      if (guard > pivot_cap) {
        if (lane == 0) atomicOr(P.err, ERR_BAD_LAUNCH);
        act = false;
        status = LPB_ITER_LIMIT;
        break;
      }
      // Step 1: lane S-1 publishes the objective row; lane c judges column c.
      if (sl == S - 1) {
#pragma unroll
        for (int c = 0; c < S; c += 4)
          *reinterpret_cast<float4 *>(&sh.objv[seg][c]) = make_float4(T[c], T[c + 1], T[c + 2], T[c + 3]);
      }
      __syncwarp();
      float cv = __int_as_float(0x7fffffff);
      int ck = kNone;
      if (act && sl < S - 1 && nv < (kNone >> kIdxBits)) {
        const float rj = sh.objv[seg][sl];
        if (rj < -eps_d) {
          cv = bland ? 0.f
             : P.rule == LPB_PIVOT_RPC ? __uint_as_float(rpc_key(P.seed, P.lp_base + lp, iters, nv) >> 1) : rj;
          ck = (nv << kIdxBits) | sl;
        }
      }
      seg_argmin<S>(cv, ck);
      // Step 2 on the entering column.
      const int ce = ck & kIdxMask;
      const float col = pick<S>(T, ck == kNone ? 0 : ce);
      float tv = __int_as_float(0x7f800000);
      int tk = kNone;
      if (act && ck != kNone && sl < m && col > eps_p)
        tv = T[S - 1] * __frcp_rn(col), tk = (bvar << kIdxBits) | sl;
      seg_argmin<S>(tv, tk);
      const int l = tk & kIdxMask;
      if (act) {
        if (ck == kNone) act = false;                                  // optimal
        else if (tk == kNone) { act = false; status = LPB_UNBOUNDED; }
        else if (iters >= max_iter) { act = false; status = LPB_ITER_LIMIT; }
      }
      // Step 3: the pivot row from lane l, T -= (column / p) (x) row, the
      // pivot row scaled by 1/p, the new column e = -t_ie / p (1/p at the pivot).
      const float p = __shfl_sync(kFull, col, base + (tk == kNone ? 0 : l));
      const int leave_var = __shfl_sync(kFull, bvar, base + (tk == kNone ? 0 : l));
      const float rp = __frcp_rn(p);
      const float g = col * rp;
#pragma unroll
      for (int c = 0; c < S; ++c) {
        const float pr = __shfl_sync(kFull, T[c], base + (tk == kNone ? 0 : l));
        if (act) {
          const float nt = sl == l ? T[c] * rp : fmaf(-g, pr, T[c]);
          T[c] = c == ce ? (sl == l ? rp : -g) : nt;
        }
      }
      if (act) {
        if (sl == l) bvar = ck >> kIdxBits;
        if (sl == ce) nv = leave_var;
        ++iters;
        if (tv <= eps_p) {
          if (++degenerate_run >= m + n) bland = true;
        } else {
          degenerate_run = 0;
          bland = false;
        }
      }
    }
    // The final objective row was published by the last Step 1.
    const int64_t yoff = lp >= 0 ? (P.R.y_off ? P.R.y_off[lp] : boff) : 0;
    int32_t *bp = (lp >= 0 && P.bbuf) ? P.bbuf + (P.bpacked ? yoff : int64_t(lp) * P.B.max_m) : nullptr;
    const bool solved = fits && !defer;
    if (solved && bp && sl < m) bp[sl] = bvar;
    sh.nvs[seg][sl] = nv;
    // Compact lists for the FP64 residuals: A x needs only the basic
    // structural columns, A^T y only the binding rows (y is zero elsewhere).
    const unsigned below = segmask & ((1u << lane) - 1u);
    const unsigned sb_lanes = __ballot_sync(kFull, sl < m && bvar < n) & segmask;
    const unsigned nk_lanes = __ballot_sync(kFull, sl < S - 1 && nv >= n && nv < n + m) & segmask;
    if (sl < m && bvar < n) sh.sbj[seg][__popc(sb_lanes & below)] = bvar;
    if (sl < S - 1 && nv >= n && nv < n + m) {
      sh.nsk[seg][__popc(nk_lanes & below)] = nv - n;
      sh.nsc[seg][__popc(nk_lanes & below)] = sl;
    }
    // The refinement reads the final tableau from shared memory with runtime
    // indices: its loops then stay rolled (the unrolled register form of every
    // S-wide loop made the code outgrow the instruction cache at S = 32).
    if (refine) {
#pragma unroll
      for (int c = 0; c < S; ++c) sh.tf[seg][sl][c] = T[c];
    }
    const int nsb = __popc(sb_lanes), nnk = __popc(nk_lanes);
    __syncwarp();

    // ---- results: plain FP32, or FP64 refinement and certificate ----
    bool cert = solved && status == LPB_OPTIMAL && refine;
    if (solved && !cert) {
      if (status == LPB_OPTIMAL) {                 // plain FP32: straight from the tableau
        if (sl < n) P.R.x[coff + sl] = 0.0;
        __syncwarp(segmask);
        if (sl < m && bvar < n) P.R.x[coff + bvar] = double(T[S - 1]);
        if (P.R.y && sl < m) P.R.y[yoff + sl] = 0.0;
        __syncwarp(segmask);
        if (P.R.y && sl < S - 1 && nv >= n && nv < n + m) P.R.y[yoff + (nv - n)] = double(sh.objv[seg][sl]);
        if (sl == S - 1) {
          P.R.status[lp] = LPB_OPTIMAL;
          P.R.obj[lp] = double(T[S - 1]);
          if (P.R.iters) P.R.iters[lp] = iters;
        }
      } else if (refine) {                         // unbounded / capped: confirm in FP64
        if (sl == 0) {
          P.R.status[lp] = STATUS_PENDING;
          if (P.R.iters) P.R.iters[lp] = iters;
          list_push(P.resolve_items, P.resolve_count, P.list_cap, lp, P.err);
        }
      } else {
        if (sl < n) P.R.x[coff + sl] = 0.0;
        if (P.R.y && sl < m) P.R.y[yoff + sl] = 0.0;
        if (sl == 0) {
          P.R.status[lp] = status;
          if (P.R.iters) P.R.iters[lp] = iters;
          P.R.obj[lp] = status == LPB_UNBOUNDED ? INFINITY : NAN;
        }
      }
    }
    // Refinement: x_B and y start from the FP32 tableau; each round forms the
    // FP64 residuals at the current point, checks the certificate (from the
    // second round on: x >= 0, A x <= b, y >= 0, A^T y >= c, c^T x = b^T y,
    // each to feas_tol scaled by the data), and if it fails applies one
    // correction with the FP32 basis inverse held in the registers: B^{-1} e_k
    // is the tableau column of slack k when k is non-basic, else the unit
    // vector of its row.
    const double tp = P.feas_tol * (1.0 + __longlong_as_double(static_cast<long long>(bmax) << 32));
    const double td = P.feas_tol * (1.0 + __longlong_as_double(static_cast<long long>(cmax) << 32));
    const double mtp = neg_bits(tp), mtd = neg_bits(td);
    double xb = (cert && sl < m) ? f2d_exact(T[S - 1]) : 0.0;       // value of the basic variable of row sl
    if (cert && sl < m) sh.yv[seg][sl] = 0.0;
    __syncwarp();
    if (cert && sl < S - 1 && nv >= n && nv < n + m) sh.yv[seg][nv - n] = f2d_exact(sh.objv[seg][sl]);
    bool ok = false;
    double cx = 0.0;
    for (int round = 0; __any_sync(kFull, cert); ++round) {
      if (round > kPackRounds + 1) {
        if (lane == 0) atomicOr(P.err, ERR_BAD_LAUNCH);
        cert = false;
        break;
      }
      // every variable's value at the current point
      if (cert) {
        sh.xv[seg][sl] = 0.0;
        sh.xv[seg][S + sl] = 0.0;
      }
      __syncwarp();
      if (cert && sl < m) sh.xv[seg][bvar < n ? bvar : S + (bvar - n)] = xb;
      __syncwarp();
      // rows: s_i = b_i - A_i x and r_i = s_i - x_slack(i); columns: d_j = A_j^T y - c_j.
      // (The FP64 unit is what bounds tiny LPs: sums start from -b_i and -c_j,
      // signs flip on the bits, and the checks compare doubles as integers.)
      double sax = 0.0, dj = 0.0;
      int fail = 0;
      if (cert && sl < m) {
        double nax = neg_bits(bk);                     // -(b_i - A_i x)
        for (int q = 0; q < nsb; ++q) {
          const int j = sh.sbj[seg][q];
          nax = fma(ld_in(P.B.A, aoff + int64_t(sl) * n + j, dt), sh.xv[seg][j], nax);
        }
        sax = neg_bits(nax);
        const double r = sax - sh.xv[seg][S + sl];
        sh.rr[seg][sl] = r;
        sh.rf[seg][sl] = d2f_rn(r);
        fail |= !dge(sax, mtp) || !dge(sh.yv[seg][sl], mtd) || (bvar < n && !dge(xb, mtp));
      }
      if (cert && sl < n) {
        double ay = neg_bits(cj);
        for (int q = 0; q < nnk; ++q) {
          const int k = sh.nsk[seg][q];
          ay = fma(ld_in(P.B.A, aoff + int64_t(k) * n + sl, dt), sh.yv[seg][k], ay);
        }
        dj = ay;
        fail |= !dge(dj, mtd);
      }
      // duality gap c^T x = b^T y (a segment that has passed keeps its c^T x)
      const double cxr = seg_sum<S>(cert && sl < n ? cj * sh.xv[seg][sl] : 0.0);
      const double by = seg_sum<S>(cert && sl < m ? bk * sh.yv[seg][sl] : 0.0);
      if (cert) cx = cxr;
      if (cert && sl == 0 && round > 0) {
        const double gap = cx - by, lim = P.feas_tol * (1.0 + abs_bits(cx));
        fail |= !dge(lim, abs_bits(gap));
      }
      // The FP32 point itself is never accepted: the certificate bounds the
      // residuals, not the error of x (a small c_j lets x_j err by the FP32
      // rounding), so at least one correction runs first.
      const unsigned fail_lanes = __ballot_sync(kFull, fail);
      const bool segfail = round == 0 || (fail_lanes & segmask) != 0u;
      if (cert && !segfail) { ok = true; cert = false; }
      if (cert && round == kPackRounds) cert = false;          // to the FP64 re-solve
      if (!__any_sync(kFull, cert)) break;
      // Corrections.  Primal: dx_i = sum_c T[i][c] r_k(c) over the non-basic
      // slack columns c (FP32) plus r_k for the basic slack of row i (FP64).
      // Dual: rho_i = -d_j for the basic structural j of row i; dy_k = sum_i
      // T[i][c(k)] rho_i for every non-basic slack k.
      const double djb = __shfl_sync(kFull, dj, base + (bvar < n ? bvar : 0));
      sh.rh[seg][sl] = (cert && sl < m && bvar < n) ? -d2f_rn(djb) : 0.f;
      __syncwarp();
      if (cert && sl < m) {
        float dxf = 0.f;
        for (int q = 0; q < nnk; ++q) dxf = fmaf(sh.tf[seg][sl][sh.nsc[seg][q]], sh.rf[seg][sh.nsk[seg][q]], dxf);
        xb += bvar >= n ? f2d_exact(dxf) + sh.rr[seg][bvar - n] : f2d_exact(dxf);
      }
      if (cert && sl < S - 1 && nv >= n && nv < n + m) {
        float s = 0.f;
        for (int i = 0; i < m; ++i) s = fmaf(sh.tf[seg][i][sl], sh.rh[seg][i], s);
        sh.yv[seg][nv - n] += f2d_exact(s);
      }
      __syncwarp();
    }
    if (solved && status == LPB_OPTIMAL && refine) {
      if (ok) {
        if (sl < n) P.R.x[coff + sl] = sh.xv[seg][sl];
        if (P.R.y && sl < m) P.R.y[yoff + sl] = sh.yv[seg][sl];
        if (sl == 0) {
          P.R.status[lp] = LPB_OPTIMAL;
          P.R.obj[lp] = cx;
        }
      } else if (sl == 0) {
        P.R.status[lp] = STATUS_PENDING;
        list_push(P.resolve_items, P.resolve_count, P.list_cap, lp, P.err);
      }
      if (sl == 0 && P.R.iters) P.R.iters[lp] = iters;
    }
    __syncwarp();
  }
}

}  // namespace

// Lanes per LP for batches whose LPs all have m, n <= max_m, max_n: 8 (four
// LPs per warp) up to 7, 16 (two per warp) up to 15, 32 (one) up to 31; 0 when
// none fits.
int pack_lanes(int max_m, int max_n) {
  if (max_m <= 7 && max_n <= 7) return 8;
  if (max_m <= 15 && max_n <= 15) return 16;
  if (max_m <= 31 && max_n <= 31) return 32;
  return 0;
}

cudaError_t pack_occupancy(int lanes, int *ctas, int *threads) {
  *threads = kPackWarps * 32;
  const void *fn = lanes == 8 ? reinterpret_cast<const void *>(&pack_kernel<8>)
                 : lanes == 16 ? reinterpret_cast<const void *>(&pack_kernel<16>)
                               : reinterpret_cast<const void *>(&pack_kernel<32>);
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas, fn, *threads, 0);
}

cudaError_t launch_pack(const TableauParams &p, int lanes, int grid, cudaStream_t s) {
  if (lanes == 8) pack_kernel<8><<<grid, kPackWarps * 32, 0, s>>>(p);
  else if (lanes == 16) pack_kernel<16><<<grid, kPackWarps * 32, 0, s>>>(p);
  else if (lanes == 32) pack_kernel<32><<<grid, kPackWarps * 32, 0, s>>>(p);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

}  // namespace lpb
