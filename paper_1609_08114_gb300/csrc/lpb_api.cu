// lpb_api.cu -- the C ABI of liblpb (declared in include/lpb.h).
//
// Host side only: argument validation, the pass plan of a solve, workspace
// carving and kernel launches.  Every pass is a fixed-size persistent launch
// whose work list length lives on the device, so a whole lpb_solve is a
// static sequence of memset + kernels with no host synchronisation (it can be
// captured in a CUDA graph).
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "lpb_internal.cuh"

struct lpb_handle {
  int device;
  int sms;
  size_t smem_optin;
  size_t l2_bytes;
  uint32_t *d_err;
  int32_t *d_ctr;   // work queues and list lengths, zeroed by every lpb_solve
  // Kernel timing (lpb_profile_*): one event pair per pass per recorded call.
  static constexpr int kProfMax = 256;
  cudaEvent_t *prof_ev = nullptr;   // [kProfMax * 3 * 2]
  bool prof_ran[kProfMax * 3] = {};
  int prof_cap = 0, prof_n = 0;
  int last_kernels = 0;             // kernel launches of the last lpb_solve
  // Autotuned schedules (lpb_autotune), by batch shape.
  struct Tuned {
    int max_m, max_n, dtype, prec;
    int kernel, threads, reg_warps;
  };
  std::vector<Tuned> tuned;
  // Host-memory pipeline (lpb_solve_host): copy-in and copy-out streams and
  // events per buffer set (input ready, solve done, results out) plus a start
  // event on the caller's stream.
  cudaStream_t s_in = nullptr, s_out = nullptr;
  cudaEvent_t ev_in[2] = {}, ev_comp[2] = {}, ev_out[2] = {}, ev_start = nullptr;
};

namespace {

using namespace lpb;

// Handle counters (the per-pass work queues live in the workspace).
enum { CTR_DEFER = 4, CTR_RESOLVE = 5, CTR_BWD = 6, CTR_N = kCounters };

class DeviceScope {
 public:
  explicit DeviceScope(int dev) {
    cudaGetDevice(&prev_);
    ok_ = cudaSetDevice(dev) == cudaSuccess;
  }
  ~DeviceScope() { cudaSetDevice(prev_); }
  bool ok() const { return ok_; }

 private:
  int prev_ = 0;
  bool ok_ = false;
};

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

enum ListKind { LIST_ALL = 0, LIST_CLASS = 1, LIST_DEFER = 2, LIST_RESOLVE = 3 };

struct Pass {
  bool fp64 = false, gmem = false;
  int kcap = 0, mode = MODE_FP64, grid = 0, threads = 128;
  int reg = -1;              // >= 0: register-resident kernel configuration
  int pack = 0;              // > 0: several LPs per warp, this many lanes per LP
  bool warp = false;         // one warp per LP, the tableau in shared memory
  int list = LIST_ALL, cls = 0;
  int lim_m = 0, lim_n = 0;  // size bounds of the launch
  int group = 0;             // timing group: 0 first solve, 1 Phase-I pass, 2 FP64 re-solve
  size_t smem = 0, slot_bytes = 0, tab_smem = 0;
};

constexpr int kMaxPasses = kMaxClasses + 2;

struct Plan {
  Pass pass[kMaxPasses];
  int npass = 0;
  bool classes = false;      // a classify step splits the batch into size classes
  int nclass = 0;
  int cls_m[kMaxClasses] = {}, cls_n[kMaxClasses] = {};
  bool resolve = false;      // the last pass re-solves FP32 failures in FP64
  bool own_basis = false;    // basis lives in the workspace
  size_t off_defer = 0, off_resolve = 0, off_basis = 0, off_lists = 0, off_hist = 0, off_cctr = 0,
         off_slots = 0, total = 0;
  double eps_p = 0, eps_d = 0, feas_tol = 0;
  double eps_p64 = 0, eps_d64 = 0;     // the FP64 re-solve's: FP64 defaults unless given
};

// Threads per CTA of the tableau kernel: about 1024 threads per SM (512 for
// FP64, whose update is bound by the FP64 pipe and whose per-warp divisions
// cost more with more warps) over the CTAs that fit by shared memory, and no
// more than one thread per 8 tableau elements for small LPs.  The kernel is compiled for up to 1024 threads of
// at most 64 registers, so 1024 threads fill the register file.
int auto_threads(int eb, int rows, int cols, size_t smem) {
  int ctas = int(size_t(232448) / (smem + 1024));
  if (ctas < 1) ctas = 1;
  if (ctas > 8) ctas = 8;
  int t = (eb == 8 ? 512 : 1024) / ctas;
  const long long per8 = (static_cast<long long>(rows) * cols / 8 + 31) & ~31LL;
  if (per8 < t) t = int(per8);
  t &= ~31;
  if (t < 64) t = 64;
  return t;
}

// A pass of the tableau kernel.  Its tableau rows go to shared memory as far
// as they fit (all of them for the SMEM class), the rest to a per-CTA slot of
// the workspace, sized so that the slots of all CTAs stay within about 3/4 of
// L2; LPB_KERNEL_GMEM puts every row in the slot.
lpb_err make_pass(const DeviceInfo &d, const lpb_batch *b, const lpb_options *o, bool fp64, int kcap,
                  int mode, Pass *p) {
  const int eb = fp64 ? 8 : 4;
  const bool refine = (mode == MODE_FP32_REFINE) && !fp64;
  p->fp64 = fp64;
  p->kcap = kcap;
  p->mode = mode;
  const size_t fixed = tableau_fixed_bytes(eb, b->max_m, b->max_n, kcap, refine);
  const size_t rowb = tableau_row_bytes(eb, b->max_n, kcap);
  const size_t rows = size_t(b->max_m) + 2;
  // Leave room for the kernel's static shared memory.
  const size_t budget = d.smem_optin > 2048 ? d.smem_optin - 2048 : 0;
  if (fixed + 16 > budget) return LPB_EUNSUPPORTED;
  size_t fit_rows = (budget - fixed) / rowb;
  if (fit_rows > rows) fit_rows = rows;
  if (o->kernel == LPB_KERNEL_SMEM && fit_rows < rows) return LPB_EUNSUPPORTED;
  if (o->kernel == LPB_KERNEL_GMEM) fit_rows = 0;
  // With many LPs, two CTAs per SM hide more latency than one CTA with more
  // rows in shared memory: when the whole tableau would leave room for fewer
  // than two CTAs per SM, the CTAs take 512 threads (two per SM) and keep in
  // shared memory the leading rows that two CTAs per SM leave room for; the
  // rest go to the L2 slot.
  int auto_threads_override = 0;
  if (o->kernel == LPB_KERNEL_AUTO && o->threads == 0 && b->count >= 16 * d.sms) {
    const size_t all_smem = fixed + rows * rowb;
    const int ctas = all_smem <= budget ? int(size_t(232448) / (all_smem + 1024)) : 0;
    if (ctas < 2) {
      const size_t half = size_t(232448) / 2 - 1024 - 1024;   // per CTA, less the kernel's static shared memory
      fit_rows = half > fixed ? (half - fixed) / rowb : 0;
      if (fit_rows > rows) fit_rows = rows;
      auto_threads_override = 512;
    }
  }
  p->tab_smem = fit_rows * rowb;
  p->slot_bytes = ((rows - fit_rows) * rowb + 127) & ~size_t(127);
  p->gmem = p->slot_bytes > 0;
  p->smem = fixed + p->tab_smem;
  if (p->smem < 16) p->smem = 16;
  p->threads = o->threads > 0 ? o->threads
             : auto_threads_override ? auto_threads_override : auto_threads(eb, int(rows), int(rowb / eb), p->smem);
  if (p->threads < 32 || p->threads > 1024 || (p->threads & 31)) return LPB_EINVAL;
  int occ = 0;
  if (tableau_max_ctas_per_sm(eb, p->threads, p->smem, &occ) != cudaSuccess) return LPB_ECUDA;
  if (occ < 1) return LPB_EUNSUPPORTED;
  p->grid = occ * d.sms;
  if (p->gmem) {
    size_t fit = (d.l2_bytes * 3 / 4) / p->slot_bytes;
    if (fit < size_t(d.sms)) fit = size_t(d.sms);
    if (fit < size_t(p->grid)) p->grid = int(fit);
  }
  if (p->grid > b->count) p->grid = b->count > 0 ? b->count : 1;
  return LPB_OK;
}

lpb_err reg_pass(const DeviceInfo &d, const lpb_batch *b, int cfg, int lim_m, int lim_n, int mode, int rule,
                 Pass *p) {
  int occ = 0;
  if (reg_occupancy(cfg, lim_m, lim_n, b->dtype, rule, &occ, &p->threads, &p->smem) != cudaSuccess)
    return LPB_ECUDA;
  if (p->smem > d.smem_optin || occ < 1) return LPB_EUNSUPPORTED;   // the input does not fit on chip
  p->fp64 = false;
  p->mode = mode;
  p->reg = cfg;
  p->lim_m = lim_m;
  p->lim_n = lim_n;
  p->grid = occ * d.sms;
  if (p->grid > b->count) p->grid = b->count > 0 ? b->count : 1;
  return LPB_OK;
}

lpb_err pack_pass(const DeviceInfo &d, const lpb_batch *b, int lanes, int mode, Pass *p) {
  int occ = 0;
  if (pack_occupancy(lanes, &occ, &p->threads) != cudaSuccess) return LPB_ECUDA;
  if (occ < 1) return LPB_EUNSUPPORTED;
  p->fp64 = false;
  p->mode = mode;
  p->pack = lanes;
  p->lim_m = b->max_m;
  p->lim_n = b->max_n;
  // Each warp takes 32 / lanes LPs at a time: no more warps than groups of LPs.
  const long long groups = (static_cast<long long>(b->count) * lanes + 31) / 32;
  const long long warps_per_cta = p->threads / 32;
  const long long need = (groups + warps_per_cta - 1) / warps_per_cta;
  p->grid = occ * d.sms;
  if (need < p->grid) p->grid = int(need > 0 ? need : 1);
  return LPB_OK;
}

lpb_err warp_pass(const DeviceInfo &d, const lpb_batch *b, int lim_m, int lim_n, int mode, Pass *p) {
  int occ = 0;
  if (warp_occupancy(lim_m, lim_n, &occ, &p->threads, &p->smem) != cudaSuccess) return LPB_ECUDA;
  if (occ < 1 || p->smem > d.smem_optin) return LPB_EUNSUPPORTED;
  p->fp64 = false;
  p->mode = mode;
  p->warp = true;
  p->lim_m = lim_m;
  p->lim_n = lim_n;
  // Each warp takes one LP at a time: no more CTAs than groups of LPs.
  const long long warps_per_cta = p->threads / 32;
  const long long need = (static_cast<long long>(b->count) + warps_per_cta - 1) / warps_per_cta;
  p->grid = occ * d.sms;
  if (need < p->grid) p->grid = int(need > 0 ? need : 1);
  return LPB_OK;
}

// Whether the planner gives LPs up to lim_m x lim_n the one-warp-per-LP
// shared-memory kernel: FP32 modes with FP64 input, the largest-coefficient or
// random rule, no kernel shape asked for, m and n from 32 (smaller LPs go
// several per warp) up to where it is measured faster than the register
// kernel (50,000 or 30,000 type-1 LPs): up to m n = 10,000 (100 x 100: 4.46
// against 4.66 ms with the FP64 refinement), and beyond that where an SM holds
// at least four of its regions while, with the refinement, the register kernel
// fits one CTA per SM (110 x 100: 3.28 against 4.80 ms; 100 x 110, two register
// CTAs per SM: 3.32 against 3.10; 127 x 127, three regions: 5.38 against 4.35).
bool warp_auto(const lpb_batch *b, const lpb_options *o, int mode, int lim_m, int lim_n) {
  if (o->kernel != LPB_KERNEL_AUTO || o->threads != 0 || o->reg_warps != 0) return false;
  if (mode == MODE_FP64 || b->dtype != LPB_DTYPE_F64 || o->pivot_rule == LPB_PIVOT_STEEPEST) return false;
  if (!warp_fits(lim_m, lim_n) || (lim_m < 32 && lim_n < 32)) return false;
  if (lim_m * lim_n <= 10000) return true;
  int wc = 0, wt = 0;
  size_t ws = 0;
  if (warp_occupancy(lim_m, lim_n, &wc, &wt, &ws) != cudaSuccess || wc * (wt / 32) < 4) return false;
  if (mode == MODE_FP32) return true;
  const int cfg = reg_pick(lim_m, lim_n, 8, false);
  if (cfg < 0) return true;
  int rc = 0, rt = 0;
  size_t rs = 0;
  if (reg_occupancy(cfg, lim_m, lim_n, b->dtype, o->pivot_rule, &rc, &rt, &rs) != cudaSuccess) return false;
  return rc <= 1;
}

lpb_err make_plan(const DeviceInfo &d, const lpb_batch *b, const lpb_options *o, bool basis_given,
                  Plan *pl) {
  if (!b || !o) return LPB_EINVAL;
  if (b->count < 0) return LPB_EINVAL;
  if (b->max_m < 1 || b->max_n < 1 || b->max_m > kMaxDim || b->max_n > kMaxDim) return LPB_EUNSUPPORTED;
  if (b->dtype != LPB_DTYPE_F32 && b->dtype != LPB_DTYPE_F64) return LPB_EINVAL;
  if (o->prec < LPB_FP64 || o->prec > LPB_FP32) return LPB_EINVAL;
  if (o->max_iter < 0 || o->eps_p < 0 || o->eps_d < 0 || o->feas_tol < 0) return LPB_EINVAL;
  if (o->pivot_rule != LPB_PIVOT_LPC && o->pivot_rule != LPB_PIVOT_RPC && o->pivot_rule != LPB_PIVOT_STEEPEST)
    return LPB_EINVAL;
  if (o->kernel < LPB_KERNEL_AUTO || o->kernel > LPB_KERNEL_WARP) return LPB_EINVAL;
  // Steepest edge has register-kernel instantiations for the 8-warp templates only.
  const bool se = o->pivot_rule == LPB_PIVOT_STEEPEST;
  const bool fp32 = o->prec != LPB_FP64;
  pl->eps_p = o->eps_p > 0 ? o->eps_p : (fp32 ? 1e-6 : 1e-9);
  pl->eps_d = o->eps_d > 0 ? o->eps_d : (fp32 ? 1e-6 : 1e-9);
  pl->eps_p64 = o->eps_p > 0 ? o->eps_p : 1e-9;
  pl->eps_d64 = o->eps_d > 0 ? o->eps_d : 1e-9;
  pl->feas_tol = o->feas_tol > 0 ? o->feas_tol : 1e-9;
  lpb_err e;
  const int mode = o->prec == LPB_FP64 ? MODE_FP64 : o->prec == LPB_FP32 ? MODE_FP32 : MODE_FP32_REFINE;
  // Warps per LP of the register templates: as asked; else one warp per LP
  // when every LP has m, n <= 31 (many tiny LPs in flight per SM), else 8.
  const int want_w = o->reg_warps > 0 ? o->reg_warps
                   : (o->kernel == LPB_KERNEL_REG && o->threads > 0) ? o->threads / 32
                   : (b->max_m <= 31 && b->max_n <= 31) ? 1 : 8;
  // Every LP of the same size (the caller's hint): one pass, no size classes.
  const bool uniform = b->min_m > 0 && b->min_m == b->max_m && b->min_n == b->max_n;
  lpb_options og = *o;          // options of the shared-memory / L2-slot kernel passes
  if (og.kernel == LPB_KERNEL_REG) { og.kernel = LPB_KERNEL_AUTO; og.threads = 0; }
  int np = 0;
  // Several tiny LPs per warp (one per warp up to 31): asked for, or the
  // default for batches of LPs with m, n <= 31 when no register-kernel shape is
  // asked for.
  const int lanes = (fp32 && !se) ? pack_lanes(b->max_m, b->max_n) : 0;
  if (o->kernel == LPB_KERNEL_PACK && lanes == 0) return LPB_EUNSUPPORTED;
  if (lanes > 0 && (o->kernel == LPB_KERNEL_PACK ||
                    (o->kernel == LPB_KERNEL_AUTO && o->reg_warps == 0 && o->threads == 0))) {
    Pass &p = pl->pass[0];
    if ((e = pack_pass(d, b, lanes, mode, &p)) != LPB_OK) return e;
    p.list = LIST_ALL;
    np = 1;
  }
  if (og.kernel == LPB_KERNEL_PACK) { og.kernel = LPB_KERNEL_AUTO; og.threads = 0; }
  // One warp per LP with the tableau in shared memory: asked for.
  if (o->kernel == LPB_KERNEL_WARP) {
    if (!fp32 || se || b->dtype != LPB_DTYPE_F64 || !warp_fits(b->max_m, b->max_n)) return LPB_EUNSUPPORTED;
    Pass &p = pl->pass[0];
    if ((e = warp_pass(d, b, b->max_m, b->max_n, mode, &p)) != LPB_OK) return e;
    p.list = LIST_ALL;
    np = 1;
    og.kernel = LPB_KERNEL_AUTO;
    og.threads = 0;
  }
  // ... and the planner's choice for batches of one size where it is faster.
  if (np == 0 && uniform && warp_auto(b, o, mode, b->max_m, b->max_n)) {
    Pass &p = pl->pass[0];
    if ((e = warp_pass(d, b, b->max_m, b->max_n, mode, &p)) != LPB_OK) return e;
    p.list = LIST_ALL;
    np = 1;
  }
  if (np == 0 && fp32 && o->kernel == LPB_KERNEL_AUTO && !uniform) {
    // Size classes: the register-tableau templates with `want_w` warps in
    // increasing size (a class the one-warp-per-LP kernel is faster for takes
    // that kernel), then the shared-memory / L2-slot kernel for the rest.
    Pass regp[kMaxClasses];
    int nreg = 0;
    bool covered = false;
    int order[16], cnt = 0;
    for (int i = 0; i < reg_count() && cnt < 16; ++i) {
      int mm, nn, ww;
      reg_limits(i, &mm, &nn, &ww);
      if (ww == want_w && (!se || reg_has_se(i))) order[cnt++] = i;
    }
    for (int a = 0; a < cnt; ++a)        // by capacity, smallest first
      for (int c = a + 1; c < cnt; ++c) {
        int ma, na, mc, nc, w0;
        reg_limits(order[a], &ma, &na, &w0);
        reg_limits(order[c], &mc, &nc, &w0);
        if (mc * nc < ma * na) { const int t = order[a]; order[a] = order[c]; order[c] = t; }
      }
    for (int a = 0; a < cnt && !covered && nreg < kMaxClasses - 1; ++a) {
      int mm, nn, ww;
      reg_limits(order[a], &mm, &nn, &ww);
      const int lm = mm < b->max_m ? mm : b->max_m, ln = nn < b->max_n ? nn : b->max_n;
      if (nreg > 0 && lm <= pl->cls_m[nreg - 1] && ln <= pl->cls_n[nreg - 1]) continue;
      Pass p;
      // A class the one-warp-per-LP kernel is faster for takes it instead.
      if (warp_auto(b, o, mode, lm, ln)) {
        if (warp_pass(d, b, lm, ln, mode, &p) != LPB_OK) continue;
      } else if (reg_pass(d, b, order[a], lm, ln, mode, o->pivot_rule, &p) != LPB_OK) {
        continue;
      }
      p.list = LIST_CLASS;
      p.cls = nreg;
      pl->cls_m[nreg] = lm;
      pl->cls_n[nreg] = ln;
      regp[nreg++] = p;
      covered = lm >= b->max_m && ln >= b->max_n;
    }
    if (nreg > 0) {
      pl->classes = true;
      pl->nclass = nreg + (covered ? 0 : 1);
      if (!covered) {              // the largest LPs first: the tableau kernel's class
        Pass &p = pl->pass[np];
        if ((e = make_pass(d, b, &og, false, 0, mode, &p)) != LPB_OK) return e;
        p.list = LIST_CLASS;
        p.cls = nreg;
        p.lim_m = b->max_m;
        p.lim_n = b->max_n;
        pl->cls_m[nreg] = b->max_m;
        pl->cls_n[nreg] = b->max_n;
        ++np;
      }
      for (int c = nreg - 1; c >= 0; --c) pl->pass[np++] = regp[c];
    }
  }
  if (np == 0) {                   // one first pass over every LP
    Pass &p = pl->pass[0];
    const int reg = fp32 && (o->kernel == LPB_KERNEL_REG || (o->kernel == LPB_KERNEL_AUTO && uniform))
                        ? reg_pick(b->max_m, b->max_n, want_w, se) : -1;
    if (o->kernel == LPB_KERNEL_REG && reg < 0) return LPB_EUNSUPPORTED;
    if (reg >= 0) {
      if ((e = reg_pass(d, b, reg, b->max_m, b->max_n, mode, o->pivot_rule, &p)) != LPB_OK) return e;
    } else if ((e = make_pass(d, b, &og, !fp32, 0, mode, &p)) != LPB_OK) {
      return e;
    }
    p.list = LIST_ALL;
    p.lim_m = b->max_m;
    p.lim_n = b->max_n;
    np = 1;
  }
  {                                // LPs that need more artificial columns (Phase I)
    Pass &p = pl->pass[np];
    if ((e = make_pass(d, b, &og, !fp32, b->max_m, mode, &p)) != LPB_OK) return e;
    p.list = LIST_DEFER;
    p.group = 1;
    p.lim_m = b->max_m;
    p.lim_n = b->max_n;
    ++np;
  }
  pl->resolve = o->prec == LPB_FP32_REFINE;
  if (pl->resolve) {               // FP64 re-solve of the LPs that failed the FP32 certificate
    Pass &p = pl->pass[np];
    if ((e = make_pass(d, b, &og, true, b->max_m, MODE_FP64, &p)) != LPB_OK) return e;
    p.list = LIST_RESOLVE;
    p.group = 2;
    p.lim_m = b->max_m;
    p.lim_n = b->max_n;
    ++np;
  }
  pl->npass = np;
  pl->own_basis = pl->resolve && !basis_given;
  size_t off = 0;
  const size_t cnt = size_t(b->count > 0 ? b->count : 1);
  pl->off_defer = off;   off = align256(off + cnt * 4);
  pl->off_resolve = off; off = align256(off + cnt * 4);
  pl->off_basis = off;   off = align256(off + (pl->own_basis ? cnt * size_t(b->max_m) * 4 : 0));
  pl->off_lists = off;   off = align256(off + (pl->classes ? cnt * size_t(pl->nclass) * 4 : 0));
  pl->off_hist = off;    off = align256(off + (pl->classes ? classify_hist_bytes(pl->nclass) : 0));
  pl->off_cctr = off;    off = align256(off + (kMaxPasses + kMaxClasses) * sizeof(int32_t));
  pl->off_slots = off;
  size_t slots = 0;
  for (int i = 0; i < pl->npass; ++i)
    if (pl->pass[i].gmem) {
      const size_t sz = size_t(pl->pass[i].grid) * pl->pass[i].slot_bytes;
      if (sz > slots) slots = sz;
    }
  pl->total = align256(off + slots);
  return LPB_OK;
}

TableauParams base_params(int32_t *ctr, uint32_t *err, const lpb_batch *b, const lpb_result *r,
                          const lpb_options *o, const Plan &pl, unsigned char *ws) {
  TableauParams p{};
  p.B = BatchDev{b->count, b->max_m, b->max_n, b->dtype, b->m, b->n, b->a_off, b->b_off, b->c_off,
                 b->A, b->b, b->c};
  p.R = ResultDev{r->status, r->iters, r->obj, r->x, r->y, r->basis, nullptr};
  p.defer_items = reinterpret_cast<int32_t *>(ws + pl.off_defer);
  p.defer_count = ctr + CTR_DEFER;
  p.resolve_items = reinterpret_cast<int32_t *>(ws + pl.off_resolve);
  p.resolve_count = ctr + CTR_RESOLVE;
  p.list_cap = b->count;
  p.bbuf = pl.own_basis ? reinterpret_cast<int32_t *>(ws + pl.off_basis) : r->basis;
  p.bpacked = pl.own_basis ? 0 : 1;
  p.slots = ws + pl.off_slots;
  p.max_iter = o->max_iter;
  p.eps_p = pl.eps_p;
  p.eps_d = pl.eps_d;
  p.feas_tol = pl.feas_tol;
  p.err = err;
  p.rule = o->pivot_rule;
  p.seed = o->seed;
  return p;
}

DeviceInfo device_info(const lpb_handle *h) { return DeviceInfo{h->sms, h->smem_optin, h->l2_bytes}; }

}  // namespace

namespace lpb {

lpb_err solve_workspace_bytes(const DeviceInfo &d, const lpb_batch *b, const lpb_options *o,
                              bool basis_given, size_t *bytes) {
  Plan pl;
  const lpb_err e = make_plan(d, b, o, basis_given, &pl);
  if (e != LPB_OK) return e;
  *bytes = pl.total;
  return LPB_OK;
}

lpb_err run_solve(const DeviceInfo &d, int32_t *ctr, uint32_t *err, const lpb_batch *b,
                  const lpb_options *o, const lpb_result *r, void *ws, size_t ws_bytes, cudaStream_t s,
                  cudaEvent_t *prof_ev, bool *prof_ran, int *kernels, long long lp_base, const int64_t *y_off,
                  int shared) {
  if (kernels) *kernels = 0;
  Plan pl;
  lpb_err e = make_plan(d, b, o, r->basis != nullptr, &pl);
  if (e != LPB_OK) return e;
  if (ws_bytes < pl.total || (pl.total > 0 && !ws)) return LPB_ENOMEM;
  if (reinterpret_cast<uintptr_t>(ws) & 255) return LPB_EINVAL;
  unsigned char *w = static_cast<unsigned char *>(ws);
  int32_t *queues = reinterpret_cast<int32_t *>(w + pl.off_cctr);   // one per pass
  int32_t *class_count = queues + kMaxPasses;
  if (cudaMemsetAsync(ctr, 0, kCounters * sizeof(int32_t), s) != cudaSuccess) return LPB_ECUDA;
  if (cudaMemsetAsync(queues, 0, (kMaxPasses + kMaxClasses) * sizeof(int32_t), s) != cudaSuccess) return LPB_ECUDA;
  int group = -1;
  for (int i = 0; i < pl.npass; ++i) {
    const Pass &ps = pl.pass[i];
    if (ps.group != group) {     // timing: one event pair around each group of passes
      if (prof_ev && group >= 0 && cudaEventRecord(prof_ev[group * 2 + 1], s) != cudaSuccess) return LPB_ECUDA;
      group = ps.group;
      if (prof_ev) {
        if (cudaEventRecord(prof_ev[group * 2], s) != cudaSuccess) return LPB_ECUDA;
        prof_ran[group] = true;
      }
      if (group == 0 && pl.classes) {
        ClassPlanParams cp{};
        cp.count = b->count;
        cp.nclass = pl.nclass;
        cp.m = b->m;
        cp.n = b->n;
        for (int c = 0; c < pl.nclass; ++c) { cp.max_m[c] = pl.cls_m[c]; cp.max_n[c] = pl.cls_n[c]; }
        cp.hist = reinterpret_cast<int32_t *>(w + pl.off_hist);
        cp.lists = reinterpret_cast<int32_t *>(w + pl.off_lists);
        cp.class_count = class_count;
        if (launch_classify(cp, d.sms, s) != cudaSuccess) return LPB_ECUDA;
        if (kernels) *kernels += 3;
      }
    }
    TableauParams p = base_params(ctr, err, b, r, o, pl, w);
    p.lp_base = lp_base;
    p.R.y_off = y_off;
    p.shared = shared;
    p.kcap = ps.kcap;
    p.mode = ps.mode;
    p.slot_bytes = ps.slot_bytes;
    p.tab_smem = ps.tab_smem;
    p.lim_m = ps.lim_m;
    p.lim_n = ps.lim_n;
    p.queue = queues + i;
    switch (ps.list) {
      case LIST_ALL:
        p.in = WorkList{nullptr, nullptr};
        break;
      case LIST_CLASS:
        p.in = WorkList{reinterpret_cast<int32_t *>(w + pl.off_lists) + size_t(ps.cls) * size_t(b->count),
                        class_count + ps.cls};
        break;
      case LIST_DEFER:
        p.in = WorkList{p.defer_items, p.defer_count};
        p.defer_items = nullptr;   // kcap = max_m: nothing is deferred again
        break;
      default:                 // FP64 re-solve: FP64 tolerances
        p.in = WorkList{p.resolve_items, p.resolve_count};
        p.warm = 1;
        p.eps_p = pl.eps_p64;
        p.eps_d = pl.eps_d64;
        break;
    }
    const cudaError_t ce = ps.pack > 0 ? launch_pack(p, ps.pack, ps.grid, s)
                         : ps.warp ? launch_warp(p, ps.grid, ps.threads, ps.smem, s)
                         : ps.reg >= 0 ? launch_reg(p, ps.reg, ps.grid, ps.smem, s)
                                       : launch_tableau(p, ps.fp64, ps.grid, ps.threads, ps.smem, s);
    if (ce != cudaSuccess) return LPB_ECUDA;
    if (kernels) *kernels += 1;
  }
  if (prof_ev && group >= 0 && cudaEventRecord(prof_ev[group * 2 + 1], s) != cudaSuccess) return LPB_ECUDA;
  return LPB_OK;
}

}  // namespace lpb

// ---- host-memory pipeline (Section 4.5: CUDA streams) ----------------------

namespace {

// Rebases the offsets of a chunk to its own buffers.
__global__ void rebase_offsets(int64_t *a_off, int64_t *b_off, int64_t *c_off, int cnt, int64_t a0, int64_t b0,
                               int64_t c0) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < cnt; k += gridDim.x * blockDim.x) {
    a_off[k] -= a0;
    b_off[k] -= b0;
    c_off[k] -= c0;
  }
}

// Chunks of a host batch: LP ranges, their element ranges in A, b, c, and the
// carving of the workspace into one solve workspace and two buffer sets.
struct HostPlan {
  int chunk = 0, nchunk = 0;
  size_t a_max = 0, b_max = 0, c_max = 0;   // largest element ranges of a chunk
  size_t solve_ws = 0;
  size_t set_bytes = 0;
  size_t o_A = 0, o_b = 0, o_c = 0, o_m = 0, o_n = 0, o_ao = 0, o_bo = 0, o_co = 0;
  size_t o_st = 0, o_it = 0, o_obj = 0, o_x = 0, o_y = 0, o_bs = 0;
  size_t total = 0;
};

// Element range [lo, hi) of LPs k0..k1-1 in an array with offsets `off` and
// lengths len(k).
template <typename F>
void chunk_range(const int64_t *off, int k0, int k1, F len, int64_t *lo, int64_t *hi) {
  *lo = off[k0];
  *hi = off[k1 - 1] + len(k1 - 1);
}

lpb_err make_host_plan(const DeviceInfo &d, const lpb_batch *b, const lpb_options *o, int chunk, HostPlan *hp) {
  if (!b || !o || chunk < 1) return LPB_EINVAL;
  if (b->count < 0) return LPB_EINVAL;
  if (b->count > 0 && (!b->m || !b->n || !b->a_off || !b->b_off || !b->c_off || !b->A || !b->b || !b->c))
    return LPB_EINVAL;
  const int cnt = b->count;
  hp->chunk = cnt > 0 && chunk > cnt ? cnt : chunk;
  hp->nchunk = cnt > 0 ? (cnt + hp->chunk - 1) / hp->chunk : 0;
  // Offsets must follow the LP order with no overlap (each array packed in order).
  for (int k = 0; k < cnt; ++k) {
    const int64_t mk = b->m[k], nk = b->n[k];
    if (mk < 0 || nk < 0 || b->a_off[k] < 0 || b->b_off[k] < 0 || b->c_off[k] < 0) return LPB_EINVAL;
    if (k + 1 < cnt && (b->a_off[k + 1] < b->a_off[k] + mk * nk || b->b_off[k + 1] < b->b_off[k] + mk ||
                        b->c_off[k + 1] < b->c_off[k] + nk))
      return LPB_EINVAL;
  }
  for (int i = 0; i < hp->nchunk; ++i) {
    const int k0 = i * hp->chunk, k1 = (k0 + hp->chunk < cnt) ? k0 + hp->chunk : cnt;
    int64_t lo, hi;
    chunk_range(b->a_off, k0, k1, [&](int k) { return int64_t(b->m[k]) * b->n[k]; }, &lo, &hi);
    if (size_t(hi - lo) > hp->a_max) hp->a_max = size_t(hi - lo);
    chunk_range(b->b_off, k0, k1, [&](int k) { return int64_t(b->m[k]); }, &lo, &hi);
    if (size_t(hi - lo) > hp->b_max) hp->b_max = size_t(hi - lo);
    chunk_range(b->c_off, k0, k1, [&](int k) { return int64_t(b->n[k]); }, &lo, &hi);
    if (size_t(hi - lo) > hp->c_max) hp->c_max = size_t(hi - lo);
  }
  lpb_batch cb = *b;
  cb.count = hp->chunk;
  const lpb_err e = solve_workspace_bytes(d, &cb, o, false, &hp->solve_ws);
  if (e != LPB_OK) return e;
  const size_t es = b->dtype == LPB_DTYPE_F64 ? 8 : 4;
  const size_t ch = size_t(hp->chunk);
  size_t off = 0;
  auto take = [&](size_t bytes) { const size_t at = off; off = align256(off + (bytes ? bytes : 1)); return at; };
  hp->o_A = take(hp->a_max * es);
  hp->o_b = take(hp->b_max * es);
  hp->o_c = take(hp->c_max * es);
  hp->o_m = take(ch * 4);
  hp->o_n = take(ch * 4);
  hp->o_ao = take(ch * 8);
  hp->o_bo = take(ch * 8);
  hp->o_co = take(ch * 8);
  hp->o_st = take(ch * 4);
  hp->o_it = take(ch * 4);
  hp->o_obj = take(ch * 8);
  hp->o_x = take(hp->c_max * 8);
  hp->o_y = take(hp->b_max * 8);
  hp->o_bs = take(hp->b_max * 4);
  hp->set_bytes = off;
  hp->total = align256(hp->solve_ws) + 2 * hp->set_bytes;
  return LPB_OK;
}

}  // namespace

// ---- shared-constraint batches: one A and b, many objectives ----------------

namespace {

// Sizes and offsets of `count` LPs that share A and b (offset 0) and read
// objective k at k n; y and basis of LP k go to k m of the result.
__global__ void fill_shared_meta(int32_t *m, int32_t *n, int64_t *a_off, int64_t *b_off, int64_t *c_off,
                                 int64_t *y_off, int count, int mm, int nn) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < count; k += gridDim.x * blockDim.x) {
    m[k] = mm;
    n[k] = nn;
    a_off[k] = 0;
    b_off[k] = 0;
    c_off[k] = int64_t(k) * nn;
    y_off[k] = int64_t(k) * mm;
  }
}

// Options of a shared-constraint solve: FP32 solves that fit a register
// template run on the register kernel over the identity work list, so that
// each CTA takes consecutive objectives and can start each from the basis of
// the one before.
lpb_options shared_options(const lpb_options *o, int m, int n) {
  lpb_options os = *o;
  if (o->prec != LPB_FP64 && o->kernel == LPB_KERNEL_AUTO && o->threads == 0 &&
      reg_pick(m, n, o->reg_warps > 0 ? o->reg_warps : 8, o->pivot_rule == LPB_PIVOT_STEEPEST) >= 0)
    os.kernel = LPB_KERNEL_REG;
  return os;
}

struct SharedPlan {
  size_t o_m = 0, o_n = 0, o_ao = 0, o_bo = 0, o_co = 0, o_yo = 0, o_ws = 0, solve_ws = 0, total = 0;
};

lpb_err make_shared_plan(const DeviceInfo &d, int m, int n, int dtype, int64_t count, const lpb_options *o,
                         SharedPlan *sp) {
  if (!o || m < 1 || n < 1 || count < 0 || count > INT32_MAX) return LPB_EINVAL;
  lpb_batch pb{};
  pb.count = int32_t(count);
  pb.max_m = m;
  pb.max_n = n;
  pb.min_m = m;            // every LP of the batch has the one size m x n
  pb.min_n = n;
  pb.dtype = dtype;
  const lpb_err e = solve_workspace_bytes(d, &pb, o, false, &sp->solve_ws);
  if (e != LPB_OK) return e;
  const size_t c = size_t(count > 0 ? count : 1);
  size_t off = 0;
  auto take = [&](size_t bytes) { const size_t at = off; off = align256(off + bytes); return at; };
  sp->o_m = take(c * 4);
  sp->o_n = take(c * 4);
  sp->o_ao = take(c * 8);
  sp->o_bo = take(c * 8);
  sp->o_co = take(c * 8);
  sp->o_yo = take(c * 8);
  sp->o_ws = take(sp->solve_ws);
  sp->total = off;
  return LPB_OK;
}

}  // namespace

// ---- bounded variables: l <= x <= u in place of x >= 0 ----------------------

namespace {

// Change of variables x = l + z: LP k becomes max c^T z subject to
// A z <= b - A l and z_j <= u_j - l_j (the row 0 <= 1 when u_j = +inf), z >= 0,
// written in FP64 at a fixed stride per LP.  One CTA per LP (grid-stride).
template <typename T>
__global__ void bounded_transform(BatchDev B, const T *l, const T *u, int mm, int nn, double *A2, double *b2,
                                  int32_t *m2, int32_t *n2, int64_t *a2_off, int64_t *b2_off, int64_t *c2_off) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const T *A = static_cast<const T *>(B.A), *b = static_cast<const T *>(B.b);
  for (int k = blockIdx.x; k < B.count; k += gridDim.x) {
    const int m = B.m[k], n = B.n[k];
    const int64_t ao = B.a_off[k], bo = B.b_off[k], co = B.c_off[k];
    const int64_t sa = int64_t(k) * (mm + nn) * nn, sb = int64_t(k) * (mm + nn);
    const bool ok = m >= 1 && n >= 1 && m <= mm && n <= nn;
    if (threadIdx.x == 0) {
      m2[k] = ok ? m + n : 0;         // a size of 0 reports LPB_BAD_SIZE
      n2[k] = ok ? n : 0;
      a2_off[k] = sa;
      b2_off[k] = sb;
      c2_off[k] = co;
    }
    if (!ok) continue;
    for (int64_t t = threadIdx.x; t < int64_t(m) * n; t += blockDim.x) A2[sa + t] = double(A[ao + t]);
    for (int64_t t = threadIdx.x; t < int64_t(n) * n; t += blockDim.x) {   // row z_j <= u_j - l_j, or 0 <= 1
      const int j = int(t / n);
      const double uj = double(u[co + j]);
      A2[sa + int64_t(m) * n + t] = (j == int(t % n) && !(isinf(uj) && uj > 0.0)) ? 1.0 : 0.0;
    }
    for (int i = wid; i < m; i += nw) {          // b_i - A_i l in FP64, one warp per row
      double s = 0.0;
      for (int j = lane; j < n; j += 32) s = fma(double(A[ao + int64_t(i) * n + j]), double(l[co + j]), s);
      s = warp_sum(s);
      if (lane == 0) b2[sb + i] = double(b[bo + i]) - s;
    }
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
      const double uj = double(u[co + j]), lj = double(l[co + j]);
      b2[sb + m + j] = (isinf(uj) && uj > 0.0) ? 1.0 : uj - lj;
    }
  }
}

// Back to the bounded LP: x = l + z and obj + c^T l for optimal LPs; the duals
// of the rows of A are the first m duals of the reduced LP.
template <typename T>
__global__ void bounded_finish(BatchDev B, const T *l, lpb_result R, const double *y2, int mm, int nn) {
  const int lane = threadIdx.x & 31;
  const T *c = static_cast<const T *>(B.c);
  for (int k = blockIdx.x; k < B.count; k += gridDim.x) {
    const int m = B.m[k], n = B.n[k];
    if (m < 1 || n < 1 || m > mm || n > nn) continue;
    const int64_t bo = B.b_off[k], co = B.c_off[k], sb = int64_t(k) * (mm + nn);
    const bool opt = R.status[k] == LPB_OPTIMAL;
    if (threadIdx.x < 32) {
      double s = 0.0;
      for (int j = lane; j < n; j += 32) s = fma(double(c[co + j]), double(l[co + j]), s);
      s = warp_sum(s);
      if (lane == 0 && opt) R.obj[k] += s;
    }
    for (int j = threadIdx.x; j < n; j += blockDim.x) R.x[co + j] = opt ? R.x[co + j] + double(l[co + j]) : 0.0;
    if (R.y)
      for (int i = threadIdx.x; i < m; i += blockDim.x) R.y[bo + i] = opt ? y2[sb + i] : 0.0;
  }
}

struct BoundedPlan {
  size_t o_A = 0, o_b = 0, o_y = 0, o_m = 0, o_n = 0, o_ao = 0, o_bo = 0, o_co = 0, o_ws = 0, solve_ws = 0, total = 0;
};

lpb_err make_bounded_plan(const DeviceInfo &d, const lpb_batch *b, const lpb_options *o, BoundedPlan *bp) {
  if (!b || !o || b->count < 0 || b->max_m < 1 || b->max_n < 1) return LPB_EINVAL;
  if (b->dtype != LPB_DTYPE_F64) return LPB_EUNSUPPORTED;   // the reduced LP reads the caller's c as FP64
  if (b->max_m + b->max_n > kMaxDim) return LPB_EUNSUPPORTED;
  lpb_batch rb = *b;
  rb.min_m = rb.min_n = 0;      // the reduced LPs have m + n rows
  rb.max_m = b->max_m + b->max_n;
  rb.dtype = LPB_DTYPE_F64;
  const lpb_err e = solve_workspace_bytes(d, &rb, o, false, &bp->solve_ws);
  if (e != LPB_OK) return e;
  const size_t c = size_t(b->count > 0 ? b->count : 1), rows = size_t(b->max_m + b->max_n);
  size_t off = 0;
  auto take = [&](size_t bytes) { const size_t at = off; off = align256(off + bytes); return at; };
  bp->o_A = take(c * rows * size_t(b->max_n) * 8);
  bp->o_b = take(c * rows * 8);
  bp->o_y = take(c * rows * 8);
  bp->o_m = take(c * 4);
  bp->o_n = take(c * 4);
  bp->o_ao = take(c * 8);
  bp->o_bo = take(c * 8);
  bp->o_co = take(c * 8);
  bp->o_ws = take(bp->solve_ws);
  bp->total = off;
  return LPB_OK;
}

}  // namespace

extern "C" {

const char *lpb_version(void) { return "liblpb 0.1 (sm_103a)"; }

const char *lpb_strerror(lpb_err err) {
  switch (err) {
    case LPB_OK: return "ok";
    case LPB_EINVAL: return "invalid argument";
    case LPB_ENOMEM: return "workspace too small";
    case LPB_ECUDA: return "CUDA runtime error";
    case LPB_EUNSUPPORTED: return "unsupported size or mode";
    case LPB_EDEVICE: return "a kernel recorded a device-side fault";
  }
  return "unknown error";
}

lpb_err lpb_create(lpb_handle **handle, int device) {
  if (!handle) return LPB_EINVAL;
  *handle = nullptr;
  DeviceScope ds(device);
  if (!ds.ok()) return LPB_ECUDA;
  lpb_handle *h = new (std::nothrow) lpb_handle{};
  if (!h) return LPB_ENOMEM;
  h->device = device;
  int v = 0;
  cudaError_t e = cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
  h->smem_optin = size_t(v);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&v, cudaDevAttrL2CacheSize, device);
  h->l2_bytes = size_t(v);
  if (e == cudaSuccess) e = cudaMalloc(&h->d_err, sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMalloc(&h->d_ctr, CTR_N * sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMemset(h->d_err, 0, sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMemset(h->d_ctr, 0, CTR_N * sizeof(int32_t));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->s_in, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->s_out, cudaStreamNonBlocking);
  for (int j = 0; j < 2 && e == cudaSuccess; ++j) {
    e = cudaEventCreateWithFlags(&h->ev_in[j], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_comp[j], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_out[j], cudaEventDisableTiming);
  }
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_start, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    cudaFree(h->d_err);
    cudaFree(h->d_ctr);
    for (int j = 0; j < 2; ++j) {
      if (h->ev_in[j]) cudaEventDestroy(h->ev_in[j]);
      if (h->ev_comp[j]) cudaEventDestroy(h->ev_comp[j]);
      if (h->ev_out[j]) cudaEventDestroy(h->ev_out[j]);
    }
    if (h->ev_start) cudaEventDestroy(h->ev_start);
    if (h->s_in) cudaStreamDestroy(h->s_in);
    if (h->s_out) cudaStreamDestroy(h->s_out);
    delete h;
    return LPB_ECUDA;
  }
  *handle = h;
  return LPB_OK;
}

lpb_err lpb_destroy(lpb_handle *h) {
  if (!h) return LPB_EINVAL;
  {
    DeviceScope ds(h->device);
    cudaDeviceSynchronize();
    cudaFree(h->d_err);
    cudaFree(h->d_ctr);
    if (h->prof_ev) {
      for (int i = 0; i < lpb_handle::kProfMax * 3 * 2; ++i) cudaEventDestroy(h->prof_ev[i]);
      delete[] h->prof_ev;
    }
    for (int j = 0; j < 2; ++j) {
      cudaEventDestroy(h->ev_in[j]);
      cudaEventDestroy(h->ev_comp[j]);
      cudaEventDestroy(h->ev_out[j]);
    }
    cudaEventDestroy(h->ev_start);
    cudaStreamDestroy(h->s_in);
    cudaStreamDestroy(h->s_out);
  }
  delete h;
  return LPB_OK;
}

lpb_err lpb_workspace_size(lpb_handle *h, const lpb_batch *b, const lpb_options *o, size_t *bytes) {
  if (!h || !b || !o || !bytes) return LPB_EINVAL;
  DeviceScope ds(h->device);
  if (!ds.ok()) return LPB_ECUDA;
  // Size for the worst case: the basis may have to live in the workspace.
  const lpb_err e = solve_workspace_bytes(device_info(h), b, o, false, bytes);
  if (e != LPB_OK) return e;
  // lpb_solve_backward needs FP64 elimination slots only for large systems.
  const size_t smem = backward_smem_bytes(b->max_m, b->max_n);
  int grid = 0;
  if (smem <= h->smem_optin && backward_grid(h->sms, smem, &grid) == cudaSuccess) {
    const size_t need = backward_slot_bytes(b->max_m, b->max_n) * size_t(grid);
    if (need > *bytes) *bytes = need;
  }
  return LPB_OK;
}

lpb_err lpb_solve(lpb_handle *h, const lpb_batch *b, const lpb_options *o, const lpb_result *r,
                  void *ws, size_t ws_bytes, void *stream) {
  if (!h || !b || !o || !r) return LPB_EINVAL;
  if (b->count < 0) return LPB_EINVAL;
  if (b->count == 0) return LPB_OK;
  if (!b->m || !b->n || !b->a_off || !b->b_off || !b->c_off || !b->A || !b->b || !b->c) return LPB_EINVAL;
  if (!r->status || !r->obj || !r->x) return LPB_EINVAL;
  DeviceScope ds(h->device);
  if (!ds.ok()) return LPB_ECUDA;
  lpb_options tuned_opt;
  if (o->kernel == LPB_KERNEL_AUTO && o->threads == 0 && o->reg_warps == 0 &&
      o->pivot_rule != LPB_PIVOT_STEEPEST)     // tuned register kernels may lack a steepest-edge instantiation
    for (const auto &t : h->tuned)
      if (t.max_m == b->max_m && t.max_n == b->max_n && t.dtype == b->dtype && t.prec == o->prec) {
        tuned_opt = *o;
        tuned_opt.kernel = t.kernel;
        tuned_opt.threads = t.threads;
        tuned_opt.reg_warps = t.reg_warps;
        o = &tuned_opt;
        break;
      }
  const bool prof = h->prof_ev && h->prof_n < h->prof_cap;
  const lpb_err e = run_solve(device_info(h), h->d_ctr, h->d_err, b, o, r, ws, ws_bytes,
                              static_cast<cudaStream_t>(stream),
                              prof ? h->prof_ev + size_t(h->prof_n) * 3 * 2 : nullptr,
                              prof ? h->prof_ran + h->prof_n * 3 : nullptr, &h->last_kernels);
  if (e == LPB_OK && prof) ++h->prof_n;
  return e;
}

lpb_err lpb_workspace_size_host(lpb_handle *h, const lpb_batch *b, const lpb_options *o, int32_t chunk,
                                size_t *bytes) {
  if (!h || !b || !o || !bytes) return LPB_EINVAL;
  DeviceScope ds(h->device);
  if (!ds.ok()) return LPB_ECUDA;
  HostPlan hp;
  const lpb_err e = make_host_plan(device_info(h), b, o, chunk, &hp);
  if (e != LPB_OK) return e;
  *bytes = hp.total;
  return LPB_OK;
}

lpb_err lpb_solve_host(lpb_handle *h, const lpb_batch *b, const lpb_options *o, const lpb_result *r, int32_t chunk,
                       void *ws, size_t ws_bytes, void *stream) {
  if (!h || !b || !o || !r) return LPB_EINVAL;
  if (b->count == 0) return b->count < 0 ? LPB_EINVAL : LPB_OK;
  if (!r->status || !r->obj || !r->x) return LPB_EINVAL;
  DeviceScope ds(h->device);
  if (!ds.ok()) return LPB_ECUDA;
  const DeviceInfo d = device_info(h);
  HostPlan hp;
  lpb_err e = make_host_plan(d, b, o, chunk, &hp);
  if (e != LPB_OK) return e;
  if (ws_bytes < hp.total || !ws) return LPB_ENOMEM;
  if (reinterpret_cast<uintptr_t>(ws) & 255) return LPB_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  unsigned char *w = static_cast<unsigned char *>(ws);
  unsigned char *solve_ws = w;
  unsigned char *sets[2] = {w + align256(hp.solve_ws), w + align256(hp.solve_ws) + hp.set_bytes};
  const size_t es = b->dtype == LPB_DTYPE_F64 ? 8 : 4;
  auto ok = [](cudaError_t ce) { return ce == cudaSuccess; };
  // Work already queued on the caller's stream may still use the workspace.
  if (!ok(cudaEventRecord(h->ev_start, s)) || !ok(cudaStreamWaitEvent(h->s_in, h->ev_start, 0)) ||
      !ok(cudaStreamWaitEvent(h->s_out, h->ev_start, 0)))
    return LPB_ECUDA;
  const unsigned char *hA = static_cast<const unsigned char *>(b->A), *hb = static_cast<const unsigned char *>(b->b),
                      *hc = static_cast<const unsigned char *>(b->c);
  for (int i = 0; i < hp.nchunk; ++i) {
    const int j = i & 1;
    unsigned char *set = sets[j];
    const int k0 = i * hp.chunk, k1 = (k0 + hp.chunk < b->count) ? k0 + hp.chunk : b->count, cnt = k1 - k0;
    int64_t a0, a1, b0, b1, c0, c1;
    chunk_range(b->a_off, k0, k1, [&](int k) { return int64_t(b->m[k]) * b->n[k]; }, &a0, &a1);
    chunk_range(b->b_off, k0, k1, [&](int k) { return int64_t(b->m[k]); }, &b0, &b1);
    chunk_range(b->c_off, k0, k1, [&](int k) { return int64_t(b->n[k]); }, &c0, &c1);
    // Copy in: once the solve of chunk i - 2 has consumed this buffer set.
    if (i >= 2 && !ok(cudaStreamWaitEvent(h->s_in, h->ev_comp[j], 0))) return LPB_ECUDA;
    const bool in_ok =
        ok(cudaMemcpyAsync(set + hp.o_A, hA + size_t(a0) * es, size_t(a1 - a0) * es, cudaMemcpyHostToDevice, h->s_in)) &&
        ok(cudaMemcpyAsync(set + hp.o_b, hb + size_t(b0) * es, size_t(b1 - b0) * es, cudaMemcpyHostToDevice, h->s_in)) &&
        ok(cudaMemcpyAsync(set + hp.o_c, hc + size_t(c0) * es, size_t(c1 - c0) * es, cudaMemcpyHostToDevice, h->s_in)) &&
        ok(cudaMemcpyAsync(set + hp.o_m, b->m + k0, size_t(cnt) * 4, cudaMemcpyHostToDevice, h->s_in)) &&
        ok(cudaMemcpyAsync(set + hp.o_n, b->n + k0, size_t(cnt) * 4, cudaMemcpyHostToDevice, h->s_in)) &&
        ok(cudaMemcpyAsync(set + hp.o_ao, b->a_off + k0, size_t(cnt) * 8, cudaMemcpyHostToDevice, h->s_in)) &&
        ok(cudaMemcpyAsync(set + hp.o_bo, b->b_off + k0, size_t(cnt) * 8, cudaMemcpyHostToDevice, h->s_in)) &&
        ok(cudaMemcpyAsync(set + hp.o_co, b->c_off + k0, size_t(cnt) * 8, cudaMemcpyHostToDevice, h->s_in));
    if (!in_ok) return LPB_ECUDA;
    rebase_offsets<<<(cnt + 255) / 256, 256, 0, h->s_in>>>(
        reinterpret_cast<int64_t *>(set + hp.o_ao), reinterpret_cast<int64_t *>(set + hp.o_bo),
        reinterpret_cast<int64_t *>(set + hp.o_co), cnt, a0, b0, c0);
    if (!ok(cudaGetLastError()) || !ok(cudaEventRecord(h->ev_in[j], h->s_in))) return LPB_ECUDA;
    // Solve on the caller's stream, once the inputs are in and the results of
    // chunk i - 2 have left this buffer set.
    if (!ok(cudaStreamWaitEvent(s, h->ev_in[j], 0))) return LPB_ECUDA;
    if (i >= 2 && !ok(cudaStreamWaitEvent(s, h->ev_out[j], 0))) return LPB_ECUDA;
    lpb_batch cb = *b;
    cb.count = cnt;
    cb.m = reinterpret_cast<const int32_t *>(set + hp.o_m);
    cb.n = reinterpret_cast<const int32_t *>(set + hp.o_n);
    cb.a_off = reinterpret_cast<const int64_t *>(set + hp.o_ao);
    cb.b_off = reinterpret_cast<const int64_t *>(set + hp.o_bo);
    cb.c_off = reinterpret_cast<const int64_t *>(set + hp.o_co);
    cb.A = set + hp.o_A;
    cb.b = set + hp.o_b;
    cb.c = set + hp.o_c;
    lpb_result cr{};
    cr.status = reinterpret_cast<int32_t *>(set + hp.o_st);
    cr.iters = r->iters ? reinterpret_cast<int32_t *>(set + hp.o_it) : nullptr;
    cr.obj = reinterpret_cast<double *>(set + hp.o_obj);
    cr.x = reinterpret_cast<double *>(set + hp.o_x);
    cr.y = r->y ? reinterpret_cast<double *>(set + hp.o_y) : nullptr;
    cr.basis = r->basis ? reinterpret_cast<int32_t *>(set + hp.o_bs) : nullptr;
    e = run_solve(d, h->d_ctr, h->d_err, &cb, o, &cr, solve_ws, hp.solve_ws, s, nullptr, nullptr,
                  &h->last_kernels, k0);
    if (e != LPB_OK) return e;
    if (!ok(cudaEventRecord(h->ev_comp[j], s))) return LPB_ECUDA;
    // Copy out.
    if (!ok(cudaStreamWaitEvent(h->s_out, h->ev_comp[j], 0))) return LPB_ECUDA;
    bool out_ok =
        ok(cudaMemcpyAsync(r->status + k0, cr.status, size_t(cnt) * 4, cudaMemcpyDeviceToHost, h->s_out)) &&
        ok(cudaMemcpyAsync(r->obj + k0, cr.obj, size_t(cnt) * 8, cudaMemcpyDeviceToHost, h->s_out)) &&
        ok(cudaMemcpyAsync(r->x + c0, cr.x, size_t(c1 - c0) * 8, cudaMemcpyDeviceToHost, h->s_out));
    if (out_ok && r->iters)
      out_ok = ok(cudaMemcpyAsync(r->iters + k0, cr.iters, size_t(cnt) * 4, cudaMemcpyDeviceToHost, h->s_out));
    if (out_ok && r->y)
      out_ok = ok(cudaMemcpyAsync(r->y + b0, cr.y, size_t(b1 - b0) * 8, cudaMemcpyDeviceToHost, h->s_out));
    if (out_ok && r->basis)
      out_ok = ok(cudaMemcpyAsync(r->basis + b0, cr.basis, size_t(b1 - b0) * 4, cudaMemcpyDeviceToHost, h->s_out));
    if (!out_ok || !ok(cudaEventRecord(h->ev_out[j], h->s_out))) return LPB_ECUDA;
  }
  // The caller's stream passes this point once every result is in host memory.
  for (int j = 0; j < 2 && j < hp.nchunk; ++j)
    if (!ok(cudaStreamWaitEvent(s, h->ev_out[j], 0))) return LPB_ECUDA;
  return LPB_OK;
}

lpb_err lpb_workspace_size_shared(lpb_handle *h, int32_t m, int32_t n, int32_t dtype, int64_t count,
                                  const lpb_options *o, size_t *bytes) {
  if (!h || !o || !bytes) return LPB_EINVAL;
  DeviceScope ds(h->device);
  if (!ds.ok()) return LPB_ECUDA;
  SharedPlan sp;
  const lpb_options os = shared_options(o, m, n);
  const lpb_err e = make_shared_plan(device_info(h), m, n, dtype, count, &os, &sp);
  if (e != LPB_OK) return e;
  *bytes = sp.total;
  return LPB_OK;
}

lpb_err lpb_solve_shared(lpb_handle *h, int32_t m, int32_t n, int32_t dtype, const void *A, const void *b,
                         int64_t count, const void *C, const lpb_options *o, const lpb_result *r, void *ws,
                         size_t ws_bytes, void *stream) {
  if (!h || !o || !r) return LPB_EINVAL;
  if (count == 0) return LPB_OK;
  if (!A || !b || !C || !r->status || !r->obj || !r->x) return LPB_EINVAL;
  if (dtype != LPB_DTYPE_F32 && dtype != LPB_DTYPE_F64) return LPB_EINVAL;
  DeviceScope ds(h->device);
  if (!ds.ok()) return LPB_ECUDA;
  const DeviceInfo d = device_info(h);
  SharedPlan sp;
  const lpb_options os = shared_options(o, m, n);
  o = &os;
  lpb_err e = make_shared_plan(d, m, n, dtype, count, o, &sp);
  if (e != LPB_OK) return e;
  if (ws_bytes < sp.total || !ws) return LPB_ENOMEM;
  if (reinterpret_cast<uintptr_t>(ws) & 255) return LPB_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  unsigned char *w = static_cast<unsigned char *>(ws);
  int32_t *dm = reinterpret_cast<int32_t *>(w + sp.o_m), *dn = reinterpret_cast<int32_t *>(w + sp.o_n);
  int64_t *dao = reinterpret_cast<int64_t *>(w + sp.o_ao), *dbo = reinterpret_cast<int64_t *>(w + sp.o_bo);
  int64_t *dco = reinterpret_cast<int64_t *>(w + sp.o_co), *dyo = reinterpret_cast<int64_t *>(w + sp.o_yo);
  const int cnt = int(count);
  const int grid = (cnt + 255) / 256 < 4 * d.sms ? (cnt + 255) / 256 : 4 * d.sms;
  fill_shared_meta<<<grid, 256, 0, s>>>(dm, dn, dao, dbo, dco, dyo, cnt, m, n);
  if (cudaGetLastError() != cudaSuccess) return LPB_ECUDA;
  lpb_batch bt{};
  bt.count = cnt;
  bt.max_m = m;
  bt.max_n = n;
  bt.min_m = m;
  bt.min_n = n;
  bt.dtype = dtype;
  bt.m = dm;
  bt.n = dn;
  bt.a_off = dao;
  bt.b_off = dbo;
  bt.c_off = dco;
  bt.A = A;
  bt.b = b;
  bt.c = C;
  return run_solve(d, h->d_ctr, h->d_err, &bt, o, r, w + sp.o_ws, sp.solve_ws, s, nullptr, nullptr,
                   &h->last_kernels, 0, dyo, 1);
}

lpb_err lpb_workspace_size_bounded(lpb_handle *h, const lpb_batch *b, const lpb_options *o, size_t *bytes) {
  if (!h || !b || !o || !bytes) return LPB_EINVAL;
  DeviceScope ds(h->device);
  if (!ds.ok()) return LPB_ECUDA;
  BoundedPlan bp;
  const lpb_err e = make_bounded_plan(device_info(h), b, o, &bp);
  if (e != LPB_OK) return e;
  *bytes = bp.total;
  return LPB_OK;
}

lpb_err lpb_solve_bounded(lpb_handle *h, const lpb_batch *b, const void *l, const void *u, const lpb_options *o,
                          const lpb_result *r, void *ws, size_t ws_bytes, void *stream) {
  if (!h || !b || !o || !r) return LPB_EINVAL;
  if (b->count < 0) return LPB_EINVAL;
  if (b->count == 0) return LPB_OK;
  if (!b->m || !b->n || !b->a_off || !b->b_off || !b->c_off || !b->A || !b->b || !b->c || !l || !u)
    return LPB_EINVAL;
  if (!r->status || !r->obj || !r->x || r->basis) return LPB_EINVAL;   // the basis has m + n rows here
  if (b->dtype != LPB_DTYPE_F64) return b->dtype == LPB_DTYPE_F32 ? LPB_EUNSUPPORTED : LPB_EINVAL;
  DeviceScope ds(h->device);
  if (!ds.ok()) return LPB_ECUDA;
  const DeviceInfo d = device_info(h);
  BoundedPlan bp;
  lpb_err e = make_bounded_plan(d, b, o, &bp);
  if (e != LPB_OK) return e;
  if (ws_bytes < bp.total || !ws) return LPB_ENOMEM;
  if (reinterpret_cast<uintptr_t>(ws) & 255) return LPB_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  unsigned char *w = static_cast<unsigned char *>(ws);
  double *A2 = reinterpret_cast<double *>(w + bp.o_A), *b2 = reinterpret_cast<double *>(w + bp.o_b);
  double *y2 = reinterpret_cast<double *>(w + bp.o_y);
  int32_t *m2 = reinterpret_cast<int32_t *>(w + bp.o_m), *n2 = reinterpret_cast<int32_t *>(w + bp.o_n);
  int64_t *ao = reinterpret_cast<int64_t *>(w + bp.o_ao), *bo = reinterpret_cast<int64_t *>(w + bp.o_bo);
  int64_t *co = reinterpret_cast<int64_t *>(w + bp.o_co);
  const BatchDev bd{b->count, b->max_m, b->max_n, b->dtype, b->m, b->n, b->a_off, b->b_off, b->c_off, b->A, b->b, b->c};
  const int grid = b->count < 8 * d.sms ? b->count : 8 * d.sms;
  bounded_transform<double><<<grid, 256, 0, s>>>(bd, static_cast<const double *>(l), static_cast<const double *>(u),
                                                 b->max_m, b->max_n, A2, b2, m2, n2, ao, bo, co);
  if (cudaGetLastError() != cudaSuccess) return LPB_ECUDA;
  // The reduced batch: FP64 data (A is exact, b - A l is formed in FP64), the
  // caller's objectives (c offsets unchanged), results into the caller's x.
  lpb_batch rb{};
  rb.count = b->count;
  rb.max_m = b->max_m + b->max_n;
  rb.max_n = b->max_n;
  rb.dtype = LPB_DTYPE_F64;
  rb.m = m2;
  rb.n = n2;
  rb.a_off = ao;
  rb.b_off = bo;
  rb.c_off = co;
  rb.A = A2;
  rb.b = b2;
  rb.c = b->c;
  lpb_result rr = *r;
  rr.y = y2;
  rr.basis = nullptr;
  e = run_solve(d, h->d_ctr, h->d_err, &rb, o, &rr, w + bp.o_ws, bp.solve_ws, s, nullptr, nullptr,
                &h->last_kernels);
  if (e != LPB_OK) return e;
  bounded_finish<double><<<grid, 256, 0, s>>>(bd, static_cast<const double *>(l), *r, y2, b->max_m, b->max_n);
  return cudaGetLastError() == cudaSuccess ? LPB_OK : LPB_ECUDA;
}

lpb_err lpb_autotune(lpb_handle *h, const lpb_batch *b, const lpb_options *o, const lpb_result *r,
                     void *ws, size_t ws_bytes, const char *table_path, void *stream, float *best_ms) {
  if (!h || !b || !o || !r) return LPB_EINVAL;
  if (best_ms) *best_ms = 0.f;
  DeviceScope ds(h->device);
  if (!ds.ok()) return LPB_ECUDA;
  lpb_handle::Tuned key{b->max_m, b->max_n, b->dtype, o->prec, 0, 0, 0};
  auto store = [&](const lpb_handle::Tuned &t) {
    for (auto &e : h->tuned)
      if (e.max_m == t.max_m && e.max_n == t.max_n && e.dtype == t.dtype && e.prec == t.prec) { e = t; return; }
    h->tuned.push_back(t);
  };
  if (table_path) {                     // a stored entry for this shape wins
    if (FILE *f = std::fopen(table_path, "r")) {
      char tag[16];
      lpb_handle::Tuned t{};
      float ms = 0.f;
      bool found = false;
      while (std::fscanf(f, "%15s %d %d %d %d %d %d %d %f", tag, &t.max_m, &t.max_n, &t.dtype, &t.prec, &t.kernel,
                         &t.threads, &t.reg_warps, &ms) == 9)
        if (!std::strcmp(tag, "lpb-tune") && t.max_m == key.max_m && t.max_n == key.max_n &&
            t.dtype == key.dtype && t.prec == key.prec) {
          store(t);
          found = true;
        }
      std::fclose(f);
      if (found) return LPB_OK;
    }
  }
  if (b->count <= 0) return LPB_EINVAL;
  struct Cand { int kernel, threads, reg_warps; };
  const bool fp32 = o->prec != LPB_FP64;
  const Cand cands[] = {
      {LPB_KERNEL_AUTO, 0, fp32 ? 8 : 0}, {LPB_KERNEL_AUTO, 0, fp32 ? 4 : 0}, {LPB_KERNEL_AUTO, 0, fp32 ? 1 : 0},
      {LPB_KERNEL_AUTO, 256, fp32 ? 8 : 0},
      {LPB_KERNEL_AUTO, 512, fp32 ? 8 : 0}, {LPB_KERNEL_AUTO, 1024, fp32 ? 8 : 0}, {LPB_KERNEL_SMEM, 0, 0},
      {LPB_KERNEL_GMEM, 0, 0}, {fp32 ? LPB_KERNEL_PACK : LPB_KERNEL_AUTO, 0, 0},
      {fp32 ? LPB_KERNEL_WARP : LPB_KERNEL_AUTO, 0, 0}};
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return LPB_ECUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return LPB_ECUDA; }
  const DeviceInfo d = device_info(h);
  float best = -1.f;
  lpb_handle::Tuned win = key;
  lpb_err status = LPB_OK;
  for (const Cand &c : cands) {
    lpb_options oc = *o;
    oc.kernel = c.kernel;
    oc.threads = c.threads;
    oc.reg_warps = c.reg_warps;
    size_t need = 0;
    if (solve_workspace_bytes(d, b, &oc, r->basis != nullptr, &need) != LPB_OK || need > ws_bytes) continue;
    if (run_solve(d, h->d_ctr, h->d_err, b, &oc, r, ws, ws_bytes, s, nullptr, nullptr) != LPB_OK) continue;
    if (cudaEventRecord(e0, s) != cudaSuccess) { status = LPB_ECUDA; break; }
    lpb_err er = LPB_OK;
    for (int rep = 0; rep < 2 && er == LPB_OK; ++rep)
      er = run_solve(d, h->d_ctr, h->d_err, b, &oc, r, ws, ws_bytes, s, nullptr, nullptr);
    if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) { status = LPB_ECUDA; break; }
    float ms = 0.f;
    if (er != LPB_OK || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) continue;
    ms *= 0.5f;
    if (best < 0.f || ms < best) {
      best = ms;
      win.kernel = c.kernel;
      win.threads = c.threads;
      win.reg_warps = c.reg_warps;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (status != LPB_OK) return status;
  if (best < 0.f) return LPB_EUNSUPPORTED;
  store(win);
  if (best_ms) *best_ms = best;
  if (table_path)
    if (FILE *f = std::fopen(table_path, "a")) {
      std::fprintf(f, "lpb-tune %d %d %d %d %d %d %d %.6f\n", win.max_m, win.max_n, win.dtype, win.prec, win.kernel,
                   win.threads, win.reg_warps, best);
      std::fclose(f);
    }
  return LPB_OK;
}

lpb_err lpb_profile_start(lpb_handle *h, int32_t calls) {
  if (!h || calls < 1 || calls > lpb_handle::kProfMax) return LPB_EINVAL;
  DeviceScope ds(h->device);
  if (!ds.ok()) return LPB_ECUDA;
  if (!h->prof_ev) {
    h->prof_ev = new (std::nothrow) cudaEvent_t[lpb_handle::kProfMax * 3 * 2];
    if (!h->prof_ev) return LPB_ENOMEM;
    for (int i = 0; i < lpb_handle::kProfMax * 3 * 2; ++i)
      if (cudaEventCreate(&h->prof_ev[i]) != cudaSuccess) return LPB_ECUDA;
  }
  std::memset(h->prof_ran, 0, sizeof(h->prof_ran));
  h->prof_cap = calls;
  h->prof_n = 0;
  return LPB_OK;
}

lpb_err lpb_profile_read(lpb_handle *h, float *ms, int32_t max_calls, int32_t *ncalls) {
  if (!h || !ms || !ncalls || max_calls < 0) return LPB_EINVAL;
  DeviceScope ds(h->device);
  if (!ds.ok()) return LPB_ECUDA;
  const int n = h->prof_n < max_calls ? h->prof_n : max_calls;
  for (int i = 0; i < n; ++i)
    for (int p = 0; p < 3; ++p) {
      ms[3 * i + p] = 0.f;
      if (!h->prof_ran[i * 3 + p]) continue;
      cudaEvent_t *ev = h->prof_ev + (size_t(i) * 3 + p) * 2;
      if (cudaEventSynchronize(ev[1]) != cudaSuccess) return LPB_ECUDA;
      if (cudaEventElapsedTime(&ms[3 * i + p], ev[0], ev[1]) != cudaSuccess) return LPB_ECUDA;
    }
  *ncalls = n;
  h->prof_cap = 0;
  h->prof_n = 0;
  return LPB_OK;
}

lpb_err lpb_solve_backward(lpb_handle *h, const lpb_batch *b, const lpb_options *o,
                           const lpb_result *r, const double *g_obj, const double *g_x, double *g_c,
                           double *g_b, double *g_A, void *ws, size_t ws_bytes, void *stream) {
  if (!h || !b || !o || !r) return LPB_EINVAL;
  if (b->count < 0) return LPB_EINVAL;
  if (b->count == 0) return LPB_OK;
  if (!b->m || !b->n || !b->a_off || !b->b_off || !b->c_off || !b->A) return LPB_EINVAL;
  if (!r->status || !r->x || !r->y || !r->basis || !g_c || !g_b || !g_A) return LPB_EINVAL;
  if (b->max_m < 1 || b->max_n < 1 || b->max_m > kMaxDim || b->max_n > kMaxDim) return LPB_EUNSUPPORTED;
  if (b->dtype != LPB_DTYPE_F32 && b->dtype != LPB_DTYPE_F64) return LPB_EINVAL;
  DeviceScope ds(h->device);
  if (!ds.ok()) return LPB_ECUDA;
  const size_t smem = backward_smem_bytes(b->max_m, b->max_n);
  if (smem > h->smem_optin) return LPB_EUNSUPPORTED;
  int grid = 0;
  if (backward_grid(h->sms, smem, &grid) != cudaSuccess) return LPB_ECUDA;
  if (grid > b->count) grid = b->count;
  const size_t slot = backward_slot_bytes(b->max_m, b->max_n);
  if (slot * size_t(grid) > ws_bytes || (slot && !ws)) return LPB_ENOMEM;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  BackwardParams p{};
  p.B = BatchDev{b->count, b->max_m, b->max_n, b->dtype, b->m, b->n, b->a_off, b->b_off, b->c_off,
                 b->A, b->b, b->c};
  p.status = r->status;
  p.basis = r->basis;
  p.x = r->x;
  p.y = r->y;
  p.g_obj = g_obj;
  p.g_x = g_x;
  p.g_c = g_c;
  p.g_b = g_b;
  p.g_A = g_A;
  p.slots = ws;
  p.slot_bytes = slot;
  p.queue = h->d_ctr + CTR_BWD;
  p.err = h->d_err;
  if (cudaMemsetAsync(p.queue, 0, sizeof(int32_t), s) != cudaSuccess) return LPB_ECUDA;
  return launch_backward(p, grid, smem, s) == cudaSuccess ? LPB_OK : LPB_ECUDA;
}

lpb_err lpb_hyperbox(lpb_handle *h, int64_t count, int32_t n, int32_t dtype, const void *c,
                     const void *l, const void *u, int32_t shared_box, void *obj, void *x,
                     void *stream) {
  if (!h || count < 0 || n < 1) return LPB_EINVAL;
  if (dtype != LPB_DTYPE_F32 && dtype != LPB_DTYPE_F64) return LPB_EINVAL;
  if (count == 0) return LPB_OK;
  if (!c || !l || !u || !obj) return LPB_EINVAL;
  DeviceScope ds(h->device);
  if (!ds.ok()) return LPB_ECUDA;
  const size_t smem = hyperbox_smem_bytes(n, dtype == LPB_DTYPE_F64 ? 8 : 4, shared_box != 0);
  if (smem > h->smem_optin) return LPB_EUNSUPPORTED;
  HyperboxParams p{count, n, dtype, shared_box != 0, c, l, u, obj, x};
  return launch_hyperbox(p, h->d_err, static_cast<cudaStream_t>(stream)) == cudaSuccess ? LPB_OK : LPB_ECUDA;
}

lpb_err lpb_sync_error(lpb_handle *h, void *stream, uint32_t *word) {
  if (!h) return LPB_EINVAL;
  DeviceScope ds(h->device);
  if (!ds.ok()) return LPB_ECUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  uint32_t v = 0;
  if (cudaStreamSynchronize(s) != cudaSuccess) return LPB_ECUDA;
  if (cudaMemcpy(&v, h->d_err, sizeof(v), cudaMemcpyDeviceToHost) != cudaSuccess) return LPB_ECUDA;
  if (cudaMemset(h->d_err, 0, sizeof(v)) != cudaSuccess) return LPB_ECUDA;
  if (word) *word = v;
  return v ? LPB_EDEVICE : LPB_OK;
}

lpb_err lpb_get_stats(lpb_handle *h, void *stream, lpb_stats *st) {
  if (!h || !st) return LPB_EINVAL;
  DeviceScope ds(h->device);
  if (!ds.ok()) return LPB_ECUDA;
  int32_t c[CTR_N];
  if (cudaStreamSynchronize(static_cast<cudaStream_t>(stream)) != cudaSuccess) return LPB_ECUDA;
  if (cudaMemcpy(c, h->d_ctr, sizeof(c), cudaMemcpyDeviceToHost) != cudaSuccess) return LPB_ECUDA;
  std::memset(st, 0, sizeof(*st));
  st->deferred = c[CTR_DEFER];
  st->resolved_fp64 = c[CTR_RESOLVE];
  st->kernels = h->last_kernels;
  return LPB_OK;
}

}  // extern "C"
