// backward.cu -- vector-Jacobian products of obj and x* through the optimal basis.
//
// For max c^T x, A x <= b, x >= 0 (Section 3, Eq. 1-3) at an optimal basis B:
// let S be the basic structural variables and N the rows whose slack is
// non-basic (the binding rows).  Every other row's slack is basic, so
//   x_S solves A[N,S] x_S = b_N,   y_N solves A[N,S]^T y_N = c_S,  y = 0 off N,
// and for upstream gradients g_obj (a scalar per LP) and g_x (one per x_j):
//   v_N solves A[N,S]^T v_N = g_x[S]   (v = B^{-T} g_B, zero off N),
//   d/dc = g_obj x*,   d/db = g_obj y + v,   d/dA = -(g_obj y + v) x*^T.
// (x* does not move with c while the basis stays optimal.)  The k x k system
// (k = |S| = |N|) is rebuilt from the stored basis indices and solved in FP64
// by Gaussian elimination with partial pivoting -- about k^3/3 FP64 FMAs, small
// because k, the number of basic structurals, is small at these optima.
// LPs that are not optimal, or whose basis is not square on (N, S) (a
// redundant row was dropped) or is singular, get zero gradients.
#include "lpb_internal.cuh"

namespace lpb {
namespace {

constexpr int kBwdThreads = 256;
constexpr int kSmemK = 64;      // systems up to this size are eliminated in shared memory

struct BwdLayout {
  size_t w, flag, slist, nlist, v, mt, total;
};

__host__ __device__ inline size_t al16(size_t x) { return (x + 15) & ~size_t(15); }

__host__ __device__ inline BwdLayout bwd_layout(int max_m, int kmax) {
  BwdLayout L{};
  const int ks = kmax < kSmemK ? kmax : kSmemK;
  size_t o = 0;
  L.w = o;     o = al16(o + size_t(max_m) * 8);
  L.flag = o;  o = al16(o + size_t(max_m) * 4);
  L.slist = o; o = al16(o + size_t(kmax) * 4);
  L.nlist = o; o = al16(o + size_t(kmax) * 4);
  L.v = o;     o = al16(o + size_t(kmax) * 8);
  L.mt = o;    o = al16(o + size_t(ks) * size_t(ks + 1) * 8);
  L.total = o;
  return L;
}

// Solve the k x k system held as [M | g] (row-major, leading dimension k + 1)
// for k <= 32 in one warp: lane r owns row r.  Gaussian elimination with
// partial pivoting (the largest |M[r][p]|, ties to the lowest row, found on
// the magnitude bits with integer warp reductions), one division per row and
// step, then back substitution by columns (each lane updates its own right-
// hand side).  FP64 is the scarce unit here, so no FP64 work is spent on
// reductions.  Returns false (warp-uniform) if a pivot is zero.
__device__ bool warp_solve(double *mt, int k, double *v) {
  const int lane = threadIdx.x & 31, ld = k + 1;
  for (int p = 0; p < k; ++p) {
    const unsigned long long mag =
        (lane >= p && lane < k) ? static_cast<unsigned long long>(__double_as_longlong(mt[lane * ld + p])) &
                                      0x7fffffffffffffffull
                                : 0ull;
    const unsigned hi = __reduce_max_sync(kFull, unsigned(mag >> 32));
    const unsigned lo = __reduce_max_sync(kFull, unsigned(mag >> 32) == hi ? unsigned(mag) : 0u);
    const bool top = unsigned(mag >> 32) == hi && unsigned(mag) == lo && lane >= p && lane < k;
    const int bk = int(__reduce_min_sync(kFull, top ? unsigned(lane) : 0xffffffffu));
    if ((hi | lo) == 0u) return false;                 // a zero column: singular
    if (bk != p)
      for (int c = p + lane; c < ld; c += 32) {
        const double t0 = mt[p * ld + c];
        mt[p * ld + c] = mt[bk * ld + c];
        mt[bk * ld + c] = t0;
      }
    __syncwarp();
    const double piv = mt[p * ld + p];
    if (lane > p && lane < k) {
      const double l = mt[lane * ld + p] / piv;
      for (int c = p + 1; c < ld; ++c) mt[lane * ld + c] = fma(-l, mt[p * ld + c], mt[lane * ld + c]);
    }
    __syncwarp();
  }
  for (int b = k - 1; b >= 0; --b) {
    double vb = 0.0;
    if (lane == b) vb = mt[b * ld + k] / mt[b * ld + b];
    vb = __shfl_sync(kFull, vb, b);
    if (lane < b) mt[lane * ld + k] = fma(-mt[lane * ld + b], vb, mt[lane * ld + k]);
    if (lane == 0) v[b] = vb;
    __syncwarp();
  }
  return true;
}

__global__ void __launch_bounds__(kBwdThreads) backward_kernel(BackwardParams P) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
  const int kmax = P.B.max_m < P.B.max_n ? P.B.max_m : P.B.max_n;
  const BwdLayout L = bwd_layout(P.B.max_m, kmax);
  double *w = reinterpret_cast<double *>(smem + L.w);
  int *flag = reinterpret_cast<int *>(smem + L.flag);
  int *slist = reinterpret_cast<int *>(smem + L.slist);
  int *nlist = reinterpret_cast<int *>(smem + L.nlist);
  double *vN = reinterpret_cast<double *>(smem + L.v);
  __shared__ int s_item, s_k, s_kn, s_ok;
  __shared__ double s_redv[32];
  __shared__ int s_redk[32];
  const int dt = P.B.dtype;

  for (;;) {
    if (tid == 0) s_item = atomicAdd(P.queue, 1);
    __syncthreads();
    const int lp = s_item;
    if (lp >= P.B.count) break;
    const int m = P.B.m[lp], n = P.B.n[lp];
    if (m < 1 || n < 1 || m > P.B.max_m || n > P.B.max_n) { __syncthreads(); continue; }
    const int64_t aoff = P.B.a_off[lp], boff = P.B.b_off[lp], coff = P.B.c_off[lp];
    const double go = P.g_obj ? P.g_obj[lp] : 0.0;
    bool ok = P.status[lp] == LPB_OPTIMAL;
    bool zeroed = false;                // the zeros of g_A are written
    // S: structural basic variables (in row order), N: rows whose slack is not basic.
    for (int i = tid; i < m; i += nt) flag[i] = 0;
    __syncthreads();
    for (int t = tid; t < m; t += nt) {
      const int v = P.basis[boff + t];
      if (v >= n && v < n + m) flag[v - n] = 1;
      if (v < 0) ok = false;
    }
    ok = __syncthreads_and(ok);
    if (wid == 0) {
      int base = 0, basen = 0;
      for (int i0 = 0; i0 < m; i0 += 32) {
        const int i = i0 + lane;
        const int v = i < m ? P.basis[boff + i] : -1;
        const bool s = i < m && v >= 0 && v < n;
        const bool nn = i < m && !flag[i];
        const unsigned ms = __ballot_sync(kFull, s), mn = __ballot_sync(kFull, nn);
        const unsigned below = (1u << lane) - 1u;
        if (s && base + __popc(ms & below) < kmax) slist[base + __popc(ms & below)] = v;
        if (nn && basen + __popc(mn & below) < kmax) nlist[basen + __popc(mn & below)] = i;
        base += __popc(ms);
        basen += __popc(mn);
      }
      if (lane == 0) { s_k = base; s_kn = basen; }
    }
    __syncthreads();
    const int k = s_k;
    ok = ok && k == s_kn && k <= kmax;
    // v_N from A[N,S]^T v_N = g_x[S] by elimination on [M^T | g].
    if (ok && P.g_x && k > 0) {
      double *mt = k <= kSmemK ? reinterpret_cast<double *>(smem + L.mt)
                               : reinterpret_cast<double *>(static_cast<unsigned char *>(P.slots) +
                                                            size_t(blockIdx.x) * P.slot_bytes);
      const int ld = k + 1;
      for (int idx = tid; idx < k * ld; idx += nt) {
        const int a = idx / ld, c = idx - a * ld;
        mt[idx] = c < k ? ld_in(P.B.A, aoff + int64_t(nlist[c]) * n + slist[a], dt)
                        : P.g_x[coff + slist[a]];
      }
      if (tid == 0) s_ok = 1;
      __syncthreads();
      if (k <= 32) {                    // small systems (the usual case): one warp
        if (wid == 0) {
          const bool solved = warp_solve(mt, k, vN);
          if (lane == 0 && !solved) s_ok = 0;
        } else {                        // meanwhile the other warps write the zeros of g_A
          for (int i = wid - 1; i < m; i += nw - 1) {
            double *row = P.g_A + aoff + int64_t(i) * n;
            for (int j = lane; j < n; j += 32) row[j] = 0.0;
          }
        }
        zeroed = true;
        __syncthreads();
        if (!s_ok) ok = false;
      } else {
      for (int p = 0; p < k; ++p) {
        // partial pivoting: the largest |mt[r][p]|, r >= p
        double bv = 1.0;     // compared as -|value| so the arg-min picks the largest
        int bk = INT_MAX;
        for (int r = p + tid; r < k; r += nt) {
          const double a = fabs(mt[r * ld + p]);
          keep_better(bv, bk, -a, r);
        }
        block_argmin(bv, bk, s_redv, s_redk);
        if (bk == INT_MAX || -bv <= 1e-300) { if (tid == 0) s_ok = 0; __syncthreads(); break; }
        if (bk != p)
          for (int c = p + tid; c < ld; c += nt) {
            const double t0 = mt[p * ld + c];
            mt[p * ld + c] = mt[bk * ld + c];
            mt[bk * ld + c] = t0;
          }
        __syncthreads();
        // One division per row for the multipliers (kept in column p, which
        // the later steps no longer read), then the rank-1 update: FP64
        // division is a long instruction sequence on this GPU's slow FP64 unit.
        const double piv = mt[p * ld + p];
        const int rows = k - p - 1, cols = ld - p - 1;
        for (int r = p + 1 + tid; r < k; r += nt) mt[r * ld + p] = mt[r * ld + p] / piv;
        __syncthreads();
        for (int idx = tid; idx < rows * cols; idx += nt) {
          const int r = p + 1 + idx / cols, c = p + 1 + idx % cols;
          mt[r * ld + c] = fma(-mt[r * ld + p], mt[p * ld + c], mt[r * ld + c]);
        }
        __syncthreads();
      }
      if (s_ok) {
        // back substitution, one unknown at a time (k is small)
        for (int b = k - 1; b >= 0; --b) {
          double s = 0.0;
          for (int c = b + 1 + tid; c < k; c += nt) s = fma(mt[b * ld + c], vN[c], s);
          s = warp_sum(s);
          if (lane == 0) s_redv[wid] = s;
          __syncthreads();
          if (tid == 0) {
            double t = 0.0;
            for (int q = 0; q < nw; ++q) t += s_redv[q];
            vN[b] = (mt[b * ld + k] - t) / mt[b * ld + b];
          }
          __syncthreads();
        }
      } else {
        ok = false;
      }
      }
    } else if (ok) {
      for (int b = tid; b < k; b += nt) vN[b] = 0.0;
    }
    __syncthreads();
    // w = g_obj y + v; then g_b = w, g_c = g_obj x, g_A = -w x^T.
    for (int i = tid; i < m; i += nt) w[i] = ok ? go * P.y[boff + i] : 0.0;
    __syncthreads();
    if (ok)
      for (int b = tid; b < k; b += nt) w[nlist[b]] += vN[b];
    __syncthreads();
    for (int i = tid; i < m; i += nt) P.g_b[boff + i] = w[i];
    for (int j = tid; j < n; j += nt) P.g_c[coff + j] = ok ? go * P.x[coff + j] : 0.0;
    // g_A = -w x*^T: x* is zero off the basic structurals, so the rows are
    // written as zeros (unless that was done during the elimination) and only
    // those k columns take an FP64 product.
    if (!zeroed) {
      for (int i = wid; i < m; i += nw) {
        double *row = P.g_A + aoff + int64_t(i) * n;
        for (int j = lane; j < n; j += 32) row[j] = 0.0;
      }
      __syncthreads();
    }
    if (ok)
      for (int q = wid; q < k; q += nw) {
        const int j = slist[q];
        const double xj = P.x[coff + j];
        for (int i = lane; i < m; i += 32) P.g_A[aoff + int64_t(i) * n + j] = -w[i] * xj;
      }
    __syncthreads();
  }
}

}  // namespace

size_t backward_smem_bytes(int max_m, int max_n) {
  return bwd_layout(max_m, max_m < max_n ? max_m : max_n).total;
}

size_t backward_slot_bytes(int max_m, int max_n) {
  const int kmax = max_m < max_n ? max_m : max_n;
  return kmax > kSmemK ? al16(size_t(kmax) * size_t(kmax + 1) * 8) : 0;
}

cudaError_t backward_grid(int sms, size_t smem, int *grid) {
  cudaError_t e = cudaFuncSetAttribute(backward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (e != cudaSuccess) return e;
  int occ = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, backward_kernel, kBwdThreads, smem);
  if (e != cudaSuccess) return e;
  *grid = occ * sms;
  return occ > 0 ? cudaSuccess : cudaErrorInvalidConfiguration;
}

cudaError_t launch_backward(const BackwardParams &p, int grid, size_t smem, cudaStream_t s) {
  cudaError_t e = cudaFuncSetAttribute(backward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (e != cudaSuccess) return e;
  backward_kernel<<<grid, kBwdThreads, smem, s>>>(p);
  return cudaGetLastError();
}

}  // namespace lpb
