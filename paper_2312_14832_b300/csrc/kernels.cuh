// Device kernels of the restarted-PDHG hot path (arXiv 2312.14832, Section 2).
//
// Everything runs in FP64 on the solver's internal numbering (rows and columns
// sorted by length, see layout.h) and on the scaled problem
// Kt = Dr K Dc, ct = Dc c, qt = Dr q, lt = l/Dc, ut = u/Dc.
//
// FP64 on this part issues one warp instruction per ~16 SM cycles whatever the
// number of active lanes, so the kernels keep every lane of every FP64
// instruction busy (one row per lane) and do comparisons, clamps and sign
// projections with integer operations on the bit patterns instead of FP64
// min/max.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include <type_traits>

#include "layout.h"

namespace pdlp {

// ------------------------------------------------------------------ state

// Scalars of a solve that live on the device, so that a captured check
// interval needs no host involvement.
struct DevState {
  double tau, sigma, omega, eta;   // tau = eta/omega, sigma = eta*omega
  double kkt_anchor, kkt_prev;     // KKT_omega(z^{n,0}) and of the previous candidate
  double inv_t;                    // 1/t at the current check (0 when t = 0)
  double out_pobj, out_dobj, out_rel_p, out_rel_d, out_rel_g, out_kkt;  // returned point
  double last_err;                 // largest relative error of the better point at the last check
  long long k, t, nrestart, ncheck;
  int done, status, which, restart_flag, cand_avg, final_force;
  // adaptive step rule: weight sum of the running sums, weight of the current iterate
  // not yet added to them, steps accepted, rejections in a row, last attempt accepted
  double wsum, pw;
  long long accepted;
  int rejects, accept;
  double p3, p6;   // (s+1)^-0.3 and (s+1)^-0.6 for the next acceptance decision
  int suspended;   // batched solver: stopped at a check by its iteration slice, resumable
  int reject_cap;  // adaptive step rule: an attempt is kept after this many rejections in a row
  long long k32;   // batched mixed precision: iterations run in FP32
};

struct DevParams {
  double tol, beta_suff, beta_nec, beta_art, theta;
  double qnorm, cnorm;            // unscaled ||q||_2, ||c||_2
  long long max_iter;
  int log_cap, restart_cap;
};

struct CheckRecord {              // same layout as pdlp_check_record
  long long k, t;
  int restart, candidate;
  double omega, kkt_cur, kkt_avg, kkt_anchor, rel_p, rel_d, rel_g;
};

// quantities reduced at a check (current point "C", average "A")
enum {
  Q_PRS_C = 0, Q_PRU_C, Q_QY_C, Q_DY_C,            // from the rows of K
  Q_PRS_A, Q_PRU_A, Q_QY_A, Q_DY_A,
  Q_DRS_C, Q_DRU_C, Q_LT_C, Q_CX_C, Q_DX_C,        // from the columns
  Q_DRS_A, Q_DRU_A, Q_LT_A, Q_CX_A, Q_DX_A,
  NQ
};

// ------------------------------------------------------------------ helpers

// Order-preserving map of a double to int64 (for non-NaN values).
__device__ __forceinline__ long long okey(double d) {
  long long b = __double_as_longlong(d);
  return b ^ ((b >> 63) & 0x7fffffffffffffffLL);
}
// proj onto [l, u] with integer comparisons.
__device__ __forceinline__ double clamp_box(double x, double l, double u) {
  long long kx = okey(x);
  double r = x;
  if (kx < okey(l)) r = l;
  if (kx > okey(u)) r = u;
  return r;
}
// max(y, 0) and min(y, 0) by the sign bit.
__device__ __forceinline__ double max0(double y) { return (__double2hiint(y) < 0) ? 0.0 : y; }
__device__ __forceinline__ double min0(double y) { return (__double2hiint(y) < 0) ? y : 0.0; }
__device__ __forceinline__ bool is_neg_inf(double v) {
  return __double_as_longlong(v) == (long long)0xFFF0000000000000ULL;
}
__device__ __forceinline__ bool is_pos_inf(double v) {
  return __double_as_longlong(v) == (long long)0x7FF0000000000000ULL;
}
__device__ __forceinline__ bool is_zero(double v) {
  return (__double_as_longlong(v) & 0x7fffffffffffffffLL) == 0;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

#define PDLP_GRID_STRIDE(i, n) \
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (n); i += (int64_t)gridDim.x * blockDim.x)

// ------------------------------------------------------------------ SELL SpMV

struct SellView {
  const int32_t* __restrict__ chunk_ptr;
  const int32_t* __restrict__ col;
  const double* __restrict__ val;
  const float* __restrict__ val32;   // FP32 copy of val (mixed precision), or null
  const SellTask* __restrict__ tasks;
  int32_t ntasks;
  int32_t nchunks;
  double* gpart;   // ntasks * 32 partial sums of split-chunk pieces
  int32_t* cnt;    // arrival counters (index: first piece task), zero between launches
  // K with entries +-1 only (mixed precision): per slot, the column index in bits 0..30
  // and the sign of the entry in bit 31; padding slots hold the index of an entry of the
  // gathered vector that stays zero.  Null otherwise.
  const int32_t* __restrict__ ucol;
};

// Row-sum operations: SpMV (gathered), and the infinity / 1-norms used by scaling.
struct OpSpmv {
  static constexpr bool kGather = true;
  __device__ static double step(double acc, double v, double x) { return fma(v, x, acc); }
  __device__ static double join(double a, double b) { return a + b; }
};
struct OpMaxAbs {
  static constexpr bool kGather = false;
  __device__ static double step(double acc, double v, double) {
    long long a = __double_as_longlong(v) & 0x7fffffffffffffffLL;
    long long b = __double_as_longlong(acc);
    return __longlong_as_double(a > b ? a : b);
  }
  __device__ static double join(double a, double b) { return step(a, b, 0.0); }
};
struct OpSumAbs {
  static constexpr bool kGather = false;
  __device__ static double step(double acc, double v, double) { return acc + fabs(v); }
  __device__ static double join(double a, double b) { return a + b; }
};
// FP32 SpMV (mixed precision iterations).
struct OpSpmvF {
  static constexpr bool kGather = true;
  __device__ static float step(float acc, float v, float x) { return fmaf(v, x, acc); }
};
// FP32 row sums of the unscaled signs of a K whose entries are all +-1 (SellView::ucol):
// sum_j s_ij x_j, with x_j taken with its sign flipped where s_ij = -1 (exact).
struct OpUnitF {
  static constexpr bool kGather = true;
};

// Combination of split-chunk partial sums (kept in FP64 for every value type).
template <class Op> __device__ __forceinline__ double join_of(double a, double b) { return a + b; }
template <> __device__ __forceinline__ double join_of<OpMaxAbs>(double a, double b) { return OpMaxAbs::join(a, b); }

template <class T> __device__ __forceinline__ const T* sell_values(const SellView& A);
template <> __device__ __forceinline__ const double* sell_values<double>(const SellView& A) { return A.val; }
template <> __device__ __forceinline__ const float* sell_values<float>(const SellView& A) { return A.val32; }

// OpUnitF's sum of slots [s, e) of one chunk for this lane's row: only the 4-byte
// column words are streamed; the batching is chunk_sum's.
template <int kBatch>
__device__ __forceinline__ float chunk_sum_unit(const SellView& A, const float* __restrict__ xg, int s, int e,
                                                int lane) {
  const int32_t* cp = A.ucol + (size_t)s * 32 + lane;
  float acc = 0.0f;
  for (int k = s; k < e; k += kBatch) {
    const int nb = min(kBatch, e - k);
    uint32_t w[kBatch];
    float xv[kBatch];
#pragma unroll
    for (int j = 0; j < kBatch; ++j) {
      w[j] = 0u;
      if (j < nb) w[j] = (uint32_t)__ldcs(cp + 32 * j);
    }
#pragma unroll
    for (int j = 0; j < kBatch; ++j) {
      xv[j] = 0.0f;
      if (j < nb) xv[j] = __ldg(xg + (w[j] & 0x7fffffffu));
    }
#pragma unroll
    for (int j = 0; j < kBatch; ++j)
      if (j < nb) acc += __uint_as_float(__float_as_uint(xv[j]) ^ (w[j] & 0x80000000u));
    cp += 32 * kBatch;
  }
  return acc;
}

// Sum of slots [s, e) of one chunk for this lane's row.  Loads of a batch of up to
// kBatch slots are issued before any of its FMAs; `nb` is warp-uniform, so the
// guards do not diverge and no FP64 instruction is spent on a missing slot.
template <class T, class Op, int kBatch>
__device__ __forceinline__ T chunk_sum_vals(const SellView& A, const T* __restrict__ xg, int s, int e, int lane) {
  const int32_t* cp = A.col + (size_t)s * 32 + lane;
  const T* vp = sell_values<T>(A) + (size_t)s * 32 + lane;
  T acc = T(0);
  for (int k = s; k < e; k += kBatch) {
    const int nb = min(kBatch, e - k);
    T v[kBatch], xv[kBatch];
    int ci[kBatch];
#pragma unroll
    for (int j = 0; j < kBatch; ++j) {
      if (j < nb) {
        v[j] = __ldcs(vp + 32 * j);
        if (Op::kGather) ci[j] = __ldcs(cp + 32 * j);
      }
    }
#pragma unroll
    for (int j = 0; j < kBatch; ++j) {
      xv[j] = T(0);
      if (Op::kGather && j < nb) xv[j] = __ldg(xg + ci[j]);
    }
#pragma unroll
    for (int j = 0; j < kBatch; ++j)
      if (j < nb) acc = Op::step(acc, v[j], xv[j]);
    vp += 32 * kBatch;
    cp += 32 * kBatch;
  }
  return acc;
}

template <class T, class Op, int kBatch>
__device__ __forceinline__ T chunk_sum(const SellView& A, const T* __restrict__ xg, int s, int e, int lane) {
  if constexpr (std::is_same<Op, OpUnitF>::value)
    return chunk_sum_unit<kBatch>(A, xg, s, e, lane);
  else
    return chunk_sum_vals<T, Op, kBatch>(A, xg, s, e, lane);
}

// A wide chunk's row sum: the lanes' partial sums combined by a fixed butterfly, the
// total in lane 0 (the row), 0 in the padding rows of lanes 1..31.
template <class Op, class T>
__device__ __forceinline__ T wide_total(T part, int lane) {
  double v = (double)part;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = join_of<Op>(v, __shfl_xor_sync(0xffffffffu, v, o));
  return lane == 0 ? (T)v : T(0);
}

// One warp per task; lane = row of the chunk.  Epi::finish(row, sum, pre) receives the
// complete row sum exactly once per row; Epi::load(row) fetches, before the row's
// SpMV loop, the operands the epilogue needs, so their latency overlaps it.
template <class Op, class Epi, int kBatch>
__global__ void __launch_bounds__(256) sell_rows_kernel(SellView A, const typename Epi::T* __restrict__ xg,
                                                        Epi epi, const DevState* __restrict__ st) {
  using T = typename Epi::T;
  if (st != nullptr && st->done) return;
  const int lane = threadIdx.x & 31;
  const int w = (int)((blockIdx.x * (unsigned)blockDim.x + threadIdx.x) >> 5);
  if (w >= A.ntasks) return;
  const SellTask Tk = A.tasks[w];
  epi.prepare(st);
  if (Tk.np == 0) {
    // whole chunks T.chunk .. T.chunk + nc - 1; lane j holds the start of chunk j
    const int cb = A.chunk_ptr[min(Tk.chunk + lane, A.nchunks)];
    for (int j = 0; j < Tk.nc; ++j) {
      const int s = __shfl_sync(0xffffffffu, cb, j);
      const int e = __shfl_sync(0xffffffffu, cb, j + 1);
      const int row = (Tk.chunk + j) * 32 + lane;
      const typename Epi::Pre pre = epi.load(row);
      T acc = chunk_sum<T, Op, kBatch>(A, xg, s, e, lane);
      if (Tk.wide) acc = wide_total<Op>(acc, lane);
      epi.finish(row, acc, pre);
    }
    epi.task_end(w, lane);
  } else {
    // piece of a split chunk: publish, count arrivals, the last arrival combines
    const T acc = chunk_sum<T, Op, kBatch>(A, xg, Tk.s0, Tk.s1, lane);
    const int row = Tk.chunk * 32 + lane;
    A.gpart[(size_t)w * 32 + lane] = (double)acc;
    __threadfence();
    int old = 0;
    if (lane == 0) old = atomicAdd(A.cnt + Tk.t0, 1);
    old = __shfl_sync(0xffffffffu, old, 0);
    if (old == Tk.np - 1) {
      __threadfence();
      const typename Epi::Pre pre = epi.load(row);
      double sum = __ldcg(A.gpart + (size_t)Tk.t0 * 32 + lane);
      for (int i = 1; i < Tk.np; ++i) sum = join_of<Op>(sum, __ldcg(A.gpart + (size_t)(Tk.t0 + i) * 32 + lane));
      if (lane == 0) A.cnt[Tk.t0] = 0;
      if (Tk.wide) sum = wide_total<Op>(sum, lane);
      epi.finish(row, (T)sum, pre);
    }
    epi.task_end(w, lane);
  }
}

// out[row] = sum (optionally times the state's 1/t, for products of the average).
struct EpiStore {
  using T = double;
  double* out;
  int use_inv_t;
  double scale;
  struct Pre {};
  __device__ void prepare(const DevState* st) { scale = (use_inv_t && st) ? st->inv_t : 1.0; }
  __device__ Pre load(int) const { return Pre{}; }
  __device__ void finish(int r, double s, const Pre&) { out[r] = use_inv_t ? s * scale : s; }
  __device__ void task_end(int, int) {}
};

// Primal step fused on g = (K'y)_j (Section 2, primal update):
//   x_j <- proj_[l_j,u_j](x_j - tau (c_j - g_j)),  sx_j += x_j.
struct EpiPrimal {
  using T = double;
  double* __restrict__ x;
  double* __restrict__ sx;
  const double* __restrict__ c;
  const double* __restrict__ l;
  const double* __restrict__ u;
  double tau;
  struct Pre { double xo, c, l, u, sx; };
  __device__ void prepare(const DevState* st) { tau = st->tau; }
  __device__ Pre load(int j) const { return Pre{x[j], c[j], l[j], u[j], sx[j]}; }
  __device__ void finish(int j, double g, const Pre& p) {
    const double d = p.c - g;
    const double xn = clamp_box(fma(-tau, d, p.xo), p.l, p.u);
    x[j] = xn;
    sx[j] = p.sx + xn;
  }
  __device__ void task_end(int, int) {}
};

// Dual step fused on v = (K x_new)_i (Section 2, dual update with extrapolation,
// using K(2 x_new - x_old) = 2 v - K x_old):
//   y_i <- y_i + sigma (q_i - 2 v + (K x_old)_i), projected onto y_i >= 0 for i >= m1;
//   sy_i += y_i;  (K x_old)_i <- v.
struct EpiDual {
  using T = double;
  double* __restrict__ y;
  double* __restrict__ sy;
  double* __restrict__ kxp;
  const double* __restrict__ q;
  int m1;
  double sigma;
  struct Pre { double q, kxp, y, sy; };
  __device__ void prepare(const DevState* st) { sigma = st->sigma; }
  __device__ Pre load(int i) const { return Pre{q[i], kxp[i], y[i], sy[i]}; }
  __device__ void finish(int i, double v, const Pre& p) {
    const double e = p.q + p.kxp;
    double yn = fma(sigma, fma(-2.0, v, e), p.y);
    if (i >= m1) yn = max0(yn);
    y[i] = yn;
    sy[i] = p.sy + yn;
    kxp[i] = v;
  }
  __device__ void task_end(int, int) {}
};

// Adaptive step rule (the cited PDLP paper; an option beside the constant eta of
// Section 2).  One attempt is the primal and dual step of Section 2 computed in place,
// with the previous point kept in backups (xb, yb, kxb) for a rejected attempt, and
// per-warp-task partial sums of ||dx||^2, ||dy||^2 and dy'(K dx) for the acceptance
// test.  The running sums receive the previous point with its pending weight pw (the
// step size that produced it; 0 once added or after a rejection).
struct EpiPrimalA {
  using T = double;
  double* __restrict__ x;
  double* __restrict__ xb;
  double* __restrict__ sx;
  const double* __restrict__ c;
  const double* __restrict__ l;
  const double* __restrict__ u;
  double* __restrict__ part;   // ||dx||^2 per warp task
  double tau, pw, acc;
  struct Pre { double xo, c, l, u, sx; };
  __device__ void prepare(const DevState* st) {
    tau = st->tau;
    pw = st->pw;
    acc = 0.0;
  }
  __device__ Pre load(int j) const { return Pre{x[j], c[j], l[j], u[j], sx[j]}; }
  __device__ void finish(int j, double g, const Pre& p) {
    const double xn = clamp_box(fma(-tau, p.c - g, p.xo), p.l, p.u);
    x[j] = xn;
    xb[j] = p.xo;
    sx[j] = fma(pw, p.xo, p.sx);
    const double d = xn - p.xo;
    acc = fma(d, d, acc);
  }
  __device__ void task_end(int w, int lane) {
    const double s = warp_sum(acc);
    if (lane == 0) part[w] = s;
  }
};

struct EpiDualA {
  using T = double;
  double* __restrict__ y;
  double* __restrict__ yb;
  double* __restrict__ sy;
  double* __restrict__ kxp;
  double* __restrict__ kxb;
  const double* __restrict__ q;
  double* __restrict__ part;   // ||dy||^2 and dy'(K dx) per warp task
  int m1;
  double sigma, pw, a2, ai;
  struct Pre { double q, kxp, y, sy; };
  __device__ void prepare(const DevState* st) {
    sigma = st->sigma;
    pw = st->pw;
    a2 = 0.0;
    ai = 0.0;
  }
  __device__ Pre load(int i) const { return Pre{q[i], kxp[i], y[i], sy[i]}; }
  __device__ void finish(int i, double v, const Pre& p) {
    double yn = fma(sigma, fma(-2.0, v, p.q + p.kxp), p.y);
    if (i >= m1) yn = max0(yn);
    y[i] = yn;
    yb[i] = p.y;
    sy[i] = fma(pw, p.y, p.sy);
    kxp[i] = v;
    kxb[i] = p.kxp;
    const double dy = yn - p.y;
    a2 = fma(dy, dy, a2);
    ai = fma(dy, v - p.kxp, ai);
  }
  __device__ void task_end(int w, int lane) {
    const double s2 = warp_sum(a2), si = warp_sum(ai);
    if (lane == 0) {
      part[2 * w] = s2;
      part[2 * w + 1] = si;
    }
  }
};

// Partial sums of the attempt's per-task partials: block b < kStepParts adds a fixed
// contiguous segment of px (||dx||^2) and of py (||dy||^2, dy'K dx pairs) into
// out[3 b .. 3 b + 2]; the extra block kStepParts computes the two powers of the
// step-size update meanwhile (they depend only on the count of kept steps).
constexpr int kStepParts = 128;
__global__ void __launch_bounds__(256) k_step_partial(const double* __restrict__ px, int ntx,
                                                      const double* __restrict__ py, int nty, double* __restrict__ out,
                                                      DevState* st) {
  if (st->done) return;
  if (blockIdx.x == kStepParts) {
    if (threadIdx.x == 0) {
      const double sidx = (double)(st->accepted + 2);
      st->p3 = pow(sidx, -0.3);
      st->p6 = pow(sidx, -0.6);
    }
    return;
  }
  __shared__ double red[3][8];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int cx = (ntx + kStepParts - 1) / kStepParts, cy = (nty + kStepParts - 1) / kStepParts;
  const int x0 = blockIdx.x * cx, x1 = min(ntx, x0 + cx), y0 = blockIdx.x * cy, y1 = min(nty, y0 + cy);
  double a = 0.0, b = 0.0, c = 0.0;
  for (int i = x0 + (int)threadIdx.x; i < x1; i += blockDim.x) a += px[i];
  for (int i = y0 + (int)threadIdx.x; i < y1; i += blockDim.x) {
    b += py[2 * i];
    c += py[2 * i + 1];
  }
  a = warp_sum(a);
  b = warp_sum(b);
  c = warp_sum(c);
  if (lane == 0) {
    red[0][wid] = a;
    red[1][wid] = b;
    red[2][wid] = c;
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[threadIdx.x][w];
    out[3 * blockIdx.x + threadIdx.x] = t;
  }
}

// Acceptance test and next step size of the adaptive rule, after one attempt (one warp,
// the kStepParts block sums added in a fixed order):
//   eta_max = (omega ||dx||^2 + ||dy||^2 / omega) / (2 |dy'K dx|)   (+inf when 0),
//   accept when eta <= eta_max (or after reject_cap rejections in a row, 64 by default:
//   a safeguard of this implementation, the cited rule has none),
//   next eta = min((1 - (s+1)^-0.3) eta_max, (1 + (s+1)^-0.6) eta), s = accepted + 1.
__global__ void __launch_bounds__(32) k_step_decide(const double* __restrict__ parts, DevState* st) {
  if (st->done) return;
  const int lane = threadIdx.x;
  double a = 0.0, b = 0.0, c = 0.0;
  for (int p = lane; p < kStepParts; p += 32) {
    a += parts[3 * p];
    b += parts[3 * p + 1];
    c += parts[3 * p + 2];
  }
  const double dx2 = warp_sum(a), dy2 = warp_sum(b), inter = warp_sum(c);
  if (lane != 0) return;
  st->wsum += st->pw;   // the pending weight went into the sums in this attempt
  const double eta = st->eta, w = st->omega;
  const double emax = inter == 0.0 ? __longlong_as_double(0x7FF0000000000000LL)
                                   : (w * dx2 + dy2 / w) / (2.0 * fabs(inter));
  const double e1 = (1.0 - st->p3) * emax, e2 = (1.0 + st->p6) * eta;
  const double enext = e1 < e2 ? e1 : e2;
  const bool acc = eta <= emax || st->rejects >= st->reject_cap;
  st->accept = acc ? 1 : 0;
  if (acc) {
    st->pw = eta;
    st->accepted += 1;
    st->rejects = 0;
  } else {
    st->pw = 0.0;
    st->rejects += 1;
  }
  st->eta = enext;
  st->tau = enext / w;
  st->sigma = enext * w;
}

// A rejected attempt: back to the previous point (and its K x).
__global__ void k_step_restore(double* __restrict__ x, const double* __restrict__ xb, int64_t npad,
                               double* __restrict__ y, const double* __restrict__ yb, double* __restrict__ kxp,
                               const double* __restrict__ kxb, int64_t mpad, const DevState* st) {
  if (st->done || st->accept) return;
  const int64_t tot = npad > mpad ? npad : mpad;
  PDLP_GRID_STRIDE(i, tot) {
    if (i < npad) x[i] = xb[i];
    if (i < mpad) {
      y[i] = yb[i];
      kxp[i] = kxb[i];
    }
  }
}

// Before a check: the pending weight of the current iterate goes into the sums.
__global__ void k_flush_pending(double* __restrict__ sx, const double* __restrict__ x, int64_t npad,
                                double* __restrict__ sy, const double* __restrict__ y, int64_t mpad,
                                const DevState* st) {
  if (st->done) return;
  const double pw = st->pw;
  if (pw == 0.0) return;
  const int64_t tot = npad > mpad ? npad : mpad;
  PDLP_GRID_STRIDE(i, tot) {
    if (i < npad) sx[i] = fma(pw, x[i], sx[i]);
    if (i < mpad) sy[i] = fma(pw, y[i], sy[i]);
  }
}

// Largest |K_ij| (bit patterns of non-negative doubles order like the values).
__global__ void k_absmax(const double* __restrict__ v, int64_t len, unsigned long long* out) {
  double mx = 0.0;
  PDLP_GRID_STRIDE(i, len) mx = fmax(mx, fabs(v[i]));
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(mx));
}

// Mixed precision (an extension, not in the paper): the same primal and dual
// steps with FP32 iterates and FP32 arithmetic; the running sums of the inner loop
// are FP32 over one check interval and folded into FP64 at every check.
struct EpiPrimal32 {
  using T = float;
  float* __restrict__ x;
  float* __restrict__ sx;
  const float* __restrict__ c;
  const float* __restrict__ l;
  const float* __restrict__ u;
  float tau;
  struct Pre { float xo, c, l, u, sx; };
  __device__ void prepare(const DevState* st) { tau = (float)st->tau; }
  __device__ Pre load(int j) const { return Pre{x[j], c[j], l[j], u[j], sx[j]}; }
  __device__ void finish(int j, float g, const Pre& p) {
    float xn = fmaf(-tau, p.c - g, p.xo);
    xn = fminf(fmaxf(xn, p.l), p.u);
    x[j] = xn;
    sx[j] = p.sx + xn;
  }
  __device__ void task_end(int, int) {}
};
struct EpiDual32 {
  using T = float;
  float* __restrict__ y;
  float* __restrict__ sy;
  float* __restrict__ kxp;
  const float* __restrict__ q;
  int m1;
  float sigma;
  struct Pre { float q, kxp, y, sy; };
  __device__ void prepare(const DevState* st) { sigma = (float)st->sigma; }
  __device__ Pre load(int i) const { return Pre{q[i], kxp[i], y[i], sy[i]}; }
  __device__ void finish(int i, float v, const Pre& p) {
    float yn = fmaf(sigma, fmaf(-2.0f, v, p.q + p.kxp), p.y);
    if (i >= m1) yn = fmaxf(yn, 0.0f);
    y[i] = yn;
    sy[i] = p.sy + yn;
    kxp[i] = v;
  }
  __device__ void task_end(int, int) {}
};

// Mixed precision with the +-1 entries of K stored as sign bits (OpUnitF).  The FP32
// iterations then run in the unscaled variables: for the scaled LP (K = D_r K0 D_c,
// c = D_c c0, q = D_r q0, bounds l0 / D_c, u0 / D_c) and xu = D_c x, yu = D_r y, the
// steps of Section 2 become
//   xu <- proj_[l0,u0](xu - tau D_c^2 (c0 - K0' yu)),
//   yu <- yu + sigma D_r^2 (q0 - 2 K0 xu_new + K0 xu_old), yu_i >= 0 for i >= m1,
// so the products gather the iterates themselves and the scaling costs one per-row
// factor (D_c^2, D_r^2) instead of a stored value per entry.  kxp holds K0 xu_old.
struct EpiPrimal32U {
  using T = float;
  float* __restrict__ x;
  float* __restrict__ sx;
  const float* __restrict__ c;
  const float* __restrict__ l;
  const float* __restrict__ u;
  const float* __restrict__ d2;   // D_c^2
  float tau;
  struct Pre { float xo, c, l, u, sx, d2; };
  __device__ void prepare(const DevState* st) { tau = (float)st->tau; }
  __device__ Pre load(int j) const { return Pre{x[j], c[j], l[j], u[j], sx[j], d2[j]}; }
  __device__ void finish(int j, float g, const Pre& p) {
    float xn = fmaf(-(tau * p.d2), p.c - g, p.xo);
    xn = fminf(fmaxf(xn, p.l), p.u);
    x[j] = xn;
    sx[j] = p.sx + xn;
  }
  __device__ void task_end(int, int) {}
};
struct EpiDual32U {
  using T = float;
  float* __restrict__ y;
  float* __restrict__ sy;
  float* __restrict__ kxp;
  const float* __restrict__ q;
  const float* __restrict__ d2;   // D_r^2
  int m1;
  float sigma;
  struct Pre { float q, kxp, y, sy, d2; };
  __device__ void prepare(const DevState* st) { sigma = (float)st->sigma; }
  __device__ Pre load(int i) const { return Pre{q[i], kxp[i], y[i], sy[i], d2[i]}; }
  __device__ void finish(int i, float v, const Pre& p) {
    float yn = fmaf(sigma * p.d2, fmaf(-2.0f, v, p.q + p.kxp), p.y);
    if (i >= m1) yn = fmaxf(yn, 0.0f);
    y[i] = yn;
    sy[i] = p.sy + yn;
    kxp[i] = v;
  }
  __device__ void task_end(int, int) {}
};

// FP32 problem data of the unscaled variables: c0 = c / D_c, l0 = l D_c, u0 = u D_c,
// D_c^2 (columns, n entries) and q0 = q / D_r, D_r^2 (rows, m entries).
__global__ void k_unit_vectors(float* c0, float* l0, float* u0, float* dc2, const double* c, const double* l,
                               const double* u, const double* Dc, const double* invDc, int64_t n, float* q0,
                               float* dr2, const double* q, const double* Dr, const double* invDr, int64_t m) {
  const int64_t tot = n > m ? n : m;
  PDLP_GRID_STRIDE(i, tot) {
    if (i < n) {
      c0[i] = (float)(c[i] * invDc[i]);
      l0[i] = (float)(l[i] * Dc[i]);
      u0[i] = (float)(u[i] * Dc[i]);
      dc2[i] = (float)(Dc[i] * Dc[i]);
    }
    if (i < m) {
      q0[i] = (float)(q[i] * invDr[i]);
      dr2[i] = (float)(Dr[i] * Dr[i]);
    }
  }
}

// Entries of K (a layout's value array, padding included) that are neither 0 nor +-1.
__global__ void k_count_nonunit(const double* val, int64_t n, unsigned long long* count) {
  unsigned long long c = 0;
  PDLP_GRID_STRIDE(i, n) {
    const double v = val[i];
    if (v != 0.0 && fabs(v) != 1.0) ++c;
  }
  if (c) atomicAdd(count, c);
}
// Sign-bit column words of a layout whose entries are all +-1 after positive scaling:
// val[i] < 0 sets bit 31, a zero value (padding) points at index `zero`.
__global__ void k_unit_cols(int32_t* ucol, const int32_t* col, const double* val, int64_t n, int32_t zero) {
  PDLP_GRID_STRIDE(i, n) {
    const double v = val[i];
    ucol[i] = v == 0.0 ? zero : (v < 0.0 ? (int32_t)((uint32_t)col[i] | 0x80000000u) : col[i]);
  }
}

// Scale factors between the FP32 iterates and the FP64 (scaled) ones: all null when
// the FP32 iterates are the scaled ones; with sign-bit storage x = xu / D_c, y = yu / D_r
// and K x = D_r (K0 xu).
struct MixedScale {
  const double* Dc;
  const double* invDc;
  const double* Dr;
  const double* invDr;
};

// Check in mixed precision: FP64 copies of the FP32 iterates, interval sums folded
// into the FP64 sums and cleared.
__global__ void k_mixed_to64(double* x, double* sx, const float* x32, float* sx32, int64_t npad, double* y,
                             double* sy, const float* y32, float* sy32, int64_t mpad, const DevState* st,
                             MixedScale ms) {
  if (st->done) return;
  const int64_t tot = npad > mpad ? npad : mpad;
  PDLP_GRID_STRIDE(i, tot) {
    if (i < npad) {
      const double f = ms.invDc ? ms.invDc[i] : 1.0;
      x[i] = (double)x32[i] * f;
      sx[i] += (double)sx32[i] * f;
      sx32[i] = 0.0f;
    }
    if (i < mpad) {
      const double f = ms.invDr ? ms.invDr[i] : 1.0;
      y[i] = (double)y32[i] * f;
      sy[i] += (double)sy32[i] * f;
      sy32[i] = 0.0f;
    }
  }
}
// After the check (and a restart, if one happened): FP32 iterates from the FP64 ones.
__global__ void k_mixed_to32(float* x32, const double* x, int64_t npad, float* y32, const double* y,
                             float* kxp32, const double* kxp, int64_t mpad, const DevState* st, MixedScale ms) {
  if (st->done) return;
  const int64_t tot = npad > mpad ? npad : mpad;
  PDLP_GRID_STRIDE(i, tot) {
    if (i < npad) x32[i] = (float)(ms.Dc ? x[i] * ms.Dc[i] : x[i]);
    if (i < mpad) {
      y32[i] = (float)(ms.Dr ? y[i] * ms.Dr[i] : y[i]);
      kxp32[i] = (float)(ms.invDr ? kxp[i] * ms.invDr[i] : kxp[i]);
    }
  }
}
__global__ void k_to_float(float* dst, const double* src, int64_t n) {
  PDLP_GRID_STRIDE(i, n) dst[i] = (float)src[i];
}

// ------------------------------------------------------------------ vector kernels

__global__ void k_fill(double* a, double v, int64_t n) {
  PDLP_GRID_STRIDE(i, n) a[i] = v;
}
__global__ void k_copy(double* dst, const double* src, int64_t n) {
  PDLP_GRID_STRIDE(i, n) dst[i] = src[i];
}

// dst[p] = src[perm[p]] (divided by div[p] if given); pad where perm[p] < 0 (padding).
__global__ void k_permute_in(double* dst, const double* src, const int32_t* perm, const double* div, int64_t npad,
                             double pad) {
  PDLP_GRID_STRIDE(p, npad) {
    const int32_t q = perm[p];
    if (q >= 0) {
      const double v = src[q];
      dst[p] = div ? v / div[p] : v;
    } else {
      dst[p] = pad;
    }
  }
}

// out[i] = a[pos[i]] * d[pos[i]] (unscale and return to the caller's order)
__global__ void k_unpermute_scale(double* out, const double* a, const double* d, const int32_t* pos,
                                  int64_t n) {
  PDLP_GRID_STRIDE(i, n) {
    int32_t p = pos[i];
    out[i] = d[p] * a[p];
  }
}

// SELL values from the input CSR values: v[e] = src[e] >= 0 ? csr[src[e]] : 0
__global__ void k_gather_values(double* v, const int32_t* src, const double* csr, int64_t total) {
  PDLP_GRID_STRIDE(e, total) {
    int32_t s = src[e];
    v[e] = s >= 0 ? csr[s] : 0.0;
  }
}

// Scaling factor from a row norm: f = 1/sqrt(norm) (1 for an empty row); D *= f.
__global__ void k_scale_factor(double* f, double* D, const double* norm, int64_t n) {
  PDLP_GRID_STRIDE(i, n) {
    double r = norm[i];
    double fi = r > 0.0 ? 1.0 / sqrt(r) : 1.0;
    f[i] = fi;
    D[i] *= fi;
  }
}

// v <- (v * fr[row]) * fc[col] over a SELL matrix (padding entries stay 0); one warp per chunk.
__global__ void k_scale_sell(double* v, const int32_t* col, const int32_t* chunk_ptr, int64_t nchunks,
                             const double* frow, const double* fcol) {
  const int lane = threadIdx.x & 31;
  for (int64_t ch = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; ch < nchunks;
       ch += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const double fr = frow[ch * 32 + lane];
    for (int64_t s = chunk_ptr[ch]; s < chunk_ptr[ch + 1]; ++s) {
      size_t e = (size_t)s * 32 + lane;
      v[e] = (v[e] * fr) * fcol[col[e]];
    }
  }
}

// Problem vectors of the scaled problem: c <- Dc c, l <- l/Dc, u <- u/Dc (columns),
// q <- Dr q (rows); inverse factors kept for the unscaled residuals.
__global__ void k_scale_cols(double* c, double* l, double* u, double* invD, const double* D, int64_t n) {
  PDLP_GRID_STRIDE(j, n) {
    double d = D[j];
    c[j] = d * c[j];
    l[j] = l[j] / d;
    u[j] = u[j] / d;
    invD[j] = 1.0 / d;
  }
}
__global__ void k_scale_rows(double* q, double* invD, const double* D, int64_t m) {
  PDLP_GRID_STRIDE(i, m) {
    double d = D[i];
    q[i] = d * q[i];
    invD[i] = 1.0 / d;
  }
}

// Deterministic 2-norm in two levels: per-block partial sums of squares, then one warp.
__global__ void k_sumsq_partial(double* part, const double* a, int64_t n) {
  double s = 0.0;
  PDLP_GRID_STRIDE(i, n) s = fma(a[i], a[i], s);
  s = warp_sum(s);
  __shared__ double sh[32];
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
    v = warp_sum(v);
    if (threadIdx.x == 0) part[blockIdx.x] = v;
  }
}
// out[0] = sqrt(sum of part[0..nb)), one warp.
__global__ void k_sum_sqrt(double* out, const double* part, int nb) {
  double s = 0.0;
  for (int i = threadIdx.x; i < nb; i += 32) s += part[i];
  s = warp_sum(s);
  if (threadIdx.x == 0) out[0] = sqrt(s);
}
// a <- a / s[0] unless s[0] == 0 (power-iteration normalisation).
__global__ void k_div_by(double* a, const double* s, int64_t n) {
  const double d = s[0];
  if (d == 0.0) return;
  PDLP_GRID_STRIDE(i, n) a[i] = a[i] / d;
}

// ------------------------------------------------------------------ solve kernels

// Initial point: x = proj_X(x0), y = proj_Y(y0) (x0, y0 already scaled; null = 0).
__global__ void k_init_point(double* x, const double* x0, const double* l, const double* u, int64_t n,
                             int64_t npad, double* y, const double* y0, int64_t m, int64_t mpad, int m1) {
  const int64_t tot = npad > mpad ? npad : mpad;
  PDLP_GRID_STRIDE(i, tot) {
    if (i < npad) x[i] = i < n ? clamp_box(x0 ? x0[i] : 0.0, l[i], u[i]) : 0.0;
    if (i < mpad) {
      double yi = y0 ? y0[i] : 0.0;   // y0 is in internal order, zero in padding rows
      y[i] = (i >= m1) ? max0(yi) : yi;
    }
  }
}

// Before a check: advance k and t by the interval just run, 1/t for the average.
// adaptive: the average is weighted by the step sizes (weight sum wsum, after the
// pending weight has been flushed into the sums)
__global__ void k_precheck(DevState* st, int len, int adaptive) {
  if (st->done) return;
  st->k += len;
  st->t += len;
  if (adaptive) {
    st->wsum += st->pw;
    st->pw = 0.0;
    st->inv_t = st->wsum > 0.0 ? 1.0 / st->wsum : 0.0;
  } else {
    st->inv_t = st->t > 0 ? 1.0 / (double)st->t : 0.0;
  }
}

struct KktInputs {
  // rows (length m): scaled q, K x (current), K x (average, already times 1/t), y, sy, anchor y, 1/Dr
  const double *q, *kx_c, *kx_a, *y, *sy, *ya, *invDr;
  // columns (length n): scaled c, l, u, K'y current and average (times 1/t), x, sx, anchor x, 1/Dc
  const double *c, *l, *u, *g_c, *g_a, *x, *sx, *xa, *invDc;
  int64_t m, n;
  int m1;
  int rows_blocks;   // blocks [0, rows_blocks) reduce rows, the rest reduce columns
};

// Per-block partial sums of the NQ check quantities (Section 2: primal residual
// ||(Ax-b, [h-Gx]^+)||, dual residual ||c - K'y - lambda|| with lambda = proj_Lambda,
// objectives q'y + l'lambda^+ - u'lambda^- and c'x, and distances to the anchor),
// residuals both on the scaled problem and on the unscaled one.
__global__ void __launch_bounds__(256) k_kkt_partials(KktInputs in, const DevState* st, double* part) {
  if (st->done) return;
  const bool avg_is_cur = st->t == 0;
  const double it = st->inv_t;
  double acc[10];
#pragma unroll
  for (int i = 0; i < 10; ++i) acc[i] = 0.0;
  const bool rows = (int)blockIdx.x < in.rows_blocks;
  if (rows) {
    const int64_t nthr = (int64_t)in.rows_blocks * blockDim.x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < in.m; i += nthr) {
      const double qi = in.q[i], id = in.invDr[i], yai = in.ya[i];
      const bool ineq = i >= in.m1;
#pragma unroll
      for (int p = 0; p < 2; ++p) {
        const bool avg = (p == 1) && !avg_is_cur;
        const double kx = avg ? in.kx_a[i] : in.kx_c[i];
        const double yi = avg ? in.sy[i] * it : in.y[i];
        double r = kx - qi;
        if (ineq) r = min0(r);   // [h - Gx]^+ enters squared as min(Gx - h, 0)^2
        const double ru = r * id;
        acc[4 * p + 0] = fma(r, r, acc[4 * p + 0]);
        acc[4 * p + 1] = fma(ru, ru, acc[4 * p + 1]);
        acc[4 * p + 2] = fma(qi, yi, acc[4 * p + 2]);
        const double dy = yi - yai;
        acc[4 * p + 3] = fma(dy, dy, acc[4 * p + 3]);
      }
    }
  } else {
    const int64_t nthr = (int64_t)(gridDim.x - in.rows_blocks) * blockDim.x;
    for (int64_t j = (blockIdx.x - in.rows_blocks) * (int64_t)blockDim.x + threadIdx.x; j < in.n; j += nthr) {
      const double cj = in.c[j], lj = in.l[j], uj = in.u[j], id = in.invDc[j], xaj = in.xa[j];
      const bool lf = !is_neg_inf(lj), uf = !is_pos_inf(uj);
#pragma unroll
      for (int p = 0; p < 2; ++p) {
        const bool avg = (p == 1) && !avg_is_cur;
        const double g = avg ? in.g_a[j] : in.g_c[j];
        const double xj = avg ? in.sx[j] * it : in.x[j];
        const double d = cj - g;
        // lambda = proj_Lambda(d): {0}, R^-, R^+ or R by which bounds are finite;
        // d - lambda is then either 0 or d, so no FP64 subtraction is needed
        const bool neg = __double2hiint(d) < 0;
        double lam, rd;
        if (lf && uf) { lam = d; rd = 0.0; }
        else if (lf) { lam = neg ? 0.0 : d; rd = neg ? d : 0.0; }
        else if (uf) { lam = neg ? d : 0.0; rd = neg ? 0.0 : d; }
        else { lam = 0.0; rd = d; }
        const double rdu = rd * id;
        // l'lambda^+ - u'lambda^-: the bound on lambda's side times lambda (0 when lambda = 0)
        const double bnd = is_zero(lam) ? 0.0 : (__double2hiint(lam) < 0 ? uj : lj);
        acc[5 * p + 0] = fma(rd, rd, acc[5 * p + 0]);
        acc[5 * p + 1] = fma(rdu, rdu, acc[5 * p + 1]);
        acc[5 * p + 2] = fma(bnd, lam, acc[5 * p + 2]);
        acc[5 * p + 3] = fma(cj, xj, acc[5 * p + 3]);
        const double dx = xj - xaj;
        acc[5 * p + 4] = fma(dx, dx, acc[5 * p + 4]);
      }
    }
  }
  __shared__ double sh[8][10];
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int i = 0; i < 10; ++i) {
    double v = warp_sum(acc[i]);
    if (lane == 0) sh[wid][i] = v;
  }
  __syncthreads();
  if (threadIdx.x < 10) {
    double v = 0.0;
    for (int w2 = 0; w2 < (int)(blockDim.x >> 5); ++w2) v += sh[w2][threadIdx.x];
    const int base = rows ? 0 : 8;
    const int nq = rows ? 8 : 10;
    if ((int)threadIdx.x < nq) part[(size_t)blockIdx.x * NQ + base + threadIdx.x] = v;
  }
}

__device__ __forceinline__ double kkt_w(double prs, double drs, double gap, double w) {
  return sqrt(w * w * prs + drs / (w * w) + gap * gap);
}

// The restart / termination logic of Section 2 on the reduced totals of one check,
// run by one thread.  Termination (the three relative tests, or the iteration limit
// when `last`) is tested first; otherwise the candidate (Section 2: the current
// iterate if its KKT_omega is strictly smaller, else the average) is checked against
// restart conditions 1-3; on a restart omega, tau, sigma and the KKT anchor are
// updated and st->restart_flag / st->cand_avg tell the caller what to copy.
// `restarts` (may be null) receives the iteration count of each restart.
__device__ inline CheckRecord decide_core(const double* tot, DevState* st, const DevParams& P, bool last,
                                          long long* restarts) {
  const double w = st->omega;
  const double pobj_c = tot[Q_CX_C], dobj_c = tot[Q_QY_C] + tot[Q_LT_C];
  const double gap_c = dobj_c - pobj_c;
  const double pobj_a = tot[Q_CX_A], dobj_a = tot[Q_QY_A] + tot[Q_LT_A];
  const double gap_a = dobj_a - pobj_a;
  const double kc = kkt_w(tot[Q_PRS_C], tot[Q_DRS_C], gap_c, w);
  const double ka = kkt_w(tot[Q_PRS_A], tot[Q_DRS_A], gap_a, w);
  const double inf = __longlong_as_double(0x7FF0000000000000LL);
  const double rp_c = sqrt(tot[Q_PRU_C]) / (1.0 + P.qnorm), rd_c = sqrt(tot[Q_DRU_C]) / (1.0 + P.cnorm);
  const double rg_c = fabs(gap_c) / (1.0 + fabs(dobj_c) + fabs(pobj_c));
  const double rp_a = sqrt(tot[Q_PRU_A]) / (1.0 + P.qnorm), rd_a = sqrt(tot[Q_DRU_A]) / (1.0 + P.cnorm);
  const double rg_a = fabs(gap_a) / (1.0 + fabs(dobj_a) + fabs(pobj_a));
  const double ec = fmax(rp_c, fmax(rd_c, rg_c)), ea = fmax(rp_a, fmax(rd_a, rg_a));
  const bool pass_c = ec <= P.tol, pass_a = ea <= P.tol;
  const bool finite = isfinite(kc) && isfinite(ka) && isfinite(ec) && isfinite(ea);
  const bool better_c = ec < ea;

  CheckRecord rec;
  rec.k = st->k;
  rec.t = st->t;
  rec.restart = 0;
  rec.candidate = !(kc < ka);
  rec.omega = w;
  rec.kkt_cur = kc;
  rec.kkt_avg = ka;
  rec.kkt_anchor = st->kkt_anchor;
  rec.rel_p = better_c ? rp_c : rp_a;
  rec.rel_d = better_c ? rd_c : rd_a;
  rec.rel_g = better_c ? rg_c : rg_a;
  st->last_err = fmin(ec, ea);

  st->restart_flag = 0;
  if (!finite || pass_c || pass_a || last) {
    int which;
    if (pass_c && !pass_a) which = 0;
    else if (pass_a && !pass_c) which = 1;
    else which = better_c ? 0 : 1;
    st->which = which;
    st->status = !finite ? 3 : ((pass_c || pass_a) ? 0 : 1);
    st->out_pobj = which ? pobj_a : pobj_c;
    st->out_dobj = which ? dobj_a : dobj_c;
    st->out_rel_p = which ? rp_a : rp_c;
    st->out_rel_d = which ? rd_a : rd_c;
    st->out_rel_g = which ? rg_a : rg_c;
    st->out_kkt = which ? ka : kc;
    st->done = 1;
  } else {
    const int cand_avg = !(kc < ka);
    const double kkt_c = cand_avg ? ka : kc;
    int why = 0;
    if (kkt_c <= P.beta_suff * st->kkt_anchor) why = 1;
    else if (kkt_c <= P.beta_nec * st->kkt_anchor && kkt_c > st->kkt_prev) why = 2;
    else if ((double)st->t >= P.beta_art * (double)st->k) why = 3;
    rec.restart = why;
    if (why) {
      const double dx = sqrt(cand_avg ? tot[Q_DX_A] : tot[Q_DX_C]);
      const double dy = sqrt(cand_avg ? tot[Q_DY_A] : tot[Q_DY_C]);
      double wn = w;
      if (dx > 1e-10 && dy > 1e-10) wn = exp(P.theta * log(dy / dx) + (1.0 - P.theta) * log(w));
      st->omega = wn;
      st->tau = st->eta / wn;
      st->sigma = st->eta * wn;
      st->kkt_anchor = cand_avg ? kkt_w(tot[Q_PRS_A], tot[Q_DRS_A], gap_a, wn)
                                : kkt_w(tot[Q_PRS_C], tot[Q_DRS_C], gap_c, wn);
      st->kkt_prev = inf;
      st->restart_flag = 1;
      st->cand_avg = cand_avg;
      if (restarts != nullptr && st->nrestart < P.restart_cap) restarts[st->nrestart] = st->k;
      st->nrestart += 1;
    } else {
      st->kkt_prev = kkt_c;
    }
  }
  st->ncheck += 1;
  return rec;
}

// Sum the partials (fixed order), then decide_core on one thread.
// mode 1: initialisation (KKT_omega of the anchor only).  final_check = 1 forces
// termination at this check (iteration-limit semantics).
__global__ void k_decide(const double* part, int nb_rows, int nb_cols, DevState* st, const DevParams* Pp,
                         CheckRecord* logbuf, long long* restarts, int mode, int final_check) {
  if (st->done) return;
  __shared__ double tot[NQ];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int qd = wid; qd < NQ; qd += (int)(blockDim.x >> 5)) {
    const bool rowq = qd < 8;
    const int b0 = rowq ? 0 : nb_rows, nb = rowq ? nb_rows : nb_cols;
    double s = 0.0;
    for (int b = lane; b < nb; b += 32) s += part[(size_t)(b0 + b) * NQ + qd];
    s = warp_sum(s);
    if (lane == 0) tot[qd] = s;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  const DevParams P = *Pp;
  if (mode == 1) {
    const double gap_c = tot[Q_QY_C] + tot[Q_LT_C] - tot[Q_CX_C];
    st->kkt_anchor = kkt_w(tot[Q_PRS_C], tot[Q_DRS_C], gap_c, st->omega);
    st->kkt_prev = __longlong_as_double(0x7FF0000000000000LL);
    return;
  }
  const long long ncheck = st->ncheck;
  const bool last = final_check || st->k >= P.max_iter || st->final_force;
  const CheckRecord rec = decide_core(tot, st, P, last, restarts);
  if (ncheck < P.log_cap) logbuf[ncheck] = rec;
}

struct RestartArgs {
  double *x, *sx, *xa, *y, *sy, *ya, *kxp;
  const double* kx_a;
  int64_t npad, mpad;
};

// Restart (Section 2): the next inner loop starts from the candidate; the anchor
// becomes that point and the running sums are cleared.
__global__ void k_restart_apply(RestartArgs a, const DevState* st) {
  if (!st->restart_flag || st->done) return;
  const bool avg = st->cand_avg;
  const double it = st->inv_t;
  const int64_t tot = a.npad > a.mpad ? a.npad : a.mpad;
  PDLP_GRID_STRIDE(i, tot) {
    if (i < a.npad) {
      double xi = avg ? a.sx[i] * it : a.x[i];
      a.x[i] = xi;
      a.xa[i] = xi;
      a.sx[i] = 0.0;
    }
    if (i < a.mpad) {
      double yi = avg ? a.sy[i] * it : a.y[i];
      a.y[i] = yi;
      a.ya[i] = yi;
      a.sy[i] = 0.0;
      if (avg) a.kxp[i] = a.kx_a[i];
    }
  }
}

// After the restart kernel: t <- 0 (separate so that every block of the restart
// kernel reads the same 1/t).
__global__ void k_post_restart(DevState* st) {
  if (st->done || !st->restart_flag) return;
  st->t = 0;
  st->inv_t = 0.0;
  st->wsum = 0.0;
  st->pw = 0.0;
}

}  // namespace pdlp
