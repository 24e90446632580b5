// Persistent batched restarted PDHG: many independent LPs in one launch.
//
// The batch is stored as one block-diagonal LP: every LP owns a contiguous, 32-aligned
// range of internal rows and columns, and its chunks in the SELL-32 layouts of K and
// K' (layout.h).  Each CTA takes LPs from a work queue (largest first) and runs the
// whole method of Section 2 on one LP at a time: the step size by power iteration,
// the PDHG iterations, and the checks with the restart rule and the termination
// tests, all without leaving the CTA.  The two iterates live in shared memory, so
// the random gathers of both SpMVs are shared-memory loads; the matrix and the other
// per-row vectors stream from global memory.  Phases are separated by __syncthreads:
// the primal phase reads y and writes x, the dual phase reads x and writes y.
#pragma once
#include "kernels.cuh"

namespace pdlp {

struct LpDesc {
  int32_t m, n, m1, pad0;   // rows, columns, equality rows
  int32_t kc0, kc1;         // chunks of K (rows of this LP)
  int32_t tc0, tc1;         // chunks of K' (columns of this LP)
  int64_t r0, c0;           // first internal row / column (multiples of 32)
  int32_t mpad, npad;       // padded row / column counts
};

struct BatchArgs {
  const LpDesc* desc;
  const int32_t* order;      // LPs in the order the queue hands them out
  int32_t count;
  int32_t* next;             // queue position (left at zero after the launch)
  const int32_t* k_cptr;     // K: chunk_ptr, col, val (rows)
  const int32_t* k_col;
  const double* k_val;
  const int32_t* t_cptr;     // K': chunk_ptr, col, val (columns)
  const int32_t* t_col;
  const double* t_val;
  const double *c, *l, *u, *q, *invDr, *invDc;   // scaled problem, internal order
  double *sx, *sy, *xa, *ya, *kxp, *g, *kx_a, *g_a;
  double *xout, *yout;       // returned point per LP (scaled, internal order)
  const double *x0, *y0;     // warm start (scaled, internal order) or null
  const double* omega0;      // initial primal weight per LP (<= 0: the default) or null
  DevState* st;              // per LP
  DevParams P;
  int check_every;
  long long max_iter;
  int power_iters;
  double step_scale, eta_fixed, omega_fixed;
  int xs_off, ys_off, red_off;   // offsets (doubles) of x, y and the reduction area in shared memory
};

// Gather source of a batched SpMV: the shared-memory x or y, or a global vector.
enum BatchSrc { kSrcSmemX, kSrcSmemY, kSrcGlobal };

// Rows in chunks [c0, c1) of a SELL matrix; warp w of the CTA takes chunks c0+w,
// c0+w+nw, ...  Each lane sums its row, gathering src[col - base], then calls
// epi(local_row, sum).  Loads of kBB slots are issued together.
constexpr int kBB = 4;
template <int SRC, class F>
__device__ __forceinline__ void batch_rows(const int32_t* __restrict__ cptr, const int32_t* __restrict__ col,
                                           const double* __restrict__ val, int c0, int c1, int64_t base,
                                           const double* gsrc, const BatchArgs& A, F epi) {
  extern __shared__ double bsm[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const double* xs = bsm + A.xs_off;
  const double* ys = bsm + A.ys_off;
  for (int ch = c0 + wid; ch < c1; ch += nw) {
    const int s0 = cptr[ch], s1 = cptr[ch + 1];
    double acc = 0.0;
    for (int s = s0; s < s1; s += kBB) {
      const int nb = min(kBB, s1 - s);
      double v[kBB], xv[kBB];
      int ci[kBB];
#pragma unroll
      for (int j = 0; j < kBB; ++j)
        if (j < nb) {
          v[j] = __ldcs(val + (size_t)(s + j) * 32 + lane);
          ci[j] = __ldcs(col + (size_t)(s + j) * 32 + lane) - (int)base;
        }
#pragma unroll
      for (int j = 0; j < kBB; ++j) {
        xv[j] = 0.0;
        if (j < nb) {
          if (SRC == kSrcSmemX) xv[j] = xs[ci[j]];
          else if (SRC == kSrcSmemY) xv[j] = ys[ci[j]];
          else xv[j] = __ldcg(gsrc + ci[j]);
        }
      }
#pragma unroll
      for (int j = 0; j < kBB; ++j)
        if (j < nb) acc = fma(v[j], xv[j], acc);
    }
    epi((ch - c0) * 32 + lane, acc);
  }
}

// Deterministic CTA sum of NV values per thread into red[0..NV) (shared memory):
// warp shuffles, then warp partials added in warp order by the first NV threads.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    const double s = warp_sum(v[i]);
    if (lane == 0) red[NV + wid * NV + i] = s;
  }
  __syncthreads();
  if ((int)threadIdx.x < NV) {
    double s = 0.0;
    for (int w = 0; w < nw; ++w) s += red[NV + w * NV + threadIdx.x];
    red[threadIdx.x] = s;
  }
  __syncthreads();
}

// The 18 check quantities of the LP (same definitions as k_kkt_partials), reduced
// over the CTA into tot[0..NQ).  avg_is_cur: the average equals the current point.
__device__ __forceinline__ void batch_kkt(const BatchArgs& A, const LpDesc& D, bool avg_is_cur, double it,
                                          double* red, double* tot) {
  extern __shared__ double bsm[];
  const double* xs = bsm + A.xs_off;
  const double* ys = bsm + A.ys_off;
  {
    double acc[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) acc[i] = 0.0;
    for (int i = threadIdx.x; i < D.m; i += blockDim.x) {
      const int64_t gi = D.r0 + i;
      const double qi = A.q[gi], id = A.invDr[gi], yai = A.ya[gi];
      const bool ineq = i >= D.m1;
#pragma unroll
      for (int p = 0; p < 2; ++p) {
        const bool avg = (p == 1) && !avg_is_cur;
        const double kx = avg ? A.kx_a[gi] : A.kxp[gi];
        const double yi = avg ? A.sy[gi] * it : ys[i];
        double r = kx - qi;
        if (ineq) r = min0(r);
        const double ru = r * id;
        acc[4 * p + 0] = fma(r, r, acc[4 * p + 0]);
        acc[4 * p + 1] = fma(ru, ru, acc[4 * p + 1]);
        acc[4 * p + 2] = fma(qi, yi, acc[4 * p + 2]);
        const double dy = yi - yai;
        acc[4 * p + 3] = fma(dy, dy, acc[4 * p + 3]);
      }
    }
    block_sum<8>(acc, red);
    if ((int)threadIdx.x < 8) tot[threadIdx.x] = red[threadIdx.x];
    __syncthreads();
  }
  {
    double acc[10];
#pragma unroll
    for (int i = 0; i < 10; ++i) acc[i] = 0.0;
    for (int j = threadIdx.x; j < D.n; j += blockDim.x) {
      const int64_t gj = D.c0 + j;
      const double cj = A.c[gj], lj = A.l[gj], uj = A.u[gj], id = A.invDc[gj], xaj = A.xa[gj];
      const bool lf = !is_neg_inf(lj), uf = !is_pos_inf(uj);
#pragma unroll
      for (int p = 0; p < 2; ++p) {
        const bool avg = (p == 1) && !avg_is_cur;
        const double g = avg ? A.g_a[gj] : A.g[gj];
        const double xj = avg ? A.sx[gj] * it : xs[j];
        const double d = cj - g;
        const bool neg = __double2hiint(d) < 0;
        double lam, rd;
        if (lf && uf) { lam = d; rd = 0.0; }
        else if (lf) { lam = neg ? 0.0 : d; rd = neg ? d : 0.0; }
        else if (uf) { lam = neg ? d : 0.0; rd = neg ? 0.0 : d; }
        else { lam = 0.0; rd = d; }
        const double rdu = rd * id;
        const double bnd = is_zero(lam) ? 0.0 : (__double2hiint(lam) < 0 ? uj : lj);
        acc[5 * p + 0] = fma(rd, rd, acc[5 * p + 0]);
        acc[5 * p + 1] = fma(rdu, rdu, acc[5 * p + 1]);
        acc[5 * p + 2] = fma(bnd, lam, acc[5 * p + 2]);
        acc[5 * p + 3] = fma(cj, xj, acc[5 * p + 3]);
        const double dx = xj - xaj;
        acc[5 * p + 4] = fma(dx, dx, acc[5 * p + 4]);
      }
    }
    block_sum<10>(acc, red);
    if ((int)threadIdx.x < 10) tot[8 + threadIdx.x] = red[threadIdx.x];
    __syncthreads();
  }
}

__device__ __forceinline__ double block_norm(const double* v, int64_t base, int n, double* red, bool smem) {
  double a[1] = {0.0};
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    const double t = smem ? v[j] : v[base + j];
    a[0] = fma(t, t, a[0]);
  }
  block_sum<1>(a, red);
  return sqrt(red[0]);
}

// Runs restarted PDHG on LP b with the whole CTA.
__device__ void batch_solve_one(const BatchArgs& A, int b) {
  extern __shared__ double bsm[];
  double* xs = bsm + A.xs_off;
  double* ys = bsm + A.ys_off;
  double* red = bsm + A.red_off;
  __shared__ DevState S;
  __shared__ double tot[NQ];
  __shared__ double scal[4];
  const LpDesc D = A.desc[b];
  const int n = D.n, m = D.m;
  const int tid = threadIdx.x, nt = blockDim.x;

  // ---- step size: power iteration on K'K from v0 = 1/sqrt(n)
  double eta = A.eta_fixed;
  if (!(eta > 0.0)) {
    const double v0 = 1.0 / sqrt((double)n);
    for (int j = tid; j < D.npad; j += nt) xs[j] = j < n ? v0 : 0.0;
    __syncthreads();
    for (int it = 0; it < A.power_iters; ++it) {
      batch_rows<kSrcSmemX>(A.k_cptr, A.k_col, A.k_val, D.kc0, D.kc1, D.c0, nullptr, A,
                            [&](int i, double s) { ys[i] = s; });
      __syncthreads();
      batch_rows<kSrcSmemY>(A.t_cptr, A.t_col, A.t_val, D.tc0, D.tc1, D.r0, nullptr, A,
                            [&](int j, double s) { A.g[D.c0 + j] = s; });
      __syncthreads();
      const double nw = block_norm(A.g, D.c0, D.npad, red, false);
      if (nw != 0.0)
        for (int j = tid; j < D.npad; j += nt) xs[j] = A.g[D.c0 + j] / nw;
      __syncthreads();
    }
    batch_rows<kSrcSmemX>(A.k_cptr, A.k_col, A.k_val, D.kc0, D.kc1, D.c0, nullptr, A,
                          [&](int i, double s) { ys[i] = s; });
    __syncthreads();
    const double sn = m > 0 ? block_norm(ys, 0, D.mpad, red, true) : 0.0;
    eta = sn > 0.0 ? A.step_scale / sn : 1.0;
  }
  // ---- initial primal weight ||c||/||q|| and the unscaled norms for termination
  double omega = A.omega_fixed;
  {
    double a[4] = {0.0, 0.0, 0.0, 0.0};
    for (int j = tid; j < n; j += nt) {
      const double cj = A.c[D.c0 + j];
      const double cu = cj * A.invDc[D.c0 + j];
      a[0] = fma(cj, cj, a[0]);
      a[2] = fma(cu, cu, a[2]);
    }
    for (int i = tid; i < m; i += nt) {
      const double qi = A.q[D.r0 + i];
      const double qu = qi * A.invDr[D.r0 + i];
      a[1] = fma(qi, qi, a[1]);
      a[3] = fma(qu, qu, a[3]);
    }
    block_sum<4>(a, red);
    if (tid == 0) {
      const double cn = sqrt(red[0]), qn = sqrt(red[1]);
      scal[0] = (cn > 1e-10 && qn > 1e-10) ? cn / qn : 1.0;
      scal[1] = sqrt(red[2]);
      scal[2] = sqrt(red[3]);
    }
    __syncthreads();
    if (!(omega > 0.0)) omega = scal[0];
    if (A.omega0 != nullptr && A.omega0[b] > 0.0) omega = A.omega0[b];
  }
  DevParams P = A.P;
  P.cnorm = scal[1];
  P.qnorm = scal[2];

  // ---- initial point (the warm start or 0, projected onto X and Y) and anchor
  for (int j = tid; j < D.npad; j += nt) {
    const int64_t gj = D.c0 + j;
    const double x0 = j < n ? clamp_box(A.x0 ? A.x0[gj] : 0.0, A.l[gj], A.u[gj]) : 0.0;
    xs[j] = x0;
    A.xa[gj] = x0;
    A.sx[gj] = 0.0;
  }
  for (int i = tid; i < D.mpad; i += nt) {
    const int64_t gi = D.r0 + i;
    double y0 = (A.y0 && i < m) ? A.y0[gi] : 0.0;
    if (i >= D.m1) y0 = max0(y0);
    ys[i] = y0;
    A.ya[gi] = y0;
    A.sy[gi] = 0.0;
  }
  __syncthreads();
  batch_rows<kSrcSmemX>(A.k_cptr, A.k_col, A.k_val, D.kc0, D.kc1, D.c0, nullptr, A,
                        [&](int i, double s) { A.kxp[D.r0 + i] = s; });
  batch_rows<kSrcSmemY>(A.t_cptr, A.t_col, A.t_val, D.tc0, D.tc1, D.r0, nullptr, A,
                        [&](int j, double s) { A.g[D.c0 + j] = s; });
  __syncthreads();
  if (tid == 0) {
    memset(&S, 0, sizeof(S));
    S.eta = eta;
    S.omega = omega;
    S.tau = eta / omega;
    S.sigma = eta * omega;
  }
  __syncthreads();
  batch_kkt(A, D, true, 0.0, red, tot);
  if (tid == 0) {
    const double gap = tot[Q_QY_C] + tot[Q_LT_C] - tot[Q_CX_C];
    S.kkt_anchor = kkt_w(tot[Q_PRS_C], tot[Q_DRS_C], gap, S.omega);
    S.kkt_prev = __longlong_as_double(0x7FF0000000000000LL);
  }
  __syncthreads();

  // ---- iterations (Section 2: primal step, dual step with extrapolation) and checks
  long long k = 0, t = 0;
  const double* c = A.c;
  const double* l = A.l;
  const double* u = A.u;
  const double* q = A.q;
  for (;;) {
    const bool at_limit = k >= A.max_iter;
    if (!at_limit) {
      const double tau = S.tau, sigma = S.sigma;
      batch_rows<kSrcSmemY>(A.t_cptr, A.t_col, A.t_val, D.tc0, D.tc1, D.r0, nullptr, A, [&](int j, double gsum) {
        const int64_t gj = D.c0 + j;
        const double xn = clamp_box(fma(-tau, c[gj] - gsum, xs[j]), l[gj], u[gj]);
        xs[j] = xn;
        A.sx[gj] = A.sx[gj] + xn;
      });
      __syncthreads();
      batch_rows<kSrcSmemX>(A.k_cptr, A.k_col, A.k_val, D.kc0, D.kc1, D.c0, nullptr, A, [&](int i, double v) {
        const int64_t gi = D.r0 + i;
        const double e = q[gi] + A.kxp[gi];
        double yn = fma(sigma, fma(-2.0, v, e), ys[i]);
        if (i >= D.m1) yn = max0(yn);
        ys[i] = yn;
        A.sy[gi] = A.sy[gi] + yn;
        A.kxp[gi] = v;
      });
      __syncthreads();
      ++k;
      ++t;
      if (!(k % A.check_every == 0 || k >= A.max_iter)) continue;
    }
    // ---- check
    const double it = t > 0 ? 1.0 / (double)t : 0.0;
    batch_rows<kSrcSmemY>(A.t_cptr, A.t_col, A.t_val, D.tc0, D.tc1, D.r0, nullptr, A,
                          [&](int j, double s) { A.g[D.c0 + j] = s; });
    batch_rows<kSrcGlobal>(A.k_cptr, A.k_col, A.k_val, D.kc0, D.kc1, D.c0, A.sx + D.c0, A,
                           [&](int i, double s) { A.kx_a[D.r0 + i] = s * it; });
    batch_rows<kSrcGlobal>(A.t_cptr, A.t_col, A.t_val, D.tc0, D.tc1, D.r0, A.sy + D.r0, A,
                           [&](int j, double s) { A.g_a[D.c0 + j] = s * it; });
    __syncthreads();
    batch_kkt(A, D, t == 0, it, red, tot);
    if (tid == 0) {
      S.k = k;
      S.t = t;
      S.inv_t = it;
      decide_core(tot, &S, P, k >= A.max_iter, nullptr);
    }
    __syncthreads();
    if (S.done) break;
    if (S.restart_flag) {
      const bool avg = S.cand_avg;
      for (int j = tid; j < D.npad; j += nt) {
        const int64_t gj = D.c0 + j;
        const double xv = avg ? A.sx[gj] * it : xs[j];
        xs[j] = xv;
        A.xa[gj] = xv;
        A.sx[gj] = 0.0;
      }
      for (int i = tid; i < D.mpad; i += nt) {
        const int64_t gi = D.r0 + i;
        const double yv = avg ? A.sy[gi] * it : ys[i];
        ys[i] = yv;
        A.ya[gi] = yv;
        A.sy[gi] = 0.0;
        if (avg) A.kxp[gi] = A.kx_a[gi];
      }
      t = 0;
      __syncthreads();
    }
  }
  // ---- returned point and state
  const bool avg = S.which == 1 && t > 0;
  const double it = t > 0 ? 1.0 / (double)t : 0.0;
  for (int j = tid; j < D.npad; j += nt) A.xout[D.c0 + j] = avg ? A.sx[D.c0 + j] * it : xs[j];
  for (int i = tid; i < D.mpad; i += nt) A.yout[D.r0 + i] = avg ? A.sy[D.r0 + i] * it : ys[i];
  if (tid == 0) A.st[b] = S;
  __syncthreads();
}

__global__ void __launch_bounds__(256, 2) k_batch_solve(BatchArgs A) {
  __shared__ int lp;
  for (;;) {
    if (threadIdx.x == 0) {
      const int v = atomicAdd(A.next, 1);
      lp = v;
      // the last of the gridDim.x failing draws is the last access of this launch
      if (v == A.count + (int)gridDim.x - 1) *A.next = 0;
    }
    __syncthreads();
    const int v = lp;
    __syncthreads();
    if (v >= A.count) break;
    batch_solve_one(A, A.order[v]);
  }
}

}  // namespace pdlp
