// Host side and C ABI of the restarted-PDHG solver (declarations and contract in
// include/pdlp.h; method: arXiv 2312.14832, Section 2).
//
// pdlp_setup orders rows and columns by length on the host (O(m + n) work), builds the
// SELL-32 layouts of K and K' on the device from the caller's CSR arrays
// (layout_kernels.cuh: checks, CSC order by radix sort, per-slot fill), scales
// (Ruiz + Pock-Chambolle) and estimates ||K||_2 with device kernels.  Batches keep
// the host builder of layout.cpp (their LPs are small), which yields the same layouts.  pdlp_solve has two engines.  The kernels launched per
// iteration run as CUDA graphs, one graph per check interval: check_every x (primal
// kernel, dual kernel) followed by the check (three SpMVs, the KKT reductions, the
// restart decision and the restart itself), all state on the device; the host only
// launches graphs and reads a small status record a few intervals behind the device.
// The persistent engine (small LPs) runs the batched kernel of batch_kernel.cuh on the
// handle's own arrays: one thread-block cluster, the whole solve in one launch.
// pdlp_batch_setup / pdlp_batch_solve run many LPs through that kernel.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <limits>
#include <string>
#include <type_traits>
#include <vector>

#include "batch_kernel.cuh"
#include "kernels.cuh"
#include "layout.h"
#include "layout_kernels.cuh"
#include "pdlp.h"
#include "spmv_stage.cuh"

namespace pdlp {

static thread_local std::string g_setup_error;

// Records the text returned by pdlp_last_error(NULL) for handle-less calls.
void set_thread_error(const std::string& msg) { g_setup_error = msg; }

struct Failure {
  int code;
  std::string msg;
};

static void check_cuda(cudaError_t e, const char* what, int line) {
  if (e == cudaSuccess) return;
  char buf[512];
  snprintf(buf, sizeof(buf), "%s failed (line %d): %s", what, line, cudaGetErrorString(e));
  throw Failure{e == cudaErrorMemoryAllocation ? PDLP_ENOMEM : PDLP_ECUDA, buf};
}
#define CK(call) check_cuda((call), #call, __LINE__)
#define CKL(what) check_cuda(cudaGetLastError(), what, __LINE__)

static void invalid(const std::string& msg) { throw Failure{PDLP_EINVAL, msg}; }

struct DevSell {
  int32_t* chunk_ptr = nullptr;
  int32_t* col = nullptr;
  double* val = nullptr;
  float* val32 = nullptr;   // mixed precision only
  int32_t* ucol = nullptr;  // mixed precision, K with +-1 entries: sign-bit column words
  SellTask* tasks = nullptr;
  double* gpart = nullptr;
  int32_t* cnt = nullptr;
  uint8_t* wide = nullptr;   // per chunk, or null when no chunk is wide
  int32_t nwide = 0;
  int32_t ntasks = 0;
  int32_t tile = 0, tchunks = 0, batch = 8;
  int32_t staged = 0;   // FP64 products: 0 plain loads, 1 / 2 stream staged by bulk copies (2 / 3 buffers)
  int64_t rows = 0, rows_pad = 0, nchunks = 0, slots = 0, split = 0;
  SellView view() const {
    return SellView{chunk_ptr, col, val, val32, tasks, ntasks, (int32_t)nchunks, gpart, cnt, ucol};
  }
};

constexpr int kRing = 4;        // pinned status records in flight
constexpr int kLookahead = 2;   // intervals queued ahead of the one being read
constexpr int kVecGridMax = 148 * 8;
constexpr int64_t kAutotuneMinNnz = 1 << 20;   // smaller matrices keep the default schedule

}  // namespace pdlp

using namespace pdlp;

struct pdlp_ctx {
  pdlp_params p{};
  int64_t m = 0, n = 0, m1 = 0, nnz = 0, mpad = 0, npad = 0;
  int64_t m1_int = 0;   // internal rows [0, m1_int) are equality rows (padding rows included)
  int dev = 0;
  cudaStream_t s = nullptr;
  cudaEvent_t ev_user = nullptr, ev_done = nullptr, ev_t0 = nullptr, ev_t1 = nullptr;
  cudaEvent_t ev_ring[kRing] = {};
  std::vector<void*> allocs;
  DevSell K, Kt;
  int32_t *perm_r = nullptr, *pos_r = nullptr, *perm_c = nullptr, *pos_c = nullptr;
  double *c = nullptr, *l = nullptr, *u = nullptr, *q = nullptr;
  double *Dr = nullptr, *Dc = nullptr, *invDr = nullptr, *invDc = nullptr;
  double *x = nullptr, *y = nullptr, *sx = nullptr, *sy = nullptr, *xa = nullptr, *ya = nullptr;
  double *kxp = nullptr, *g_c = nullptr, *g_a = nullptr, *kx_a = nullptr;
  double *tn = nullptr, *tm = nullptr, *stage_n = nullptr, *stage_m = nullptr;
  double* part = nullptr;
  int nb_rows = 1, nb_cols = 1;
  double *red_part = nullptr, *red_out = nullptr;
  int red_blocks = 1;
  DevState* st = nullptr;
  DevState* st_tmp = nullptr;
  DevParams* dp = nullptr;
  CheckRecord* log = nullptr;
  long long* restarts = nullptr;
  int log_cap = 4096, restart_cap = 1 << 16;
  DevState* st_host = nullptr;   // pinned ring
  DevState st_init{};
  DevParams dp_host{};
  double eta = 1.0, omega0 = 1.0, normK = 0.0, qnorm = 0.0, cnorm = 0.0;
  std::string err;
  int* d_err = nullptr;   // set by a staged SpMV kernel whose bounded wait gave up
  bool broken = false;    // after such a failure the handle refuses further calls
  int64_t last_ncheck = 0, last_nrestart = 0;
  bool solved = false;
  bool resumable = false;   // the last solve ran the FP64 kernels per iteration (pdlp_get_state)
  cudaGraphExec_t g_full = nullptr, g_rem = nullptr;
  int g_full_len = -1, g_rem_len = -1;
  std::vector<cudaEvent_t> timing_events;
  // batch handles (pdlp_batch_setup): one block-diagonal layout, one LP per team of CTAs
  bool is_batch = false;
  int64_t count = 0;
  LpDesc* desc = nullptr;
  int32_t* order = nullptr;
  int32_t* next = nullptr;
  DevState* bstate = nullptr;
  double *bx = nullptr, *by = nullptr, *bomega = nullptr;
  int batch_grid = 0;        // CTAs of a one-CTA-per-LP launch
  int batch_resident = 0;    // CTAs of the batched kernel resident on the whole GPU
  int64_t team_npad_max = 0;
  int part_off = 0;
  size_t batch_smem = 0;
  int last_team = 0;         // CTAs per LP and resident mode of the last batched launch
  bool last_resident = false;
  bool last_glob = false;
  int32_t* order2 = nullptr; // queue of the second stage (LPs stopped by the slice)
  bool small_engine = false; // single-LP handle that can run the persistent engine
  bool batch_glob = false;   // x and y of the largest LP do not fit in shared memory
  size_t glob_smem = 0;      // shared memory of a launch with global iterates
  double *xg = nullptr, *yg = nullptr;      // global iterates (allocated on first use)
  float *xg32 = nullptr, *yg32 = nullptr;
  int64_t last_resumed = 0;  // LPs continued in the second stage of the last solve
  int64_t last_launches = 0; // batched launches of the last solve
  cudaGraphExec_t bgraph = nullptr;   // the device part of a batched solve (see batch_solve_impl)
  long long bgraph_key = -1;          // its launch configuration
  int last_grid = 0;                  // grid and shared memory of the last batched launch
  size_t last_smem = 0;
  bool last_graph = false;
  bool last_tuned = false;   // the last solve ran the online autotuner
  long long* brestarts = nullptr;   // batches: kBatchRestartCap restart iterations per LP
  // online autotuner of the batched launch: the kept choice and what the tuning timed
  bool tuned = false;
  int tuned_team = 0, tuned_resident = 0;
  int32_t tune_candidates = 0;
  double tune_rates[8] = {};
  int tune_team[8] = {}, tune_res[8] = {};
  double setup_ms[5] = {};   // setup phases (pdlp_info)
  std::vector<int32_t> hk_cptr, ht_cptr;  // host copies of the chunk pointers of K and K'
  int dev_smem_optin = 0;
  int xs_off = 0, ys_off = 0, red_off = 0;
  std::vector<LpDesc> hdesc;
  std::vector<DevState> hstate;
  // mixed precision (params.precision = 1): FP32 iterates, values and problem vectors
  float *x32 = nullptr, *y32 = nullptr, *sx32 = nullptr, *sy32 = nullptr, *kxp32 = nullptr;
  float *c32 = nullptr, *l32 = nullptr, *u32 = nullptr, *q32 = nullptr;
  // +-1 entries as sign bits (mixed_values): the FP32 iterates are D_c x and D_r y;
  // D_c^2 and D_r^2 in FP32 (c32, l32, u32, q32 then hold the unscaled data)
  float *dc2 = nullptr, *dr2 = nullptr;
  bool unit_ok = false;     // every entry of K is +-1 (checked at setup when mixed_values != 1)
  int32_t mixed_values = 0; // 0 FP64 handle, 1 FP32 value copies, 2 sign bits
  cudaGraphExec_t gm_full = nullptr, gm_rem = nullptr;
  int gm_full_len = -1, gm_rem_len = -1;
  int64_t fp32_iters = 0;   // iterations of the last solve run in FP32
  // adaptive step rule (params.step_rule = 1): backups of the point, per-task partials
  double *xb = nullptr, *yb = nullptr, *kxb = nullptr, *part_x = nullptr, *part_y = nullptr, *part_s = nullptr;
  double eta_adapt0 = 1.0;   // 1 / max |K_ij| of the scaled K
  bool power_done = false;   // the power-iteration step size has been computed
  cudaGraphExec_t ga_full = nullptr, ga_rem = nullptr;
  int ga_full_len = -1, ga_rem_len = -1;
};

namespace pdlp {

static int grid_for(int64_t n) {
  int64_t g = (n + 255) / 256;
  if (g < 1) g = 1;
  if (g > kVecGridMax) g = kVecGridMax;
  return (int)g;
}

template <class T>
static T* dalloc(pdlp_ctx* h, size_t count) {
  void* p = nullptr;
  size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
  CK(cudaMalloc(&p, bytes));
  h->allocs.push_back(p);
  CK(cudaMemsetAsync(p, 0, bytes, h->s));
  return (T*)p;
}

template <class T>
static T* upload(pdlp_ctx* h, const std::vector<T>& v) {
  T* d = dalloc<T>(h, v.size());
  if (!v.empty()) CK(cudaMemcpyAsync(d, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, h->s));
  CK(cudaStreamSynchronize(h->s));   // host vectors may be released after return
  return d;
}

static void dfree(pdlp_ctx* h, void* p) {
  auto it = std::find(h->allocs.begin(), h->allocs.end(), p);
  if (it != h->allocs.end()) {
    cudaFree(p);
    h->allocs.erase(it);
  }
}

// Staged-stream SpMV shapes: kStageSB slots per buffer, 2 or 3 buffers per warp.
constexpr int kStageSB = 8;
using StageA = StageShape<kStageSB, 2>;
using StageB = StageShape<kStageSB, 3>;

template <class Op, class Epi>
static void launch_rows(pdlp_ctx* h, const DevSell& S, const typename Epi::T* xg, Epi epi, const DevState* st) {
  const int blocks = (S.ntasks + 7) / 8;
  if constexpr (std::is_same<Op, OpSpmv>::value && std::is_same<typename Epi::T, double>::value) {
    if (S.staged == 1) {
      if (S.batch == 4)
        sell_rows_staged_kernel<Op, Epi, 4, kStageSB, 2><<<blocks, 256, StageA::kCtaBytes, h->s>>>(S.view(), xg, epi, st, h->d_err);
      else
        sell_rows_staged_kernel<Op, Epi, 8, kStageSB, 2><<<blocks, 256, StageA::kCtaBytes, h->s>>>(S.view(), xg, epi, st, h->d_err);
      return;
    }
    if (S.staged == 2) {
      if (S.batch == 4)
        sell_rows_staged_kernel<Op, Epi, 4, kStageSB, 3><<<blocks, 256, StageB::kCtaBytes, h->s>>>(S.view(), xg, epi, st, h->d_err);
      else
        sell_rows_staged_kernel<Op, Epi, 8, kStageSB, 3><<<blocks, 256, StageB::kCtaBytes, h->s>>>(S.view(), xg, epi, st, h->d_err);
      return;
    }
  }
  if (S.batch == 4) sell_rows_kernel<Op, Epi, 4><<<blocks, 256, 0, h->s>>>(S.view(), xg, epi, st);
  else sell_rows_kernel<Op, Epi, 8><<<blocks, 256, 0, h->s>>>(S.view(), xg, epi, st);
}

// Opt-in shared memory of every staged SpMV instantiation (on the current device).
template <class Epi>
static void stage_attrs_for() {
  CK(cudaFuncSetAttribute(sell_rows_staged_kernel<OpSpmv, Epi, 4, kStageSB, 2>,
                          cudaFuncAttributeMaxDynamicSharedMemorySize, StageA::kCtaBytes));
  CK(cudaFuncSetAttribute(sell_rows_staged_kernel<OpSpmv, Epi, 8, kStageSB, 2>,
                          cudaFuncAttributeMaxDynamicSharedMemorySize, StageA::kCtaBytes));
  CK(cudaFuncSetAttribute(sell_rows_staged_kernel<OpSpmv, Epi, 4, kStageSB, 3>,
                          cudaFuncAttributeMaxDynamicSharedMemorySize, StageB::kCtaBytes));
  CK(cudaFuncSetAttribute(sell_rows_staged_kernel<OpSpmv, Epi, 8, kStageSB, 3>,
                          cudaFuncAttributeMaxDynamicSharedMemorySize, StageB::kCtaBytes));
}
static void stage_attrs() {
  stage_attrs_for<EpiStore>();
  stage_attrs_for<EpiPrimal>();
  stage_attrs_for<EpiDual>();
  stage_attrs_for<EpiPrimalA>();
  stage_attrs_for<EpiDualA>();
}

// A staged SpMV kernel sets *d_err when a bounded wait gave up; the handle's device
// state is then undefined, so the handle refuses every later call.
static void check_stage_err(pdlp_ctx* h) {
  if (!h->d_err) return;
  int e = 0;
  CK(cudaMemcpyAsync(&e, h->d_err, sizeof(int), cudaMemcpyDeviceToHost, h->s));
  CK(cudaStreamSynchronize(h->s));
  if (e) {
    h->broken = true;
    throw Failure{PDLP_ETIMEOUT, "a bounded wait of the staged SpMV kernel gave up; free this handle"};
  }
}

// The caller's matrix on the device, with what the device layout builder derives from
// it: tp = column starts of the CSC order (n + 1), csc = entry indices in CSC order,
// rowof = the row of each entry.
struct DevCsr {
  const int64_t* rp;
  const int32_t* col;
  const double* val;
  const int32_t* tp;
  const int32_t* csc;
  const int32_t* rowof;
  const int32_t* kpad;   // padding column of each K chunk (first internal column of its LP)
  const int32_t* tpad;   // padding column of each K' chunk (first internal row of its LP)
};

// Uploads the shape and task plan of a layout and allocates its arrays.
static void alloc_device_sell(pdlp_ctx* h, DevSell& D, const SellHost& S, const TaskPlan& P) {
  D.rows = S.rows;
  D.rows_pad = S.rows_pad;
  D.nchunks = S.nchunks;
  D.slots = S.slots();
  D.split = P.split_chunks;
  D.ntasks = (int32_t)P.tasks.size();
  D.chunk_ptr = upload(h, S.chunk_ptr);
  D.tasks = upload(h, P.tasks);
  D.gpart = dalloc<double>(h, (size_t)D.ntasks * 32);
  D.cnt = dalloc<int32_t>(h, (size_t)D.ntasks);
  D.val = dalloc<double>(h, (size_t)D.slots * 32);
  D.nwide = 0;
  for (uint8_t f : S.wide) D.nwide += f != 0;
  D.wide = D.nwide > 0 ? upload(h, S.wide) : nullptr;
}

// Layout built on the host (S.col, S.src): upload, then gather the values.
static void build_device_sell(pdlp_ctx* h, DevSell& D, const SellHost& S, const TaskPlan& P,
                              const double* d_csr_val) {
  alloc_device_sell(h, D, S, P);
  D.col = upload(h, S.col);
  int32_t* d_src = upload(h, S.src);
  k_gather_values<<<grid_for(D.slots * 32), 256, 0, h->s>>>(D.val, d_src, d_csr_val, D.slots * 32);
  CKL("k_gather_values");
  CK(cudaStreamSynchronize(h->s));
  dfree(h, d_src);
}

// Layout filled on the device from the caller's matrix (S holds the shape only): K rows
// from the CSR rows, K' rows from the CSC order.  Needs perm_* and pos_* on the device.
static void fill_device_sell(pdlp_ctx* h, DevSell& D, const SellHost& S, const TaskPlan& P, const DevCsr& C,
                             bool transpose) {
  alloc_device_sell(h, D, S, P);
  const int64_t total = D.slots * 32;
  D.col = dalloc<int32_t>(h, (size_t)total);
  if (!transpose)
    k_fill_sell<int64_t><<<grid_for(total), 256, 0, h->s>>>(D.chunk_ptr, D.nchunks, D.wide, total, h->perm_r, C.rp,
                                                           nullptr, C.col, h->pos_c, C.val, C.kpad, D.col, D.val);
  else
    k_fill_sell<int32_t><<<grid_for(total), 256, 0, h->s>>>(D.chunk_ptr, D.nchunks, D.wide, total, h->perm_c, C.tp,
                                                           C.csc, C.rowof, h->pos_r, C.val, C.tpad, D.col, D.val);
  CKL("k_fill_sell");
}

// Replaces the warp-task plan of a device layout (the arrays of values and indices stay).
static void set_plan(pdlp_ctx* h, DevSell& D, const TaskPlan& P, int32_t tile, int32_t tchunks, int32_t batch) {
  CK(cudaStreamSynchronize(h->s));
  dfree(h, D.tasks);
  dfree(h, D.gpart);
  dfree(h, D.cnt);
  D.ntasks = (int32_t)P.tasks.size();
  D.split = P.split_chunks;
  D.tasks = upload(h, P.tasks);
  D.gpart = dalloc<double>(h, (size_t)D.ntasks * 32);
  D.cnt = dalloc<int32_t>(h, (size_t)D.ntasks);
  D.tile = tile;
  D.tchunks = tchunks;
  D.batch = batch;
}

static void norm2_dev(pdlp_ctx* h, const double* a, int64_t n) {
  k_sumsq_partial<<<h->red_blocks, 256, 0, h->s>>>(h->red_part, a, n);
  k_sum_sqrt<<<1, 32, 0, h->s>>>(h->red_out, h->red_part, h->red_blocks);
}

static double norm2_host(pdlp_ctx* h, const double* a, int64_t n) {
  norm2_dev(h, a, n);
  double v = 0.0;
  CK(cudaMemcpyAsync(&v, h->red_out, sizeof(double), cudaMemcpyDeviceToHost, h->s));
  CK(cudaStreamSynchronize(h->s));
  return v;
}

// k_div_into: a <- w / s[0] when s[0] != 0 (otherwise a keeps the last unit vector)
__global__ void k_div_into(double* a, const double* w, const double* s, int64_t n) {
  const double d = s[0];
  if (d == 0.0) return;
  PDLP_GRID_STRIDE(i, n) a[i] = w[i] / d;
}

// v <- (v * fr[i]) * fc[j] for K (transposed = 0: chunk rows are i, columns j) and for
// K' (transposed = 1: chunk rows are j, columns i), so both copies round identically.
// One thread per (slot, lane) of the total = slots * 32 entries; a warp's slot is found
// in chunk_ptr by binary search, so long chunks take no longer than short ones.  A wide
// chunk (wide[ch] != 0) holds one row, the chunk's first.
__global__ void k_scale_sell2(double* v, const int32_t* col, const int32_t* chunk_ptr, int64_t nchunks, int64_t total,
                              const double* fr, const double* fc, int transposed, const uint8_t* wide) {
  PDLP_GRID_STRIDE(e, total) {
    const int64_t s = e >> 5;
    int64_t lo = 0, hi = nchunks - 1;
    while (lo < hi) {
      const int64_t mid = (lo + hi + 1) >> 1;
      if (chunk_ptr[mid] <= s) lo = mid;
      else hi = mid - 1;
    }
    const int64_t row = lo * 32 + ((wide != nullptr && wide[lo]) ? 0 : (e & 31));
    const double a = transposed ? fr[col[e]] : fr[row];
    const double b = transposed ? fc[row] : fc[col[e]];
    v[e] = (v[e] * a) * b;
  }
}

// Bound duals in scaled, internal order: lam = proj_Lambda(c - g) (Section 2: Lambda_j is
// {0}, R^-, R^+ or R as l_j, u_j are infinite or finite); positive scalings keep the cone.
__global__ void k_bound_duals(double* lam, const double* c, const double* g, const double* l, const double* u,
                              int64_t n) {
  PDLP_GRID_STRIDE(j, n) {
    const double d = c[j] - g[j];
    const bool lf = !is_neg_inf(l[j]), uf = !is_pos_inf(u[j]);
    const bool neg = __double2hiint(d) < 0;
    double v;
    if (lf && uf) v = d;
    else if (lf) v = neg ? 0.0 : d;
    else if (uf) v = neg ? d : 0.0;
    else v = 0.0;
    lam[j] = v;
  }
}

// dst = average of the inner loop (sum * 1/t), or the current iterate when t = 0
__global__ void k_average(double* dst, const double* sum, const double* cur, const DevState* st, int64_t n) {
  const bool empty = st->t == 0;
  const double it = st->inv_t;
  PDLP_GRID_STRIDE(i, n) dst[i] = empty ? cur[i] : sum[i] * it;
}

// copy of the state with done cleared (for pdlp_time_iterations)
__global__ void k_copy_state(DevState* dst, const DevState* src) {
  *dst = *src;
  dst->done = 0;
}

static void enqueue_iteration(pdlp_ctx* h, const DevState* st) {
  launch_rows<OpSpmv>(h, h->Kt, h->y, EpiPrimal{h->x, h->sx, h->c, h->l, h->u, 0.0}, st);
  launch_rows<OpSpmv>(h, h->K, h->x, EpiDual{h->y, h->sy, h->kxp, h->q, (int)h->m1_int, 0.0}, st);
}

// One attempt of the adaptive step rule (launch count: 5).
static void enqueue_attempt(pdlp_ctx* h, DevState* st) {
  launch_rows<OpSpmv>(h, h->Kt, h->y, EpiPrimalA{h->x, h->xb, h->sx, h->c, h->l, h->u, h->part_x, 0.0, 0.0, 0.0}, st);
  launch_rows<OpSpmv>(h, h->K, h->x,
                      EpiDualA{h->y, h->yb, h->sy, h->kxp, h->kxb, h->q, h->part_y, (int)h->m1_int, 0.0, 0.0, 0.0, 0.0},
                      st);
  k_step_partial<<<kStepParts + 1, 256, 0, h->s>>>(h->part_x, h->Kt.ntasks, h->part_y, h->K.ntasks, h->part_s, st);
  k_step_decide<<<1, 32, 0, h->s>>>(h->part_s, st);
  // a kept step (most attempts) makes this a no-op, so it gets one block per SM
  k_step_restore<<<std::min(grid_for(std::max(h->npad, h->mpad)), 148), 256, 0, h->s>>>(
      h->x, h->xb, h->npad, h->y, h->yb, h->kxp, h->kxb, h->mpad, st);
}

static void launch_primal32(pdlp_ctx* h, const DevState* st) {
  if (h->mixed_values == 2)
    launch_rows<OpUnitF>(h, h->Kt, h->y32, EpiPrimal32U{h->x32, h->sx32, h->c32, h->l32, h->u32, h->dc2, 0.f}, st);
  else
    launch_rows<OpSpmvF>(h, h->Kt, h->y32, EpiPrimal32{h->x32, h->sx32, h->c32, h->l32, h->u32, 0.f}, st);
}
static void launch_dual32(pdlp_ctx* h, const DevState* st) {
  if (h->mixed_values == 2)
    launch_rows<OpUnitF>(h, h->K, h->x32, EpiDual32U{h->y32, h->sy32, h->kxp32, h->q32, h->dr2, (int)h->m1_int, 0.f},
                         st);
  else
    launch_rows<OpSpmvF>(h, h->K, h->x32, EpiDual32{h->y32, h->sy32, h->kxp32, h->q32, (int)h->m1_int, 0.f}, st);
}

static void enqueue_iteration32(pdlp_ctx* h, const DevState* st) {
  launch_primal32(h, st);
  launch_dual32(h, st);
}

static MixedScale mixed_scale(pdlp_ctx* h) {
  if (h->mixed_values != 2) return MixedScale{nullptr, nullptr, nullptr, nullptr};
  return MixedScale{h->Dc, h->invDc, h->Dr, h->invDr};
}

static KktInputs kkt_inputs(pdlp_ctx* h) {
  KktInputs in;
  in.q = h->q; in.kx_c = h->kxp; in.kx_a = h->kx_a; in.y = h->y; in.sy = h->sy; in.ya = h->ya;
  in.invDr = h->invDr;
  in.c = h->c; in.l = h->l; in.u = h->u; in.g_c = h->g_c; in.g_a = h->g_a; in.x = h->x; in.sx = h->sx;
  in.xa = h->xa; in.invDc = h->invDc;
  in.m = h->mpad; in.n = h->n; in.m1 = (int)h->m1_int; in.rows_blocks = h->nb_rows;
  return in;
}

// The check (launch count: 8; 9 with the adaptive rule, whose pending weight goes
// into the running sums first).
static void enqueue_check(pdlp_ctx* h, int len, int final_check, bool adaptive = false) {
  if (adaptive)
    k_flush_pending<<<grid_for(std::max(h->npad, h->mpad)), 256, 0, h->s>>>(h->sx, h->x, h->npad, h->sy, h->y,
                                                                            h->mpad, h->st);
  k_precheck<<<1, 1, 0, h->s>>>(h->st, len, adaptive ? 1 : 0);
  launch_rows<OpSpmv>(h, h->Kt, h->y, EpiStore{h->g_c, 0, 1.0}, h->st);
  launch_rows<OpSpmv>(h, h->K, h->sx, EpiStore{h->kx_a, 1, 1.0}, h->st);
  launch_rows<OpSpmv>(h, h->Kt, h->sy, EpiStore{h->g_a, 1, 1.0}, h->st);
  k_kkt_partials<<<h->nb_rows + h->nb_cols, 256, 0, h->s>>>(kkt_inputs(h), h->st, h->part);
  k_decide<<<1, 256, 0, h->s>>>(h->part, h->nb_rows, h->nb_cols, h->st, h->dp, h->log, h->restarts, 0,
                                final_check);
  RestartArgs ra{h->x, h->sx, h->xa, h->y, h->sy, h->ya, h->kxp, h->kx_a, h->npad, h->mpad};
  k_restart_apply<<<grid_for(std::max(h->npad, h->mpad)), 256, 0, h->s>>>(ra, h->st);
  k_post_restart<<<1, 1, 0, h->s>>>(h->st);
}

// Mixed-precision check: FP64 copies of the FP32 iterates and sums, K x in FP64, the
// FP64 check, FP32 iterates back from the (possibly restarted) FP64 ones (launches: 12).
static void enqueue_check_mixed(pdlp_ctx* h, int len, int final_check) {
  k_mixed_to64<<<grid_for(std::max(h->npad, h->mpad)), 256, 0, h->s>>>(h->x, h->sx, h->x32, h->sx32, h->npad, h->y,
                                                                       h->sy, h->y32, h->sy32, h->mpad, h->st,
                                                                       mixed_scale(h));
  launch_rows<OpSpmv>(h, h->K, h->x, EpiStore{h->kxp, 0, 1.0}, h->st);
  enqueue_check(h, len, final_check);
  k_mixed_to32<<<grid_for(std::max(h->npad, h->mpad)), 256, 0, h->s>>>(h->x32, h->x, h->npad, h->y32, h->y,
                                                                       h->kxp32, h->kxp, h->mpad, h->st,
                                                                       mixed_scale(h));
}

enum { kModeFp64 = 0, kModeMixed = 1, kModeAdaptive = 2 };

static cudaGraphExec_t capture_interval(pdlp_ctx* h, int len, int mode = kModeFp64) {
  cudaGraph_t g = nullptr;
  cudaGraphExec_t ex = nullptr;
  CK(cudaStreamBeginCapture(h->s, cudaStreamCaptureModeThreadLocal));
  if (mode == kModeMixed) {
    for (int i = 0; i < len; ++i) enqueue_iteration32(h, h->st);
    enqueue_check_mixed(h, len, 0);
  } else if (mode == kModeAdaptive) {
    for (int i = 0; i < len; ++i) enqueue_attempt(h, h->st);
    enqueue_check(h, len, 0, true);
  } else {
    for (int i = 0; i < len; ++i) enqueue_iteration(h, h->st);
    enqueue_check(h, len, 0);
  }
  cudaError_t e = cudaStreamEndCapture(h->s, &g);
  CK(e);
  e = cudaGraphInstantiate(&ex, g, 0);
  cudaGraphDestroy(g);
  CK(e);
  return ex;
}

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

struct StreamOrder {
  pdlp_ctx* h;
  cudaStream_t user;
  StreamOrder(pdlp_ctx* h_, void* user_stream) : h(h_), user((cudaStream_t)user_stream) {
    if (user) {
      CK(cudaEventRecord(h->ev_user, user));
      CK(cudaStreamWaitEvent(h->s, h->ev_user, 0));
    }
  }
  ~StreamOrder() {
    if (user) {
      cudaEventRecord(h->ev_done, h->s);
      cudaStreamWaitEvent(user, h->ev_done, 0);
    }
  }
};

static void copy_in(pdlp_ctx* h, double* dst, const double* src, int64_t count) {
  if (count <= 0) return;
  CK(cudaMemcpyAsync(dst, src, (size_t)count * sizeof(double),
                     h->p.inputs_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->s));
}
static void copy_out(pdlp_ctx* h, double* dst, const double* src, int64_t count) {
  if (count <= 0 || dst == nullptr) return;
  CK(cudaMemcpyAsync(dst, src, (size_t)count * sizeof(double),
                     h->p.inputs_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->s));
}

// Unscaled, original-order copy of an internal (x, y) pair to caller buffers.
static void export_point(pdlp_ctx* h, const double* xi, const double* yi, double* x_out, double* y_out) {
  if (x_out) {
    k_unpermute_scale<<<grid_for(h->n), 256, 0, h->s>>>(h->stage_n, xi, h->Dc, h->pos_c, h->n);
    copy_out(h, x_out, h->stage_n, h->n);
  }
  if (y_out && h->m > 0) {
    k_unpermute_scale<<<grid_for(h->m), 256, 0, h->s>>>(h->stage_m, yi, h->Dr, h->pos_r, h->m);
    copy_out(h, y_out, h->stage_m, h->m);
  }
  CK(cudaStreamSynchronize(h->s));
}

static void destroy(pdlp_ctx* h) {
  if (!h) return;
  if (h->s) cudaStreamSynchronize(h->s);
  if (h->g_full) cudaGraphExecDestroy(h->g_full);
  if (h->g_rem) cudaGraphExecDestroy(h->g_rem);
  if (h->gm_full) cudaGraphExecDestroy(h->gm_full);
  if (h->gm_rem) cudaGraphExecDestroy(h->gm_rem);
  if (h->ga_full) cudaGraphExecDestroy(h->ga_full);
  if (h->ga_rem) cudaGraphExecDestroy(h->ga_rem);
  if (h->bgraph) cudaGraphExecDestroy(h->bgraph);
  for (void* p : h->allocs) cudaFree(p);
  h->allocs.clear();
  if (h->st_host) cudaFreeHost(h->st_host);
  for (auto e : h->timing_events) cudaEventDestroy(e);
  for (auto& e : h->ev_ring)
    if (e) cudaEventDestroy(e);
  if (h->ev_user) cudaEventDestroy(h->ev_user);
  if (h->ev_done) cudaEventDestroy(h->ev_done);
  if (h->ev_t0) cudaEventDestroy(h->ev_t0);
  if (h->ev_t1) cudaEventDestroy(h->ev_t1);
  if (h->s) cudaStreamDestroy(h->s);
  delete h;
}

// ------------------------------------------------------------------ autotuner

// Chooses (tile_slots, tile_chunks, batch) for one layout by timing the production
// iteration kernel (fused epilogue included) on the handle's own buffers, which the
// next pdlp_solve re-initialises; tau = sigma = 0 so the iterate does not move.  Then,
// for that plan, the kernels whose value / index stream is staged in shared memory by
// bulk copies (two or three buffers per warp, both batch sizes) compete with it, unless
// stage_fixed >= 0 fixes the kind (0 plain loads, 1 / 2 staged).
static void autotune(pdlp_ctx* h, DevSell& D, const SellHost& S, bool primal, int stage_fixed) {
  static const int32_t tiles[] = {32, 64};
  static const int32_t chunks[] = {1, 2, 4, 8};
  static const int32_t batches[] = {4, 8};
  DevState zs{};
  CK(cudaMemcpyAsync(h->st_tmp, &zs, sizeof(DevState), cudaMemcpyHostToDevice, h->s));
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  auto time_plan = [&]() {
    float tot = 0.f;
    for (int rep = 0; rep < 4; ++rep) {
      if (rep == 1) CK(cudaEventRecord(e0, h->s));
      if (primal)
        launch_rows<OpSpmv>(h, D, h->y, EpiPrimal{h->x, h->sx, h->c, h->l, h->u, 0.0}, h->st_tmp);
      else
        launch_rows<OpSpmv>(h, D, h->x, EpiDual{h->y, h->sy, h->kxp, h->q, (int)h->m1_int, 0.0}, h->st_tmp);
    }
    CK(cudaEventRecord(e1, h->s));
    CKL("autotune launch");
    CK(cudaEventSynchronize(e1));
    CK(cudaEventElapsedTime(&tot, e0, e1));
    return tot;
  };
  float best = 1e30f;
  int32_t bt = D.tile, bc = D.tchunks, bb = D.batch, bs = 0;
  D.staged = stage_fixed > 0 ? stage_fixed : 0;
  for (int32_t t : tiles)
    for (int32_t c : chunks) {
      TaskPlan P = plan_tasks(S, t, c);
      for (int32_t b : batches) {
        set_plan(h, D, P, t, c, b);
        const float tot = time_plan();
        if (tot < best) {
          best = tot;
          bt = t;
          bc = c;
          bb = b;
        }
      }
    }
  bs = D.staged;
  set_plan(h, D, plan_tasks(S, bt, bc), bt, bc, bb);
  if (stage_fixed < 0) {
    for (int32_t sg : {1, 2})
      for (int32_t b : batches) {
        D.staged = sg;
        D.batch = b;
        const float tot = time_plan();
        if (tot < best) {
          best = tot;
          bs = sg;
          bb = b;
        }
      }
  }
  D.staged = bs;
  D.batch = bb;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  check_stage_err(h);
}

// ------------------------------------------------------------------ setup

// Host copy of the matrix of an LP (one LP, or the concatenation of a batch) for the
// host builder.
struct HostLP {
  std::vector<int64_t> rp;   // row pointers (per LP restarting at 0 for a batch)
  std::vector<int32_t> col;
  std::vector<double> val;
};

static void init_handle_resources(pdlp_ctx* h) {
  CK(cudaGetDevice(&h->dev));
  CK(cudaStreamCreateWithFlags(&h->s, cudaStreamNonBlocking));
  CK(cudaEventCreateWithFlags(&h->ev_user, cudaEventDisableTiming));
  CK(cudaEventCreateWithFlags(&h->ev_done, cudaEventDisableTiming));
  CK(cudaEventCreate(&h->ev_t0));
  CK(cudaEventCreate(&h->ev_t1));
  for (auto& e : h->ev_ring) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  CK(cudaMallocHost(&h->st_host, sizeof(DevState) * kRing));
  h->d_err = dalloc<int>(h, 1);
  stage_attrs();
}

static void check_params(const pdlp_params& P) {
  if (P.check_every < 1) invalid("check_every must be >= 1");
  if (P.spmv_stage < 0 || P.spmv_stage > 3) invalid("spmv_stage must be 0, 1, 2 or 3");
  if (!(P.step_scale > 0.0) || P.ruiz_iters < 0 || P.power_iters < 0) invalid("bad scaling/step parameters");
  if (P.cluster_ctas < 0 || P.cluster_ctas > kMaxTeam) invalid("cluster_ctas must be in [0, 16]");
  if (P.resident < 0 || P.resident > 3) invalid("resident must be 0, 1, 2 or 3");
  if (P.step_rule < 0 || P.step_rule > 1) invalid("step_rule must be 0 or 1");
  if (P.engine < 0 || P.engine > 2) invalid("engine must be 0, 1 or 2");
  if (P.host_layout < 0 || P.host_layout > 1) invalid("host_layout must be 0 or 1");
  if (P.mixed_values < 0 || P.mixed_values > 2) invalid("mixed_values must be 0, 1 or 2");
  if (P.adaptive_reject_cap < 0) invalid("adaptive_reject_cap must be >= 0");
}

// True when pred(i) holds for every i in [0, n) (checked in parallel ranges).
template <class P>
static bool all_of_range(int64_t n, P pred) {
  std::atomic<int> bad{0};
  parallel_ranges(n, [&](int64_t a, int64_t b) {
    for (int64_t i = a; i < b; ++i)
      if (!pred(i)) {
        bad.store(1, std::memory_order_relaxed);
        return;
      }
  });
  return bad.load() == 0;
}

// The host builder's inputs (host_layout = 1): copies the row pointers (rp_count of
// them), column indices and values of the matrix (h->nnz entries) to the host and checks
// that the values are finite; the vectors are checked by check_vectors.
static void fetch_matrix(pdlp_ctx* h, const int64_t* row_ptr_in, const int32_t* col_in, const double* val_in,
                         HostLP& H, int64_t rp_count) {
  const bool dev_in = h->p.inputs_on_device != 0;
  auto fetch = [&](void* dst, const void* src, size_t bytes) {
    if (bytes == 0) return;
    if (dev_in) {
      CK(cudaMemcpy(dst, src, bytes, cudaMemcpyDeviceToHost));
    } else {
      parallel_ranges((int64_t)bytes, [&](int64_t a, int64_t b) {
        std::memcpy(static_cast<char*>(dst) + a, static_cast<const char*>(src) + a, (size_t)(b - a));
      }, (int64_t)1 << 22);
    }
  };
  const int64_t nnz = h->nnz;
  H.rp.resize((size_t)rp_count);
  H.col.resize((size_t)nnz);
  H.val.resize((size_t)nnz);
  fetch(H.rp.data(), row_ptr_in, sizeof(int64_t) * rp_count);
  fetch(H.col.data(), col_in, sizeof(int32_t) * nnz);
  fetch(H.val.data(), val_in, sizeof(double) * nnz);
  if (!all_of_range(nnz, [&](int64_t k) { return std::isfinite(H.val[(size_t)k]); }))
    invalid("non-finite matrix value");
}

// Checks row pointers [rp0, rp0 + m] of one LP (starting at 0) and its column indices.
static int64_t check_csr(const HostLP& H, int64_t rp0, int64_t m, int64_t n, int64_t nnz0) {
  if (H.rp[(size_t)rp0] != 0) invalid("row_ptr[0] must be 0");
  for (int64_t i = 0; i < m; ++i)
    if (H.rp[(size_t)(rp0 + i + 1)] < H.rp[(size_t)(rp0 + i)]) invalid("row_ptr must be nondecreasing");
  const int64_t nnz = H.rp[(size_t)(rp0 + m)];
  if (!all_of_range(nnz, [&](int64_t k) {
        const int32_t cc = H.col[(size_t)(nnz0 + k)];
        return cc >= 0 && cc < n;
      }))
    invalid("column index out of range");
  return nnz;
}

// Internal numbering and SELL layouts.  perm_* have one entry per internal (padded)
// position: the caller's index, or -1 in padding; pos_* map the caller's index to
// the internal position.
struct Layout {
  SellHost SK, SKt;
  std::vector<int32_t> perm_r, pos_r, perm_c, pos_c;
  int64_t mpad = 0, npad = 0;
};

// Single-LP handles up to this many nonzeros get the persistent engine (when x and y fit
// in one CTA's shared memory and no row is wide).
constexpr int64_t kSmallEngineNnz = (int64_t)1 << 18;

// Rows at least this long that are more than 4 times longer than the next row in
// length order are stored as wide rows (layout.h).
constexpr int64_t kWideMin = 1024;

// Row and column order of one LP inside a layout (local indices count from the LP's
// first row / column; internal ones from its first internal row / column).
struct LpOrder {
  std::vector<int32_t> ord;      // internal row -> local row, -1 for padding (mp entries)
  std::vector<int32_t> pc;       // internal column -> local column (n entries)
  std::vector<int32_t> lpos_r;   // local row -> internal row
  std::vector<int32_t> lpos_c;   // local column -> internal column
  std::vector<int32_t> rlen, clen;
  int64_t m = 0, n = 0, rbase = 0, cbase = 0, mp = 0, np = 0;
};

// Orders the rows and columns of one LP (row pointers rp[0..m], starting at 0; column
// counts clen) and appends them to L at internal offsets L.mpad / L.npad: rows are
// equality rows, then inequality rows, each by decreasing length; columns by decreasing
// length; both padded to a multiple of 32 (at least 32).  A wide row (wide_ok) starts a
// chunk and is followed by 31 empty padding rows.  Appends the entry counts of the
// internal rows of K (k_eln) and of K' (t_eln).  O(m + n) work.
static void order_lp(Layout& L, LpOrder& O, const int64_t* rp, std::vector<int32_t>&& clen, int64_t m, int64_t n,
                     int64_t m1, int64_t row0, int64_t col0, std::vector<int32_t>& k_eln, std::vector<int32_t>& t_eln,
                     bool wide_ok = false, std::vector<uint8_t>* k_wide = nullptr, int64_t* m1_int = nullptr) {
  O.m = m;
  O.n = n;
  O.rbase = L.mpad;
  O.cbase = L.npad;
  O.np = std::max<int64_t>(32, (n + 31) / 32 * 32);
  O.clen = std::move(clen);
  O.rlen.resize((size_t)m);
  for (int64_t i = 0; i < m; ++i) O.rlen[(size_t)i] = (int32_t)(rp[i + 1] - rp[i]);
  const std::vector<int32_t>& rlen = O.rlen;
  std::vector<int32_t> pr((size_t)std::max<int64_t>(m, 1));
  O.pc.resize((size_t)n);
  sort_by_length_desc(rlen, 0, m1, pr);
  sort_by_length_desc(rlen, m1, m, pr);
  sort_by_length_desc(O.clen, 0, n, O.pc);
  std::vector<int32_t>& ord = O.ord;
  std::vector<uint8_t> wflag;
  ord.reserve((size_t)m + 64);
  auto emit_block = [&](int64_t p0, int64_t p1) {
    int64_t p = p0;
    while (wide_ok && p < p1) {
      const int64_t len = rlen[(size_t)pr[(size_t)p]];
      const int64_t next = p + 1 < p1 ? rlen[(size_t)pr[(size_t)p + 1]] : 0;
      if (len < kWideMin || len <= 4 * next) break;
      while (ord.size() % 32) {
        ord.push_back(-1);
        wflag.push_back(0);
      }
      ord.push_back(pr[(size_t)p]);
      wflag.push_back(1);
      for (int k = 0; k < 31; ++k) {
        ord.push_back(-1);
        wflag.push_back(0);
      }
      ++p;
    }
    for (; p < p1; ++p) {
      ord.push_back(pr[(size_t)p]);
      wflag.push_back(0);
    }
  };
  emit_block(0, m1);
  if (m1_int) *m1_int = (int64_t)ord.size();
  emit_block(m1, m);
  const int64_t mint = (int64_t)ord.size();
  O.mp = std::max<int64_t>(32, (mint + 31) / 32 * 32);
  const int64_t mp = O.mp, np = O.np;
  ord.resize((size_t)mp, -1);
  wflag.resize((size_t)mp, 0);
  if (k_wide) *k_wide = std::move(wflag);
  O.lpos_r.resize((size_t)std::max<int64_t>(m, 1));
  O.lpos_c.resize((size_t)n);
  for (int64_t p = 0; p < mp; ++p)
    if (ord[(size_t)p] >= 0) O.lpos_r[(size_t)ord[(size_t)p]] = (int32_t)p;
  for (int64_t p = 0; p < n; ++p) O.lpos_c[(size_t)O.pc[(size_t)p]] = (int32_t)p;
  for (int64_t p = 0; p < mp; ++p) L.perm_r.push_back(ord[(size_t)p] >= 0 ? (int32_t)(row0 + ord[(size_t)p]) : -1);
  for (int64_t p = 0; p < np; ++p) L.perm_c.push_back(p < n ? (int32_t)(col0 + O.pc[(size_t)p]) : -1);
  for (int64_t i = 0; i < m; ++i) L.pos_r[(size_t)(row0 + i)] = (int32_t)(O.rbase + O.lpos_r[(size_t)i]);
  for (int64_t j = 0; j < n; ++j) L.pos_c[(size_t)(col0 + j)] = (int32_t)(O.cbase + O.lpos_c[(size_t)j]);
  for (int64_t p = 0; p < mp; ++p) k_eln.push_back(ord[(size_t)p] >= 0 ? rlen[(size_t)ord[(size_t)p]] : 0);
  for (int64_t p = 0; p < np; ++p) t_eln.push_back(p < n ? O.clen[(size_t)O.pc[(size_t)p]] : 0);
  L.mpad += mp;
  L.npad += np;
}

// Host entry lists of one LP for build_sell: internal K row p has the entries
// k_est[p] .. of (k_ecol, k_esrc) in the caller's order, with columns renumbered;
// internal K' row p (a column of K) has the column's entries by increasing row.  col
// holds the LP's nnz column indices, which are entries nnz0 .. of the caller's arrays.
static void host_entries(const LpOrder& O, const int64_t* rp, const int32_t* col, int64_t nnz0, int64_t nnz,
                         std::vector<int64_t>& k_est, std::vector<int32_t>& k_ecol, std::vector<int32_t>& k_esrc,
                         std::vector<int64_t>& t_est, std::vector<int32_t>& t_ecol, std::vector<int32_t>& t_esrc) {
  const int64_t m = O.m, n = O.n;
  k_ecol.resize((size_t)nnz);
  k_esrc.resize((size_t)nnz);
  t_ecol.resize((size_t)nnz);
  t_esrc.resize((size_t)nnz);
  for (int64_t p = 0; p < O.mp; ++p) k_est.push_back(O.ord[(size_t)p] >= 0 ? rp[O.ord[(size_t)p]] : 0);
  for (int64_t k = 0; k < nnz; ++k) {
    k_ecol[(size_t)k] = (int32_t)(O.cbase + O.lpos_c[(size_t)col[k]]);
    k_esrc[(size_t)k] = (int32_t)(nnz0 + k);
  }
  std::vector<int64_t> tp((size_t)n + 1, 0);
  for (int64_t j = 0; j < n; ++j) tp[(size_t)j + 1] = tp[(size_t)j] + O.clen[(size_t)j];
  std::vector<int64_t> fill(tp.begin(), tp.end() - 1);
  for (int64_t i = 0; i < m; ++i)
    for (int64_t k = rp[i]; k < rp[i + 1]; ++k) {
      const int64_t at = fill[(size_t)col[k]]++;
      t_ecol[(size_t)at] = (int32_t)(O.rbase + O.lpos_r[(size_t)i]);
      t_esrc[(size_t)at] = (int32_t)(nnz0 + k);
    }
  for (int64_t p = 0; p < O.np; ++p) t_est.push_back(p < n ? tp[(size_t)O.pc[(size_t)p]] : 0);
}

// Checks c, l, u (n entries) and q (m entries): read in place from host inputs, from a
// host copy of device inputs.
static void check_vectors(pdlp_ctx* h, int64_t n, int64_t m, const double* c_in, const double* q_in,
                          const double* l_in, const double* u_in) {
  std::vector<double> hc, hl, hu, hq;
  const double *c = c_in, *l = l_in, *u = u_in, *q = q_in;
  if (h->p.inputs_on_device) {
    auto fetch = [](std::vector<double>& v, const double* src, int64_t count) {
      v.resize((size_t)count);
      if (count > 0) CK(cudaMemcpy(v.data(), src, sizeof(double) * count, cudaMemcpyDeviceToHost));
      return v.data();
    };
    c = fetch(hc, c_in, n);
    l = fetch(hl, l_in, n);
    u = fetch(hu, u_in, n);
    q = fetch(hq, q_in, m);
  }
  for (int64_t j = 0; j < n; ++j) {
    const double a = l[j], b = u[j];
    if (!std::isfinite(c[j])) invalid("non-finite c");
    if (std::isnan(a) || std::isnan(b) || a == INFINITY || b == -INFINITY || a > b)
      invalid("bounds must satisfy l <= u, l < +inf, u > -inf");
  }
  for (int64_t i = 0; i < m; ++i)
    if (!std::isfinite(q[i])) invalid("non-finite q");
}

// In-place exclusive prefix sums of a[0, n) on the handle's stream (total below 2^31).
static void dev_exclusive_scan(pdlp_ctx* h, int32_t* a, int64_t n) {
  if (n <= 0) return;
  const int64_t tiles = (n + kScanTile - 1) / kScanTile;
  int32_t* sums = dalloc<int32_t>(h, (size_t)tiles);
  k_scan_tiles<<<(unsigned)tiles, kScanThreads, 0, h->s>>>(a, n, sums);
  CKL("k_scan_tiles");
  if (tiles > 1) {
    dev_exclusive_scan(h, sums, tiles);
    k_scan_add<<<grid_for(n), 256, 0, h->s>>>(a, n, sums);
    CKL("k_scan_add");
  }
  CK(cudaStreamSynchronize(h->s));
  dfree(h, sums);
}

// The entry indices 0 .. nnz-1 sorted by their column col[k] in [0, n), equal columns in
// increasing index: the CSC order of a CSR matrix.  ceil(log2 n / 8) stable radix passes
// of 8 bits (at least one).  The result is an allocation of the handle.
static int32_t* dev_csc_order(pdlp_ctx* h, const int32_t* d_col, int64_t nnz, int64_t n) {
  if (nnz == 0) return dalloc<int32_t>(h, 1);
  int bits = 0;
  while (bits < 31 && ((int64_t)1 << bits) < n) ++bits;
  const int passes = std::max(1, (bits + 7) / 8);
  const int64_t tiles = (nnz + kRadixTile - 1) / kRadixTile;
  int32_t* hist = dalloc<int32_t>(h, (size_t)(256 * tiles));
  int32_t* kb[2] = {dalloc<int32_t>(h, (size_t)nnz), dalloc<int32_t>(h, (size_t)nnz)};
  int32_t* vb[2] = {dalloc<int32_t>(h, (size_t)nnz), dalloc<int32_t>(h, (size_t)nnz)};
  const int32_t* kin = d_col;
  const int32_t* vin = nullptr;
  int cur = 0;
  for (int ps = 0; ps < passes; ++ps) {
    k_radix_hist<<<(unsigned)tiles, kRadixThreads, 0, h->s>>>(kin, nnz, 8 * ps, hist, tiles);
    CKL("k_radix_hist");
    dev_exclusive_scan(h, hist, 256 * tiles);
    k_radix_scatter<<<(unsigned)tiles, kRadixThreads, 0, h->s>>>(kin, vin, nnz, 8 * ps, hist, tiles, kb[cur],
                                                                    vb[cur]);
    CKL("k_radix_scatter");
    kin = kb[cur];
    vin = vb[cur];
    cur ^= 1;
  }
  CK(cudaStreamSynchronize(h->s));
  int32_t* out = vb[cur ^ 1];
  for (void* v : {(void*)hist, (void*)kb[0], (void*)kb[1], (void*)vb[cur]}) dfree(h, v);
  return out;
}

// The caller's matrix on the device: count LPs back to back in one global numbering of
// rows and columns, and what the device builder derives from it (DevCsr).
struct DevMatrix {
  int64_t* rp = nullptr;     // global row pointers (M + 1)
  int32_t* col = nullptr;    // global column of each entry
  double* val = nullptr;
  int32_t* tp = nullptr;     // entries per global column, then column starts (N + 1)
  int32_t* csc = nullptr;
  int32_t* rowof = nullptr;
  int32_t* kpad = nullptr;
  int32_t* tpad = nullptr;
  DevCsr csr() const { return DevCsr{rp, col, val, tp, csc, rowof, kpad, tpad}; }
};

// Copies the matrix of count = ent0.size() - 1 LPs to the device (LP b: entries
// ent0[b] .. ent0[b+1] - 1 with local columns, its columns col0[b] .. col0[b+1] - 1 of
// the global numbering; grp: global row pointers, host), checks the entries there and
// counts the entries of each global column (clen, host).  Throws on a bad entry.
static DevMatrix upload_matrix(pdlp_ctx* h, int64_t M, int64_t N, int64_t nnz, const int64_t* grp,
                               const std::vector<int64_t>& ent0, const std::vector<int64_t>& col0,
                               const int32_t* col_in, const double* val_in, std::vector<int32_t>& clen) {
  DevMatrix A;
  const cudaMemcpyKind kind = h->p.inputs_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  A.rp = dalloc<int64_t>(h, (size_t)M + 1);
  A.col = dalloc<int32_t>(h, (size_t)nnz);
  A.val = dalloc<double>(h, (size_t)nnz);
  A.tp = dalloc<int32_t>(h, (size_t)N + 1);
  int64_t* d_ent0 = upload(h, ent0);
  int64_t* d_col0 = upload(h, col0);
  int* d_flags = dalloc<int>(h, 1);
  CK(cudaMemcpyAsync(A.rp, grp, sizeof(int64_t) * (M + 1), cudaMemcpyHostToDevice, h->s));
  if (nnz > 0) {
    CK(cudaMemcpyAsync(A.col, col_in, sizeof(int32_t) * nnz, kind, h->s));
    CK(cudaMemcpyAsync(A.val, val_in, sizeof(double) * nnz, kind, h->s));
  }
  k_check_count<<<grid_for(nnz), 256, 0, h->s>>>(A.col, A.val, nnz, d_ent0, d_col0, (int64_t)ent0.size() - 1, A.tp,
                                                 d_flags);
  CKL("k_check_count");
  int flags = 0;
  clen.resize((size_t)N);
  CK(cudaMemcpyAsync(&flags, d_flags, sizeof(int), cudaMemcpyDeviceToHost, h->s));
  CK(cudaMemcpyAsync(clen.data(), A.tp, sizeof(int32_t) * N, cudaMemcpyDeviceToHost, h->s));
  CK(cudaStreamSynchronize(h->s));
  for (void* v : {(void*)d_ent0, (void*)d_col0, (void*)d_flags}) dfree(h, v);
  if (flags & kBadVal) invalid("non-finite matrix value");
  if (flags & kBadCol) invalid("column index out of range");
  return A;
}

// What K' needs: column starts (in place of the counts), the CSC order and the row of
// each entry; and the padding column of each chunk of both layouts.
static void finish_matrix(pdlp_ctx* h, DevMatrix& A, int64_t M, int64_t N, int64_t nnz,
                          const std::vector<int32_t>& kpad, const std::vector<int32_t>& tpad) {
  dev_exclusive_scan(h, A.tp, N + 1);
  A.csc = dev_csc_order(h, A.col, nnz, N);
  A.rowof = dalloc<int32_t>(h, (size_t)nnz);
  k_row_of<<<grid_for(M * 32), 256, 0, h->s>>>(A.rp, M, A.rowof);
  CKL("k_row_of");
  A.kpad = upload(h, kpad);
  A.tpad = upload(h, tpad);
}

static void free_matrix(pdlp_ctx* h, DevMatrix& A) {
  CK(cudaStreamSynchronize(h->s));
  for (void* v : {(void*)A.rp, (void*)A.col, (void*)A.val, (void*)A.tp, (void*)A.csc, (void*)A.rowof, (void*)A.kpad,
                  (void*)A.tpad})
    if (v) dfree(h, v);
  A = DevMatrix{};
}

// Upload of the layouts and values, problem vectors in internal order, unscaled norms,
// scaling and the scaled problem vectors: everything both handle kinds share.
static void device_setup_common(pdlp_ctx* h, Layout& Lo, const DevCsr* dc, const std::vector<double>* hval,
                                const double* c_in, const double* q_in, const double* l_in, const double* u_in);
static void estimate_step_and_weight(pdlp_ctx* h);
static void setup_mixed(pdlp_ctx* h);
static void init_batch_launch(pdlp_ctx* h, const Layout& Lo, int64_t npad_max, int64_t mpad_max);
static int batch_solve_impl(pdlp_ctx* h, const pdlp_params& sp, const double* x0, const double* y0,
                            const double* omega0, pdlp_result* res, double* x_out, double* y_out, bool single,
                            double omega0_single);

static void setup_impl(pdlp_ctx* h, int64_t m, int64_t n, int64_t m1, const int64_t* row_ptr_in,
                       const int32_t* col_in, const double* val_in, const double* c_in,
                       const double* q_in, const double* l_in, const double* u_in) {
  const pdlp_params& P = h->p;
  if (m < 0 || n < 1 || m1 < 0 || m1 > m) invalid("sizes must satisfy m >= 0, n >= 1, 0 <= m1 <= m");
  if (m >= (int64_t)1 << 31 || n >= (int64_t)1 << 31) invalid("m and n must be below 2^31");
  check_params(P);
  if (!row_ptr_in || !c_in || !l_in || !u_in || (m > 0 && !q_in)) invalid("null input array");
  init_handle_resources(h);
  using clk = std::chrono::steady_clock;
  auto ms_since = [](clk::time_point a) { return std::chrono::duration<double, std::milli>(clk::now() - a).count(); };
  auto tp = clk::now();
  h->m = m;
  h->n = n;
  h->m1 = m1;
  const bool dev_in = P.inputs_on_device != 0;
  // device inputs are read on this handle's stream and by copies to the host: the
  // caller's stream must have finished writing them
  if (dev_in && P.stream) CK(cudaStreamSynchronize((cudaStream_t)P.stream));
  // row pointers on the host: the caller's array, or a copy of the device array
  std::vector<int64_t> rp_copy;
  const int64_t* rp = row_ptr_in;
  if (dev_in) {
    rp_copy.resize((size_t)m + 1);
    CK(cudaMemcpy(rp_copy.data(), row_ptr_in, sizeof(int64_t) * (m + 1), cudaMemcpyDeviceToHost));
    rp = rp_copy.data();
  }
  if (rp[m] < 0 || rp[m] >= ((int64_t)1 << 31)) invalid("nnz must be in [0, 2^31)");
  if (rp[0] != 0) invalid("row_ptr[0] must be 0");
  for (int64_t i = 0; i < m; ++i)
    if (rp[i + 1] < rp[i]) invalid("row_ptr must be nondecreasing");
  const int64_t nnz = rp[m];
  h->nnz = nnz;
  if (nnz > 0 && (!col_in || !val_in)) invalid("null col_idx/val with nnz > 0");
  check_vectors(h, n, m, c_in, q_in, l_in, u_in);

  Layout Lo;
  Lo.pos_r.assign((size_t)m, 0);
  Lo.pos_c.assign((size_t)n, 0);
  std::vector<int32_t> k_eln, t_eln;
  std::vector<uint8_t> k_wide;
  int64_t m1i = m1;
  LpOrder O;
  if (P.host_layout) {
    // the reference builder: entries copied, checked and laid out on the host
    HostLP H;
    fetch_matrix(h, row_ptr_in, col_in, val_in, H, m + 1);
    check_csr(H, 0, m, n, 0);
    std::vector<int32_t> clen((size_t)n, 0);
    for (int64_t k = 0; k < nnz; ++k) clen[(size_t)H.col[(size_t)k]]++;
    h->setup_ms[0] = ms_since(tp);
    tp = clk::now();
    order_lp(Lo, O, rp, std::move(clen), m, n, m1, 0, 0, k_eln, t_eln, true, &k_wide, &m1i);
    std::vector<int64_t> k_est, t_est;
    std::vector<int32_t> k_ecol, k_esrc, t_ecol, t_esrc;
    host_entries(O, rp, H.col.data(), 0, nnz, k_est, k_ecol, k_esrc, t_est, t_ecol, t_esrc);
    Lo.SK = build_sell(Lo.mpad, k_est, k_eln, k_ecol, k_esrc, 0, &k_wide);
    Lo.SKt = build_sell(Lo.npad, t_est, t_eln, t_ecol, t_esrc);
    h->m1_int = m1i;
    h->setup_ms[1] = ms_since(tp);
    tp = clk::now();
    device_setup_common(h, Lo, nullptr, &H.val, c_in, q_in, l_in, u_in);
  } else {
    // the matrix goes to the device as it is: entries checked and columns counted there;
    // the host orders rows and columns (O(m + n)); the device fills the layouts
    std::vector<int32_t> clen;
    DevMatrix A = upload_matrix(h, m, n, nnz, rp, {0, nnz}, {0, n}, col_in, val_in, clen);
    h->setup_ms[0] = ms_since(tp);
    tp = clk::now();
    order_lp(Lo, O, rp, std::move(clen), m, n, m1, 0, 0, k_eln, t_eln, true, &k_wide, &m1i);
    h->m1_int = m1i;
    Lo.SK = sell_shape(Lo.mpad, k_eln, &k_wide);
    Lo.SKt = sell_shape(Lo.npad, t_eln);
    h->setup_ms[1] = ms_since(tp);
    tp = clk::now();
    finish_matrix(h, A, m, n, nnz, std::vector<int32_t>((size_t)Lo.SK.nchunks, 0),
                  std::vector<int32_t>((size_t)Lo.SKt.nchunks, 0));
    const DevCsr dc = A.csr();
    device_setup_common(h, Lo, &dc, nullptr, c_in, q_in, l_in, u_in);
    free_matrix(h, A);
  }
  CK(cudaStreamSynchronize(h->s));
  h->setup_ms[2] = ms_since(tp);
  tp = clk::now();

  // ---- SpMV schedule per layout: explicit parameters, or timed candidates for large K
  const bool auto_tile = P.tile_slots == 0 && P.tile_chunks == 0 && P.spmv_batch == 0;
  const int stage_fixed = P.spmv_stage - 1;   // -1: chosen by the autotuner (plain below its size)
  if (auto_tile && h->nnz >= kAutotuneMinNnz) {
    autotune(h, h->Kt, Lo.SKt, true, stage_fixed);
    autotune(h, h->K, Lo.SK, false, stage_fixed);
  } else if (stage_fixed > 0) {
    h->K.staged = h->Kt.staged = stage_fixed;
  }
  h->setup_ms[3] = ms_since(tp);
  tp = clk::now();
  estimate_step_and_weight(h);
  if (P.precision == PDLP_MIXED) setup_mixed(h);
  else if (P.precision != PDLP_FP64) invalid("precision must be PDLP_FP64 or PDLP_MIXED");
  // persistent engine for a small LP: the batched kernel on this handle's own layout and
  // vectors (same internal order when no row is wide), x and y in shared memory
  h->small_engine = false;
  if (P.engine != 1 && P.precision == PDLP_FP64 && h->K.nwide == 0 && h->nnz <= kSmallEngineNnz) {
    LpDesc D{};
    D.m = (int32_t)m;
    D.n = (int32_t)n;
    D.m1 = (int32_t)h->m1_int;
    D.kc0 = 0;
    D.kc1 = (int32_t)Lo.SK.nchunks;
    D.tc0 = 0;
    D.tc1 = (int32_t)Lo.SKt.nchunks;
    D.r0 = 0;
    D.c0 = 0;
    D.mpad = (int32_t)Lo.mpad;
    D.npad = (int32_t)Lo.npad;
    h->hdesc.assign(1, D);
    h->count = 1;
    try {
      init_batch_launch(h, Lo, Lo.npad, Lo.mpad);
      h->small_engine = !h->batch_glob;
    } catch (const std::string&) {
      h->small_engine = false;   // the kernels launched per iteration remain
    }
  }
  if (P.engine == 2 && !h->small_engine) invalid("engine 2: this LP does not fit the persistent engine");
  CK(cudaStreamSynchronize(h->s));
  h->setup_ms[4] = ms_since(tp);
}

// FP32 iterates and problem vectors; FP32 copies of the scaled matrix values, or, for a
// K with +-1 entries, sign-bit column words with the unscaled problem data and D_c^2,
// D_r^2 (the iterations then run in the unscaled variables).
static void setup_mixed(pdlp_ctx* h) {
  const int64_t np = h->npad, mp = h->mpad;
  // the iterates get 32 more entries: with sign-bit storage entry np (mp) stays zero and
  // is what the padding slots of K (K') point at
  for (float** v : {&h->x32, &h->sx32, &h->c32, &h->l32, &h->u32}) *v = dalloc<float>(h, np + 32);
  for (float** v : {&h->y32, &h->sy32, &h->kxp32, &h->q32}) *v = dalloc<float>(h, mp + 32);
  if (h->unit_ok) {
    h->K.ucol = dalloc<int32_t>(h, (size_t)h->K.slots * 32);
    k_unit_cols<<<grid_for(h->K.slots * 32), 256, 0, h->s>>>(h->K.ucol, h->K.col, h->K.val, h->K.slots * 32,
                                                             (int32_t)np);
    h->Kt.ucol = dalloc<int32_t>(h, (size_t)h->Kt.slots * 32);
    k_unit_cols<<<grid_for(h->Kt.slots * 32), 256, 0, h->s>>>(h->Kt.ucol, h->Kt.col, h->Kt.val, h->Kt.slots * 32,
                                                              (int32_t)mp);
    h->dc2 = dalloc<float>(h, np);
    h->dr2 = dalloc<float>(h, mp);
    k_unit_vectors<<<grid_for(std::max(np, mp)), 256, 0, h->s>>>(h->c32, h->l32, h->u32, h->dc2, h->c, h->l, h->u,
                                                                h->Dc, h->invDc, np, h->q32, h->dr2, h->q, h->Dr,
                                                                h->invDr, mp);
    h->mixed_values = 2;
  } else {
    for (DevSell* S : {&h->K, &h->Kt}) {
      S->val32 = dalloc<float>(h, (size_t)S->slots * 32);
      k_to_float<<<grid_for(S->slots * 32), 256, 0, h->s>>>(S->val32, S->val, S->slots * 32);
    }
    k_to_float<<<grid_for(np), 256, 0, h->s>>>(h->c32, h->c, np);
    k_to_float<<<grid_for(np), 256, 0, h->s>>>(h->l32, h->l, np);
    k_to_float<<<grid_for(np), 256, 0, h->s>>>(h->u32, h->u, np);
    k_to_float<<<grid_for(mp), 256, 0, h->s>>>(h->q32, h->q, mp);
    h->mixed_values = 1;
  }
  CKL("mixed setup");
  CK(cudaStreamSynchronize(h->s));
}

static void device_setup_common(pdlp_ctx* h, Layout& Lo, const DevCsr* dc, const std::vector<double>* hval,
                                const double* c_in, const double* q_in, const double* l_in, const double* u_in) {
  const pdlp_params& P = h->p;
  const int64_t m = h->m, n = h->n;
  h->mpad = Lo.mpad;
  h->npad = Lo.npad;
  const int32_t tile = P.tile_slots > 0 ? P.tile_slots : 64;
  const int32_t tchunks = P.tile_chunks > 0 ? std::min(P.tile_chunks, 32) : 4;
  TaskPlan PK = plan_tasks(Lo.SK, tile, tchunks), PKt = plan_tasks(Lo.SKt, tile, tchunks);
  h->K.tile = h->Kt.tile = tile;
  h->K.tchunks = h->Kt.tchunks = tchunks;
  h->K.batch = h->Kt.batch = (P.spmv_batch == 4) ? 4 : 8;

  h->perm_r = upload(h, Lo.perm_r);
  h->pos_r = upload(h, Lo.pos_r);
  h->perm_c = upload(h, Lo.perm_c);
  h->pos_c = upload(h, Lo.pos_c);
  if (dc) {
    fill_device_sell(h, h->K, Lo.SK, PK, *dc, false);
    fill_device_sell(h, h->Kt, Lo.SKt, PKt, *dc, true);
  } else {
    double* d_val = upload(h, *hval);
    build_device_sell(h, h->K, Lo.SK, PK, d_val);
    build_device_sell(h, h->Kt, Lo.SKt, PKt, d_val);
    dfree(h, d_val);
  }
  // mixed precision: are the (unscaled) entries all +-1?  Then the FP32 products keep
  // signs instead of values (mixed_values); the gathered vectors' zero entry np (mp)
  // must be a valid 31-bit index
  h->unit_ok = false;
  if (!h->is_batch && P.precision == PDLP_MIXED && P.mixed_values != 1) {
    unsigned long long* cnt = dalloc<unsigned long long>(h, 1);
    k_count_nonunit<<<grid_for(h->K.slots * 32), 256, 0, h->s>>>(h->K.val, h->K.slots * 32, cnt);
    CKL("entry check");
    unsigned long long bad = 0;
    CK(cudaMemcpyAsync(&bad, cnt, sizeof(bad), cudaMemcpyDeviceToHost, h->s));
    CK(cudaStreamSynchronize(h->s));
    dfree(h, cnt);
    const int64_t lim = ((int64_t)1 << 31) - 64;
    h->unit_ok = bad == 0 && Lo.npad < lim && Lo.mpad < lim;
    if (P.mixed_values == 2 && !h->unit_ok)
      invalid("mixed_values = 2 needs every entry of K to be +1 or -1 (and fewer than 2^31 - 64 rows and columns)");
  }

  const int64_t mp = h->mpad, np = h->npad;
  h->c = dalloc<double>(h, np);
  h->l = dalloc<double>(h, np);
  h->u = dalloc<double>(h, np);
  h->q = dalloc<double>(h, mp);
  h->Dr = dalloc<double>(h, mp);
  h->Dc = dalloc<double>(h, np);
  h->invDr = dalloc<double>(h, mp);
  h->invDc = dalloc<double>(h, np);
  for (double** v : {&h->x, &h->sx, &h->xa, &h->g_c, &h->g_a, &h->tn}) *v = dalloc<double>(h, np);
  for (double** v : {&h->y, &h->sy, &h->ya, &h->kxp, &h->kx_a, &h->tm}) *v = dalloc<double>(h, mp);
  h->stage_n = dalloc<double>(h, n);
  h->stage_m = dalloc<double>(h, std::max<int64_t>(m, 1));
  h->red_blocks = grid_for(std::max(np, mp));
  h->red_part = dalloc<double>(h, h->red_blocks);
  h->red_out = dalloc<double>(h, 1);
  h->nb_rows = std::min<int>(296, std::max<int>(1, (int)((m + 255) / 256)));
  h->nb_cols = std::min<int>(296, std::max<int>(1, (int)((n + 255) / 256)));
  h->part = dalloc<double>(h, (size_t)(h->nb_rows + h->nb_cols) * NQ);
  h->st = dalloc<DevState>(h, 1);
  h->st_tmp = dalloc<DevState>(h, 1);
  h->dp = dalloc<DevParams>(h, 1);
  h->log_cap = P.log_capacity > 0 ? P.log_capacity : 1;
  h->log = dalloc<CheckRecord>(h, (size_t)h->log_cap);
  h->restarts = dalloc<long long>(h, (size_t)h->restart_cap);

  // ---- problem vectors in internal order; unscaled norms for the termination tests
  copy_in(h, h->stage_n, c_in, n);
  h->cnorm = norm2_host(h, h->stage_n, n);
  k_permute_in<<<grid_for(np), 256, 0, h->s>>>(h->c, h->stage_n, h->perm_c, nullptr, np, 0.0);
  copy_in(h, h->stage_n, l_in, n);
  k_permute_in<<<grid_for(np), 256, 0, h->s>>>(h->l, h->stage_n, h->perm_c, nullptr, np, 0.0);
  copy_in(h, h->stage_n, u_in, n);
  k_permute_in<<<grid_for(np), 256, 0, h->s>>>(h->u, h->stage_n, h->perm_c, nullptr, np, 0.0);
  if (m > 0) {
    copy_in(h, h->stage_m, q_in, m);
    h->qnorm = norm2_host(h, h->stage_m, m);
  }
  k_permute_in<<<grid_for(mp), 256, 0, h->s>>>(h->q, h->stage_m, h->perm_r, nullptr, mp, 0.0);
  k_fill<<<grid_for(mp), 256, 0, h->s>>>(h->Dr, 1.0, mp);
  k_fill<<<grid_for(np), 256, 0, h->s>>>(h->Dc, 1.0, np);
  CKL("setup vectors");

  // ---- scaling: ruiz_iters Ruiz passes, then one Pock-Chambolle pass
  if (P.scaling) {
    for (int pass = 0; pass <= P.ruiz_iters; ++pass) {
      const bool pc = pass == P.ruiz_iters;
      if (pc) {
        launch_rows<OpSumAbs>(h, h->K, nullptr, EpiStore{h->tm, 0, 1.0}, nullptr);
        launch_rows<OpSumAbs>(h, h->Kt, nullptr, EpiStore{h->tn, 0, 1.0}, nullptr);
      } else {
        launch_rows<OpMaxAbs>(h, h->K, nullptr, EpiStore{h->tm, 0, 1.0}, nullptr);
        launch_rows<OpMaxAbs>(h, h->Kt, nullptr, EpiStore{h->tn, 0, 1.0}, nullptr);
      }
      k_scale_factor<<<grid_for(mp), 256, 0, h->s>>>(h->tm, h->Dr, h->tm, mp);
      k_scale_factor<<<grid_for(np), 256, 0, h->s>>>(h->tn, h->Dc, h->tn, np);
      k_scale_sell2<<<grid_for(h->K.slots * 32), 256, 0, h->s>>>(h->K.val, h->K.col, h->K.chunk_ptr, h->K.nchunks,
                                                                h->K.slots * 32, h->tm, h->tn, 0, h->K.wide);
      k_scale_sell2<<<grid_for(h->Kt.slots * 32), 256, 0, h->s>>>(h->Kt.val, h->Kt.col, h->Kt.chunk_ptr,
                                                                 h->Kt.nchunks, h->Kt.slots * 32, h->tm, h->tn, 1,
                                                                 h->Kt.wide);
      CKL("scaling pass");
    }
  }
  k_scale_cols<<<grid_for(np), 256, 0, h->s>>>(h->c, h->l, h->u, h->invDc, h->Dc, np);
  k_scale_rows<<<grid_for(mp), 256, 0, h->s>>>(h->q, h->invDr, h->Dr, mp);
  CKL("scale vectors");

  CK(cudaStreamSynchronize(h->s));
}

// ||K||_2 by power iteration on K'K (v0 = 1/sqrt(n)) -> eta; omega0 = ||c||/||q||.
// Power-iteration step size eta = step_scale / ||K||_2 (Section 2, constant step).
static void power_step(pdlp_ctx* h) {
  const pdlp_params& P = h->p;
  const int64_t m = h->m, n = h->n, mp = h->mpad, np = h->npad;
  if (P.eta > 0.0) {
    h->eta = P.eta;
  } else {
    double* a = h->tn;
    double* w = h->g_a;
    k_fill<<<grid_for(np), 256, 0, h->s>>>(a, 0.0, np);
    k_fill<<<grid_for(n), 256, 0, h->s>>>(a, 1.0 / std::sqrt((double)n), n);
    for (int it = 0; it < P.power_iters; ++it) {
      launch_rows<OpSpmv>(h, h->K, a, EpiStore{h->tm, 0, 1.0}, nullptr);
      launch_rows<OpSpmv>(h, h->Kt, h->tm, EpiStore{w, 0, 1.0}, nullptr);
      norm2_dev(h, w, np);
      k_div_into<<<grid_for(np), 256, 0, h->s>>>(a, w, h->red_out, np);
    }
    launch_rows<OpSpmv>(h, h->K, a, EpiStore{h->tm, 0, 1.0}, nullptr);
    CKL("power iteration");
    h->normK = m > 0 ? norm2_host(h, h->tm, mp) : 0.0;
    h->eta = h->normK > 0.0 ? P.step_scale / h->normK : 1.0;
  }
  h->power_done = true;
}

static void estimate_step_and_weight(pdlp_ctx* h) {
  const pdlp_params& P = h->p;
  const int64_t mp = h->mpad, np = h->npad;
  // the power iteration is skipped for a handle set up for the adaptive rule (it runs
  // on the first constant-step solve instead)
  if (P.step_rule != 1) power_step(h);
  {
    // first step of the adaptive rule: 1 / max |K_ij| (1 when K = 0)
    unsigned long long* mx = reinterpret_cast<unsigned long long*>(h->red_out);
    CK(cudaMemsetAsync(mx, 0, sizeof(unsigned long long), h->s));
    const int64_t len = h->K.slots * 32;
    if (len > 0) k_absmax<<<std::max(1, std::min(grid_for(len), 1184)), 256, 0, h->s>>>(h->K.val, len, mx);
    unsigned long long bits = 0;
    CK(cudaMemcpyAsync(&bits, mx, sizeof(bits), cudaMemcpyDeviceToHost, h->s));
    CK(cudaStreamSynchronize(h->s));
    double v;
    std::memcpy(&v, &bits, sizeof(v));
    h->eta_adapt0 = v > 0.0 ? 1.0 / v : 1.0;
  }
  {
    const double cn = norm2_host(h, h->c, np), qn = norm2_host(h, h->q, mp);
    h->omega0 = (cn > 1e-10 && qn > 1e-10) ? cn / qn : 1.0;
  }
  CK(cudaStreamSynchronize(h->s));
}

static void ensure_graphs(pdlp_ctx* h, int full, int rem) {
  if (h->g_full_len != full) {
    if (h->g_full) cudaGraphExecDestroy(h->g_full);
    h->g_full = nullptr;
    h->g_full_len = -1;
    if (full > 0) {
      h->g_full = capture_interval(h, full);
      h->g_full_len = full;
    }
  }
  if (rem > 0 && h->g_rem_len != rem) {
    if (h->g_rem) cudaGraphExecDestroy(h->g_rem);
    h->g_rem = nullptr;
    h->g_rem_len = -1;
    h->g_rem = capture_interval(h, rem);
    h->g_rem_len = rem;
  }
}

static void ensure_graphs_mixed(pdlp_ctx* h, int full, int rem) {
  if (h->gm_full_len != full) {
    if (h->gm_full) cudaGraphExecDestroy(h->gm_full);
    h->gm_full = nullptr;
    h->gm_full_len = -1;
    if (full > 0) {
      h->gm_full = capture_interval(h, full, kModeMixed);
      h->gm_full_len = full;
    }
  }
  if (rem > 0 && h->gm_rem_len != rem) {
    if (h->gm_rem) cudaGraphExecDestroy(h->gm_rem);
    h->gm_rem = nullptr;
    h->gm_rem_len = -1;
    h->gm_rem = capture_interval(h, rem, kModeMixed);
    h->gm_rem_len = rem;
  }
}

static void ensure_graphs_adaptive(pdlp_ctx* h, int full, int rem) {
  if (h->ga_full_len != full) {
    if (h->ga_full) cudaGraphExecDestroy(h->ga_full);
    h->ga_full = nullptr;
    h->ga_full_len = -1;
    if (full > 0) {
      h->ga_full = capture_interval(h, full, kModeAdaptive);
      h->ga_full_len = full;
    }
  }
  if (rem > 0 && h->ga_rem_len != rem) {
    if (h->ga_rem) cudaGraphExecDestroy(h->ga_rem);
    h->ga_rem = nullptr;
    h->ga_rem_len = -1;
    h->ga_rem = capture_interval(h, rem, kModeAdaptive);
    h->ga_rem_len = rem;
  }
}

// Buffers of the adaptive rule, allocated on its first use.
static void ensure_adaptive_buffers(pdlp_ctx* h) {
  if (h->xb) return;
  h->xb = dalloc<double>(h, h->npad);
  h->yb = dalloc<double>(h, h->mpad);
  h->kxb = dalloc<double>(h, h->mpad);
  h->part_x = dalloc<double>(h, std::max<int64_t>(1, h->Kt.ntasks));
  h->part_y = dalloc<double>(h, 2 * std::max<int64_t>(1, h->K.ntasks));
  h->part_s = dalloc<double>(h, 3 * kStepParts);
}

// Continuing a solve (pdlp_solve_resume): the handle's device state is the one its last
// solve ended with, or one loaded by load_state; the check that ended it is repeated as
// an ordinary check, then the intervals go on from its iteration count.
__global__ void k_resume_state(DevState* st, int reject_cap) {
  st->done = 0;
  st->status = 0;
  st->final_force = 0;
  if (st->ncheck > 0) st->ncheck -= 1;
  st->reject_cap = reject_cap;
}

static int solve_impl(pdlp_ctx* h, const pdlp_params& sp, const double* x0, const double* y0, double omega0,
                      pdlp_result* res, double* x_out, double* y_out, bool resume = false) {
  if (sp.check_every < 1 || sp.max_iter < 0 || !(sp.tol >= 0.0)) invalid("bad solve parameters");
  if (sp.step_rule < 0 || sp.step_rule > 1) invalid("step_rule must be 0 or 1");
  if (sp.adaptive_reject_cap < 0) invalid("adaptive_reject_cap must be >= 0");
  const bool adaptive = sp.step_rule == 1;
  if (adaptive && h->p.precision == PDLP_MIXED) invalid("the adaptive step rule runs in FP64 only");
  if (adaptive) ensure_adaptive_buffers(h);
  if (!adaptive && !h->power_done) power_step(h);
  if (sp.engine < 0 || sp.engine > 2) invalid("engine must be 0, 1 or 2");
  {
    // the persistent engine: automatic for a small LP with the constant step in FP64 and
    // no time limit, or when asked for
    const bool can = h->small_engine && !adaptive && h->p.precision == PDLP_FP64 && !resume;
    if (sp.engine == 2 && !can) invalid("engine 2 needs a small FP64 LP with the constant step (and no resume)");
    if (can && (sp.engine == 2 || (sp.engine == 0 && !std::isfinite(sp.time_limit_s)))) {
      pdlp_params bp = sp;
      bp.resident = 0;
      bp.batch_tail_iters = 0;
      return batch_solve_impl(h, bp, x0, y0, nullptr, res, x_out, y_out, true, omega0);
    }
  }
  auto t_start = std::chrono::steady_clock::now();
  const int64_t n = h->n, m = h->m, np = h->npad, mp = h->mpad;
  int64_t launches = 0;
  h->fp32_iters = 0;

  // device parameters of the decision kernel
  h->dp_host.tol = sp.tol;
  h->dp_host.beta_suff = sp.beta_suff;
  h->dp_host.beta_nec = sp.beta_nec;
  h->dp_host.beta_art = sp.beta_art;
  h->dp_host.theta = sp.omega_theta;
  h->dp_host.qnorm = h->qnorm;
  h->dp_host.cnorm = h->cnorm;
  h->dp_host.max_iter = sp.max_iter;
  h->dp_host.log_cap = h->log_cap;
  h->dp_host.restart_cap = h->restart_cap;
  CK(cudaMemcpyAsync(h->dp, &h->dp_host, sizeof(DevParams), cudaMemcpyHostToDevice, h->s));

  int64_t k0 = 0;   // iterations already done (resume)
  const bool mixed = h->p.precision == PDLP_MIXED;
  if (resume) {
    if (mixed) invalid("resume: FP64 handles only");
    CK(cudaEventRecord(h->ev_t0, h->s));
    k_resume_state<<<1, 1, 0, h->s>>>(h->st, sp.adaptive_reject_cap);
    DevState cur{};
    CK(cudaMemcpyAsync(&cur, h->st, sizeof(DevState), cudaMemcpyDeviceToHost, h->s));
    CK(cudaStreamSynchronize(h->s));
    k0 = cur.k;
    enqueue_check(h, 0, k0 >= sp.max_iter ? 1 : 0, adaptive);
    launches += adaptive ? 10 : 9;
    CKL("resume check");
  } else {
  // initial point (Section 2: x in X, y in Y), anchor z^{0,0} = (x0, y0)
  const double* xs = nullptr;
  const double* ys = nullptr;
  if (x0) {
    copy_in(h, h->stage_n, x0, n);
    k_permute_in<<<grid_for(np), 256, 0, h->s>>>(h->tn, h->stage_n, h->perm_c, h->Dc, np, 0.0);
    xs = h->tn;
    launches++;
  }
  if (y0 && m > 0) {
    copy_in(h, h->stage_m, y0, m);
    k_permute_in<<<grid_for(mp), 256, 0, h->s>>>(h->tm, h->stage_m, h->perm_r, h->Dr, mp, 0.0);
    ys = h->tm;
    launches++;
  }
  CK(cudaEventRecord(h->ev_t0, h->s));
  k_init_point<<<grid_for(std::max(np, mp)), 256, 0, h->s>>>(h->x, xs, h->l, h->u, n, np, h->y, ys, m, mp,
                                                              (int)h->m1_int);
  const double w0 = omega0 > 0.0 ? omega0 : h->omega0;
  DevState& s0 = h->st_init;
  std::memset(&s0, 0, sizeof(s0));
  const double eta0 = adaptive ? (sp.eta > 0.0 ? sp.eta : h->eta_adapt0) : h->eta;
  s0.eta = eta0;
  s0.omega = w0;
  s0.tau = eta0 / w0;
  s0.sigma = eta0 * w0;
  s0.kkt_prev = std::numeric_limits<double>::infinity();
  s0.reject_cap = sp.adaptive_reject_cap;
  CK(cudaMemcpyAsync(h->st, &s0, sizeof(DevState), cudaMemcpyHostToDevice, h->s));
  launch_rows<OpSpmv>(h, h->K, h->x, EpiStore{h->kxp, 0, 1.0}, h->st);
  launch_rows<OpSpmv>(h, h->Kt, h->y, EpiStore{h->g_c, 0, 1.0}, h->st);
  k_copy<<<grid_for(np), 256, 0, h->s>>>(h->xa, h->x, np);
  k_copy<<<grid_for(mp), 256, 0, h->s>>>(h->ya, h->y, mp);
  k_fill<<<grid_for(np), 256, 0, h->s>>>(h->sx, 0.0, np);
  k_fill<<<grid_for(mp), 256, 0, h->s>>>(h->sy, 0.0, mp);
  k_kkt_partials<<<h->nb_rows + h->nb_cols, 256, 0, h->s>>>(kkt_inputs(h), h->st, h->part);
  k_decide<<<1, 256, 0, h->s>>>(h->part, h->nb_rows, h->nb_cols, h->st, h->dp, h->log, h->restarts, 1, 0);
  launches += 9;
  if (mixed) {
    CK(cudaMemsetAsync(h->sx32, 0, sizeof(float) * np, h->s));
    CK(cudaMemsetAsync(h->sy32, 0, sizeof(float) * mp, h->s));
    k_mixed_to32<<<grid_for(std::max(np, mp)), 256, 0, h->s>>>(h->x32, h->x, np, h->y32, h->y, h->kxp32, h->kxp, mp,
                                                                 h->st, mixed_scale(h));
    launches += 1;
  }
  CKL("solve init");
  }

  const int L = sp.check_every;
  const int64_t todo = std::max<int64_t>(0, sp.max_iter - k0);
  const int64_t nfull = todo / L;
  const int rem = (int)(todo % L);
  const int64_t nint = nfull + (rem > 0 ? 1 : 0);
  bool timed_out = false;
  DevState fin{};
  if (nint == 0 && resume) {
    // the repeated check was the last one
  } else if (nint == 0) {
    enqueue_check(h, 0, 1, adaptive);
    launches += adaptive ? 9 : 8;
    CKL("final check");
  } else {
    if (adaptive) ensure_graphs_adaptive(h, nfull > 0 ? L : 0, rem);
    else ensure_graphs(h, nfull > 0 ? L : 0, rem);
    if (mixed) ensure_graphs_mixed(h, nfull > 0 ? L : 0, rem);
    // mixed precision: FP32 intervals until the FP64-measured relative error reaches
    // the switch tolerance or stops improving, then FP64 intervals (refinement)
    bool phase32 = mixed;
    const double switch_tol = sp.mixed_switch_tol > 0.0 ? sp.mixed_switch_tol : std::max(sp.tol, 1e-5);
    double best_err = INFINITY;
    int since_best = 0;
    int64_t issued = 0, read = 0, issued_k = 0;
    std::vector<std::pair<int64_t, int>> fp32_intervals;   // (first iteration, length) of FP32 intervals
    bool done = false;
    while (!done && read < nint) {
      while (issued < nint && issued - read < kLookahead) {
        const bool fullint = issued < nfull;
        cudaGraphExec_t g = phase32    ? (fullint ? h->gm_full : h->gm_rem)
                            : adaptive ? (fullint ? h->ga_full : h->ga_rem)
                                       : (fullint ? h->g_full : h->g_rem);
        const int len = fullint ? L : rem;
        CK(cudaGraphLaunch(g, h->s));
        launches += adaptive ? 5 * len + 9 : 2 * len + (phase32 ? 12 : 8);
        if (phase32) fp32_intervals.emplace_back(issued_k, len);
        issued_k += len;
        const int slot = (int)(issued % kRing);
        CK(cudaMemcpyAsync(h->st_host + slot, h->st, sizeof(DevState), cudaMemcpyDeviceToHost, h->s));
        CK(cudaEventRecord(h->ev_ring[slot], h->s));
        ++issued;
      }
      const int slot = (int)(read % kRing);
      CK(cudaEventSynchronize(h->ev_ring[slot]));
      done = h->st_host[slot].done != 0;
      ++read;
      if (phase32 && !done) {
        const double e = h->st_host[slot].last_err;
        if (e < 0.9 * best_err) {
          best_err = e;
          since_best = 0;
        } else {
          ++since_best;
        }
        if (e <= switch_tol || since_best >= 16) phase32 = false;
      }
      if (!done && std::isfinite(sp.time_limit_s)) {
        double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
        if (el > sp.time_limit_s) {
          timed_out = true;
          break;
        }
      }
    }
    CK(cudaStreamSynchronize(h->s));
    CK(cudaMemcpy(&fin, h->st, sizeof(DevState), cudaMemcpyDeviceToHost));
    // intervals queued after the solve finished did nothing
    for (const auto& iv : fp32_intervals) h->fp32_iters += std::max<int64_t>(0, std::min<int64_t>(iv.second, fin.k - iv.first));
    if (!fin.done) {
      // time limit: one more check that must terminate
      int one = 1;
      CK(cudaMemcpyAsync(&h->st->final_force, &one, sizeof(int), cudaMemcpyHostToDevice, h->s));
      CK(cudaStreamSynchronize(h->s));
      enqueue_check(h, 0, 1, adaptive);
      launches += adaptive ? 9 : 8;
      CKL("time-limit check");
    }
  }
  CK(cudaEventRecord(h->ev_t1, h->s));
  CK(cudaStreamSynchronize(h->s));
  CK(cudaMemcpy(&fin, h->st, sizeof(DevState), cudaMemcpyDeviceToHost));
  check_stage_err(h);
  float dev_ms = 0.f;
  CK(cudaEventElapsedTime(&dev_ms, h->ev_t0, h->ev_t1));
  h->last_ncheck = fin.ncheck;
  h->last_nrestart = fin.nrestart;
  h->solved = true;
  h->resumable = !mixed;

  // returned point
  if (x_out || y_out) {
    const double* xo = h->x;
    const double* yo = h->y;
    if (fin.which == 1) {
      k_average<<<grid_for(np), 256, 0, h->s>>>(h->tn, h->sx, h->x, h->st, np);
      k_average<<<grid_for(mp), 256, 0, h->s>>>(h->tm, h->sy, h->y, h->st, mp);
      xo = h->tn;
      yo = h->tm;
    }
    export_point(h, xo, yo, x_out, y_out);
  }
  if (res) {
    res->status = fin.status;
    if (timed_out && fin.status != PDLP_OPTIMAL && fin.status != PDLP_NUMERICAL) res->status = PDLP_TIME_LIMIT;
    res->which = fin.which;
    res->iters = fin.k;
    res->restarts = fin.nrestart;
    res->primal_obj = fin.out_pobj;
    res->dual_obj = fin.out_dobj;
    res->rel_primal = fin.out_rel_p;
    res->rel_dual = fin.out_rel_d;
    res->rel_gap = fin.out_rel_g;
    res->kkt_omega = fin.out_kkt;
    res->omega = fin.omega;
    res->eta = fin.eta;
    res->device_ms = dev_ms;
    res->launches = launches;
    res->accepted = adaptive ? fin.accepted : fin.k;
    res->fp32_iters = h->fp32_iters;
    res->solve_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
  }
  return PDLP_OK;
}

template <class F>
static int guarded(pdlp_ctx* h, F&& f) {
  if (!h) return PDLP_EINVAL;
  if (h->broken) {
    h->err = "a bounded device wait gave up earlier on this handle; free it";
    return PDLP_ETIMEOUT;
  }
  h->err.clear();
  try {
    DeviceGuard dg(h->dev);
    StreamOrder so(h, h->p.stream);
    return f();
  } catch (const Failure& e) {
    h->err = e.msg;
    return e.code;
  } catch (const std::bad_alloc&) {
    h->err = "host allocation failed";
    return PDLP_ENOMEM;
  } catch (...) {
    h->err = "unexpected internal error";
    return PDLP_EINTERNAL;
  }
}


// ------------------------------------------------------------------ batches

constexpr int kBatchThreads = 256;
constexpr int kBatchRed = NQ * (1 + kBatchThreads / 32);   // block_sum scratch (doubles)

// Launch resources of the persistent batched kernel for the h->count LPs described by
// h->hdesc over the layout Lo: shared-memory plan, kernel attributes, occupancy, the
// queue (largest LP first) and the per-LP state and output arrays.
static void init_batch_launch(pdlp_ctx* h, const Layout& Lo, int64_t npad_max, int64_t mpad_max) {
  const int64_t count = h->count;
  // shared memory per CTA: x and y of the largest LP plus the reduction scratch; when
  // they do not fit, the iterates go to global memory (one copy per LP)
  h->xs_off = 0;
  h->ys_off = (int)npad_max;
  h->red_off = (int)(npad_max + mpad_max);
  h->part_off = h->red_off + kBatchRed;
  h->batch_smem = (size_t)(npad_max + mpad_max + kBatchRed + kPartBuf) * sizeof(double);
  h->glob_smem = (size_t)(kBatchRed + kPartBuf) * sizeof(double);
  int dev_smem = 0;
  CK(cudaDeviceGetAttribute(&dev_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->dev));
  int static_max = 0;
  const void* kernels[] = {(const void*)k_batch_solve<false, false, false>, (const void*)k_batch_solve<false, true, false>,
                           (const void*)k_batch_solve<true, false, false>,  (const void*)k_batch_solve<true, true, false>,
                           (const void*)k_batch_solve<false, false, true>,  (const void*)k_batch_solve<true, false, true>,
                           (const void*)k_batch_solve32<false, false>,      (const void*)k_batch_solve32<true, false>,
                           (const void*)k_batch_solve32<false, true>,       (const void*)k_batch_solve32<true, true>};
  for (const void* f : kernels) {
    cudaFuncAttributes fa;
    CK(cudaFuncGetAttributes(&fa, f));
    static_max = std::max(static_max, (int)fa.sharedSizeBytes);
  }
  const int smem_cap = dev_smem - static_max;
  h->batch_glob = smem_cap < (int)h->batch_smem;
  h->dev_smem_optin = smem_cap;
  for (const void* f : kernels) CK(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_cap));
  for (int i = 2; i < 10; ++i)
    if (i != 4 && i != 6 && i != 8)   // the cluster (team) kernels
      CK(cudaFuncSetAttribute(kernels[i], cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
  h->hk_cptr = Lo.SK.chunk_ptr;
  h->ht_cptr = Lo.SKt.chunk_ptr;
  int per_sm = 0, sms = 0;
  CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
      &per_sm, h->batch_glob ? (const void*)k_batch_solve<false, false, true> : (const void*)k_batch_solve<false, false, false>,
      kBatchThreads, h->batch_glob ? h->glob_smem : h->batch_smem));
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->dev));
  if (per_sm < 1) invalid("batched kernel does not fit on an SM");
  h->batch_resident = per_sm * sms;
  h->batch_grid = (int)std::min<int64_t>((int64_t)per_sm * sms, count);
  h->team_npad_max = npad_max;

  // queue order: largest LP (most nonzeros) first
  std::vector<int32_t> ord((size_t)count);
  for (int64_t b = 0; b < count; ++b) ord[(size_t)b] = (int32_t)b;
  std::vector<int64_t> work((size_t)count);
  for (int64_t b = 0; b < count; ++b) {
    const LpDesc& D = h->hdesc[(size_t)b];
    std::vector<int32_t> dummy;
    work[(size_t)b] = (int64_t)(Lo.SK.chunk_ptr[(size_t)D.kc1] - Lo.SK.chunk_ptr[(size_t)D.kc0]) + D.mpad + D.npad;
  }
  std::stable_sort(ord.begin(), ord.end(), [&](int32_t a, int32_t b2) { return work[(size_t)a] > work[(size_t)b2]; });
  h->desc = upload(h, h->hdesc);
  h->order = upload(h, ord);
  h->next = dalloc<int32_t>(h, 1);
  h->bstate = dalloc<DevState>(h, (size_t)count);
  h->bx = dalloc<double>(h, h->npad);
  h->by = dalloc<double>(h, h->mpad);
  h->hstate.resize((size_t)count);
  CK(cudaStreamSynchronize(h->s));
}

static void batch_setup_impl(pdlp_ctx* h, int64_t count, const int64_t* m_in, const int64_t* n_in,
                             const int64_t* m1_in, const int64_t* row_ptr_in, const int32_t* col_in,
                             const double* val_in, const double* c_in, const double* q_in, const double* l_in,
                             const double* u_in) {
  const pdlp_params& P = h->p;
  check_params(P);
  if (count < 1 || count >= ((int64_t)1 << 31)) invalid("batch count must be in [1, 2^31)");
  if (!m_in || !n_in || !m1_in || !row_ptr_in || !c_in || !l_in || !u_in) invalid("null input array");
  std::vector<int64_t> lm((size_t)count), ln((size_t)count), lm1((size_t)count);
  std::memcpy(lm.data(), m_in, sizeof(int64_t) * count);   // sizes are host arrays
  std::memcpy(ln.data(), n_in, sizeof(int64_t) * count);
  std::memcpy(lm1.data(), m1_in, sizeof(int64_t) * count);
  int64_t M = 0, N = 0, R = 0;
  for (int64_t b = 0; b < count; ++b) {
    if (lm[(size_t)b] < 0 || ln[(size_t)b] < 1 || lm1[(size_t)b] < 0 || lm1[(size_t)b] > lm[(size_t)b])
      invalid("each LP needs m >= 0, n >= 1, 0 <= m1 <= m");
    M += lm[(size_t)b];
    N += ln[(size_t)b];
    R += lm[(size_t)b] + 1;
  }
  if (M >= ((int64_t)1 << 31) || N >= ((int64_t)1 << 31)) invalid("total rows and columns must be below 2^31");
  if (M > 0 && !q_in) invalid("null q");
  init_handle_resources(h);
  h->is_batch = true;
  h->count = count;
  h->m = M;
  h->n = N;
  h->m1 = 0;
  using clk = std::chrono::steady_clock;
  auto ms_since = [](clk::time_point a) { return std::chrono::duration<double, std::milli>(clk::now() - a).count(); };
  auto t0 = clk::now();
  const bool dev_in = P.inputs_on_device != 0;
  if (dev_in && P.stream) CK(cudaStreamSynchronize((cudaStream_t)P.stream));
  // row pointers on the host (the caller's array or a copy); each LP's start at 0 and
  // nondecreasing; nonzeros from each LP's last row pointer
  std::vector<int64_t> rp_copy;
  const int64_t* rp = row_ptr_in;
  if (dev_in) {
    rp_copy.resize((size_t)R);
    CK(cudaMemcpy(rp_copy.data(), row_ptr_in, sizeof(int64_t) * R, cudaMemcpyDeviceToHost));
    rp = rp_copy.data();
  }
  std::vector<int64_t> ent0((size_t)count + 1, 0), col0v((size_t)count + 1, 0);
  int64_t nnz = 0;
  for (int64_t b = 0, r = 0; b < count; ++b) {
    const int64_t m = lm[(size_t)b];
    if (rp[r + m] < 0) invalid("negative row pointer");
    if (rp[r] != 0) invalid("row_ptr[0] must be 0");
    for (int64_t i = 0; i < m; ++i)
      if (rp[r + i + 1] < rp[r + i]) invalid("row_ptr must be nondecreasing");
    nnz += rp[r + m];
    if (nnz >= ((int64_t)1 << 31)) invalid("total nnz must be below 2^31");
    ent0[(size_t)b + 1] = nnz;
    col0v[(size_t)b + 1] = col0v[(size_t)b] + ln[(size_t)b];
    r += m + 1;
  }
  h->nnz = nnz;
  if (nnz > 0 && (!col_in || !val_in)) invalid("null col_idx/val with nnz > 0");
  check_vectors(h, N, M, c_in, q_in, l_in, u_in);

  Layout Lo;
  Lo.pos_r.assign((size_t)M, 0);
  Lo.pos_c.assign((size_t)N, 0);
  h->hdesc.resize((size_t)count);
  int64_t npad_max = 0, mpad_max = 0;
  // appends LP b's layouts (shape only, or with host entry arrays) and its descriptor
  auto add_lp = [&](int64_t b, SellHost&& sk, SellHost&& stt, int64_t rbase, int64_t cbase) {
    const int64_t mp = Lo.mpad - rbase, np = Lo.npad - cbase;
    LpDesc& D = h->hdesc[(size_t)b];
    D.m = (int32_t)lm[(size_t)b];
    D.n = (int32_t)ln[(size_t)b];
    D.m1 = (int32_t)lm1[(size_t)b];
    D.pad0 = 0;
    D.kc0 = (int32_t)Lo.SK.nchunks;
    append_sell(Lo.SK, sk);
    D.kc1 = (int32_t)Lo.SK.nchunks;
    D.tc0 = (int32_t)Lo.SKt.nchunks;
    append_sell(Lo.SKt, stt);
    D.tc1 = (int32_t)Lo.SKt.nchunks;
    D.r0 = rbase;
    D.c0 = cbase;
    D.mpad = (int32_t)mp;
    D.npad = (int32_t)np;
    npad_max = std::max(npad_max, np);
    mpad_max = std::max(mpad_max, mp);
  };
  if (P.host_layout) {
    // the reference builder: entries copied, checked and laid out on the host
    HostLP H;
    fetch_matrix(h, row_ptr_in, col_in, val_in, H, R);
    h->setup_ms[0] = ms_since(t0);
    t0 = clk::now();
    int64_t rp0 = 0, row0 = 0;
    for (int64_t b = 0; b < count; ++b) {
      const int64_t m = lm[(size_t)b], n = ln[(size_t)b], nnz0 = ent0[(size_t)b];
      const int64_t lnnz = check_csr(H, rp0, m, n, nnz0);
      const int64_t* lrp = H.rp.data() + rp0;
      const int32_t* lcol = H.col.data() + nnz0;
      std::vector<int32_t> clen((size_t)n, 0);
      for (int64_t k = 0; k < lnnz; ++k) clen[(size_t)lcol[k]]++;
      std::vector<int64_t> k_est, t_est;
      std::vector<int32_t> k_eln, t_eln, k_ecol, k_esrc, t_ecol, t_esrc;
      const int64_t rbase = Lo.mpad, cbase = Lo.npad;
      LpOrder O;
      order_lp(Lo, O, lrp, std::move(clen), m, n, lm1[(size_t)b], row0, col0v[(size_t)b], k_eln, t_eln);
      host_entries(O, lrp, lcol, nnz0, lnnz, k_est, k_ecol, k_esrc, t_est, t_ecol, t_esrc);
      SellHost sk = build_sell(O.mp, k_est, k_eln, k_ecol, k_esrc, (int32_t)cbase);
      SellHost stt = build_sell(O.np, t_est, t_eln, t_ecol, t_esrc, (int32_t)rbase);
      add_lp(b, std::move(sk), std::move(stt), rbase, cbase);
      rp0 += m + 1;
      row0 += m;
    }
    h->setup_ms[1] = ms_since(t0);
    t0 = clk::now();
    device_setup_common(h, Lo, nullptr, &H.val, c_in, q_in, l_in, u_in);
  } else {
    // one global numbering: global row pointers, entries checked and counted on the
    // device; each LP ordered on the host; the layouts filled on the device
    std::vector<int64_t> grp((size_t)M + 1);
    for (int64_t b = 0, r = 0, g = 0; b < count; ++b) {
      const int64_t m = lm[(size_t)b];
      for (int64_t i = 0; i <= m; ++i) grp[(size_t)(g + i)] = ent0[(size_t)b] + rp[r + i];
      r += m + 1;
      g += m;
    }
    std::vector<int32_t> clen;
    DevMatrix A = upload_matrix(h, M, N, nnz, grp.data(), ent0, col0v, col_in, val_in, clen);
    h->setup_ms[0] = ms_since(t0);
    t0 = clk::now();
    std::vector<int32_t> kpad, tpad;
    int64_t r = 0, row0 = 0;
    for (int64_t b = 0; b < count; ++b) {
      const int64_t m = lm[(size_t)b], n = ln[(size_t)b], c0 = col0v[(size_t)b];
      std::vector<int32_t> k_eln, t_eln;
      const int64_t rbase = Lo.mpad, cbase = Lo.npad;
      LpOrder O;
      order_lp(Lo, O, rp + r, std::vector<int32_t>(clen.begin() + c0, clen.begin() + c0 + n), m, n,
               lm1[(size_t)b], row0, c0, k_eln, t_eln);
      SellHost sk = sell_shape(O.mp, k_eln), stt = sell_shape(O.np, t_eln);
      kpad.insert(kpad.end(), (size_t)sk.nchunks, (int32_t)cbase);
      tpad.insert(tpad.end(), (size_t)stt.nchunks, (int32_t)rbase);
      add_lp(b, std::move(sk), std::move(stt), rbase, cbase);
      r += m + 1;
      row0 += m;
    }
    h->setup_ms[1] = ms_since(t0);
    t0 = clk::now();
    finish_matrix(h, A, M, N, nnz, kpad, tpad);
    const DevCsr dc = A.csr();
    device_setup_common(h, Lo, &dc, nullptr, c_in, q_in, l_in, u_in);
    free_matrix(h, A);
  }
  CK(cudaStreamSynchronize(h->s));
  h->setup_ms[2] = ms_since(t0);
  t0 = clk::now();

  init_batch_launch(h, Lo, npad_max, mpad_max);
  if (P.precision == PDLP_MIXED) setup_mixed(h);
  else if (P.precision != PDLP_FP64) invalid("precision must be PDLP_FP64 or PDLP_MIXED");
  CK(cudaStreamSynchronize(h->s));
  h->setup_ms[4] = ms_since(t0);
}

// CTAs per LP: the requested count, else the largest power of two <= 16 whose CTAs for
// the whole batch come to at most kTeamWaves times the resident CTAs of the GPU, with at
// least 64 columns of the largest LP per CTA (one CTA per LP for a batch that fills the
// GPU several times over).  Teams finish an LP faster, and waiting teams take the SMs
// that finished LPs free, so a few waves beat one wave of smaller teams: 16..256 planted
// LPs with n ~ U(2000, 5000) chose 16, 16, 16, 8, 4 CTAs (within 4 % of the best of
// 1..16 each; the former one-wave rule, 16, 8, 4, 2, 1, was up to 3.2x slower).  With
// the iterates in global memory (four CTAs per SM) teams beyond 4 lose and one wave is
// best: 200 x 300 transportation LPs (n = 60000), 64 / 128 / 256 / 512 / 1000 of them,
// get 4 / 4 / 2 / 1 / 1 CTAs, the best of 1, 2, 4 at each count.
constexpr int64_t kTeamWaves = 4;
constexpr int kTeamGlobMax = 4;
constexpr int64_t kTeamWavesGlob = 1;
// The same cut of chunks [c0, c1) into `size` pieces as split_point on the device.
static int host_split_point(const std::vector<int32_t>& cptr, int c0, int c1, int r, int size) {
  if (r <= 0) return c0;
  if (r >= size) return c1;
  const long long s0 = cptr[(size_t)c0], s1 = cptr[(size_t)c1];
  const long long target = s0 + (s1 - s0) * r / size;
  int lo = c0, hi = c1;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (cptr[(size_t)mid] < target) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// Largest resident slice (bytes) over the LPs of the batch and the CTAs of a team.
static long long resident_need(const pdlp_ctx* h, int team) {
  long long need = 0;
  for (const LpDesc& D : h->hdesc) {
    for (int r = 0; r < team; ++r) {
      const int k0 = host_split_point(h->hk_cptr, D.kc0, D.kc1, r, team);
      const int k1 = host_split_point(h->hk_cptr, D.kc0, D.kc1, r + 1, team);
      const int t0 = host_split_point(h->ht_cptr, D.tc0, D.tc1, r, team);
      const int t1 = host_split_point(h->ht_cptr, D.tc0, D.tc1, r + 1, team);
      const long long ks = h->hk_cptr[(size_t)k1] - h->hk_cptr[(size_t)k0];
      const long long ts = h->ht_cptr[(size_t)t1] - h->ht_cptr[(size_t)t0];
      need = std::max(need, resident_bytes(k1 - k0, ks, t1 - t0, ts, 32LL * (k1 - k0), 32LL * (t1 - t0)));
    }
  }
  return need;
}

static int batch_team_size(const pdlp_ctx* h, int64_t count, int team_req, bool glob) {
  if (team_req > 0) return team_req;
  const int cap = glob ? kTeamGlobMax : kMaxTeam;
  const int64_t waves = glob ? kTeamWavesGlob : kTeamWaves;
  int team = 1;
  while (team < cap && count * (int64_t)(team * 2) <= waves * (int64_t)h->batch_resident &&
         h->team_npad_max >= (int64_t)(team * 2) * 64)
    team *= 2;
  return team;
}

// One launch of the persistent batched kernel over A.count LPs (A.order): team size,
// resident slices and grid chosen for that count.
// One launch of the persistent batched kernel over A.count LPs (A.order): team size,
// placement of the iterates (shared-memory replicas, with or without resident matrix
// slices, or global memory) and grid chosen for that count.
// Device buffers a batched launch may need, allocated before any launch (and so before a
// graph capture): global iterates and the second queue.
static void batch_buffers(pdlp_ctx* h, bool glob, bool fp32) {
  if (glob && !h->xg) {
    h->xg = dalloc<double>(h, (size_t)h->npad);
    h->yg = dalloc<double>(h, (size_t)std::max<int64_t>(h->mpad, 1));
  }
  if (glob && fp32 && !h->xg32) {
    h->xg32 = dalloc<float>(h, (size_t)h->npad);
    h->yg32 = dalloc<float>(h, (size_t)std::max<int64_t>(h->mpad, 1));
  }
  if (!h->order2) h->order2 = dalloc<int32_t>(h, (size_t)h->count);
}

static void launch_batch(pdlp_ctx* h, const BatchArgs& A0, const pdlp_params& sp, int64_t count, int team_req,
                         bool fp32 = false) {
  const bool glob = h->batch_glob || sp.resident == 3;
  const int team = batch_team_size(h, count, team_req, glob);
  BatchArgs A = A0;
  batch_buffers(h, glob, fp32);
  if (glob) {
    A.xs_off = A.ys_off = 0;
    A.red_off = 0;
    A.part_off = kBatchRed;
  }
  A.xg = h->xg;
  A.yg = h->yg;
  A.xg32 = h->xg32;
  A.yg32 = h->yg32;
  // resident slices: the largest one of any LP and CTA decides the launch's shared memory
  bool resident = false;
  size_t res_smem = 0;
  if (!glob && !fp32 && sp.resident != 1) {
    const long long res_bytes = resident_need(h, team);
    res_smem = h->batch_smem + (size_t)((res_bytes + 7) / 8 * 8);
    if (res_smem <= (size_t)h->dev_smem_optin) {
      if (sp.resident == 2) {
        resident = true;
      } else {
        // automatic: only while it keeps as many CTAs per SM as the streaming kernel
        int a = 0, r = 0;
        CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_batch_solve<false, false, false>, kBatchThreads,
                                                         h->batch_smem));
        CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&r, k_batch_solve<false, true, false>, kBatchThreads,
                                                         res_smem));
        resident = r >= a;
      }
    }
  }
  const size_t smem = glob ? h->glob_smem : resident ? res_smem : h->batch_smem;
  // the kernel: [team > 1][fp32][resident][glob]
  const void* kfn;
  if (team == 1)
    kfn = fp32       ? (glob ? (const void*)k_batch_solve32<false, true> : (const void*)k_batch_solve32<false, false>)
          : glob     ? (const void*)k_batch_solve<false, false, true>
          : resident ? (const void*)k_batch_solve<false, true, false>
                     : (const void*)k_batch_solve<false, false, false>;
  else
    kfn = fp32       ? (glob ? (const void*)k_batch_solve32<true, true> : (const void*)k_batch_solve32<true, false>)
          : glob     ? (const void*)k_batch_solve<true, false, true>
          : resident ? (const void*)k_batch_solve<true, true, false>
                     : (const void*)k_batch_solve<true, false, false>;
  int grid = 0;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = (unsigned)team;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.blockDim = dim3(kBatchThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = h->s;
  if (team == 1) {
    int per_sm = 0, sms = 0;
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kfn, kBatchThreads, smem));
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->dev));
    if (per_sm < 1) invalid("batched kernel does not fit on an SM");
    grid = (int)std::min<int64_t>((int64_t)per_sm * sms, count);
  } else {
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cfg.gridDim = dim3((unsigned)team);
    int nc = 0;
    CK(cudaOccupancyMaxActiveClusters(&nc, kfn, &cfg));
    if (nc < 1) invalid("a cluster of this many CTAs does not fit on the GPU");
    grid = (int)std::min<int64_t>((int64_t)nc, count) * team;
  }
  cfg.gridDim = dim3((unsigned)grid);
  h->last_grid = grid;
  h->last_smem = smem;
  h->last_team = team;
  h->last_resident = resident;
  h->last_glob = glob;
  void* args[] = {(void*)&A};
  CK(cudaLaunchKernelExC(&cfg, kfn, args));
  CKL("k_batch_solve");
  h->last_launches++;
}

constexpr int64_t kBatchRestartCap = 256;   // restart iterations kept per LP of a batch

// LPs of the batch whose last launch suspended them (they continue in a resumed launch).
static std::vector<int32_t> suspended_lps(pdlp_ctx* h) {
  CK(cudaMemcpyAsync(h->hstate.data(), h->bstate, sizeof(DevState) * h->count, cudaMemcpyDeviceToHost, h->s));
  CK(cudaStreamSynchronize(h->s));
  std::vector<int32_t> rest;
  for (int64_t b = 0; b < h->count; ++b)
    if (h->hstate[(size_t)b].suspended) rest.push_back((int32_t)b);
  return rest;
}

// A resumed launch over the LPs `lps` (uploaded to the second queue).
static void launch_resumed(pdlp_ctx* h, const BatchArgs& A0, const pdlp_params& sp, const std::vector<int32_t>& lps,
                           int team_req, long long slice) {
  batch_buffers(h, h->batch_glob || sp.resident == 3, false);
  CK(cudaMemcpyAsync(h->order2, lps.data(), sizeof(int32_t) * lps.size(), cudaMemcpyHostToDevice, h->s));
  BatchArgs A = A0;
  A.order = h->order2;
  A.count = (int32_t)lps.size();
  A.resume = 1;
  A.slice_iters = slice;
  launch_batch(h, A, sp, (int64_t)lps.size(), team_req);
}

// Online autotuner of the batched launch, run by the first solve of a handle whose team
// size and data placement are automatic (FP64 batches).  The first check_every
// iterations of every LP run with the rule's choice (they also hold the power
// iteration); then each candidate runs the next check_every iterations of every LP
// still running, as one resumed launch, and is scored by the work it did (iterations
// run x stored bytes of one iteration of each LP) per device second.  Candidates: the
// rule's team size with each placement that fits (iterates streamed from shared-memory
// replicas or resident matrix slices; global iterates when x and y do not fit), then a
// climb in team size with the better placement: doubling while the score improves, or
// halving when the first doubling did not.  At most 8 candidates; tuning stops early
// once fewer than half of the LPs are still running.  Nothing is repeated: the slices
// are the solve's own iterations, resumed exactly (up to summation order).  The fastest
// candidate is kept for the rest of the solve and for later solves of the handle.
// Returns the LPs left running after the slices.
static std::vector<int32_t> tune_batch(pdlp_ctx* h, const BatchArgs& A0, const pdlp_params& sp) {
  const int64_t count = h->count;
  const bool glob = h->batch_glob;
  const int rule = batch_team_size(h, count, 0, glob);
  const int cap = glob ? kTeamGlobMax : kMaxTeam;
  auto feasible = [&](int T) { return T >= 1 && T <= cap && (T == 1 || h->team_npad_max >= (int64_t)T * 64); };
  auto res_fits = [&](int T) {
    const long long need = resident_need(h, T);
    return h->batch_smem + (size_t)((need + 7) / 8 * 8) <= (size_t)h->dev_smem_optin;
  };
  std::vector<double> w((size_t)count);
  for (int64_t b = 0; b < count; ++b) {
    const LpDesc& D = h->hdesc[(size_t)b];
    const double slots = (double)(h->hk_cptr[(size_t)D.kc1] - h->hk_cptr[(size_t)D.kc0]) +
                         (double)(h->ht_cptr[(size_t)D.tc1] - h->ht_cptr[(size_t)D.tc0]);
    w[(size_t)b] = 12.0 * 32.0 * slots + 68.0 * (double)(D.mpad + D.npad);
  }
  // slice 0: the rule's choice
  BatchArgs A = A0;
  A.slice_iters = sp.check_every;
  launch_batch(h, A, sp, count, 0);
  std::vector<int32_t> active = suspended_lps(h);
  std::vector<long long> kprev((size_t)count);
  for (int64_t b = 0; b < count; ++b) kprev[(size_t)b] = h->hstate[(size_t)b].k;
  h->tune_candidates = 0;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  double best = -1.0;
  int best_team = rule, best_res = glob ? 3 : 1;
  // one timed slice of candidate (team, placement); -1 when tuning has to stop
  auto eval = [&](int team, int res) -> double {
    if (h->tune_candidates >= 8 || (int64_t)active.size() * 2 < count) return -1.0;
    pdlp_params sc = sp;
    sc.resident = res;
    CK(cudaEventRecord(e0, h->s));
    launch_resumed(h, A0, sc, active, team, sp.check_every);
    CK(cudaEventRecord(e1, h->s));
    std::vector<int32_t> next = suspended_lps(h);
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, e0, e1));
    double work = 0.0;
    for (int32_t b : active) {
      work += (double)(h->hstate[(size_t)b].k - kprev[(size_t)b]) * w[(size_t)b];
      kprev[(size_t)b] = h->hstate[(size_t)b].k;
    }
    const double rate = ms > 0.f ? work / (double)ms : 0.0;
    const int i = h->tune_candidates++;
    h->tune_rates[i] = rate * 1e-6;   // GB/s of stored bytes
    h->tune_team[i] = team;
    h->tune_res[i] = res;
    if (rate > best) {
      best = rate;
      best_team = team;
      best_res = res;
    }
    active.swap(next);
    return rate;
  };
  try {
    // the rule's team with each placement that fits
    if (glob) {
      eval(rule, 3);
    } else {
      eval(rule, 1);
      if (res_fits(rule)) eval(rule, 2);
    }
    const int mode = best_res;
    auto mode_for = [&](int T) { return (mode == 2 && !res_fits(T)) ? 1 : mode; };
    // climb: double while the score improves; if the first doubling loses, halve instead
    bool up_won = false;
    for (int T = rule * 2; feasible(T); T *= 2) {
      const double before = best;
      const double r = eval(T, mode_for(T));
      if (r < 0.0 || r <= before) break;
      up_won = true;
    }
    if (!up_won)
      for (int T = rule / 2; T >= 1 && feasible(T); T /= 2) {
        const double before = best;
        const double r = eval(T, mode_for(T));
        if (r < 0.0 || r <= before) break;
      }
  } catch (...) {
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    throw;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  // a choice needs at least two timed candidates (a solve shorter than the slices
  // leaves the handle untuned, and the next solve tries again)
  if (h->tune_candidates >= 2) {
    h->tuned = true;
    h->tuned_team = best_team;
    h->tuned_resident = best_res;
  }
  return active;
}

// single: one LP of a single-LP handle through the persistent engine (omega0_single is
// its initial primal weight, <= 0 for the handle's ω₀; the current point, restarts and
// check records go to the handle's own arrays).
static int batch_solve_impl(pdlp_ctx* h, const pdlp_params& sp, const double* x0, const double* y0,
                            const double* omega0, pdlp_result* res, double* x_out, double* y_out, bool single,
                            double omega0_single) {
  if (sp.check_every < 1 || sp.max_iter < 0 || !(sp.tol >= 0.0)) invalid("bad solve parameters");
  if (sp.cluster_ctas < 0 || sp.cluster_ctas > kMaxTeam) invalid("cluster_ctas must be in [0, 16]");
  if (sp.resident < 0 || sp.resident > 3) invalid("resident must be 0, 1, 2 or 3");
  if (sp.step_rule != 0) invalid("batches use the constant step (step_rule 0)");
  if (sp.batch_tail_iters < 0) invalid("batch_tail_iters must be >= 0");
  if (sp.batch_tune < 0 || sp.batch_tune > 2) invalid("batch_tune must be 0, 1 or 2");
  auto t_start = std::chrono::steady_clock::now();
  BatchArgs A;
  A.x0 = nullptr;
  A.y0 = nullptr;
  A.omega0 = nullptr;
  if (x0) {
    copy_in(h, h->stage_n, x0, h->n);
    k_permute_in<<<grid_for(h->npad), 256, 0, h->s>>>(h->tn, h->stage_n, h->perm_c, h->Dc, h->npad, 0.0);
    A.x0 = h->tn;
  }
  if (y0 && h->m > 0) {
    copy_in(h, h->stage_m, y0, h->m);
    k_permute_in<<<grid_for(h->mpad), 256, 0, h->s>>>(h->tm, h->stage_m, h->perm_r, h->Dr, h->mpad, 0.0);
    A.y0 = h->tm;
  }
  if (omega0) {
    if (!h->bomega) h->bomega = dalloc<double>(h, (size_t)h->count);
    copy_in(h, h->bomega, omega0, h->count);
    A.omega0 = h->bomega;
  }
  A.xcur = A.ycur = nullptr;
  A.restarts = nullptr;
  A.restart_stride = 0;
  A.log = nullptr;
  A.desc = h->desc;
  A.order = h->order;
  A.count = (int32_t)h->count;
  A.next = h->next;
  A.k_cptr = h->K.chunk_ptr;
  A.k_col = h->K.col;
  A.k_val = h->K.val;
  A.t_cptr = h->Kt.chunk_ptr;
  A.t_col = h->Kt.col;
  A.t_val = h->Kt.val;
  A.c = h->c; A.l = h->l; A.u = h->u; A.q = h->q; A.invDr = h->invDr; A.invDc = h->invDc;
  A.sx = h->sx; A.sy = h->sy; A.xa = h->xa; A.ya = h->ya; A.kxp = h->kxp; A.g = h->g_c; A.kx_a = h->kx_a;
  A.g_a = h->g_a;
  A.xout = h->bx;
  A.yout = h->by;
  A.st = h->bstate;
  A.P = DevParams{};
  A.P.tol = sp.tol;
  A.P.beta_suff = sp.beta_suff;
  A.P.beta_nec = sp.beta_nec;
  A.P.beta_art = sp.beta_art;
  A.P.theta = sp.omega_theta;
  A.P.max_iter = sp.max_iter;
  if (!single) {
    if (!h->brestarts) h->brestarts = dalloc<long long>(h, (size_t)h->count * kBatchRestartCap);
    A.restarts = h->brestarts;
    A.restart_stride = kBatchRestartCap;
    A.P.restart_cap = (int)kBatchRestartCap;
  }
  A.check_every = sp.check_every;
  A.max_iter = sp.max_iter;
  A.power_iters = h->p.power_iters;
  A.step_scale = h->p.step_scale;
  A.eta_fixed = h->p.eta;
  A.omega_fixed = 0.0;
  if (single) {
    // the same step size and primal weight as the launch-per-kernel path
    A.eta_fixed = h->eta;
    A.omega_fixed = omega0_single > 0.0 ? omega0_single : h->omega0;
    A.xcur = h->x;
    A.ycur = h->y;
    A.restarts = h->restarts;
    A.log = h->log;
    A.P.log_cap = h->log_cap;
    A.P.restart_cap = h->restart_cap;
  }
  A.xs_off = h->xs_off;
  A.ys_off = h->ys_off;
  A.red_off = h->red_off;
  A.part_off = h->part_off;
  const bool mixed = h->p.precision == PDLP_MIXED;
  A.k_val32 = h->K.val32;
  A.t_val32 = h->Kt.val32;
  A.c32 = h->c32; A.l32 = h->l32; A.u32 = h->u32; A.q32 = h->q32;
  A.sx32 = h->sx32; A.sy32 = h->sy32; A.kxp32 = h->kxp32;
  A.switch_tol = sp.mixed_switch_tol > 0.0 ? sp.mixed_switch_tol : std::max(sp.tol, 1e-5);
  A.slice_iters = (!mixed && sp.batch_tail_iters > 0) ? sp.batch_tail_iters : 0;
  A.resume = 0;
  h->last_resumed = 0;
  h->last_launches = 0;
  CK(cudaEventRecord(h->ev_t0, h->s));
  // team size and placement: the caller's, the online autotuner's (timed on the first
  // solve of the handle, on the solve's own first iterations), or the rule
  const bool auto_cfg = !single && !mixed && sp.cluster_ctas == 0 && sp.resident == 0 && sp.batch_tune != 1;
  pdlp_params sp1 = sp;
  int team1 = sp.cluster_ctas;
  bool tuned_now = false;
  std::vector<int32_t> active;
  h->last_tuned = false;
  if (auto_cfg && h->count >= 2 && (sp.batch_tune == 2 || !h->tuned)) {
    active = tune_batch(h, A, sp);
    tuned_now = true;
    h->last_tuned = true;
  }
  if (auto_cfg && h->tuned) {
    team1 = h->tuned_team;
    sp1.resident = h->tuned_resident;
  } else if (tuned_now) {
    team1 = 0;   // nothing to choose from: the rule
  }
  // mixed precision: FP32 iterations first; the LPs that leave them unfinished are
  // suspended with their FP64 state and continue in FP64 (second stage).  With
  // batch_tail_iters the LPs still running after that many iterations continue in a
  // second stage too, with teams sized for their number.
  const bool two_stage = A.slice_iters > 0 || mixed;
  h->last_graph = false;
  if (!tuned_now && !single && !two_stage) {
    // a one-stage solve: its persistent launch as a CUDA graph, instantiated once per
    // handle and updated in place when the arguments change
    batch_buffers(h, h->batch_glob || sp1.resident == 3, false);
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(h->s, cudaStreamCaptureModeThreadLocal));
    try {
      launch_batch(h, A, sp1, h->count, team1, false);
    } catch (...) {
      cudaStreamEndCapture(h->s, &g);
      if (g) cudaGraphDestroy(g);
      throw;
    }
    CK(cudaStreamEndCapture(h->s, &g));
    // an in-place update only for the same launch configuration (kernel, team size, grid,
    // shared memory); another configuration gets a new executable graph
    const long long key = ((long long)h->last_grid << 24) ^ ((long long)h->last_smem << 8) ^
                          ((long long)h->last_team << 2) ^ ((long long)h->last_resident << 1) ^ (long long)h->last_glob;
    if (h->bgraph && key != h->bgraph_key) {
      cudaGraphExecDestroy(h->bgraph);
      h->bgraph = nullptr;
    }
    if (h->bgraph) {
      cudaGraphExecUpdateResultInfo ui;
      if (cudaGraphExecUpdate(h->bgraph, g, &ui) != cudaSuccess) {
        (void)cudaGetLastError();
        cudaGraphExecDestroy(h->bgraph);
        h->bgraph = nullptr;
      }
    }
    h->bgraph_key = key;
    if (!h->bgraph) {
      const cudaError_t e = cudaGraphInstantiate(&h->bgraph, g, 0);
      cudaGraphDestroy(g);
      CK(e);
    } else {
      cudaGraphDestroy(g);
    }
    CK(cudaGraphLaunch(h->bgraph, h->s));
    h->last_graph = true;
  } else {
    if (!tuned_now) launch_batch(h, A, sp1, h->count, team1, mixed);
    else if (!active.empty()) launch_resumed(h, A, sp1, active, team1, A.slice_iters);
    if (two_stage) {
      std::vector<int32_t> rest = suspended_lps(h);
      h->last_resumed = (int64_t)rest.size();
      if (!rest.empty()) launch_resumed(h, A, sp, rest, 0, 0);
    }
  }
  CK(cudaEventRecord(h->ev_t1, h->s));
  CK(cudaStreamSynchronize(h->s));
  float dev_ms = 0.f;
  CK(cudaEventElapsedTime(&dev_ms, h->ev_t0, h->ev_t1));
  CK(cudaMemcpy(h->hstate.data(), h->bstate, sizeof(DevState) * h->count, cudaMemcpyDeviceToHost));
  if (x_out) {
    k_unpermute_scale<<<grid_for(h->n), 256, 0, h->s>>>(h->stage_n, h->bx, h->Dc, h->pos_c, h->n);
    copy_out(h, x_out, h->stage_n, h->n);
  }
  if (y_out && h->m > 0) {
    k_unpermute_scale<<<grid_for(h->m), 256, 0, h->s>>>(h->stage_m, h->by, h->Dr, h->pos_r, h->m);
    copy_out(h, y_out, h->stage_m, h->m);
  }
  CK(cudaStreamSynchronize(h->s));
  const double wall = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
  if (res) {
    for (int64_t b = 0; b < h->count; ++b) {
      const DevState& S = h->hstate[(size_t)b];
      pdlp_result& r = res[b];
      r.status = S.status;
      r.which = S.which;
      r.iters = S.k;
      r.restarts = S.nrestart;
      r.primal_obj = S.out_pobj;
      r.dual_obj = S.out_dobj;
      r.rel_primal = S.out_rel_p;
      r.rel_dual = S.out_rel_d;
      r.rel_gap = S.out_rel_g;
      r.kkt_omega = S.out_kkt;
      r.omega = S.omega;
      r.eta = S.eta;
      r.solve_s = wall;
      r.device_ms = dev_ms;
      r.launches = h->last_launches;
      r.fp32_iters = S.k32;
      r.accepted = S.k;
    }
  }
  if (single) {
    // the handle's state as the launch-per-kernel path leaves it (averages, restart and
    // check counts for pdlp_get_iterate / get_restarts / get_log)
    CK(cudaMemcpy(h->st, h->hstate.data(), sizeof(DevState), cudaMemcpyHostToDevice));
    h->last_ncheck = h->hstate[0].ncheck;
    h->last_nrestart = h->hstate[0].nrestart;
  }
  h->solved = true;
  h->resumable = false;
  return PDLP_OK;
}

}  // namespace pdlp

// ------------------------------------------------------------------ C ABI

extern "C" {

void pdlp_default_params(pdlp_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->tol = 1e-4;
  p->max_iter = 100000000;
  p->time_limit_s = INFINITY;
  p->check_every = 64;
  p->scaling = 0;
  p->beta_suff = 0.2;
  p->beta_nec = 0.8;
  p->beta_art = 0.36;
  p->step_scale = 0.9;
  p->omega_theta = 0.5;
  p->ruiz_iters = 10;
  p->power_iters = 100;
  p->eta = 0.0;
  p->tile_slots = 0;
  p->inputs_on_device = 0;
  p->stream = nullptr;
  p->log_capacity = 4096;
  p->tile_chunks = 0;
  p->spmv_batch = 0;
  p->precision = PDLP_FP64;
  p->mixed_switch_tol = 0.0;
  p->adaptive_reject_cap = 64;
}

int pdlp_setup(pdlp_handle* out, int64_t m, int64_t n, int64_t m1, const int64_t* row_ptr,
               const int32_t* col_idx, const double* val, const double* c, const double* q, const double* l,
               const double* u, const pdlp_params* p) {
  g_setup_error.clear();
  if (!out) {
    g_setup_error = "null output handle";
    return PDLP_EINVAL;
  }
  *out = nullptr;
  pdlp_ctx* h = nullptr;
  try {
    h = new pdlp_ctx();
    if (p) h->p = *p;
    else pdlp_default_params(&h->p);
    setup_impl(h, m, n, m1, row_ptr, col_idx, val, c, q, l, u);
    if (h->p.stream) {
      CK(cudaEventRecord(h->ev_done, h->s));
      CK(cudaStreamWaitEvent((cudaStream_t)h->p.stream, h->ev_done, 0));
    }
  } catch (const Failure& e) {
    g_setup_error = e.msg;
    destroy(h);
    return e.code;
  } catch (const std::bad_alloc&) {
    g_setup_error = "host allocation failed";
    destroy(h);
    return PDLP_ENOMEM;
  } catch (...) {
    g_setup_error = "unexpected internal error";
    destroy(h);
    return PDLP_EINTERNAL;
  }
  *out = h;
  return PDLP_OK;
}

int pdlp_solve(pdlp_handle h, const pdlp_params* p, const double* x0, const double* y0, double omega0,
               pdlp_result* res, double* x_out, double* y_out) {
  return guarded(h, [&]() {
    if (h->is_batch) invalid("batch handle: use pdlp_batch_solve");
    pdlp_params sp = p ? *p : h->p;
    return solve_impl(h, sp, x0, y0, omega0, res, x_out, y_out);
  });
}

// ------------------------------------------------------------------ solve state

namespace pdlp {

// Layout of a saved solve state (host bytes, this build only): the header, the device
// state record, x, y, their running sums, the restart anchor and K x (internal order,
// scaled, padded lengths), then the restart iterations and the per-check records kept.
struct StateHeader {
  char magic[8];
  int64_t version, m, n, npad, mpad, nnz, state_bytes, nrestart, nlog;
};
constexpr char kStateMagic[8] = {'P', 'D', 'L', 'P', 'S', 'T', 'A', 'T'};
constexpr int64_t kStateVersion = 1;

static int64_t state_size(const pdlp_ctx* h, int64_t nrestart, int64_t nlog) {
  return (int64_t)sizeof(StateHeader) + (int64_t)sizeof(DevState) + 8 * (3 * h->npad + 4 * h->mpad) +
         8 * nrestart + (int64_t)sizeof(CheckRecord) * nlog;
}

static void state_counts(const pdlp_ctx* h, int64_t* nrestart, int64_t* nlog) {
  *nrestart = std::min<int64_t>(h->last_nrestart, h->restart_cap);
  *nlog = std::min<int64_t>(h->last_ncheck, h->log_cap);
}

// The vectors of a state in their order in the blob, with their lengths.
static std::vector<std::pair<double*, int64_t>> state_vectors(pdlp_ctx* h) {
  return {{h->x, h->npad}, {h->sx, h->npad}, {h->xa, h->npad}, {h->y, h->mpad},
          {h->sy, h->mpad}, {h->ya, h->mpad}, {h->kxp, h->mpad}};
}

static void load_state(pdlp_ctx* h, const void* state, int64_t size) {
  if (!state || size < (int64_t)sizeof(StateHeader)) invalid("resume: state too small");
  StateHeader hd;
  std::memcpy(&hd, state, sizeof(hd));
  if (std::memcmp(hd.magic, kStateMagic, 8) != 0 || hd.version != kStateVersion)
    invalid("resume: not a solve state of this library");
  if (hd.m != h->m || hd.n != h->n || hd.npad != h->npad || hd.mpad != h->mpad || hd.nnz != h->nnz ||
      hd.state_bytes != (int64_t)sizeof(DevState))
    invalid("resume: the state belongs to an LP of other sizes");
  if (hd.nrestart < 0 || hd.nrestart > h->restart_cap || hd.nlog < 0 || hd.nlog > h->log_cap)
    invalid("resume: restart or log counts out of range for this handle");
  if (size != state_size(h, hd.nrestart, hd.nlog)) invalid("resume: state size does not match its header");
  const char* p = static_cast<const char*>(state) + sizeof(StateHeader);
  CK(cudaMemcpyAsync(h->st, p, sizeof(DevState), cudaMemcpyHostToDevice, h->s));
  p += sizeof(DevState);
  for (auto& v : state_vectors(h)) {
    CK(cudaMemcpyAsync(v.first, p, 8 * (size_t)v.second, cudaMemcpyHostToDevice, h->s));
    p += 8 * v.second;
  }
  if (hd.nrestart > 0) CK(cudaMemcpyAsync(h->restarts, p, 8 * (size_t)hd.nrestart, cudaMemcpyHostToDevice, h->s));
  p += 8 * hd.nrestart;
  if (hd.nlog > 0) CK(cudaMemcpyAsync(h->log, p, sizeof(CheckRecord) * (size_t)hd.nlog, cudaMemcpyHostToDevice, h->s));
  CK(cudaStreamSynchronize(h->s));   // the caller's buffer may be released after return
}

}  // namespace pdlp

int64_t pdlp_state_size(pdlp_handle h) {
  if (!h) return PDLP_EINVAL;
  int64_t out = 0;
  const int rc = guarded(h, [&]() {
    if (h->is_batch) invalid("batch handle");
    if (!h->solved || !h->resumable) invalid("no resumable solve on this handle (FP64, engine 1)");
    int64_t nr = 0, nl = 0;
    state_counts(h, &nr, &nl);
    out = state_size(h, nr, nl);
    return PDLP_OK;
  });
  return rc == PDLP_OK ? out : rc;
}

int pdlp_get_state(pdlp_handle h, void* buf, int64_t size) {
  return guarded(h, [&]() {
    if (h->is_batch) invalid("batch handle");
    if (!h->solved || !h->resumable) invalid("no resumable solve on this handle (FP64, engine 1)");
    int64_t nr = 0, nl = 0;
    state_counts(h, &nr, &nl);
    if (!buf || size != state_size(h, nr, nl)) invalid("buffer size must be pdlp_state_size(h)");
    StateHeader hd;
    std::memcpy(hd.magic, kStateMagic, 8);
    hd.version = kStateVersion;
    hd.m = h->m;
    hd.n = h->n;
    hd.npad = h->npad;
    hd.mpad = h->mpad;
    hd.nnz = h->nnz;
    hd.state_bytes = (int64_t)sizeof(DevState);
    hd.nrestart = nr;
    hd.nlog = nl;
    char* p = static_cast<char*>(buf);
    std::memcpy(p, &hd, sizeof(hd));
    p += sizeof(hd);
    CK(cudaMemcpyAsync(p, h->st, sizeof(DevState), cudaMemcpyDeviceToHost, h->s));
    p += sizeof(DevState);
    for (auto& v : state_vectors(h)) {
      CK(cudaMemcpyAsync(p, v.first, 8 * (size_t)v.second, cudaMemcpyDeviceToHost, h->s));
      p += 8 * v.second;
    }
    if (nr > 0) CK(cudaMemcpyAsync(p, h->restarts, 8 * (size_t)nr, cudaMemcpyDeviceToHost, h->s));
    p += 8 * nr;
    if (nl > 0) CK(cudaMemcpyAsync(p, h->log, sizeof(CheckRecord) * (size_t)nl, cudaMemcpyDeviceToHost, h->s));
    CK(cudaStreamSynchronize(h->s));
    return PDLP_OK;
  });
}

int pdlp_solve_resume(pdlp_handle h, const pdlp_params* p, const void* state, int64_t size, pdlp_result* res,
                      double* x_out, double* y_out) {
  return guarded(h, [&]() {
    if (h->is_batch) invalid("batch handle");
    pdlp_params sp = p ? *p : h->p;
    if (sp.engine == 2) invalid("resume runs the kernels per iteration (engine 0 or 1)");
    if (h->p.precision != PDLP_FP64) invalid("resume: FP64 handles only");
    if (state) {
      load_state(h, state, size);
    } else if (!h->solved || !h->resumable) {
      invalid("no resumable solve on this handle (FP64, engine 1) and no state given");
    }
    return solve_impl(h, sp, nullptr, nullptr, 0.0, res, x_out, y_out, true);
  });
}

void pdlp_free(pdlp_handle h) {
  if (!h) return;
  DeviceGuard dg(h->dev);
  destroy(h);
}

const char* pdlp_last_error(pdlp_handle h) {
  if (!h) return g_setup_error.c_str();
  return h->err.c_str();
}

int pdlp_get_iterate(pdlp_handle h, int32_t which, double* x, double* y) {
  return guarded(h, [&]() {
    if (h->is_batch) invalid("batch handle: use pdlp_batch_solve outputs");
    if (which < 0 || which > 2) invalid("which must be 0, 1 or 2");
    if (!h->solved) invalid("no solve has run on this handle");
    const double* xi = h->x;
    const double* yi = h->y;
    if (which == 1) {
      k_average<<<grid_for(h->npad), 256, 0, h->s>>>(h->tn, h->sx, h->x, h->st, h->npad);
      k_average<<<grid_for(h->mpad), 256, 0, h->s>>>(h->tm, h->sy, h->y, h->st, h->mpad);
      xi = h->tn;
      yi = h->tm;
    } else if (which == 2) {
      xi = h->xa;
      yi = h->ya;
    }
    export_point(h, xi, yi, x, y);
    return PDLP_OK;
  });
}

int64_t pdlp_get_restarts(pdlp_handle h, int64_t* iters, int64_t cap) {
  return guarded(h, [&]() -> int {
    int64_t nr = h->solved ? h->last_nrestart : 0;
    int64_t k = std::min<int64_t>({nr, cap, (int64_t)h->restart_cap});
    if (iters && k > 0) CK(cudaMemcpy(iters, h->restarts, sizeof(long long) * k, cudaMemcpyDeviceToHost));
    return (int)nr;
  });
}

int64_t pdlp_get_log(pdlp_handle h, pdlp_check_record* rec, int64_t cap) {
  static_assert(sizeof(pdlp_check_record) == sizeof(CheckRecord), "record layout");
  return guarded(h, [&]() -> int {
    int64_t nc = h->solved ? h->last_ncheck : 0;
    int64_t k = std::min<int64_t>({nc, cap, (int64_t)h->log_cap});
    if (rec && k > 0) CK(cudaMemcpy(rec, h->log, sizeof(CheckRecord) * k, cudaMemcpyDeviceToHost));
    return (int)nc;
  });
}

int pdlp_spmv(pdlp_handle h, int32_t transpose, const double* in, double* out) {
  return guarded(h, [&]() {
    if (!in || !out) invalid("null vector");
    if (!transpose) {
      copy_in(h, h->stage_n, in, h->n);
      k_permute_in<<<grid_for(h->npad), 256, 0, h->s>>>(h->tn, h->stage_n, h->perm_c, h->Dc, h->npad, 0.0);
      launch_rows<OpSpmv>(h, h->K, h->tn, EpiStore{h->tm, 0, 1.0}, nullptr);
      if (h->m > 0) {
        k_unpermute_scale<<<grid_for(h->m), 256, 0, h->s>>>(h->stage_m, h->tm, h->invDr, h->pos_r, h->m);
        copy_out(h, out, h->stage_m, h->m);
      }
    } else {
      if (h->m > 0) copy_in(h, h->stage_m, in, h->m);
      k_permute_in<<<grid_for(h->mpad), 256, 0, h->s>>>(h->tm, h->stage_m, h->perm_r, h->Dr, h->mpad, 0.0);
      launch_rows<OpSpmv>(h, h->Kt, h->tm, EpiStore{h->tn, 0, 1.0}, nullptr);
      k_unpermute_scale<<<grid_for(h->n), 256, 0, h->s>>>(h->stage_n, h->tn, h->invDc, h->pos_c, h->n);
      copy_out(h, out, h->stage_n, h->n);
    }
    CKL("pdlp_spmv");
    CK(cudaStreamSynchronize(h->s));
    check_stage_err(h);
    return PDLP_OK;
  });
}

int pdlp_bound_duals(pdlp_handle h, const double* y, double* lambda_out) {
  return guarded(h, [&]() {
    if (h->is_batch) invalid("batch handle");
    if (!lambda_out || (h->m > 0 && !y)) invalid("null array");
    if (h->m > 0) copy_in(h, h->stage_m, y, h->m);
    k_permute_in<<<grid_for(h->mpad), 256, 0, h->s>>>(h->tm, h->stage_m, h->perm_r, h->Dr, h->mpad, 0.0);
    launch_rows<OpSpmv>(h, h->Kt, h->tm, EpiStore{h->g_a, 0, 1.0}, nullptr);
    k_bound_duals<<<grid_for(h->npad), 256, 0, h->s>>>(h->tn, h->c, h->g_a, h->l, h->u, h->npad);
    k_unpermute_scale<<<grid_for(h->n), 256, 0, h->s>>>(h->stage_n, h->tn, h->invDc, h->pos_c, h->n);
    copy_out(h, lambda_out, h->stage_n, h->n);
    CK(cudaStreamSynchronize(h->s));
    check_stage_err(h);
    return PDLP_OK;
  });
}

int pdlp_get_info(pdlp_handle h, pdlp_info* info) {
  return guarded(h, [&]() {
    if (!info) invalid("null info");
    std::memset(info, 0, sizeof(*info));
    info->m = h->m;
    info->n = h->n;
    info->m1 = h->m1;
    info->nnz = h->nnz;
    info->slots_K = h->K.slots;
    info->slots_Kt = h->Kt.slots;
    info->tasks_K = h->K.ntasks;
    info->tasks_Kt = h->Kt.ntasks;
    info->split_chunks_K = h->K.split;
    info->split_chunks_Kt = h->Kt.split;
    info->tile_slots_K = h->K.tile;
    info->tile_slots_Kt = h->Kt.tile;
    info->tile_chunks_K = h->K.tchunks;
    info->tile_chunks_Kt = h->Kt.tchunks;
    info->spmv_batch_K = h->K.batch;
    info->spmv_batch_Kt = h->Kt.batch;
    info->algorithmic_bytes_per_iter = 24.0 * h->nnz + 68.0 * (h->m + h->n);
    info->stored_bytes_per_iter = 12.0 * 32.0 * (h->K.slots + h->Kt.slots) + 68.0 * (h->mpad + h->npad);
    info->eta = h->eta;
    info->omega0 = h->omega0;
    info->norm_K = h->normK;
    info->batch_team = h->last_team;
    info->batch_resident = h->last_glob ? 3 : (h->last_resident ? 1 : 0);
    info->wide_rows_K = h->K.nwide;
    info->batch_resumed = (int32_t)h->last_resumed;
    info->setup_validate_ms = h->setup_ms[0];
    info->setup_layout_ms = h->setup_ms[1];
    info->setup_device_ms = h->setup_ms[2];
    info->setup_tune_ms = h->setup_ms[3];
    info->setup_step_ms = h->setup_ms[4];
    info->spmv_stage_K = h->K.staged + 1;
    info->batch_tuned = h->last_tuned ? h->tune_candidates : 0;
    for (int i = 0; i < 8 && i < h->tune_candidates; ++i) {
      info->tune_team[i] = h->tune_team[i];
      info->tune_resident[i] = h->tune_res[i];
      info->tune_gbs[i] = h->tune_rates[i];
    }
    info->spmv_stage_Kt = h->Kt.staged + 1;
    info->mixed_values = h->mixed_values;
    return PDLP_OK;
  });
}

int64_t pdlp_batch_get_restarts(pdlp_handle h, int64_t lp, int64_t* iters, int64_t cap) {
  return guarded(h, [&]() -> int {
    if (!h->is_batch) invalid("single-LP handle: use pdlp_get_restarts");
    if (lp < 0 || lp >= h->count) invalid("lp out of range");
    if (!h->solved) invalid("no solve has run on this handle");
    const int64_t nr = h->hstate[(size_t)lp].nrestart;
    const int64_t k = std::min<int64_t>({nr, cap, kBatchRestartCap});
    if (iters && k > 0)
      CK(cudaMemcpy(iters, h->brestarts + (size_t)lp * kBatchRestartCap, sizeof(long long) * k,
                    cudaMemcpyDeviceToHost));
    return (int)nr;
  });
}

int pdlp_time_iterations(pdlp_handle h, int64_t iters, double* ms_primal, double* ms_dual) {
  return guarded(h, [&]() {
    if (h->is_batch) invalid("batch handle");
    if (iters < 1) invalid("iters must be >= 1");
    if (!h->solved) invalid("no solve has run on this handle");
    k_copy_state<<<1, 1, 0, h->s>>>(h->st_tmp, h->st);
    const int64_t chunk = 512;
    while ((int64_t)h->timing_events.size() < 2 * chunk + 1) {
      cudaEvent_t e;
      CK(cudaEventCreate(&e));
      h->timing_events.push_back(e);
    }
    double tp = 0.0, td = 0.0;
    for (int64_t done = 0; done < iters; done += chunk) {
      const int64_t cnt = std::min(chunk, iters - done);
      auto& ev = h->timing_events;
      CK(cudaEventRecord(ev[0], h->s));
      for (int64_t i = 0; i < cnt; ++i) {
        if (h->p.precision == PDLP_MIXED)
          launch_primal32(h, h->st_tmp);
        else
          launch_rows<OpSpmv>(h, h->Kt, h->y, EpiPrimal{h->x, h->sx, h->c, h->l, h->u, 0.0}, h->st_tmp);
        CK(cudaEventRecord(ev[2 * i + 1], h->s));
        if (h->p.precision == PDLP_MIXED)
          launch_dual32(h, h->st_tmp);
        else
          launch_rows<OpSpmv>(h, h->K, h->x, EpiDual{h->y, h->sy, h->kxp, h->q, (int)h->m1_int, 0.0}, h->st_tmp);
        CK(cudaEventRecord(ev[2 * i + 2], h->s));
      }
      CKL("timed iterations");
      CK(cudaStreamSynchronize(h->s));
      for (int64_t i = 0; i < cnt; ++i) {
        float a = 0.f, b = 0.f;
        CK(cudaEventElapsedTime(&a, ev[2 * i], ev[2 * i + 1]));
        CK(cudaEventElapsedTime(&b, ev[2 * i + 1], ev[2 * i + 2]));
        tp += a;
        td += b;
      }
    }
    check_stage_err(h);
    if (ms_primal) *ms_primal = tp / (double)iters;
    if (ms_dual) *ms_dual = td / (double)iters;
    return PDLP_OK;
  });
}

int pdlp_batch_setup(pdlp_handle* out, int64_t count, const int64_t* m, const int64_t* n, const int64_t* m1,
                     const int64_t* row_ptr, const int32_t* col_idx, const double* val, const double* c,
                     const double* q, const double* l, const double* u, const pdlp_params* p) {
  g_setup_error.clear();
  if (!out) {
    g_setup_error = "null output handle";
    return PDLP_EINVAL;
  }
  *out = nullptr;
  pdlp_ctx* h = nullptr;
  try {
    h = new pdlp_ctx();
    if (p) h->p = *p;
    else pdlp_default_params(&h->p);
    batch_setup_impl(h, count, m, n, m1, row_ptr, col_idx, val, c, q, l, u);
    if (h->p.stream) {
      CK(cudaEventRecord(h->ev_done, h->s));
      CK(cudaStreamWaitEvent((cudaStream_t)h->p.stream, h->ev_done, 0));
    }
  } catch (const Failure& e) {
    g_setup_error = e.msg;
    destroy(h);
    return e.code;
  } catch (const std::bad_alloc&) {
    g_setup_error = "host allocation failed";
    destroy(h);
    return PDLP_ENOMEM;
  } catch (...) {
    g_setup_error = "unexpected internal error";
    destroy(h);
    return PDLP_EINTERNAL;
  }
  *out = h;
  return PDLP_OK;
}

int pdlp_batch_solve(pdlp_handle h, const pdlp_params* p, const double* x0, const double* y0, const double* omega0,
                     pdlp_result* res, double* x_out, double* y_out) {
  return guarded(h, [&]() {
    if (!h->is_batch) invalid("not a batch handle (use pdlp_solve)");
    pdlp_params sp = p ? *p : h->p;
    return batch_solve_impl(h, sp, x0, y0, omega0, res, x_out, y_out, false, 0.0);
  });
}

}  // extern "C"
