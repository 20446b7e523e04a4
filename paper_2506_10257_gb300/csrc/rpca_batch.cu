// rpca_batch.cu -- batched persistent form: many independent windows of uneven
// pixel and frame counts solved in one cooperative launch (captured in a CUDA
// graph), with the CTA schedule chosen by a measuring autotuner.
//
// Schedule.  The grid holds every CTA the GPU can keep resident.  It is cut
// into lanes (contiguous CTA ranges); each lane runs its windows one after the
// other, all of the lane's CTAs sweeping the pixels of the current window.
// Windows go to lanes by longest-processing-time first on their per-iteration
// bytes (5 m T floats, the dominant cost), and each lane gets a CTA count
// proportional to (its load)^alpha.  The number of lanes, alpha and the CTAs
// per SM are the tuned parameters: the autotuner times every candidate on the
// caller's own windows and keeps the fastest, cached per batch signature
// (the sorted window shapes and the SM count) for the life of the process.
#include <cuda_runtime.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <numeric>
#include <string>
#include <vector>

#include "rpca_kernels.cuh"
#include "rpca_internal.h"
#include "rpca_wide.cuh"

namespace rpca {
#include "rpca_batch.cuh"

// The wide / complex batch kernel (rpca_batch_wide.cu).
void* batch_wide_kernel_fn(bool cplx);
// The tensor-core batch kernel for windows of <= tbmax frames (rpca_batch_tc.cu).
void batch_tc_kernel_info(int tbmax, bool bf16, void** fn, size_t* smem);
}  // namespace rpca

using namespace rpca;

namespace {

struct BatchConfig {
  int lanes;        // CTA ranges (<= windows)
  double alpha;     // lane CTAs ~ load^alpha
  int ctas_per_sm;  // resident CTAs per SM used by the grid
  int paired;       // lanes of >= 2 windows run them two at a time beside an eigen-step CTA
};

bool operator==(const BatchConfig& a, const BatchConfig& b) {
  return a.lanes == b.lanes && a.alpha == b.alpha && a.ctas_per_sm == b.ctas_per_sm && a.paired == b.paired;
}

std::mutex g_tune_mu;
std::map<std::string, BatchConfig> g_tune_cache;

int bucket_tb(int T) {
  if (T <= 8) return 8;
  if (T <= 12) return 12;
  if (T <= 16) return 16;
  if (T <= 20) return 20;
  if (T <= 24) return 24;
  return 32;
}

struct KernelInfo {
  void* fn;
  size_t smem;
};

// Columns per warp of the tiled pass for T real columns.
int wide_cw(int Tr) { return (Tr + 31) / 32 * 32 / 8; }

KernelInfo batch_kernel_for(int tbmax) {
  if (tbmax <= 20) return {(void*)batch_kernel<20>, batch_smem<20>()};
  return {(void*)batch_kernel<32>, batch_smem<32>()};
}

rpca_status cuda_st(cudaError_t e) {
  if (e == cudaSuccess) return RPCA_OK;
  if (e == cudaErrorMemoryAllocation) return RPCA_ERR_NOMEM;
  return RPCA_ERR_CUDA;
}

}  // namespace

struct rpca_batch_s {
  int n = 0;
  std::vector<rpca_params> p;
  std::vector<rpca_plan_t> plans;
  std::vector<PlanView> views;
  KernelInfo kern{};
  bool wide = false;           // every window runs the tiled bodies
  int vrows = 16;              // wide eigen-steps: rows of V staged per step
  int sms = 0;
  int occ_max = 0;       // resident batch CTAs per SM the kernel allows
  BatchConfig cfg{};
  std::string signature;
  int grid = 0;
  int nlanes = 0;
  std::vector<LaneDesc> lanes;
  std::vector<int> slot_win;   // window index of each descriptor slot
  std::vector<int> win_slot;   // descriptor slot of each window
  std::vector<int> win_ncta;   // CTAs each window uses
  BatchDesc* h_desc = nullptr;  // pinned
  BatchDesc* d_desc = nullptr;
  Ctrl* h_ctrl = nullptr;       // pinned [n]
  Ctrl* d_ctrl = nullptr;       // [n]
  size_t desc_bytes = 0;        // descriptor prefix copied per solve
  unsigned long long spin_limit = 4000000ull;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  bool use_graph = true;
  cudaEvent_t last = nullptr;   // end of the last launch (guards h_desc reuse)
  bool pending = false;
  // host-buffer form: two device staging sets (call parity), copy streams
  struct Stage {
    std::vector<void*> X, L, S;
    std::vector<uint8_t*> M;
    cudaEvent_t solved = nullptr, down = nullptr;
    bool used = false;
  };
  Stage stage[2];
  cudaStream_t s_up = nullptr, s_dn = nullptr;
  cudaEvent_t up_done = nullptr;
  long long host_calls = 0;
};

namespace {

double window_load(const rpca_params& p) { return (double)p.m * (double)p.T; }

// The lanes of a schedule: the windows each lane runs, in order, and its CTAs.
struct LanePlan {
  std::vector<std::vector<int>> lw;
  std::vector<int> nc;
};

// Windows go to lanes by longest-processing-time first on wload (equal loads
// keep their index order); lane CTAs ~ (lane load)^alpha, at least one, at
// most the largest wcap of the lane's windows, summing to at most C, the
// fractional shares settled by largest remainders.  L = min(lanes, n, C).
LanePlan plan_lanes(const std::vector<double>& wload, const std::vector<int>& wcap, int C, int lanes,
                    double alpha) {
  const int n = (int)wload.size();
  const int L = std::max(1, std::min({lanes, n, C}));
  std::vector<int> order(n);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return wload[a] > wload[c]; });
  std::vector<double> load(L, 0.0);
  std::vector<std::vector<int>> lw(L);
  for (int w : order) {
    int best = 0;
    for (int l = 1; l < L; ++l)
      if (load[l] < load[best]) best = l;
    load[best] += wload[w];
    lw[best].push_back(w);
  }
  // useful CTAs of a lane: its largest window's partial capacity
  std::vector<int> cap(L, 1);
  for (int l = 0; l < L; ++l)
    for (int w : lw[l]) cap[l] = std::max(cap[l], wcap[w]);
  // CTAs ~ load^alpha, at least one, at most cap, summing to <= C
  std::vector<int> nc(L, 1);
  int left = C - L;
  std::vector<double> wgt(L);
  for (int l = 0; l < L; ++l) wgt[l] = pow(std::max(load[l], 1.0), alpha);
  for (int pass = 0; pass < 4 && left > 0; ++pass) {
    double tot = 0;
    for (int l = 0; l < L; ++l)
      if (nc[l] < cap[l]) tot += wgt[l];
    if (tot <= 0) break;
    int given = 0;
    std::vector<double> frac(L, 0.0);
    for (int l = 0; l < L; ++l) {
      if (nc[l] >= cap[l]) continue;
      const double want = left * wgt[l] / tot;
      int add = std::min((int)floor(want), cap[l] - nc[l]);
      nc[l] += add;
      given += add;
      frac[l] = want - floor(want);
    }
    left -= given;
    // largest remainders
    std::vector<int> idx(L);
    std::iota(idx.begin(), idx.end(), 0);
    std::stable_sort(idx.begin(), idx.end(), [&](int a, int c) { return frac[a] > frac[c]; });
    for (int l : idx) {
      if (left <= 0) break;
      if (nc[l] < cap[l] && frac[l] > 0) {
        nc[l] += 1;
        left -= 1;
      }
    }
    if (given == 0) break;
  }
  return {std::move(lw), std::move(nc)};
}

// Lanes, their CTAs and the window order for configuration cfg.
void make_schedule(rpca_batch_s* b, const BatchConfig& cfg) {
  const int n = b->n;
  const int C = b->sms * cfg.ctas_per_sm;
  std::vector<double> wload(n);
  std::vector<int> wcap(n);
  for (int w = 0; w < n; ++w) {
    wload[w] = window_load(b->p[w]);
    // a paired lane's last CTA runs the eigen-steps beside the pass CTAs
    wcap[w] = b->views[w].max_grid + (cfg.paired ? 1 : 0);
  }
  const LanePlan lp = plan_lanes(wload, wcap, C, cfg.lanes, cfg.alpha);
  const int L = (int)lp.nc.size();
  const std::vector<std::vector<int>>& lw = lp.lw;
  const std::vector<int>& nc = lp.nc;
  b->lanes.assign(L, LaneDesc{});
  b->slot_win.clear();
  b->win_slot.assign(n, 0);
  b->win_ncta.assign(n, 1);
  int cta = 0;
  for (int l = 0; l < L; ++l) {
    LaneDesc& d = b->lanes[l];
    d.cta0 = cta;
    d.ncta = nc[l];
    d.w0 = (int)b->slot_win.size();
    d.w1 = d.w0 + (int)lw[l].size();
    const int pass_ctas = lane_is_paired(cfg.paired, d) ? nc[l] - 1 : nc[l];
    for (int w : lw[l]) {
      b->win_slot[w] = (int)b->slot_win.size();
      b->slot_win.push_back(w);
      const int64_t tiles = (b->p[w].m + b->views[w].tile - 1) / b->views[w].tile;
      b->win_ncta[w] =
          (int)std::max<int64_t>(1, std::min<int64_t>({(int64_t)pass_ctas, tiles, b->views[w].max_grid}));
    }
    cta += nc[l];
  }
  b->grid = cta;
  b->nlanes = L;
  b->cfg = cfg;
}

void drop_graph(rpca_batch_s* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
}

cudaError_t launch_batch(rpca_batch_s* b, cudaStream_t s) {
  cudaLaunchConfig_t lc;
  memset(&lc, 0, sizeof(lc));
  lc.gridDim = dim3((unsigned)b->grid);
  lc.blockDim = dim3(kBatchThreads);
  lc.dynamicSmemBytes = b->kern.smem;
  lc.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  lc.attrs = attr;
  lc.numAttrs = 1;
  void* args[] = {&b->d_desc};
  cudaError_t e = cudaLaunchKernelExC(&lc, b->kern.fn, args);
  if (e != cudaSuccess) return e;
  void* gargs[] = {&b->d_desc, &b->d_ctrl};
  return cudaLaunchKernel((void*)batch_gather_ctrl, dim3((unsigned)b->n), dim3(64), gargs, 0, s);
}

// One solve's work on stream s: descriptor upload, the persistent launch,
// the control-block gather.
cudaError_t enqueue(rpca_batch_s* b, cudaStream_t s) {
  cudaError_t e = cudaMemcpyAsync(b->d_desc, b->h_desc, b->desc_bytes, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = launch_batch(b, s);
  return e;
}

// Captures enqueue() into a graph (once per schedule); on any capture error
// the batch launches its kernels directly instead.
void ensure_graph(rpca_batch_s* b, cudaStream_t s) {
  if (!b->use_graph || b->exec) return;
  cudaStream_t cs = nullptr;
  if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
    b->use_graph = false;
    return;
  }
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    cudaError_t e2 = enqueue(b, cs);
    e = cudaStreamEndCapture(cs, &g);
    if (e2 != cudaSuccess) e = e2;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, g, 0);
  if (e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    b->exec = nullptr;
    b->use_graph = false;
    cudaGetLastError();
  } else {
    b->graph = g;
  }
  cudaStreamDestroy(cs);
  (void)s;
}

// Fixed part of the descriptor (lanes, window buffers); pointers per solve.
void write_static_desc(rpca_batch_s* b) {
  BatchDesc* d = b->h_desc;
  d->nwin = b->n;
  d->nlanes = b->nlanes;
  d->paired = b->cfg.paired;
  d->spin_limit = b->spin_limit;
  d->vrows = b->vrows;
  for (int l = 0; l < b->nlanes; ++l) d->lane[l] = b->lanes[l];
  for (int slot = 0; slot < b->n; ++slot) {
    const int w = b->slot_win[slot];
    WinDesc& wd = d->w[slot];
    memset(&wd, 0, sizeof(wd));
    wd.b = b->views[w].bufs;
    wd.b.finalize = 1;
    wd.b.grid = b->win_ncta[w];
    wd.b.ngroups = (b->win_ncta[w] + kGroup - 1) / kGroup;
    wd.TB = b->wide ? wide_cw(b->views[w].T) : bucket_tb(b->p[w].T);
  }
}

rpca_status wait_last(rpca_batch_s* b) {
  if (!b->pending) return RPCA_OK;
  cudaError_t e = cudaEventSynchronize(b->last);
  b->pending = false;
  return cuda_st(e);
}

rpca_status apply_config(rpca_batch_s* b, const BatchConfig& cfg) {
  rpca_status st = wait_last(b);
  if (st != RPCA_OK) return st;
  make_schedule(b, cfg);
  drop_graph(b);
  b->use_graph = true;
  write_static_desc(b);
  return RPCA_OK;
}

std::string make_signature(const rpca_batch_s* b) {
  std::vector<std::string> parts;
  for (const rpca_params& p : b->p)
    parts.push_back(std::to_string(p.m) + "x" + std::to_string(p.T) + "d" + std::to_string((int)p.dtype));
  std::sort(parts.begin(), parts.end());
  // the kernel (its precision, tiled or not) and its residency enter too: a
  // schedule tuned for one kernel is not valid for another
  std::string s = "sms" + std::to_string(b->sms) + "p" + std::to_string((int)b->p[0].precision) + "w" +
                  std::to_string((int)b->wide) + "o" + std::to_string(b->occ_max);
  for (auto& x : parts) s += "," + x;
  return s;
}

// Default: lanes of two windows each, run paired beside an eigen-step CTA
// (one window alone when the batch has one).
BatchConfig default_config(const rpca_batch_s* b) {
  BatchConfig c;
  c.ctas_per_sm = b->occ_max;
  c.paired = b->n >= 2 ? 1 : 0;
  c.lanes = std::min(c.paired ? (b->n + 1) / 2 : b->n, b->sms * c.ctas_per_sm);
  c.alpha = 1.0;
  return c;
}

}  // namespace

extern "C" {

rpca_status rpca_batch_create(const rpca_params* params, int32_t n, rpca_batch_t* out) {
  if (!params || !out || n < 1) return RPCA_ERR_ARG;
  *out = nullptr;
  if (n > kMaxBatch) return RPCA_ERR_UNSUPPORTED;
  bool wide = false;
  const int prec = params[0].precision;
  for (int i = 0; i < n; ++i) {
    if (params[i].precision != prec) return RPCA_ERR_UNSUPPORTED;  // one precision per batch
    if (params[i].warm_start) return RPCA_ERR_UNSUPPORTED;        // windows of a batch start cold
    if (params[i].dtype != params[0].dtype) return RPCA_ERR_UNSUPPORTED;  // one element type per batch
    if (params[i].T > kMaxT || params[i].dtype == RPCA_C64) wide = true;
  }
  if (prec != RPCA_PREC_FP32 && prec != RPCA_PREC_TF32X3 && prec != RPCA_PREC_BF16X3) return RPCA_ERR_UNSUPPORTED;
  // tensor-core batches: real windows of <= 32 frames (the narrow tensor-core pass)
  if (prec != RPCA_PREC_FP32 && wide) return RPCA_ERR_UNSUPPORTED;
  rpca_batch_s* b = new rpca_batch_s();
  b->n = n;
  b->p.assign(params, params + n);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev);
  int coop = 0;
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
  if (e != cudaSuccess || !coop) {
    delete b;
    return e != cudaSuccess ? cuda_st(e) : RPCA_ERR_UNSUPPORTED;
  }
  b->wide = wide;
  if (!wide) {
    int tbmax = 8;
    for (int i = 0; i < n; ++i) tbmax = std::max(tbmax, bucket_tb(params[i].T));
    if (prec == RPCA_PREC_FP32)
      b->kern = batch_kernel_for(tbmax);
    else
      batch_tc_kernel_info(tbmax, prec == RPCA_PREC_BF16X3, &b->kern.fn, &b->kern.smem);
  } else {
    // shared memory: the largest tiled pass or eigen-step of the batch, with
    // as many staged V rows (<= 16) as the SM leaves room for
    const bool cplx = params[0].dtype == RPCA_C64;
    b->kern.fn = batch_wide_kernel_fn(cplx);
    cudaFuncAttributes fa;
    int optin = 0;
    e = cudaFuncGetAttributes(&fa, b->kern.fn);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) {
      delete b;
      return cuda_st(e);
    }
    const size_t room = (size_t)optin > fa.sharedSizeBytes ? (size_t)optin - fa.sharedSizeBytes : 0;
    size_t need = 0;
    for (int vr = 16; vr >= 1; --vr) {
      need = 0;
      for (int i = 0; i < n; ++i) {
        const int Tr = params[i].dtype == RPCA_C64 ? 2 * params[i].T : params[i].T;
        need = std::max({need, wide_pass_smem_bytes(wide_cw(Tr)), eig_wide_smem(Tr, vr)});
      }
      b->vrows = vr;
      if (need <= room) break;
    }
    if (need > room) {
      delete b;
      return RPCA_ERR_UNSUPPORTED;
    }
    b->kern.smem = need;
  }
  e = cudaFuncSetAttribute(b->kern.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->kern.smem);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b->occ_max, b->kern.fn, kBatchThreads, b->kern.smem);
  if (e != cudaSuccess || b->occ_max < 1) {
    delete b;
    return e != cudaSuccess ? cuda_st(e) : RPCA_ERR_UNSUPPORTED;
  }
  rpca_status st = RPCA_OK;
  for (int i = 0; i < n && st == RPCA_OK; ++i) {
    rpca_params q = params[i];
    q.drive = RPCA_DRIVE_STREAM;  // the batch drives the kernels itself
    rpca_plan_t pl = nullptr;
    st = plan_create_ex(&q, wide, &pl);
    if (st == RPCA_OK) {
      b->plans.push_back(pl);
      PlanView v;
      plan_view(pl, &v);
      b->views.push_back(v);
    }
  }
  if (st == RPCA_OK) {
    e = cudaMallocHost((void**)&b->h_desc, sizeof(BatchDesc));
    if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_desc, sizeof(BatchDesc));
    if (e == cudaSuccess) e = cudaMallocHost((void**)&b->h_ctrl, sizeof(Ctrl) * n);
    if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_ctrl, sizeof(Ctrl) * n);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->last, cudaEventDisableTiming);
    st = cuda_st(e);
  }
  if (st != RPCA_OK) {
    rpca_batch_destroy(b);
    return st;
  }
  memset(b->h_desc, 0, sizeof(BatchDesc));
  b->desc_bytes = offsetof(BatchDesc, w) + sizeof(WinDesc) * (size_t)n;
  b->signature = make_signature(b);
  BatchConfig cfg = default_config(b);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_cache.find(b->signature);
    if (it != g_tune_cache.end()) cfg = it->second;
  }
  apply_config(b, cfg);
  *out = b;
  return RPCA_OK;
}

rpca_status rpca_batch_solve(rpca_batch_t b, const rpca_window* win, void* stream, rpca_result* out) {
  if (!b || !win) return RPCA_ERR_ARG;
  for (int i = 0; i < b->n; ++i) {
    const rpca_window& w = win[i];
    if (!w.X || !w.L || !w.S) return RPCA_ERR_ARG;
    if (((uintptr_t)w.X | (uintptr_t)w.L | (uintptr_t)w.S) & 15u) return RPCA_ERR_ARG;
    if (w.X == w.L || w.X == w.S || w.L == w.S) return RPCA_ERR_ARG;
  }
  rpca_status st = wait_last(b);
  if (st != RPCA_OK) return st;
  for (int i = 0; i < b->n; ++i) {
    WinDesc& wd = b->h_desc->w[b->win_slot[i]];
    wd.X = (const float*)win[i].X;
    wd.L = (float*)win[i].L;
    wd.S = (float*)win[i].S;
    wd.mask = win[i].mask;
    wd.theta = win[i].theta;
    wd.gen = 0u;
    wd.pdone = 0u;
  }
  cudaStream_t s = (cudaStream_t)stream;
  ensure_graph(b, s);
  cudaError_t e = b->exec ? cudaGraphLaunch(b->exec, s) : enqueue(b, s);
  if (e == cudaSuccess) e = cudaEventRecord(b->last, s);
  if (e != cudaSuccess) return cuda_st(e);
  b->pending = true;
  if (!out) return RPCA_OK;
  e = cudaMemcpyAsync(b->h_ctrl, b->d_ctrl, sizeof(Ctrl) * b->n, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_st(e);
  b->pending = false;
  int worst = RPCA_OK;
  for (int i = 0; i < b->n; ++i) {
    result_from_ctrl(b->views[i].lambda, b->h_ctrl[b->win_slot[i]], &out[i], b->views[i].cplx);
    if (out[i].status < 0) worst = out[i].status;
    else if (worst == RPCA_OK && out[i].status != RPCA_OK) worst = out[i].status;
  }
  return (rpca_status)worst;
}

// Bytes of one window's X (and of L, S) in the batch.
static size_t window_bytes(const rpca_params& p) {
  return sizeof(float) * (size_t)p.m * (size_t)(p.dtype == RPCA_C64 ? 2 * p.T : p.T);
}

// Staging sets, copy streams and events of the host-buffer form (first call).
static rpca_status host_stage_init(rpca_batch_t b) {
  if (b->s_up) return RPCA_OK;
  cudaError_t e = cudaStreamCreateWithFlags(&b->s_up, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->s_dn, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->up_done, cudaEventDisableTiming);
  for (int j = 0; j < 2 && e == cudaSuccess; ++j) {
    rpca_batch_s::Stage& st = b->stage[j];
    e = cudaEventCreateWithFlags(&st.solved, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&st.down, cudaEventDisableTiming);
    st.X.assign(b->n, nullptr);
    st.L.assign(b->n, nullptr);
    st.S.assign(b->n, nullptr);
    st.M.assign(b->n, nullptr);
    for (int i = 0; i < b->n && e == cudaSuccess; ++i) {
      const size_t nb = window_bytes(b->p[i]);
      e = cudaMalloc(&st.X[i], nb);
      if (e == cudaSuccess) e = cudaMalloc(&st.L[i], nb);
      if (e == cudaSuccess) e = cudaMalloc(&st.S[i], nb);
      if (e == cudaSuccess) e = cudaMalloc((void**)&st.M[i], (size_t)b->p[i].m);
    }
  }
  return cuda_st(e);
}

static void host_stage_free(rpca_batch_t b) {
  if (b->s_up) cudaStreamSynchronize(b->s_up);
  if (b->s_dn) cudaStreamSynchronize(b->s_dn);
  for (int j = 0; j < 2; ++j) {
    rpca_batch_s::Stage& st = b->stage[j];
    for (void* p : st.X) if (p) cudaFree(p);
    for (void* p : st.L) if (p) cudaFree(p);
    for (void* p : st.S) if (p) cudaFree(p);
    for (uint8_t* p : st.M) if (p) cudaFree(p);
    if (st.solved) cudaEventDestroy(st.solved);
    if (st.down) cudaEventDestroy(st.down);
  }
  if (b->up_done) cudaEventDestroy(b->up_done);
  if (b->s_up) cudaStreamDestroy(b->s_up);
  if (b->s_dn) cudaStreamDestroy(b->s_dn);
}

rpca_status rpca_batch_solve_host(rpca_batch_t b, const rpca_window* win, void* stream, rpca_result* out) {
  if (!b || !win) return RPCA_ERR_ARG;
  for (int i = 0; i < b->n; ++i)
    if (!win[i].X || !win[i].L || !win[i].S) return RPCA_ERR_ARG;
  rpca_status st = host_stage_init(b);
  if (st != RPCA_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  const int j = (int)(b->host_calls & 1);
  rpca_batch_s::Stage& sg = b->stage[j];
  // uploads into this set once the downloads of the call two before have landed
  cudaError_t e = sg.used ? cudaStreamWaitEvent(b->s_up, sg.down, 0) : cudaSuccess;
  for (int i = 0; i < b->n && e == cudaSuccess; ++i)
    e = cudaMemcpyAsync(sg.X[i], win[i].X, window_bytes(b->p[i]), cudaMemcpyHostToDevice, b->s_up);
  if (e == cudaSuccess) e = cudaEventRecord(b->up_done, b->s_up);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(s, b->up_done, 0);
  if (e != cudaSuccess) return cuda_st(e);
  std::vector<rpca_window> dw(b->n);
  for (int i = 0; i < b->n; ++i) {
    dw[i] = win[i];
    dw[i].X = sg.X[i];
    dw[i].L = sg.L[i];
    dw[i].S = sg.S[i];
    dw[i].mask = win[i].mask ? sg.M[i] : nullptr;
  }
  st = rpca_batch_solve(b, dw.data(), stream, nullptr);
  if (st != RPCA_OK) return st;
  e = cudaEventRecord(sg.solved, s);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(b->s_dn, sg.solved, 0);
  for (int i = 0; i < b->n && e == cudaSuccess; ++i) {
    const size_t nb = window_bytes(b->p[i]);
    e = cudaMemcpyAsync(win[i].L, sg.L[i], nb, cudaMemcpyDeviceToHost, b->s_dn);
    if (e == cudaSuccess) e = cudaMemcpyAsync(win[i].S, sg.S[i], nb, cudaMemcpyDeviceToHost, b->s_dn);
    if (e == cudaSuccess && win[i].mask)
      e = cudaMemcpyAsync(win[i].mask, sg.M[i], (size_t)b->p[i].m, cudaMemcpyDeviceToHost, b->s_dn);
  }
  if (e == cudaSuccess && out)
    e = cudaMemcpyAsync(b->h_ctrl, b->d_ctrl, sizeof(Ctrl) * b->n, cudaMemcpyDeviceToHost, b->s_dn);
  if (e == cudaSuccess) e = cudaEventRecord(sg.down, b->s_dn);
  if (e != cudaSuccess) return cuda_st(e);
  sg.used = true;
  ++b->host_calls;
  if (!out) return RPCA_OK;
  e = cudaEventSynchronize(sg.down);
  if (e != cudaSuccess) return cuda_st(e);
  b->pending = false;
  int worst = RPCA_OK;
  for (int i = 0; i < b->n; ++i) {
    result_from_ctrl(b->views[i].lambda, b->h_ctrl[b->win_slot[i]], &out[i], b->views[i].cplx);
    if (out[i].status < 0) worst = out[i].status;
    else if (worst == RPCA_OK && out[i].status != RPCA_OK) worst = out[i].status;
  }
  return (rpca_status)worst;
}

rpca_status rpca_batch_tune(rpca_batch_t b, const rpca_window* win, void* stream, int32_t reps, double* best_ms) {
  if (!b || !win || reps < 1) return RPCA_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<BatchConfig> cands;
  std::vector<int> lane_opts;
  for (int div : {1, 2, 4, 8})
    if (std::find(lane_opts.begin(), lane_opts.end(), std::max(1, (b->n + div - 1) / div)) == lane_opts.end())
      lane_opts.push_back(std::max(1, (b->n + div - 1) / div));
  std::vector<int> occ_opts = {1};
  if (b->occ_max > 1) occ_opts.push_back(b->occ_max);
  for (int occ : occ_opts)
    for (int L : lane_opts)
      for (double a : {1.0, 0.5})
        for (int pr : {0, 1}) {
          if (pr && b->n < 2 * L) continue;  // a paired lane needs two windows
          BatchConfig c{std::min(L, b->sms * occ), a, occ, pr};
          if (std::find(cands.begin(), cands.end(), c) == cands.end()) cands.push_back(c);
        }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e != cudaSuccess) return cuda_st(e);
  double best = 1e300;
  BatchConfig best_cfg = b->cfg;
  rpca_status st = RPCA_OK;
  for (const BatchConfig& c : cands) {
    st = apply_config(b, c);
    if (st != RPCA_OK) break;
    st = rpca_batch_solve(b, win, stream, nullptr);  // warm-up (and graph capture)
    if (st != RPCA_OK) break;
    std::vector<float> ms;
    for (int r = 0; r < reps && st == RPCA_OK; ++r) {
      e = cudaEventRecord(e0, s);
      if (e == cudaSuccess) st = rpca_batch_solve(b, win, stream, nullptr);
      if (e == cudaSuccess && st == RPCA_OK) e = cudaEventRecord(e1, s);
      if (e == cudaSuccess && st == RPCA_OK) e = cudaEventSynchronize(e1);
      float t = 0.f;
      if (e == cudaSuccess && st == RPCA_OK) e = cudaEventElapsedTime(&t, e0, e1);
      if (e != cudaSuccess) st = cuda_st(e);
      ms.push_back(t);
    }
    if (st != RPCA_OK) break;
    std::sort(ms.begin(), ms.end());
    const double med = ms[ms.size() / 2];
    if (med < best) {
      best = med;
      best_cfg = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  rpca_status st2 = apply_config(b, best_cfg);
  if (st != RPCA_OK) return st;
  if (st2 != RPCA_OK) return st2;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache[b->signature] = best_cfg;
  }
  if (best_ms) *best_ms = best;
  return RPCA_OK;
}

rpca_status rpca_batch_schedule(int32_t n, const int64_t* m, const int32_t* T, const int32_t* max_ctas,
                                int32_t ctas, int32_t lanes, double alpha, int32_t* n_lanes, int32_t* lane_ctas,
                                int32_t* order, int32_t* lane_end) {
  if (n < 1 || !m || !T || !n_lanes || !lane_ctas || !order || !lane_end || ctas < 1 || lanes < 1 ||
      !(alpha >= 0.0) || !isfinite(alpha))
    return RPCA_ERR_ARG;
  std::vector<double> wload(n);
  std::vector<int> wcap(n);
  for (int w = 0; w < n; ++w) {
    if (m[w] < 1 || T[w] < 1 || (max_ctas && max_ctas[w] < 1)) return RPCA_ERR_ARG;
    rpca_params p{};
    p.m = m[w];
    p.T = T[w];
    wload[w] = window_load(p);
    wcap[w] = max_ctas ? max_ctas[w] : ctas;
  }
  const LanePlan lp = plan_lanes(wload, wcap, ctas, lanes, alpha);
  const int L = (int)lp.nc.size();
  *n_lanes = L;
  int k = 0;
  for (int l = 0; l < L; ++l) {
    lane_ctas[l] = lp.nc[l];
    for (int w : lp.lw[l]) order[k++] = w;
    lane_end[l] = k;
  }
  return RPCA_OK;
}

rpca_status rpca_batch_set_schedule(rpca_batch_t b, int32_t lanes, double alpha, int32_t ctas_per_sm,
                                    int32_t paired) {
  if (!b || lanes < 1 || !(alpha >= 0.0) || !isfinite(alpha) || ctas_per_sm < 1 || ctas_per_sm > b->occ_max ||
      (paired != 0 && paired != 1))
    return RPCA_ERR_ARG;
  BatchConfig c{std::min(lanes, b->sms * ctas_per_sm), alpha, ctas_per_sm, paired};
  return apply_config(b, c);
}

rpca_status rpca_batch_info(rpca_batch_t b, int32_t* info, int32_t n) {
  if (!b || !info || n < 0) return RPCA_ERR_ARG;
  const int32_t v[7] = {b->grid, b->nlanes, b->cfg.ctas_per_sm, (int32_t)lround(b->cfg.alpha * 1000.0),
                        b->occ_max, b->exec ? 1 : 0, b->cfg.paired};
  for (int i = 0; i < n && i < 7; ++i) info[i] = v[i];
  return RPCA_OK;
}

rpca_status rpca_batch_window_ctas(rpca_batch_t b, int32_t* ctas, int32_t n) {
  if (!b || !ctas || n < b->n) return RPCA_ERR_ARG;
  for (int i = 0; i < b->n; ++i) ctas[i] = b->win_ncta[i];
  return RPCA_OK;
}

void rpca_batch_destroy(rpca_batch_t b) {
  if (!b) return;
  if (b->pending && b->last) cudaEventSynchronize(b->last);
  host_stage_free(b);
  drop_graph(b);
  for (rpca_plan_t pl : b->plans) rpca_plan_destroy(pl);
  if (b->h_desc) cudaFreeHost(b->h_desc);
  if (b->d_desc) cudaFree(b->d_desc);
  if (b->h_ctrl) cudaFreeHost(b->h_ctrl);
  if (b->d_ctrl) cudaFree(b->d_ctrl);
  if (b->last) cudaEventDestroy(b->last);
  delete b;
}

}  // extern "C"
