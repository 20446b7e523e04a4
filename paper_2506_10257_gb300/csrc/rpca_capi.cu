// rpca_capi.cu -- C ABI of the GB300 PCP solver: plans, CUDA-graph driver,
// host-driven plain form, kernel-level entry points.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "../../include/rpca.h"
#include "rpca_kernels.cuh"
#include "rpca_internal.h"

using namespace rpca;

namespace {

struct KernelSet {
  void* pass[4];
  size_t pass_smem;        // dynamic shared memory of the CUDA-core passes
  void* pass_tc[4];        // fused pass with tensor-core contractions, per rpca_precision (0 unused)
  size_t pass_tc_smem[4];
  void* pass_fs[4];        // CUDA-core FP32 passes fed by TMA, by mode (needs m % 4 == 0)
  size_t pass_fs_smem;
  void* eig64;       // plain smem Jacobi, FP64 rotations (rpca_eig on an external matrix)
  void* eig_fast;    // the plans' eigen-step: FP64 rotations, logged and accumulated once
  size_t eig_fast_smem;
  void* eig_fast32;  // the same with FP32 rotations and basis arithmetic (RPCA_EIG_FP32=1)
  size_t eig_fast32_smem;
  int TB;
  int eig_threads;
};

template <int TB>
KernelSet make_set() {
  KernelSet k;
  k.pass[PM_INIT] = (void*)pass_kernel<TB, PM_INIT>;
  k.pass[PM_FUSED] = (void*)pass_kernel<TB, PM_FUSED>;
  k.pass[PM_UPDATE] = (void*)pass_kernel<TB, PM_UPDATE>;
  k.pass[PM_GRAM] = (void*)pass_kernel<TB, PM_GRAM>;
  k.pass_smem = pass_simt_smem<TB>();
  k.pass_fs[PM_INIT] = (void*)pass_fs_kernel<TB, PM_INIT>;
  k.pass_fs[PM_FUSED] = (void*)pass_fs_kernel<TB, PM_FUSED>;
  k.pass_fs[PM_UPDATE] = (void*)pass_fs_kernel<TB, PM_UPDATE>;
  k.pass_fs[PM_GRAM] = (void*)pass_fs_kernel<TB, PM_GRAM>;
  k.pass_fs_smem = FsShape<TB>::SMEM;
  k.eig64 = (void*)eig_kernel<TB, double>;
  k.eig_fast = (void*)eig64_kernel<TB>;
  k.eig_fast_smem = sizeof(Eig64Smem<TB>);
  k.eig_fast32 = (void*)eig_fast_kernel<TB, float>;
  k.eig_fast32_smem = sizeof(EigFastSmem<TB, float>);
  k.TB = TB;
  k.eig_threads = TB > 20 ? 512 : 256;
  return k;
}

int bucket_of(int T) {
  if (T <= 8) return 8;
  if (T <= 12) return 12;
  if (T <= 16) return 16;
  if (T <= 20) return 20;
  if (T <= 24) return 24;
  if (T <= 32) return 32;
  return 0;
}

template <int TB>
void add_tc(KernelSet& k) {
  constexpr int KP = TB <= 16 ? 16 : 32;
  k.pass_tc[RPCA_PREC_FP32] = nullptr;
  k.pass_tc_smem[RPCA_PREC_FP32] = 0;
  k.pass_tc[RPCA_PREC_TF32X3] = (void*)pass_tc_kernel<TB, KP, false, true>;
  k.pass_tc_smem[RPCA_PREC_TF32X3] = pass_tc_smem<TB, KP, false>();
  k.pass_tc[RPCA_PREC_BF16X3] = (void*)pass_tc_kernel<TB, KP, true, true>;
  k.pass_tc_smem[RPCA_PREC_BF16X3] = pass_tc_smem<TB, KP, true>();
  k.pass_tc[RPCA_PREC_TF32] = nullptr;  // plain TF32 is not offered (validate)
  k.pass_tc_smem[RPCA_PREC_TF32] = 0;
}

// Tensor-core pass buckets: T <= 16, 20, 32.
void set_tc(int T, KernelSet* k) {
  if (T <= 16) add_tc<16>(*k);
  else if (T <= 20) add_tc<20>(*k);
  else add_tc<32>(*k);
}

bool get_set(int T, KernelSet* out) {
  switch (bucket_of(T)) {
    case 8: *out = make_set<8>(); return true;
    case 12: *out = make_set<12>(); return true;
    case 16: *out = make_set<16>(); return true;
    case 20: *out = make_set<20>(); return true;
    case 24: *out = make_set<24>(); return true;
    case 32: *out = make_set<32>(); return true;
    default: return false;
  }
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

struct Layout {
  size_t ctrl, eig, red, job, gw, ww, vw, evw, rlog, rk, rrnd, wtc, gram_part, group_part, scal_part, gscal_part, ybuf,
      total;
  int grid, ngroups;
  int ws_grid;     // CTAs of the passes with 128-pixel tiles (TMA-fed FP32, tiled tensor-core): one per SM
  int wide_grid;   // CTAs of the wide pass (T > kMaxT; one per SM, 32-pixel tiles)
};

int device_sms() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  return sms;
}

// Grid: one 256-thread CTA per SM (register bound), never more than the tiles.
// wtc_bytes: B operand images of the tiled tensor-core pass (0: none).
Layout make_layout(int64_t m, int T, int sms, bool wide, size_t wtc_bytes = 0) {
  Layout L;
  const int64_t ntiles = (m + kTile - 1) / kTile;
  int64_t grid = std::min<int64_t>(ntiles, (int64_t)std::max(sms, 1) * kPassCtasPerSm);
  grid = std::min<int64_t>(grid, (int64_t)kGroup * kMaxGroups);
  L.grid = (int)std::max<int64_t>(grid, 1);
  L.ws_grid = (int)std::max<int64_t>(std::min<int64_t>((m + 127) / 128, std::max(sms, 1)), 1);
  int wtile = 32, wper = 1;
  if (wide) wide_launch_shape(T, &wtile, &wper);
  L.wide_grid = (int)std::max<int64_t>(std::min<int64_t>((m + wtile - 1) / wtile, (int64_t)std::max(sms, 1) * wper), 1);
  const int maxgrid = std::max({L.grid, L.ws_grid, wide ? L.wide_grid : 1});
  L.ngroups = (maxgrid + kGroup - 1) / kGroup;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off = align_up(off + bytes, 256);
    return o;
  };
  L.ctrl = take(sizeof(Ctrl));
  L.eig = take(sizeof(EigState));
  L.red = take(sizeof(RedState));
  L.job = take(sizeof(Job));
  const size_t tw = wide ? (size_t)T * T : 1;   // wide-path Gram, Wbar, V
  L.gw = take(sizeof(double) * tw);
  L.ww = take(sizeof(float) * tw);
  L.vw = take(sizeof(float) * tw);
  L.evw = take(sizeof(double) * (size_t)T);
  // rotation log of the wide eigen-step: every round of kWideLogSweeps sweeps
  const size_t nrounds = wide ? (size_t)kWideLogSweeps * (size_t)(T + (T & 1)) : 1;
  const size_t npairs = wide ? (size_t)(T + (T & 1)) / 2 : 1;
  L.rlog = take(sizeof(float2) * nrounds * npairs);
  L.rk = take(sizeof(int) * nrounds * npairs);
  L.rrnd = take(sizeof(int) * 2 * nrounds);
  L.wtc = take(wtc_bytes ? wtc_bytes : 1);
  L.gram_part = take(sizeof(float) * (size_t)maxgrid * T * T);
  L.group_part = take(sizeof(float2) * (size_t)L.ngroups * T * T);
  L.scal_part = take(sizeof(double) * 2 * (size_t)maxgrid);
  L.gscal_part = take(sizeof(double) * 2 * (size_t)L.ngroups);
  L.ybuf = take(sizeof(float) * (size_t)m * T);
  L.total = off;
  return L;
}

// Real columns of the window's matrix: complex windows run as their
// interleaved real embedding with 2 x T columns.
int real_cols(const rpca_params* p) { return p->dtype == RPCA_C64 ? 2 * p->T : p->T; }
// Complex windows and windows of more than kMaxT frames run the tiled path.
bool uses_wide(const rpca_params* p) { return p->dtype == RPCA_C64 || p->T > kMaxT; }

rpca_status validate(const rpca_params* p) {
  if (!p) return RPCA_ERR_ARG;
  if (p->m < 1 || p->T < 1) return RPCA_ERR_ARG;
  if (p->T > RPCA_MAX_T) return RPCA_ERR_UNSUPPORTED;
  if (!(p->tol > 0) || p->max_iter < 1) return RPCA_ERR_ARG;
  if (p->mu_schedule != RPCA_MU_IALM && p->mu_schedule != RPCA_MU_FIXED_L1) return RPCA_ERR_ARG;
  if (p->mu_schedule == RPCA_MU_IALM && (!(p->rho >= 1.0) || !(p->mu0_scale > 0) || !(p->mu_max_factor >= 1.0)))
    return RPCA_ERR_ARG;
  if (p->drive != RPCA_DRIVE_GRAPH && p->drive != RPCA_DRIVE_HOST && p->drive != RPCA_DRIVE_STREAM)
    return RPCA_ERR_ARG;
  if (p->dtype != RPCA_R32 && p->dtype != RPCA_C64) return RPCA_ERR_ARG;
  // complex windows: the tiled path up to 112 frames; the tensor-core
  // precisions up to 64 frames (128 real columns)
  if (p->dtype == RPCA_C64 && (2 * p->T > kMaxTW || (p->precision != RPCA_PREC_FP32 && 2 * p->T > 128)))
    return RPCA_ERR_UNSUPPORTED;
  if (p->precision < RPCA_PREC_FP32 || p->precision > RPCA_PREC_TF32) return RPCA_ERR_ARG;
  // one TF32 product per contraction (10-bit mantissa) leaves L and S about
  // 7e-4 from the FP64 solution on the 262144 x 20 window, outside the 1e-4
  // bound of the reduced precisions, so it is not offered
  if (p->precision == RPCA_PREC_TF32) return RPCA_ERR_UNSUPPORTED;
  if (p->precision != RPCA_PREC_FP32 && p->drive == RPCA_DRIVE_HOST) return RPCA_ERR_UNSUPPORTED;
  // the tiled path's tensor-core pass: real windows of at most 128 frames
  // (complex ones: checked above)
  if (p->precision != RPCA_PREC_FP32 && p->dtype == RPCA_R32 && p->T > 128) return RPCA_ERR_UNSUPPORTED;
  if (p->m * (int64_t)p->T > (int64_t)1 << 40) return RPCA_ERR_ARG;
  if (p->warm_start != 0 && p->warm_start != 1) return RPCA_ERR_ARG;
  if (p->sharded != 0 && p->sharded != 1) return RPCA_ERR_ARG;
  if (p->sharded && (p->dtype != RPCA_R32 || p->T > kMaxT || p->precision != RPCA_PREC_FP32 ||
                     p->mu_schedule != RPCA_MU_IALM || p->warm_start))
    return RPCA_ERR_UNSUPPORTED;
  if (!(p->mu_init >= 0.0) || !(p->mu_prev_scale >= 0.0) || !isfinite(p->mu_init) || !isfinite(p->mu_prev_scale))
    return RPCA_ERR_ARG;
  return RPCA_OK;
}

}  // namespace

struct rpca_plan_s {
  rpca_params p;
  KernelSet ks;
  bool wide;          // T > kMaxT: shared-memory tiled passes, 1024-thread eigen-step
  WideKernels wk;
  Layout lay;
  Bufs bufs;
  char* ws;
  bool own_ws;
  double lambda;
  int eig_fp32;       // opt-in FP32 rotations in the narrow eigen-step (RPCA_EIG_FP32=1)
  cudaGraph_t graph;
  cudaGraphExec_t exec;
  Ctrl* ctrl_host;  // pinned
  bool use_fs;      // FP32 passes = TMA-fed CUDA-core kernels (narrow windows, m % 4 == 0)
  // device staging of rpca_solve_host (allocated on first use)
  float* stage_x;
  float* stage_l;
  float* stage_s;
  uint8_t* stage_mask;
};

// cuTensorMapEncodeTiled from the driver (looked up once; NULL if unavailable).
static PFN_cuTensorMapEncodeTiled_v12000 tma_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)f;
  }
  return fn;
}

// 2D map of a frame-major m x T float32 matrix, box 128 pixels x T frames.
static bool encode_map(CUtensorMap* map, const void* ptr, int64_t m, int T) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tma_encoder();
  if (!enc) return false;
  cuuint64_t gdim[2] = {(cuuint64_t)m, (cuuint64_t)T};
  cuuint64_t gstride[1] = {(cuuint64_t)m * 4};
  cuuint32_t box[2] = {128, (cuuint32_t)T};
  cuuint32_t estr[2] = {1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(ptr), gdim, gstride, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

static rpca_status cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return RPCA_OK;
  if (e == cudaErrorMemoryAllocation) return RPCA_ERR_NOMEM;
  return RPCA_ERR_CUDA;
}
#define CK(x)                                 \
  do {                                        \
    cudaError_t _e = (x);                     \
    if (_e != cudaSuccess) return cuda_status(_e); \
  } while (0)

static cudaError_t launch(void* fn, dim3 g, dim3 blk, void** args, cudaStream_t s, size_t smem = 0) {
  return cudaLaunchKernel(fn, g, blk, args, smem, s);
}

// Eigen-step kernel of a plan: FP64 Jacobi rotations and basis arithmetic,
// or FP32 ones when RPCA_EIG_FP32 is set.  Both take (Bufs, flags, handle,
// use_cond, ...); the extra pointer arguments of the argument lists below
// are ignored.
static void* eig_fn(const rpca_plan_s* pl) {
  if (pl->wide) return pl->wk.eig;
  return pl->eig_fp32 ? pl->ks.eig_fast32 : pl->ks.eig_fast;
}
static size_t eig_smem(const rpca_plan_s* pl) {
  if (pl->wide) return pl->wk.eig_smem;
  return pl->eig_fp32 ? pl->ks.eig_fast32_smem : pl->ks.eig_fast_smem;
}
static dim3 eig_block(const rpca_plan_s* pl) {
  if (pl->wide) return dim3(pl->wk.eig_threads);
  return dim3(kEigThreads);
}
// CUDA-core FP32 passes by mode (narrow: one pixel row per thread, TMA-fed when
// the plan has tensor maps; wide: tiles).
static void* pass_fn(const rpca_plan_s* pl, int mode) {
  if (pl->wide) return pl->wk.pass[mode];
  return pl->use_fs ? pl->ks.pass_fs[mode] : pl->ks.pass[mode];
}
static size_t pass_smem(const rpca_plan_s* pl) {
  if (pl->wide) return pl->wk.pass_smem;
  return pl->use_fs ? pl->ks.pass_fs_smem : pl->ks.pass_smem;
}
static dim3 pass_grid(const rpca_plan_s* pl) {
  if (pl->wide) return dim3(pl->lay.wide_grid);
  return dim3(pl->use_fs ? pl->lay.ws_grid : pl->lay.grid);
}
static dim3 pass_block(const rpca_plan_s* pl) {
  if (pl->wide) return dim3(pl->wk.pass_threads);
  return dim3(pl->use_fs ? kFsThreads : kPassThreads);
}
// Fused per-iteration pass: CUDA-core FP32 or the tensor-core form of the plan's precision.
static void* fused_fn(const rpca_plan_s* pl) {
  if (pl->p.precision == RPCA_PREC_FP32) return pass_fn(pl, PM_FUSED);
  if (pl->wide) return pl->wk.pass_tc[pl->p.precision];
  return pl->ks.pass_tc[pl->p.precision];
}
static size_t fused_smem(const rpca_plan_s* pl) {
  if (pl->p.precision == RPCA_PREC_FP32) return pass_smem(pl);
  if (pl->wide) return pl->wk.pass_tc_smem[pl->p.precision];
  return pl->ks.pass_tc_smem[pl->p.precision];
}
static dim3 fused_grid(const rpca_plan_s* pl) {
  if (pl->p.precision == RPCA_PREC_FP32) return pass_grid(pl);
  if (pl->wide) return dim3(pl->lay.ws_grid);  // one CTA per SM, 128-pixel tiles
  return dim3(pl->lay.grid);
}
static dim3 fused_block(const rpca_plan_s* pl) {
  if (pl->p.precision == RPCA_PREC_FP32) return pass_block(pl);
  if (pl->wide) return dim3(pl->wk.pass_tc_threads);
  return dim3(kPassThreads);
}

static cudaError_t add_kernel(cudaGraph_t g, cudaGraphNode_t* node, const cudaGraphNode_t* deps, size_t ndeps,
                              void* fn, dim3 grid, dim3 blk, void** args, size_t smem = 0) {
  cudaKernelNodeParams kp;
  memset(&kp, 0, sizeof(kp));
  kp.func = fn;
  kp.gridDim = grid;
  kp.blockDim = blk;
  kp.sharedMemBytes = (unsigned)smem;
  kp.kernelParams = args;
  kp.extra = nullptr;
  return cudaGraphAddKernelNode(node, g, deps, ndeps, &kp);
}

// Graph: init pass -> eig(init) -> while(cond){ fused pass -> eig(check|eig) } -> final.
static rpca_status build_graph(rpca_plan_s* pl) {
  CK(cudaGraphCreate(&pl->graph, 0));
  cudaGraphConditionalHandle h;
  CK(cudaGraphConditionalHandleCreate(&h, pl->graph, 0, cudaGraphCondAssignDefault));
  Bufs b = pl->bufs;
  const dim3 pg = pass_grid(pl), pb = pass_block(pl), eg(1), eb = eig_block(pl);
  const size_t es = eig_smem(pl);
  const double* nulld = nullptr;
  double* nullo = nullptr;
  int use_cond = 1;
  int f_init = EF_INIT | EF_EIG, f_iter = EF_CHECK | EF_EIG;

  void* a_pass[] = {&b};
  void* a_eig0[] = {&b, &f_init, &h, &use_cond, &nulld, &nullo, &nullo};
  void* a_eig1[] = {&b, &f_iter, &h, &use_cond, &nulld, &nullo, &nullo};
  cudaGraphNode_t n_init, n_eig0, n_while, n_fin, n_pass, n_eig;
  CK(add_kernel(pl->graph, &n_init, nullptr, 0, pass_fn(pl, PM_INIT), pg, pb, a_pass, pass_smem(pl)));
  CK(add_kernel(pl->graph, &n_eig0, &n_init, 1, eig_fn(pl), eg, eb, a_eig0, es));
  if (pl->p.warm_start) {
    // warm start: the first SVT needs the Gram of Z1 = X - S0 + Y0/mu1, not of X
    int f_eig = EF_EIG | EF_FULL;
    void* a_eigw[] = {&b, &f_eig, &h, &use_cond, &nulld, &nullo, &nullo};
    cudaGraphNode_t n_gw, n_ew;
    CK(add_kernel(pl->graph, &n_gw, &n_eig0, 1, pass_fn(pl, PM_GRAM), pg, pb, a_pass, pass_smem(pl)));
    CK(add_kernel(pl->graph, &n_ew, &n_gw, 1, eig_fn(pl), eg, eb, a_eigw, es));
    n_eig0 = n_ew;
  }

  alignas(cudaGraphNodeParams) unsigned char cp_raw[sizeof(cudaGraphNodeParams)];
  memset(cp_raw, 0, sizeof(cp_raw));
  cudaGraphNodeParams& cp = *reinterpret_cast<cudaGraphNodeParams*>(cp_raw);
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  CK(cudaGraphAddNode(&n_while, pl->graph, &n_eig0, nullptr, 1, &cp));
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  CK(add_kernel(body, &n_pass, nullptr, 0, fused_fn(pl), fused_grid(pl), fused_block(pl), a_pass, fused_smem(pl)));
  CK(add_kernel(body, &n_eig, &n_pass, 1, eig_fn(pl), eg, eb, a_eig1, es));

  const int fgrid = (int)std::min<int64_t>((pl->p.m + 255) / 256, 4096);
  CK(add_kernel(pl->graph, &n_fin, &n_while, 1, (void*)final_kernel, dim3(fgrid), dim3(256), a_pass));
  CK(cudaGraphInstantiate(&pl->exec, pl->graph, 0));
  return RPCA_OK;
}

namespace rpca {

void result_from_ctrl(double lambda, const Ctrl& c, rpca_result* out, int cplx) {
  memset(out, 0, sizeof(*out));
  out->status = c.status;
  out->iters = c.k;
  out->rank = cplx ? c.rank / 2 : c.rank;
  out->sweeps = c.total_sweeps;
  out->resid = c.resid;
  out->mu = c.mu_cur;
  out->normX = c.normX;
  out->lambda = lambda;
  out->pass_us = c.pass_cnt ? (double)c.pass_ns / (double)c.pass_cnt * 1e-3 : 0.0;
  out->eig_us = c.eig_cnt ? (double)c.eig_ns / (double)c.eig_cnt * 1e-3 : 0.0;
  out->init_us = (double)c.init_ns * 1e-3;
  out->passes_timed = (int32_t)c.pass_cnt;
  out->eigs_timed = (int32_t)c.eig_cnt;
}

Ctrl* plan_ctrl(rpca_plan_t pl) { return pl ? pl->bufs.ctrl : nullptr; }

rpca_status plan_view(rpca_plan_t pl, PlanView* v) {
  if (!pl || !v) return RPCA_ERR_ARG;
  v->bufs = pl->bufs;
  v->m = pl->p.m;
  v->T = real_cols(&pl->p);
  v->cplx = pl->p.dtype == RPCA_C64;
  v->max_grid = std::max({pl->lay.grid, pl->lay.ws_grid, pl->wide ? pl->lay.wide_grid : 1});
  v->tile = pl->wide ? pl->wk.tile : kTile;
  v->wide = pl->wide ? 1 : 0;
  v->lambda = pl->lambda;
  v->y1 = (float*)(pl->ws + pl->lay.ybuf);
  return RPCA_OK;
}

}  // namespace rpca

static void fill_result(const rpca_plan_s* pl, const Ctrl& c, rpca_result* out) {
  result_from_ctrl(pl->lambda, c, out, pl->p.dtype == RPCA_C64);
}

extern "C" {

rpca_status rpca_params_default(rpca_params* p, int64_t m, int32_t T) {
  if (!p) return RPCA_ERR_ARG;
  memset(p, 0, sizeof(*p));
  p->m = m;
  p->T = T;
  p->dtype = RPCA_R32;
  p->precision = RPCA_PREC_FP32;
  p->mu_schedule = RPCA_MU_IALM;
  p->drive = RPCA_DRIVE_GRAPH;
  p->max_iter = 500;
  p->lambda = 0.0;
  p->mu0_scale = 1.25;
  p->rho = 1.5;
  p->mu_max_factor = 1e7;
  p->tol = 1e-7;
  return RPCA_OK;
}

rpca_status rpca_workspace_size(const rpca_params* p, size_t* bytes) {
  rpca_status st = validate(p);
  if (st != RPCA_OK) return st;
  if (!bytes) return RPCA_ERR_ARG;
  const int sms = device_sms();
  if (sms <= 0) return RPCA_ERR_CUDA;
  *bytes = make_layout(p->m, real_cols(p), sms, uses_wide(p),
                       uses_wide(p) ? wide_tc_img_bytes(real_cols(p), p->precision) : 0).total;
  return RPCA_OK;
}

static rpca_status plan_create_impl(const rpca_params* p, void* workspace, size_t workspace_bytes, bool force_wide,
                                    rpca_plan_t* out);

rpca_status rpca_plan_create(const rpca_params* p, void* workspace, size_t workspace_bytes, rpca_plan_t* out) {
  return plan_create_impl(p, workspace, workspace_bytes, false, out);
}

}  // extern "C"

rpca_status rpca::plan_create_ex(const rpca_params* p, bool force_wide, rpca_plan_t* out) {
  return plan_create_impl(p, nullptr, 0, force_wide, out);
}

static rpca_status plan_create_impl(const rpca_params* p, void* workspace, size_t workspace_bytes, bool force_wide,
                                    rpca_plan_t* out) {
  rpca_status st = validate(p);
  if (st != RPCA_OK) return st;
  if (!out) return RPCA_ERR_ARG;
  *out = nullptr;
  const int sms = device_sms();
  if (sms <= 0) return RPCA_ERR_CUDA;
  rpca_plan_s* pl = new rpca_plan_s();
  pl->p = *p;
  const bool cplx = p->dtype == RPCA_C64;
  const int Tr = real_cols(p);
  pl->wide = uses_wide(p) || force_wide;
  if (pl->wide) {
    if (!wide_kernels(Tr, cplx, pl->wide && !uses_wide(p), &pl->wk)) {
      delete pl;
      return RPCA_ERR_UNSUPPORTED;
    }
  } else {
    if (!get_set(p->T, &pl->ks)) {
      delete pl;
      return RPCA_ERR_UNSUPPORTED;
    }
    set_tc(p->T, &pl->ks);
  }
  // The TMA-fed FP32 pass is opt-in (RPCA_PASS_TMA=1): the register-resident
  // pass measured as fast or faster.
  pl->use_fs = !pl->wide && (p->precision == RPCA_PREC_FP32) && (p->m % 4 == 0) && (p->m < ((int64_t)1 << 31)) &&
               tma_encoder() != nullptr && getenv("RPCA_PASS_TMA") && atoi(getenv("RPCA_PASS_TMA")) != 0;
  if (!pl->wide) {
    // the register-resident passes stage two tiles of Z~ rows (over 48 KB from 20 frames)
    for (int i = 0; i < 4; ++i) {
      const cudaError_t ea = cudaFuncSetAttribute(pl->ks.pass[i], cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                  (int)pl->ks.pass_smem);
      if (ea != cudaSuccess) {
        delete pl;
        return cuda_status(ea);
      }
    }
  }
  if (pl->use_fs) {
    for (int i = 0; i < 4; ++i) {
      const cudaError_t ea = cudaFuncSetAttribute(pl->ks.pass_fs[i], cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                  (int)pl->ks.pass_fs_smem);
      if (ea != cudaSuccess) {
        delete pl;
        return cuda_status(ea);
      }
    }
  }
  if (p->precision != RPCA_PREC_FP32 && pl->wide && !pl->wk.pass_tc[p->precision]) {
    delete pl;
    return RPCA_ERR_UNSUPPORTED;
  }
  if (p->precision != RPCA_PREC_FP32 && !pl->wide) {
    cudaError_t ea = cudaFuncSetAttribute(pl->ks.pass_tc[p->precision], cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)pl->ks.pass_tc_smem[p->precision]);
    if (ea != cudaSuccess) {
      delete pl;
      return cuda_status(ea);
    }
  }
  pl->lay = make_layout(p->m, Tr, sms, pl->wide, pl->wide ? wide_tc_img_bytes(Tr, p->precision) : 0);
  if (!pl->wide) {
    cudaError_t ea = cudaFuncSetAttribute(pl->ks.eig_fast, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)pl->ks.eig_fast_smem);
    if (ea == cudaSuccess)
      ea = cudaFuncSetAttribute(pl->ks.eig_fast32, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)pl->ks.eig_fast32_smem);
    if (ea != cudaSuccess) {
      delete pl;
      return cuda_status(ea);
    }
  }
  pl->eig_fp32 = (getenv("RPCA_EIG_FP32") && atoi(getenv("RPCA_EIG_FP32")) != 0) ? 1 : 0;
  if (workspace) {
    if (workspace_bytes < pl->lay.total || ((uintptr_t)workspace & 255u)) {
      delete pl;
      return RPCA_ERR_ARG;
    }
    pl->ws = (char*)workspace;
    pl->own_ws = false;
  } else {
    cudaError_t e = cudaMalloc((void**)&pl->ws, pl->lay.total);
    if (e != cudaSuccess) {
      delete pl;
      return cuda_status(e);
    }
    pl->own_ws = true;
  }
  Bufs& b = pl->bufs;
  b.ctrl = (Ctrl*)(pl->ws + pl->lay.ctrl);
  b.eig = (EigState*)(pl->ws + pl->lay.eig);
  b.red = (RedState*)(pl->ws + pl->lay.red);
  b.job = (Job*)(pl->ws + pl->lay.job);
  b.gram_part = (float*)(pl->ws + pl->lay.gram_part);
  b.group_part = (float2*)(pl->ws + pl->lay.group_part);
  b.scal_part = (double*)(pl->ws + pl->lay.scal_part);
  b.gscal_part = (double*)(pl->ws + pl->lay.gscal_part);
  b.Gw = (double*)(pl->ws + pl->lay.gw);
  b.Ww = (float*)(pl->ws + pl->lay.ww);
  b.Vw = (float*)(pl->ws + pl->lay.vw);
  b.evw = (double*)(pl->ws + pl->lay.evw);
  b.rot_log = (float2*)(pl->ws + pl->lay.rlog);
  b.rot_k = (int*)(pl->ws + pl->lay.rk);
  b.rot_rnd = (int*)(pl->ws + pl->lay.rrnd);
  b.wtc = (pl->wide && p->precision == RPCA_PREC_TF32X3) ? 1 : (pl->wide && p->precision == RPCA_PREC_BF16X3) ? 2 : 0;
  b.wtc_img = b.wtc ? (unsigned char*)(pl->ws + pl->lay.wtc) : nullptr;
  b.m = p->m;
  b.T = Tr;
  b.cplx = cplx ? 1 : 0;
  b.wide = pl->wide ? 1 : 0;
  b.grid = pl->lay.grid;
  b.ngroups = pl->lay.ngroups;
  // a sharded plan's passes finish their reduction themselves, so the summed
  // Gram and residual sums sit in the reduction record between the steps
  b.finalize = p->sharded ? 1 : 0;
  b.eig64 = pl->wide ? 0 : (pl->eig_fp32 ? 0 : 1);

  const int mT = (int)std::max<int64_t>(p->m, p->T);
  pl->lambda = p->lambda > 0 ? p->lambda : 1.0 / sqrt((double)mT);
  Ctrl c;
  memset(&c, 0, sizeof(c));
  c.max_iter = p->max_iter;
  c.schedule = p->mu_schedule == RPCA_MU_IALM ? 0 : 1;
  c.lambda = pl->lambda;
  c.rho = p->rho;
  c.mu0_scale = p->mu0_scale;
  c.mu_max_factor = p->mu_max_factor;
  c.tol = p->tol;
  // Jacobi threshold: an off-diagonal pair rotates while |g_pq| > eps sqrt(g_pp g_qq);
  // FP64 rotations stop 1e2 below the FP32 rounding of the passes' Gram entries
  c.jacobi_eps = (b.eig64 ? 1e-9 : 1e-6);
  c.warm_sweeps = 4;
  c.cold_sweeps = 30;
  c.warm = p->warm_start;
  c.mu_init = p->mu_init;
  c.mu_prev_scale = p->mu_prev_scale;
  cudaError_t e = cudaMemset(pl->ws, 0, pl->lay.gram_part);  // ctrl, eig, red (counters), job
  if (e == cudaSuccess) e = cudaMemcpy(b.ctrl, &c, sizeof(c), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMallocHost((void**)&pl->ctrl_host, sizeof(Ctrl));
  if (e != cudaSuccess) {
    if (pl->own_ws) cudaFree(pl->ws);
    delete pl;
    return cuda_status(e);
  }
  // Dual buffer 1 lives in the workspace; buffer 0 is the caller's L.
  float* y1 = (float*)(pl->ws + pl->lay.ybuf);
  e = cudaMemcpy(&b.job->Y1, &y1, sizeof(float*), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFreeHost(pl->ctrl_host);
    if (pl->own_ws) cudaFree(pl->ws);
    delete pl;
    return cuda_status(e);
  }
  if (p->drive == RPCA_DRIVE_GRAPH) {
    rpca_status gs = build_graph(pl);
    if (gs != RPCA_OK) {
      rpca_plan_destroy(pl);
      return gs;
    }
  }
  *out = pl;
  return RPCA_OK;
}

extern "C" {

// The plain form: separate Gram and update passes, residual read back by the
// host after every iteration (one host synchronisation per iteration).
static rpca_status run_host_loop(rpca_plan_s* pl, cudaStream_t s) {
  Bufs b = pl->bufs;
  const dim3 pg = pass_grid(pl), pb = pass_block(pl), eg(1), eb = eig_block(pl);
  const size_t es = eig_smem(pl);
  cudaGraphConditionalHandle h = 0;
  const double* nulld = nullptr;
  double* nullo = nullptr;
  int use_cond = 0;
  int f_init = EF_INIT | EF_EIG, f_check = EF_CHECK, f_eig = EF_EIG;
  void* a_pass[] = {&b};
  void* a_init[] = {&b, &f_init, &h, &use_cond, &nulld, &nullo, &nullo};
  void* a_check[] = {&b, &f_check, &h, &use_cond, &nulld, &nullo, &nullo};
  void* a_eig[] = {&b, &f_eig, &h, &use_cond, &nulld, &nullo, &nullo};
  CK(launch(pass_fn(pl, PM_INIT), pg, pb, a_pass, s, pass_smem(pl)));
  CK(launch(eig_fn(pl), eg, eb, a_init, s, es));
  if (pl->p.warm_start) {
    int f_full = EF_EIG | EF_FULL;
    void* a_full[] = {&b, &f_full, &h, &use_cond, &nulld, &nullo, &nullo};
    CK(launch(pass_fn(pl, PM_GRAM), pg, pb, a_pass, s, pass_smem(pl)));
    CK(launch(eig_fn(pl), eg, eb, a_full, s, es));
  }
  for (int it = 0; it <= pl->p.max_iter; ++it) {
    CK(cudaMemcpyAsync(pl->ctrl_host, b.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (pl->ctrl_host->done) break;
    CK(launch(pass_fn(pl, PM_UPDATE), pg, pb, a_pass, s, pass_smem(pl)));
    CK(launch(eig_fn(pl), eg, eb, a_check, s, es));
    CK(cudaMemcpyAsync(pl->ctrl_host, b.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (pl->ctrl_host->done) break;
    CK(launch(pass_fn(pl, PM_GRAM), pg, pb, a_pass, s, pass_smem(pl)));
    CK(launch(eig_fn(pl), eg, eb, a_eig, s, es));
  }
  const int fgrid = (int)std::min<int64_t>((pl->p.m + 255) / 256, 4096);
  CK(launch((void*)final_kernel, dim3(fgrid), dim3(256), a_pass, s));
  return RPCA_OK;
}

// The graph's kernels launched one by one (no conditional node), convergence
// flag read back every 8 iterations; kernels launched after convergence return
// at once.
static rpca_status run_stream_loop(rpca_plan_s* pl, cudaStream_t s) {
  Bufs b = pl->bufs;
  const dim3 pg = pass_grid(pl), pb = pass_block(pl), eg(1), eb = eig_block(pl);
  const size_t es = eig_smem(pl);
  cudaGraphConditionalHandle h = 0;
  const double* nulld = nullptr;
  double* nullo = nullptr;
  int use_cond = 0;
  int f_init = EF_INIT | EF_EIG, f_iter = EF_CHECK | EF_EIG;
  void* a_pass[] = {&b};
  void* a_init[] = {&b, &f_init, &h, &use_cond, &nulld, &nullo, &nullo};
  void* a_iter[] = {&b, &f_iter, &h, &use_cond, &nulld, &nullo, &nullo};
  CK(launch(pass_fn(pl, PM_INIT), pg, pb, a_pass, s, pass_smem(pl)));
  CK(launch(eig_fn(pl), eg, eb, a_init, s, es));
  if (pl->p.warm_start) {
    int f_eig = EF_EIG | EF_FULL;
    void* a_eig[] = {&b, &f_eig, &h, &use_cond, &nulld, &nullo, &nullo};
    CK(launch(pass_fn(pl, PM_GRAM), pg, pb, a_pass, s, pass_smem(pl)));
    CK(launch(eig_fn(pl), eg, eb, a_eig, s, es));
  }
  for (int it = 0; it < pl->p.max_iter; ++it) {
    if (it % 8 == 0) {
      CK(cudaMemcpyAsync(pl->ctrl_host, b.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      if (pl->ctrl_host->done) break;
    }
    CK(launch(fused_fn(pl), fused_grid(pl), fused_block(pl), a_pass, s, fused_smem(pl)));
    CK(launch(eig_fn(pl), eg, eb, a_iter, s, es));
  }
  const int fgrid = (int)std::min<int64_t>((pl->p.m + 255) / 256, 4096);
  CK(launch((void*)final_kernel, dim3(fgrid), dim3(256), a_pass, s));
  return RPCA_OK;
}

rpca_status rpca_solve(rpca_plan_t pl, const void* X, void* L, void* S, uint8_t* mask, float theta, void* stream,
                       rpca_result* out) {
  return rpca::plan_solve_ex(pl, X, L, S, mask, theta, stream, nullptr, nullptr, -1.0, out);
}

}  // extern "C"

rpca_status rpca::plan_solve_ex(rpca_plan_t pl, const void* X, void* L, void* S, uint8_t* mask, float theta,
                                void* stream, float* Sout, float* Yout, double mu_prev_scale, rpca_result* out) {
  if (!pl || !X || !L || !S) return RPCA_ERR_ARG;
  if (((uintptr_t)X | (uintptr_t)L | (uintptr_t)S) & 15u) return RPCA_ERR_ARG;
  if (X == L || X == S || L == S) return RPCA_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  Bufs b = pl->bufs;
  TmaMaps maps;
  memset(&maps, 0, sizeof(maps));
  int use_maps = 0;
  if (pl->use_fs) {
    const float* y1 = (const float*)(pl->ws + pl->lay.ybuf);
    if (!encode_map(&maps.x, X, pl->p.m, pl->p.T) || !encode_map(&maps.s, S, pl->p.m, pl->p.T) ||
        !encode_map(&maps.y0, L, pl->p.m, pl->p.T) || !encode_map(&maps.y1, y1, pl->p.m, pl->p.T))
      return RPCA_ERR_CUDA;
    use_maps = 1;
  }
  void* a_begin[] = {&b, (void*)&X, &L, &S, &mask, &theta, &Sout, &Yout, &mu_prev_scale, &maps, &use_maps};
  CK(cudaLaunchKernel((void*)begin_kernel, dim3(1), dim3(64), a_begin, 0, s));
  if (pl->p.drive == RPCA_DRIVE_GRAPH) {
    CK(cudaGraphLaunch(pl->exec, s));
  } else {
    rpca_status st = pl->p.drive == RPCA_DRIVE_HOST ? run_host_loop(pl, s) : run_stream_loop(pl, s);
    if (st != RPCA_OK) return st;
  }
  if (!out) return RPCA_OK;
  CK(cudaMemcpyAsync(pl->ctrl_host, b.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  fill_result(pl, *pl->ctrl_host, out);
  return (rpca_status)out->status;
}

extern "C" {

rpca_status rpca_plan_result(rpca_plan_t pl, rpca_result* out) {
  if (!pl || !out) return RPCA_ERR_ARG;
  CK(cudaMemcpy(pl->ctrl_host, pl->bufs.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost));
  fill_result(pl, *pl->ctrl_host, out);
  return RPCA_OK;
}

rpca_status rpca_solve_host(rpca_plan_t pl, const void* X_host, void* L_host, void* S_host, uint8_t* mask_host,
                            float theta, void* stream, rpca_result* out) {
  if (!pl || !X_host || !L_host || !S_host) return RPCA_ERR_ARG;
  const size_t bytes = sizeof(float) * (size_t)pl->p.m * real_cols(&pl->p);
  if (!pl->stage_x) {
    CK(cudaMalloc((void**)&pl->stage_x, bytes));
    CK(cudaMalloc((void**)&pl->stage_l, bytes));
    CK(cudaMalloc((void**)&pl->stage_s, bytes));
    CK(cudaMalloc((void**)&pl->stage_mask, (size_t)pl->p.m));
  }
  cudaStream_t s = (cudaStream_t)stream;
  CK(cudaMemcpyAsync(pl->stage_x, X_host, bytes, cudaMemcpyHostToDevice, s));
  rpca_status st = rpca_solve(pl, pl->stage_x, pl->stage_l, pl->stage_s, mask_host ? pl->stage_mask : nullptr, theta,
                              stream, nullptr);
  if (st != RPCA_OK) return st;
  CK(cudaMemcpyAsync(L_host, pl->stage_l, bytes, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(S_host, pl->stage_s, bytes, cudaMemcpyDeviceToHost, s));
  if (mask_host) CK(cudaMemcpyAsync(mask_host, pl->stage_mask, (size_t)pl->p.m, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(pl->ctrl_host, pl->bufs.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (!out) return (rpca_status)(pl->ctrl_host->status < 0 ? pl->ctrl_host->status : RPCA_OK);
  fill_result(pl, *pl->ctrl_host, out);
  return (rpca_status)out->status;
}

rpca_status rpca_plan_timings(rpca_plan_t pl, double* out, int32_t n) {
  if (!pl || !out || n < 0) return RPCA_ERR_ARG;
  CK(cudaMemcpy(pl->ctrl_host, pl->bufs.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost));
  const Ctrl& c = *pl->ctrl_host;
  const double cnt = c.eig_cnt ? (double)c.eig_cnt : 1.0;
  const double pcnt = c.pass_cnt ? (double)c.pass_cnt : 1.0;
  double v[9];
  for (int i = 0; i < 4; ++i) v[i] = (double)c.eig_phase_ns[i] * 1e-3 / cnt;
  v[4] = (double)c.eig_rounds / cnt;
  v[5] = (double)c.eig_cnt;
  for (int i = 0; i < 3; ++i) v[6 + i] = (double)c.pass_phase_ns[i] * 1e-3 / pcnt;
  for (int i = 0; i < n && i < 9; ++i) out[i] = v[i];
  return RPCA_OK;
}

void rpca_plan_destroy(rpca_plan_t pl) {
  if (!pl) return;
  if (pl->stage_x) cudaFree(pl->stage_x);
  if (pl->stage_l) cudaFree(pl->stage_l);
  if (pl->stage_s) cudaFree(pl->stage_s);
  if (pl->stage_mask) cudaFree(pl->stage_mask);
  if (pl->exec) cudaGraphExecDestroy(pl->exec);
  if (pl->graph) cudaGraphDestroy(pl->graph);
  if (pl->ctrl_host) cudaFreeHost(pl->ctrl_host);
  if (pl->own_ws && pl->ws) cudaFree(pl->ws);
  delete pl;
}

const char* rpca_status_str(int32_t s) {
  switch (s) {
    case RPCA_OK: return "ok";
    case RPCA_NOT_CONVERGED: return "not converged (max_iter reached)";
    case RPCA_PENDING: return "pending";
    case RPCA_ERR_ARG: return "invalid argument";
    case RPCA_ERR_CUDA: return "CUDA error";
    case RPCA_ERR_NOMEM: return "out of device memory";
    case RPCA_ERR_BUDGET: return "HBM budget exceeded";
    case RPCA_ERR_TIMEOUT: return "device wait timed out";
    case RPCA_ERR_NONFINITE: return "non-finite residual";
    case RPCA_ERR_UNSUPPORTED: return "unsupported shape or precision";
    case RPCA_ERR_NOTFOUND: return "unknown request";
    default: return "unknown status";
  }
}

rpca_status rpca_gram(const float* X, int64_t m, int32_t T, const float* V, double* G, int32_t precision,
                      void* stream) {
  if (!X || !G || m < 1 || T < 1) return RPCA_ERR_ARG;
  if (T > kMaxT) return RPCA_ERR_UNSUPPORTED;
  if (precision != RPCA_PREC_FP32) return RPCA_ERR_UNSUPPORTED;
  rpca_params p;
  rpca_params_default(&p, m, T);
  p.drive = RPCA_DRIVE_HOST;
  rpca_plan_t pl = nullptr;
  rpca_status st = rpca_plan_create(&p, nullptr, 0, &pl);
  if (st != RPCA_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<float> v32(kMaxT * kMaxT, 0.f);
  if (V) {
    std::vector<float> vh((size_t)T * T);
    cudaError_t e = cudaMemcpy(vh.data(), V, sizeof(float) * T * T, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
      rpca_plan_destroy(pl);
      return cuda_status(e);
    }
    for (int r = 0; r < T; ++r)
      for (int c = 0; c < T; ++c) v32[r * kMaxT + c] = vh[r * T + c];
  } else {
    for (int r = 0; r < T; ++r) v32[r * kMaxT + r] = 1.f;
  }
  Bufs b = pl->bufs;
  b.finalize = 1;
  Job j;
  memset(&j, 0, sizeof(j));
  j.X = X;
  float* y1 = (float*)(pl->ws + pl->lay.ybuf);
  j.Y1 = y1;
  Ctrl c;
  cudaError_t e = cudaMemcpy(&c, b.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost);
  c.k = 0;
  c.done = 0;
  c.f_inv_mu = 1.f;
  std::vector<double> gred(kMaxT * kMaxT);
  if (e == cudaSuccess) e = cudaMemcpy(b.ctrl, &c, sizeof(Ctrl), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(b.job, &j, sizeof(Job), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(b.eig->V32, v32.data(), sizeof(float) * kMaxT * kMaxT, cudaMemcpyHostToDevice);
  void* a_pass[] = {&b};
  if (e == cudaSuccess)
    e = launch(pl->ks.pass[PM_GRAM], dim3(pl->lay.grid), dim3(kPassThreads), a_pass, s, pl->ks.pass_smem);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = cudaMemcpy(gred.data(), b.red->G, sizeof(double) * kMaxT * kMaxT, cudaMemcpyDeviceToHost);
  std::vector<double> gh((size_t)T * T);
  for (int r = 0; r < T; ++r)
    for (int cc = 0; cc < T; ++cc) gh[r * T + cc] = gred[r * kMaxT + cc];
  if (e == cudaSuccess) e = cudaMemcpy(G, gh.data(), sizeof(double) * T * T, cudaMemcpyHostToDevice);
  rpca_plan_destroy(pl);
  return cuda_status(e);
}

rpca_status rpca_eig(const double* G, int32_t T, double* evals, double* evecs, void* stream) {
  if (!G || !evals || !evecs || T < 1) return RPCA_ERR_ARG;
  if (T > kMaxT) return RPCA_ERR_UNSUPPORTED;
  rpca_params p;
  rpca_params_default(&p, 1, T);
  p.drive = RPCA_DRIVE_HOST;
  rpca_plan_t pl = nullptr;
  rpca_status st = rpca_plan_create(&p, nullptr, 0, &pl);
  if (st != RPCA_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  Bufs b = pl->bufs;
  int flags = EF_RAW;
  cudaGraphConditionalHandle h = 0;
  int use_cond = 0;
  double *ev = nullptr, *vv = nullptr;
  cudaError_t e = cudaMalloc(&ev, sizeof(double) * T);
  if (e == cudaSuccess) e = cudaMalloc(&vv, sizeof(double) * T * T);
  void* args[] = {&b, &flags, &h, &use_cond, (void*)&G, &vv, &ev};
  if (e == cudaSuccess) e = launch(pl->ks.eig64, dim3(1), dim3(pl->ks.eig_threads), args, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  std::vector<double> evh(T), vvh((size_t)T * T), evs(T), vvs((size_t)T * T);
  if (e == cudaSuccess) e = cudaMemcpy(evh.data(), ev, sizeof(double) * T, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(vvh.data(), vv, sizeof(double) * T * T, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) {
    std::vector<int> idx(T);
    for (int i = 0; i < T; ++i) idx[i] = i;
    std::stable_sort(idx.begin(), idx.end(), [&](int a, int c) { return evh[a] > evh[c]; });
    for (int i = 0; i < T; ++i) {
      evs[i] = evh[idx[i]];
      for (int r = 0; r < T; ++r) vvs[r * T + i] = vvh[r * T + idx[i]];
    }
    e = cudaMemcpy(evals, evs.data(), sizeof(double) * T, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(evecs, vvs.data(), sizeof(double) * T * T, cudaMemcpyHostToDevice);
  }
  if (ev) cudaFree(ev);
  if (vv) cudaFree(vv);
  rpca_plan_destroy(pl);
  return cuda_status(e);
}

}  // extern "C"

// ---- one window split by pixel rows across processes: the steps one by one ----
static_assert(offsetof(RedState, l1) == offsetof(RedState, e2) + sizeof(double), "e2, l1 adjacent");

extern "C" {

rpca_status rpca_step_begin(rpca_plan_t pl, const float* X, float* L, float* S, uint8_t* mask, float theta,
                            void* stream) {
  if (!pl || !pl->p.sharded || !X || !L || !S) return RPCA_ERR_ARG;
  if (((uintptr_t)X | (uintptr_t)L | (uintptr_t)S) & 15u) return RPCA_ERR_ARG;
  if ((const void*)X == (const void*)L || (const void*)X == (const void*)S || L == S) return RPCA_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  Bufs b = pl->bufs;
  TmaMaps maps;
  memset(&maps, 0, sizeof(maps));
  int use_maps = 0;
  if (pl->use_fs) {
    const float* y1 = (const float*)(pl->ws + pl->lay.ybuf);
    if (!encode_map(&maps.x, X, pl->p.m, pl->p.T) || !encode_map(&maps.s, S, pl->p.m, pl->p.T) ||
        !encode_map(&maps.y0, L, pl->p.m, pl->p.T) || !encode_map(&maps.y1, y1, pl->p.m, pl->p.T))
      return RPCA_ERR_CUDA;
    use_maps = 1;
  }
  float* Sout = nullptr;
  float* Yout = nullptr;
  double mu_prev_scale = 0.0;
  void* a_begin[] = {&b, (void*)&X, &L, &S, &mask, &theta, &Sout, &Yout, &mu_prev_scale, &maps, &use_maps};
  CK(cudaLaunchKernel((void*)begin_kernel, dim3(1), dim3(64), a_begin, 0, s));
  return RPCA_OK;
}

rpca_status rpca_step_run(rpca_plan_t pl, int32_t step, void* stream) {
  if (!pl || !pl->p.sharded) return RPCA_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  Bufs b = pl->bufs;
  cudaGraphConditionalHandle h = 0;
  const double* nulld = nullptr;
  double* nullo = nullptr;
  int use_cond = 0;
  int flags = 0;
  void* a_pass[] = {&b};
  void* a_eig[] = {&b, &flags, &h, &use_cond, &nulld, &nullo, &nullo};
  switch (step) {
    case RPCA_STEP_INIT:
      CK(launch(pass_fn(pl, PM_INIT), pass_grid(pl), pass_block(pl), a_pass, s, pass_smem(pl)));
      return RPCA_OK;
    case RPCA_STEP_EIG_INIT:
      flags = EF_INIT | EF_EIG;
      CK(launch(eig_fn(pl), dim3(1), eig_block(pl), a_eig, s, eig_smem(pl)));
      return RPCA_OK;
    case RPCA_STEP_PASS:
      CK(launch(fused_fn(pl), fused_grid(pl), fused_block(pl), a_pass, s, fused_smem(pl)));
      return RPCA_OK;
    case RPCA_STEP_EIG:
      flags = EF_CHECK | EF_EIG;
      CK(launch(eig_fn(pl), dim3(1), eig_block(pl), a_eig, s, eig_smem(pl)));
      return RPCA_OK;
    case RPCA_STEP_FINAL: {
      const int fgrid = (int)std::min<int64_t>((pl->p.m + 255) / 256, 4096);
      CK(launch((void*)final_kernel, dim3(fgrid), dim3(256), a_pass, s));
      return RPCA_OK;
    }
    default:
      return RPCA_ERR_ARG;
  }
}

rpca_status rpca_step_sums(rpca_plan_t pl, double** gram, double** sums) {
  if (!pl || !pl->p.sharded || !gram || !sums) return RPCA_ERR_ARG;
  *gram = pl->bufs.red->G;
  *sums = &pl->bufs.red->e2;
  return RPCA_OK;
}

rpca_status rpca_step_done(rpca_plan_t pl, int32_t* done, rpca_result* out, void* stream) {
  if (!pl || !pl->p.sharded || !done) return RPCA_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  CK(cudaMemcpyAsync(pl->ctrl_host, pl->bufs.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  *done = pl->ctrl_host->done ? 1 : 0;
  if (out) fill_result(pl, *pl->ctrl_host, out);
  return RPCA_OK;
}

}  // extern "C"
