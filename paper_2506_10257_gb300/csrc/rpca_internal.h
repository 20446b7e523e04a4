// rpca_internal.h -- what the library's translation units share beyond the
// public C ABI: a read-only view of a plan's device buffers.
#pragma once
#include "../../include/rpca.h"
#include "rpca_device.cuh"

namespace rpca {

struct PlanView {
  Bufs bufs;          // device buffers of the plan (finalize as created)
  int64_t m;
  int T;
  int max_grid;       // CTAs whose partials fit in the plan's workspace
  int tile;           // pixels per tile of the plan's passes
  int wide;           // the plan runs the tiled path
  double lambda;      // resolved lambda
  float* y1;          // second dual buffer (workspace)
  int cplx;           // complex window (T = 2 x frames)
};

// Kernels of the wide path (kMaxT < T <= kMaxTW), defined in rpca_wide.cu.
struct WideKernels {
  void* pass[4];        // per PassMode
  size_t pass_smem;
  int pass_threads;
  int tile;             // pixels per tile
  int per_sm;           // CTAs of a pass resident per SM
  void* eig;            // (Bufs, flags, handle, use_cond)
  size_t eig_smem;
  int eig_threads;
  void* pass_tc[4];     // fused pass on the tensor cores per rpca_precision (real TP <= 128; NULL: none)
  size_t pass_tc_smem[4];
  int pass_tc_threads;
};

// Bytes of the B operand images a tiled tensor-core plan keeps (0: none).
size_t wide_tc_img_bytes(int T, int precision);

// Fills *out for T real columns (complex windows: T = 2 x frames, cplx set);
// false when T is not a wide column count (real T <= kMaxT unless force) or a
// kernel attribute cannot be set.
bool wide_kernels(int T, bool cplx, bool force, WideKernels* out);

// Pixels per tile and CTAs per SM of the tiled pass for T real columns.
void wide_launch_shape(int T, int* tile, int* per_sm);

// rpca_plan_create with the tiled path forced for any frame count (the
// batched form runs every window of a batch that holds a wide or complex
// window through the tiled bodies).
rpca_status plan_create_ex(const rpca_params* p, bool force_wide, rpca_plan_t* out);

// Fills *v from a plan; RPCA_ERR_ARG for a null plan.
rpca_status plan_view(rpca_plan_t plan, PlanView* v);

// rpca_solve with two extra outputs written by the final step (either may be
// NULL): Sout gets S, Yout the final dual Y_k (the state a warm start resumes);
// mu_prev_scale >= 0 replaces the plan's mu_prev_scale for this solve and
// later ones (< 0 keeps it).
rpca_status plan_solve_ex(rpca_plan_t plan, const void* X, void* L, void* S, uint8_t* mask, float theta,
                          void* stream, float* Sout, float* Yout, double mu_prev_scale, rpca_result* out);

// Device control block of the plan.
Ctrl* plan_ctrl(rpca_plan_t plan);

// rpca_result of a solve from its control block (cplx: the rank counts each
// complex singular value once, not twice as the real embedding does).
void result_from_ctrl(double lambda, const Ctrl& c, rpca_result* out, int cplx = 0);

}  // namespace rpca
