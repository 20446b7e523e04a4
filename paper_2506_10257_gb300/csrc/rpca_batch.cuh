// rpca_batch.cuh -- many windows in one persistent, cooperative launch
// (included inside namespace rpca).
//
// Every CTA of the grid is resident for the whole launch.  The CTAs are split
// into contiguous ranges, one per window (sizes chosen on the host from the
// windows' work); a window's CTAs run its whole solve without returning to the
// host: the init pass, then per iteration the fused pass over the window's
// pixels.  The CTA that completes a pass's cross-CTA reduction runs that
// window's eigen-step right away and publishes it by bumping the window's
// generation counter; the other CTAs of the window wait on that counter
// (bounded, with back-off) and continue with the next pass.  While one
// window's CTAs wait for its eigen-step, the other windows' CTAs on the same
// GPU keep working, so one window's latency-bound step overlaps the others'
// bandwidth-bound passes.  A final per-CTA step writes L and the mask.
#pragma once

constexpr int kMaxBatch = 1024;         // windows per launch
constexpr int kMaxLanes = 1024;         // CTA ranges per launch
constexpr int kBatchThreads = kPassThreads;
static_assert(kEigThreads <= kBatchThreads, "the eigen-step runs on one batch CTA");

struct WinDesc {
  Bufs b;              // the window's plan buffers (finalize = 1, grid = CTAs it uses)
  const float* X;      // the window's input and outputs (frame-major m x T)
  float* L;
  float* S;
  uint8_t* mask;
  float theta;
  int TB;              // frame bucket of the window's kernels
  unsigned int gen;    // publications so far (0 when the host uploads the batch)
  unsigned int pdone;  // passes whose reduction has completed (paired lanes; 0 at upload)
};

// A lane: a contiguous range of CTAs that runs windows [w0, w1) one after the other.
struct LaneDesc {
  int cta0, ncta, w0, w1;
};

struct BatchDesc {
  int nwin;
  int nlanes;
  int paired;                      // lanes of >= 2 windows and >= 3 CTAs run them two at a time (run_lane)
  unsigned long long spin_limit;   // polls of a publication wait before it gives up
  unsigned int stop;               // set once any wait ran out: every later wait gives up at once
  int vrows;                       // wide eigen-steps: rows of V staged per step
  LaneDesc lane[kMaxLanes];
  WinDesc w[kMaxBatch];
};

// largest dynamic shared memory any window's steps need
__host__ __device__ constexpr size_t cmax(size_t a, size_t b) { return a > b ? a : b; }
template <int TB>
__host__ __device__ constexpr size_t batch_smem_tb() {
  return cmax(pass_simt_smem<TB>(), cmax(sizeof(Eig64Smem<TB>), sizeof(EigFastSmem<TB, float>)));
}
template <int TBMAX>
__host__ __device__ constexpr size_t batch_smem() {
  size_t s = batch_smem_tb<8>();
  if (TBMAX >= 12) s = cmax(s, batch_smem_tb<12>());
  if (TBMAX >= 16) s = cmax(s, batch_smem_tb<16>());
  if (TBMAX >= 20) s = cmax(s, batch_smem_tb<20>());
  if (TBMAX >= 24) s = cmax(s, batch_smem_tb<24>());
  if (TBMAX >= 32) s = cmax(s, batch_smem_tb<32>());
  return s;
}

// Copies every window's control block into out[0..nwin) (one CTA per window).
static __global__ void batch_gather_ctrl(const BatchDesc* bd, Ctrl* out) {
  const int w = blockIdx.x;
  if (w >= bd->nwin) return;
  const unsigned* src = reinterpret_cast<const unsigned*>(bd->w[w].b.ctrl);
  unsigned* dst = reinterpret_cast<unsigned*>(out + w);
  for (int i = threadIdx.x; i < (int)(sizeof(Ctrl) / 4); i += blockDim.x) dst[i] = __ldcg(src + i);
}

__device__ __forceinline__ unsigned int ld_acquire_u32(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Wait until the window's publication counter reaches `target`; false if the
// wait ran out.  Publications: 1 = state reset, 2 = first eigen-step, then one
// per iteration, so every CTA knows which value to expect.
// Once a wait of the launch has run out, `stop` makes every other wait give
// up at once, so a fault costs one wait limit, not one per window.
__device__ __forceinline__ bool gen_wait(const unsigned int* gen, unsigned int target, unsigned long long limit,
                                         unsigned int* stop) {
  __shared__ int sOk;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    unsigned long long n = 0;
    unsigned int ns = 64;
    while (ld_acquire_u32(gen) < target) {
      if (++n > limit || ld_acquire_u32(stop) != 0u) {
        ok = 0;
        atomicExch(stop, 1u);
        break;
      }
      __nanosleep(ns);
      if (ns < 1024) ns <<= 1;
    }
    sOk = ok;
  }
  __syncthreads();
  return sOk != 0;
}

__device__ __forceinline__ void gen_publish(unsigned int* gen) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(gen, 1u);
  }
}

// A wait ran out: mark the window failed so its other CTAs stop as well.
__device__ __forceinline__ void window_fail(Bufs b) {
  if (threadIdx.x == 0) {
    atomicExch(&b.red->err, 1);
    atomicExch(&b.ctrl->status, ST_ERR_TIMEOUT);
    atomicExch(&b.ctrl->done, 1);
  }
  __syncthreads();
}

// Steps of one window kind: the narrow (register-resident) pass and eigen-step
// for T <= kMaxT frames, or the tiled ones (wide or complex windows).
// The eigen-step runs once per iteration and is called, not inlined, which
// keeps the batch kernels' build short; the passes stay inlined.
template <int TB>
__device__ __noinline__ void narrow_eig_call(Bufs b, int flags, unsigned char* dsm) {
  if (b.eig64)
    eig64_body<TB>(b, flags, 0, 0, dsm);
  else
    eig_fast_body<TB, float>(b, flags, 0, 0, dsm);
}

template <int TB>
struct NarrowBody {
  static __device__ bool pass(Bufs b, bool init, int lc, int nc, unsigned char* dsm) {
    return init ? pass_body<TB, PM_INIT>(b, lc, nc, dsm) : pass_body<TB, PM_FUSED>(b, lc, nc, dsm);
  }
  static __device__ void eig(Bufs b, int flags, unsigned char* dsm, int) { narrow_eig_call<TB>(b, flags, dsm); }
};

// The window's state reset before its solve (the lane's CTA 0, thread 0).
__device__ __forceinline__ void reset_window(WinDesc& wd) {
  const Bufs b = wd.b;
  Job* j = b.job;
  j->X = wd.X;
  j->S = wd.S;
  j->Y0 = wd.L;
  j->L = wd.L;
  j->mask = wd.mask;
  j->theta = wd.theta;
  j->Sout = nullptr;
  j->Yout = nullptr;
  Ctrl* c = b.ctrl;
  c->k = 0;
  c->done = 0;
  c->status = 0;
  c->rank = 0;
  c->sweeps = 0;
  c->total_sweeps = 0;
  c->resid = 0.0;
  c->pass_ns = c->pass_cnt = c->eig_ns = c->eig_cnt = c->init_ns = 0ull;
  for (int i = 0; i < 4; ++i) c->eig_phase_ns[i] = 0ull;
  for (int i = 0; i < 3; ++i) c->pass_phase_ns[i] = 0ull;
  c->eig_rounds = 0;
  b.red->t_start = ~0ull;
  b.red->t_end = 0ull;
  b.red->t_loop = 0ull;
  b.red->t_l1 = 0ull;
  b.red->err = 0;
  for (int g = 0; g <= kMaxGroups; ++g) b.red->cnt[g] = 0u;
}

// Wait until *ctr reaches target (thread 0 polls, bounded, with back-off);
// false if the wait ran out (or another wait of the launch did).
__device__ __forceinline__ bool ctr_wait(const unsigned int* ctr, unsigned int target, unsigned long long limit,
                                         unsigned int* stop) {
  return gen_wait(ctr, target, limit, stop);
}

// The window's done flag as one value for the whole CTA (read by thread 0):
// a failure elsewhere may set it at any time, and every thread must take the
// same branch around the barriers that follow.
__device__ __forceinline__ bool window_done(const Bufs& b) {
  __shared__ int sDone;
  __syncthreads();
  if (threadIdx.x == 0) sDone = __ldcg(&b.ctrl->done);
  __syncthreads();
  return sDone != 0;
}

// Whether a lane runs its windows two at a time (the host sizes the windows'
// CTA counts by the same rule).
__host__ __device__ inline bool lane_is_paired(int paired, const LaneDesc& ld) {
  return paired && ld.w1 - ld.w0 >= 2 && ld.ncta >= 3;
}

// The windows of one lane.
//
// Sequential lane (paired = false): the lane's CTAs run its windows one after
// the other; per iteration every CTA runs its share of the window's pass, the
// CTA that completes the pass's reduction runs the eigen-step at once and
// publishes it, and the others wait for the publication.
//
// Paired lane: its windows run two at a time and its last CTA runs every
// eigen-step.  The windows alternate between two slots (slot s starts with
// window w0 + s; a slot whose window has finished takes the lane's next
// unstarted window).  The other CTAs (the pass CTAs) run slot 0's pass, then
// slot 1's, then slot 0's next, ...; the CTA completing a pass's reduction
// bumps the window's pass counter and goes on at once.  The eigen-step CTA
// takes the slots in the same order: it waits for the slot's pass, runs its
// eigen-step and publishes it.  So one window's latency-bound eigen-step (one
// SM) runs while the pass CTAs stream the other window's pixels, and a pass
// waits only when an eigen-step takes longer than the other slot's pass.
//
// Both sides see the same sequence of windows and iterations (the eigen-step's
// done flag decides it), so every wait has a matching publication; all waits
// are bounded, and a window whose wait ran out is marked failed and its slot
// moves on.  Disp::pass(wd, init, lc, nc, dsm) and Disp::eig(wd, flags, dsm,
// vrows) run the window's steps for its frame bucket.
template <class Disp>
__device__ void run_lane(BatchDesc* bd, const LaneDesc& ld, int lc, unsigned char* dsm, unsigned long long limit,
                         unsigned int* stop, int vrows, bool paired) {
  const int np = paired ? ld.ncta - 1 : ld.ncta;  // pass CTAs; in a paired lane CTA np runs the eigen-steps
  const bool eigc = paired && (lc == np);
  int w[2], it[2];
  w[0] = ld.w0;
  w[1] = (paired && ld.w0 + 1 < ld.w1) ? ld.w0 + 1 : -1;
  it[0] = it[1] = 0;
  int nxt = ld.w0 + (paired ? 2 : 1);  // next window of the lane to start
  auto advance = [&](int s) {
    w[s] = (nxt < ld.w1) ? nxt++ : -1;
    it[s] = 0;
  };
  while (w[0] >= 0 || w[1] >= 0) {
    for (int s = 0; s < 2; ++s) {
      if (w[s] < 0) continue;
      WinDesc& wd = bd->w[w[s]];
      const Bufs b = wd.b;
      if (eigc) {
        // ---- the eigen-step of this slot's pass it[s] ----
        if (ctr_wait(&wd.pdone, (unsigned)it[s] + 1u, limit, stop)) {
          __syncthreads();
          Disp::eig(wd, it[s] == 0 ? (EF_INIT | EF_EIG) : (EF_CHECK | EF_EIG), dsm, vrows);
        } else {
          window_fail(b);
        }
        gen_publish(&wd.gen);
        if (window_done(b)) advance(s);
        else ++it[s];
        continue;
      }
      // ---- pass CTAs ----
      if (it[s] == 0) {
        if (lc == 0) {
          if (threadIdx.x == 0) reset_window(wd);
          gen_publish(&wd.gen);
        }
        if (!gen_wait(&wd.gen, 1u, limit, stop)) window_fail(b);
      } else {
        // the eigen-step of iteration it - 1 (publication 2 + it - 1)
        if (!gen_wait(&wd.gen, 1u + (unsigned)it[s], limit, stop)) window_fail(b);
        if (window_done(b)) {
          final_body(b, lc, np);
          __syncthreads();
          advance(s);
          continue;
        }
      }
      if (window_done(b)) {
        // failed before its first pass: nothing more to run for this window;
        // the eigen-step CTA sees the failure through its own bounded wait
        advance(s);
        continue;
      }
      if (lc < b.grid) {
        const bool fin = Disp::pass(wd, it[s] == 0, lc, b.grid, dsm);
        if (fin) {
          __syncthreads();
          if (paired) {
            if (threadIdx.x == 0) {
              __threadfence();
              atomicAdd(&wd.pdone, 1u);
            }
          } else {
            Disp::eig(wd, it[s] == 0 ? (EF_INIT | EF_EIG) : (EF_CHECK | EF_EIG), dsm, vrows);
            gen_publish(&wd.gen);
          }
        }
      }
      __syncthreads();
      ++it[s];
    }
  }
}

// The narrow steps of a window by its frame bucket (<= TBMAX).
template <int TBMAX>
struct NarrowDisp {
  static __device__ bool pass(WinDesc& wd, bool init, int lc, int nc, unsigned char* dsm) {
    switch (wd.TB) {
      case 8: return NarrowBody<8>::pass(wd.b, init, lc, nc, dsm);
      case 12: if constexpr (TBMAX >= 12) return NarrowBody<12>::pass(wd.b, init, lc, nc, dsm); break;
      case 16: if constexpr (TBMAX >= 16) return NarrowBody<16>::pass(wd.b, init, lc, nc, dsm); break;
      case 20: if constexpr (TBMAX >= 20) return NarrowBody<20>::pass(wd.b, init, lc, nc, dsm); break;
      case 24: if constexpr (TBMAX >= 24) return NarrowBody<24>::pass(wd.b, init, lc, nc, dsm); break;
      case 32: if constexpr (TBMAX >= 32) return NarrowBody<32>::pass(wd.b, init, lc, nc, dsm); break;
      default: break;
    }
    return false;
  }
  static __device__ void eig(WinDesc& wd, int flags, unsigned char* dsm, int vrows) {
    switch (wd.TB) {
      case 8: NarrowBody<8>::eig(wd.b, flags, dsm, vrows); break;
      case 12: if constexpr (TBMAX >= 12) NarrowBody<12>::eig(wd.b, flags, dsm, vrows); break;
      case 16: if constexpr (TBMAX >= 16) NarrowBody<16>::eig(wd.b, flags, dsm, vrows); break;
      case 20: if constexpr (TBMAX >= 20) NarrowBody<20>::eig(wd.b, flags, dsm, vrows); break;
      case 24: if constexpr (TBMAX >= 24) NarrowBody<24>::eig(wd.b, flags, dsm, vrows); break;
      case 32: if constexpr (TBMAX >= 32) NarrowBody<32>::eig(wd.b, flags, dsm, vrows); break;
      default: break;
    }
  }
};

// Windows of frame bucket <= TBMAX (the batch's largest), lane by lane.
// One CTA per SM: under a 128-register cap (two CTAs per SM) the kernel
// spills (measured on 16 windows of 262144 x 20: 638 against 749 solves/s).
template <int TBMAX>
__global__ void __launch_bounds__(kBatchThreads, 1) batch_kernel(BatchDesc* bd) {
  extern __shared__ __align__(16) unsigned char batch_dsm[];
  const int nl = bd->nlanes;
  int l = 0;
  while (l + 1 < nl && (int)blockIdx.x >= bd->lane[l + 1].cta0) ++l;
  const LaneDesc ld = bd->lane[l];
  const int lc = (int)blockIdx.x - ld.cta0;
  if (lc < 0 || lc >= ld.ncta) return;
  const unsigned long long limit = bd->spin_limit;
  run_lane<NarrowDisp<TBMAX>>(bd, ld, lc, batch_dsm, limit, &bd->stop, 0, lane_is_paired(bd->paired, ld));
}
