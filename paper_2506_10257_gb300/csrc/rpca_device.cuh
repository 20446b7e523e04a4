// rpca_device.cuh -- device side of the GB300 PCP solver (kernels + shared state).
//
// One iteration of the augmented-Lagrangian method (Sec. II-A, Eq. 4-6) on the
// m x T Casorati matrix X (frame-major: element (p, t) at X[t*m + p]):
//
//   Z   = X - S + Y/mu                       (argument of Eq. 4)
//   L   = D_{1/mu}(Z) = Z - Z Wbar,  Wbar = V diag(min(1, tau/sigma)) V^T,
//         with Z^T Z = V diag(sigma^2) V^T, tau = 1/mu      (Eq. 4 through the Gram)
//   R   = X - L + Y/mu  (= S + Z Wbar)       (argument of Eq. 5)
//   S'  = shrink_{lambda/mu}(R)              (Eq. 5)
//   Y'  = Y + mu (X - L - S') = mu * clip(R, +-lambda/mu)   (Eq. 6)
//   E   = X - L - S' = clip(R) - Y/mu        (stopping test, Sec. II-A)
//
// The identities on the right are exact rearrangements (R - S' = clip(R)).
// The fused pass computes all of that per pixel row in one sweep over
// X, S, Y, and in the same sweep accumulates the Gram of the NEXT iteration's
// Z' = X - S' + Y'/mu' in the basis V of the current eigenvectors, so the
// eigen-decomposition of the next iteration starts from a nearly diagonal
// matrix whose FP32 accumulation error is relative to each eigenvalue.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace rpca {

constexpr int kMaxT = 32;            // largest frame count of the register-resident passes
constexpr int kMaxTW = 224;          // largest frame count of the wide (shared-memory tiled) path
constexpr int kWideLogSweeps = 30;   // Jacobi sweeps one wide eigen-step may take (and log)
constexpr int kPassThreads = 256;    // one pixel per thread per tile
constexpr int kTile = kPassThreads;  // pixels per CTA tile
constexpr int kPassCtasPerSm = 1;    // resident CTAs of the narrow passes per SM
constexpr int kGroup = 16;           // CTAs per first-level reduction group
constexpr int kMaxGroups = 64;

// Pass kinds.
enum PassMode { PM_INIT = 0, PM_FUSED = 1, PM_UPDATE = 2, PM_GRAM = 3 };
// Eig-kernel phases.
// EF_FULL: allow the cold sweep cap while keeping the basis (first SVT of a warm start).
enum EigFlags { EF_INIT = 1, EF_CHECK = 2, EF_EIG = 4, EF_FULL = 16 };

// Iteration control block (device resident, one per plan).
struct Ctrl {
  int k;             // completed iterations
  int done;          // 1 once converged, out of iterations or failed
  int status;        // rpca_status
  int rank;          // singular values above tau in the last SVT
  int sweeps;        // Jacobi sweeps of the last eigensolve
  int total_sweeps;  // over the whole solve
  int max_iter;
  int schedule;      // 0 IALM, 1 FIXED_L1
  double mu_cur;     // mu of the next pass (iteration k+1)
  double mu_nxt;     // mu of iteration k+2 (forms Z' in the fused pass)
  double mu_max;
  double lambda;
  double rho;
  double mu0_scale;
  double mu_max_factor;
  double tol;
  double normX2;     // ||X||_F^2
  double normX;      // ||X||_F
  double normX1;     // sum |X_ij|
  double resid;      // relative residual of iteration k
  double jacobi_eps; // graded off-diagonal threshold of the Jacobi sweeps
  int warm_sweeps;   // sweep cap once warm started
  int cold_sweeps;   // sweep cap of the first eigensolve
  int warm;          // 1: the solve starts from S0 (in S) and Y0 (in the L buffer)
  int pad_w;
  double mu_init;       // > 0: first mu of the solve instead of the schedule's
  double mu_prev_scale; // > 0 with warm: first mu = this times the plan's previous final mu
  // FP32 copies used by the passes (rounded once from the FP64 values).
  float f_mu, f_inv_mu, f_gamma, f_inv_mu_nxt;
  // Device-side timing of the solve (globaltimer, ns): fused/update passes
  // after the first, eigen-steps, and the init pass.
  unsigned long long pass_ns, pass_cnt, eig_ns, eig_cnt, init_ns;
  // eigen-step phase split (ns, summed over calls): control+load, sweeps,
  // rotation product, basis update + Wbar
  unsigned long long eig_phase_ns[4];
  // pass phase split (ns, summed over the timed passes): CTA work up to the
  // last CTA's partials, first-level reduction, final reduction
  unsigned long long pass_phase_ns[3];
  int eig_rounds;    // Jacobi rounds executed (summed)
  int pad_;
};

// Eigen data handed from the eig kernel to the passes.
struct EigState {
  float Wbar[kMaxT * kMaxT];   // row-major T x T (row t, col j)
  float V32[kMaxT * kMaxT];    // basis of the next rotated Gram, row-major
  double evals[kMaxT];
};

// Cross-CTA reduction state (two levels, last-arriving CTA reduces).
struct RedState {
  double G[kMaxT * kMaxT];     // final Gram (row-major): the CTAs' FP32 partials summed in two-float
                               // arithmetic, stored in FP64
  double e2;                   // sum of E^2 (or ||X||_F^2 in the init pass)
  double l1;                   // sum |X| (init pass)
  unsigned long long t_start;  // earliest CTA start of the last pass (globaltimer)
 unsigned long long t_end;    // end of its final reduction
  unsigned long long t_loop;   // latest time a CTA finished its partials
  unsigned long long t_l1;     // latest end of a first-level group reduction
  int ngroups_last;            // group partials left by the last pass
  int gram_last;               // whether that pass produced a Gram
  int err;                     // set by a pass whose bounded device wait ran out
  unsigned int cnt[kMaxGroups + 1];
};

// Pointers of the current solve (written by a tiny kernel before each graph
// launch, so one instantiated graph serves every call).
struct Job {
  // TMA descriptors of the frame-major X, S, Y0, Y1 (box 128 pixels x T frames),
  // written per solve when the pixel count allows TMA (m % 4 == 0)
  CUtensorMap map_x, map_s, map_y0, map_y1;
  const float* X;
  float* S;
  float* Y0;        // dual ping-pong buffer 0 (the caller's L buffer)
  float* Y1;        // dual ping-pong buffer 1 (workspace)
  float* L;
  uint8_t* mask;
  float theta;
  float* Sout;      // when set, the final step also copies S here
  float* Yout;      // ... and the final dual Y_k here (the state a warm start resumes)
};

// Per-solve tensor maps handed to the begin kernel as a kernel parameter.
struct TmaMaps {
  CUtensorMap x, s, y0, y1;
};

struct Bufs {
  Ctrl* ctrl;
  EigState* eig;
  RedState* red;
  Job* job;
  float* gram_part;    // [grid][T*T] FP32 partial Gram of each CTA
  float2* group_part;  // [ngroups][T*T] sums of the partials of each group of CTAs as two-float
                       // (hi, lo) values: hi + lo carries the sum to about 2^-48 of its terms
  double* scal_part;   // [grid][2]
  double* gscal_part;  // [ngroups][2]
  int64_t m;
  int T;
  int grid;
  int ngroups;
  int cplx;            // complex window: T = 2 x frames, columns (2t, 2t + 1) = (Re, Im) of frame t
  int wide;            // tiled path: the reduced Gram goes to Gw (T x T), else to red->G (kMaxT stride)
  int finalize;        // 1: the pass itself sums the group partials into red->G, e2, l1;
                       // 0: the next eigen-step does (saves a serial reduction level)
  int eig64;           // narrow eigen-step: 1 FP64 Jacobi rotations and basis arithmetic, 0 FP32
  // T > kMaxT ("wide" windows): the reduced Gram, Wbar and V live in these
  // T x T row-major arrays of the workspace instead of red->G and EigState.
  double* Gw;          // summed partial Grams as FP64 (also scratch of the eigen-step)
  float* Ww;
  float* Vw;
  double* evw;
  unsigned char* wtc_img;  // tiled tensor-core pass: B operand images of Wbar and V (NULL: unused)
  int wtc;            // their arithmetic: 0 none, 1 TF32x3, 2 BF16x3
  float2* rot_log;    // wide eigen-step: (c, s) of every rotated pair of every executed round
  int* rot_k;         // ... its columns p | q << 8, bit 16 set on the first rotation of a round
  int* rot_rnd;       // ... per round: round number and rotated pairs
};

}  // namespace rpca
