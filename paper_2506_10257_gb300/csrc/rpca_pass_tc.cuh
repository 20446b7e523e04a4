// rpca_pass_tc.cuh -- the fused per-iteration pass with its two dense
// contractions on the 5th-generation tensor cores (included inside namespace
// rpca by rpca_kernels.cuh).
//
// Same arithmetic as pass_kernel<TB, PM_FUSED> (Eq. 4-6 in the rearranged form
// described in rpca_device.cuh) except that
//     Q  = Z Wbar        (the part of Z that SVT removes), and
//     Z~ = Z' V          (the next iteration's Z in the current eigenbasis)
// are tcgen05.mma products: each 256-pixel tile is two M = 128 tiles, the
// pixel rows are the M rows, K = N = KP (T padded to 16 or 32).  Every thread
// writes its pixel row of Z (then Z') into shared memory in the canonical
// K-major layout, one thread issues the MMAs, the accumulators live in TMEM
// and each thread reads its own row back with tcgen05.ld (TMEM lane = pixel).
//
// Precision: SPLIT = true uses three products per K step,
//   A B ~ Ahi Bhi + Alo Bhi + Ahi Blo   (A = Ahi + Alo, B = Bhi + Blo),
// with TF32 or BF16 parts and FP32 accumulation ("TF32x3", "BF16x3");
// SPLIT = false is one TF32 product.  The Gram of Z~ stays FP32 on the CUDA
// cores (the rotated basis needs its small entries to FP32 relative accuracy).
#pragma once

template <int KP, bool BF16>
struct TcShape {
  static constexpr int EB = BF16 ? 2 : 4;                       // bytes per element
  static constexpr int KC = 16 / EB;                            // elements per 16-byte core row
  static constexpr uint32_t SBO = (KP / KC) * kTcLBO;           // next 8-row group
  static constexpr int A_BYTES = 128 * KP * EB;                 // one 128-row operand tile
  static constexpr int B_BYTES = KP * KP * EB;                  // one KP x KP operand
  static constexpr int KSTEP = BF16 ? 16 : 8;                   // K per tcgen05.mma
  static constexpr int NCOL = 4 * KP;                           // TMEM columns: Q and Z~ for 2 tiles
  static constexpr int TMEM_COLS = NCOL <= 32 ? 32 : (NCOL <= 64 ? 64 : 128);
  __host__ __device__ static constexpr uint32_t off(int r, int k) {
    return (uint32_t)((r / 8) * SBO + (k / KC) * kTcLBO + (r % 8) * 16 + (k % KC) * EB);
  }
};

// A region: 2 tiles x (hi, lo), also used for the Gram staging and the
// epilogue's reduction scratch once the MMAs of a tile are done
template <int TB, int KP, bool BF16>
__host__ __device__ constexpr size_t pass_tc_aregion() {
  using S = TcShape<KP, BF16>;
  const size_t a = 4 * (size_t)S::A_BYTES, z = (size_t)kTile * (TB + 4) * sizeof(float);
  return a > z ? a : z;
}

template <int TB, int KP, bool BF16>
__host__ __device__ constexpr size_t pass_tc_smem() {
  return 4 * (size_t)TcShape<KP, BF16>::B_BYTES + pass_tc_aregion<TB, KP, BF16>();
}

constexpr uint32_t kTcWaitLimit = 1u << 21;  // tries (each may suspend ~1 us) before a wait gives up

// The fused pass with tensor-core contractions over the tiles of this CTA
// (number lc of nc), on kPassThreads threads.  `tc_smem` holds
// pass_tc_smem<TB, KP, BF16>() bytes (128-byte aligned); `tmem` is a TMEM
// allocation of TcShape<KP, BF16>::TMEM_COLS columns owned by the CTA.
// Returns true in the CTA that wrote the final reduced sums (b.finalize).
template <int TB, int KP, bool BF16, bool SPLIT>
__device__ bool pass_tc_body(Bufs b, int lc, int nc, unsigned char* tc_smem, uint32_t tmem) {
  using SH = TcShape<KP, BF16>;
  using GM = GramMap<TB>;
  constexpr int ZS = TB + 4;
  static_assert(TB <= KP, "frames exceed the MMA width");
  static_assert(pass_tc_aregion<TB, KP, BF16>() >= (size_t)GM::NGRP * GM::NBLK * 16 * sizeof(float), "scratch");
  unsigned char* sWh = tc_smem;
  unsigned char* sWl = sWh + SH::B_BYTES;
  unsigned char* sVh = sWl + SH::B_BYTES;
  unsigned char* sVl = sVh + SH::B_BYTES;
  unsigned char* sA = sVl + SH::B_BYTES;  // tile s: hi at sA + 2 s A_BYTES, lo after it
  float* sZ = reinterpret_cast<float*>(sA);
  __shared__ double sRed[2][kPassThreads / 32];
  __shared__ double sScal[2 * kMaxGroups];
  __shared__ int sLast;
  __shared__ __align__(8) uint64_t sMbar;

  const Ctrl* ctrl = b.ctrl;
  if (solve_done_uniform(ctrl)) return false;
  const int tid = threadIdx.x, warp = tid >> 5;
  if (tid == 0) atomicMin(&b.red->t_start, gtimer());
  const int T = b.T;
  const int64_t m = b.m;
  const Job job = *b.job;
  const int kc = ctrl->k;
  const bool first = (kc == 0) && !__ldcg(&ctrl->warm);  // a warm start reads S0, Y0
  const float f_mu = ctrl->f_mu, inv_mu = ctrl->f_inv_mu, gamma = ctrl->f_gamma;
  const float inv_mu_nxt = ctrl->f_inv_mu_nxt;
  const float* Yin = (kc & 1) ? job.Y1 : job.Y0;
  float* Yout = (kc & 1) ? job.Y0 : job.Y1;

  // B operands: B[n][k] = Wbar[k][n] and V[k][n] (K-major), zero outside T
  for (int i = tid; i < KP * (KP / 4); i += kPassThreads) {
    const int n = i / (KP / 4), k4 = (i % (KP / 4)) * 4;
    float w[4], v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int k = k4 + u;
      const bool in = (k < T && n < T);
      w[u] = in ? b.eig->Wbar[k * kMaxT + n] : 0.f;
      v[u] = in ? b.eig->V32[k * kMaxT + n] : 0.f;
    }
    const uint32_t o = SH::off(n, k4);
    tc_store4<BF16>(sWh, sWl, o, w[0], w[1], w[2], w[3], SPLIT);
    tc_store4<BF16>(sVh, sVl, o, v[0], v[1], v[2], v[3], SPLIT);
  }
  if (tid == 0) mbar_init(&sMbar, 1);
  fence_async_smem();
  __syncthreads();
  tc_fence_after();
  const int sub = tid >> 7;            // which 128-row tile of the 256-pixel tile
  const int row = tid & 127;           // M row = TMEM lane
  unsigned char* myAh = sA + (size_t)(2 * sub) * SH::A_BYTES;
  unsigned char* myAl = myAh + SH::A_BYTES;
  const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;
  const uint32_t colQ = (uint32_t)(sub * KP), colZ = (uint32_t)(2 * KP + sub * KP);
  constexpr uint32_t idesc = tc_idesc(BF16 ? 1u : 2u, 128, KP);

  const bool gthr = tid < GM::NBLK * GM::NGRP;
  const int gblk = tid % GM::NBLK, ggrp = tid / GM::NBLK;
  int bi, bj;
  blk_coords(gblk, GM::NB, bi, bj);
  float acc[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) acc[i] = 0.f;
  float e2 = 0.f;
  uint32_t parity = 0;
  bool ok = true;

  // thread 0: the MMAs of one product for both 128-row tiles, then commit
  auto issue = [&](const unsigned char* Bh, const unsigned char* Bl, uint32_t col0) {
    tc_fence_after();
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      const uint32_t ah = smem_u32(sA + (size_t)(2 * s) * SH::A_BYTES), al = ah + SH::A_BYTES;
      const uint32_t d = tmem + col0 + (uint32_t)(s * KP);
#pragma unroll
      for (int kk = 0; kk < KP / SH::KSTEP; ++kk) {
        const uint32_t ko = (uint32_t)kk * (SH::KSTEP / SH::KC) * kTcLBO;
        const uint64_t dah = tc_desc(ah + ko, kTcLBO, SH::SBO), dbh = tc_desc(smem_u32(Bh) + ko, kTcLBO, SH::SBO);
        tc_mma<BF16>(d, dah, dbh, idesc, kk > 0 ? 1u : 0u);
        if (SPLIT) {
          const uint64_t dal = tc_desc(al + ko, kTcLBO, SH::SBO), dbl = tc_desc(smem_u32(Bl) + ko, kTcLBO, SH::SBO);
          tc_mma<BF16>(d, dal, dbh, idesc, 1u);
          tc_mma<BF16>(d, dah, dbl, idesc, 1u);
        }
      }
    }
    tc_commit(&sMbar);
  };

  const int64_t ntiles = (m + kTile - 1) / kTile;
  for (int64_t tile = lc; tile < ntiles; tile += nc) {
    const int64_t p = tile * kTile + tid;
    const bool valid = p < m;
    float x[TB], s[TB], d[TB], z[KP];
#pragma unroll
    for (int t = 0; t < TB; ++t) {
      const bool in = valid && t < T;
      x[t] = in ? job.X[t * m + p] : 0.f;
      s[t] = (in && !first) ? job.S[t * m + p] : 0.f;
      const float y = (in && !first) ? Yin[t * m + p] : 0.f;
      d[t] = y * inv_mu;
      z[t] = form_z(x[t], s[t], y, inv_mu);
    }
#pragma unroll
    for (int t = TB; t < KP; ++t) z[t] = 0.f;
    // A = Z (this thread's row), then Q = Z Wbar
#pragma unroll
    for (int k4 = 0; k4 < KP; k4 += 4)
      tc_store4<BF16>(myAh, myAl, SH::off(row, k4), z[k4], z[k4 + 1], z[k4 + 2], z[k4 + 3], SPLIT);
    fence_async_smem();
    __syncthreads();
    if (tid == 0) issue(sWh, sWl, 0u);
    ok = mbar_wait(&sMbar, parity, kTcWaitLimit) && ok;
    parity ^= 1u;
    tc_fence_after();
    float q[KP];
    tmem_ld_row<KP>(tmem + lane_base + colQ, q);
    // Eq. 5-6 and the residual, then Z' of the next iteration
#pragma unroll
    for (int t = 0; t < TB; ++t) {
      z[t] = 0.f;
      if (t < T) {
        const float r = s[t] + q[t];                       // X - L + Y/mu
        const float c = fminf(fmaxf(r, -gamma), gamma);    // clip to +-lambda/mu
        const float sn = r - c;                            // Eq. 5
        const float yn = f_mu * c;                         // Eq. 6
        const float e = c - d[t];                          // X - L - S'
        e2 = fmaf(e, e, e2);
        if (valid) {
          job.S[t * m + p] = sn;
          Yout[t * m + p] = yn;
          z[t] = form_z(x[t], sn, yn, inv_mu_nxt);
        }
      }
    }
    // A = Z', then Z~ = Z' V
#pragma unroll
    for (int k4 = 0; k4 < KP; k4 += 4)
      tc_store4<BF16>(myAh, myAl, SH::off(row, k4), z[k4], z[k4 + 1], z[k4 + 2], z[k4 + 3], SPLIT);
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    if (tid == 0) issue(sVh, sVl, 2u * KP);
    ok = mbar_wait(&sMbar, parity, kTcWaitLimit) && ok;
    parity ^= 1u;
    tc_fence_after();
    float zt[KP];
    tmem_ld_row<KP>(tmem + lane_base + colZ, zt);
    // stage Z~ rows for the FP32 Gram (aliases the A tiles, whose MMAs are done)
    float4* dst = reinterpret_cast<float4*>(&sZ[tid * ZS]);
#pragma unroll
    for (int j4 = 0; j4 < TB / 4; ++j4)
      dst[j4] = make_float4(valid ? zt[4 * j4] : 0.f, valid ? zt[4 * j4 + 1] : 0.f, valid ? zt[4 * j4 + 2] : 0.f,
                            valid ? zt[4 * j4 + 3] : 0.f);
    tc_fence_before();
    __syncthreads();
    if (gthr) gram_tile<TB>(sZ, acc, ggrp, bi, bj);
    __syncthreads();
  }
  if (!ok) atomicExch(&b.red->err, 1);
  tc_fence_before();
  __syncthreads();
  return pass_epilogue<TB, true>(b, acc, e2, 0.f, sZ, sRed, sScal, &sLast, gthr, ggrp, gblk, lc, nc);
}

template <int TB, int KP, bool BF16, bool SPLIT>
__global__ void __launch_bounds__(kPassThreads, 1) pass_tc_kernel(Bufs b) {
  using SH = TcShape<KP, BF16>;
  extern __shared__ __align__(128) unsigned char tc_smem_k[];
  __shared__ uint32_t sTmem;
  if (solve_done_uniform(b.ctrl)) return;
  if ((threadIdx.x >> 5) == 0) tmem_alloc(&sTmem, SH::TMEM_COLS);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  pass_tc_body<TB, KP, BF16, SPLIT>(b, blockIdx.x, gridDim.x, tc_smem_k, sTmem);
  tc_fence_before();
  __syncthreads();
  if ((threadIdx.x >> 5) == 0) tmem_dealloc(sTmem, SH::TMEM_COLS);
}
