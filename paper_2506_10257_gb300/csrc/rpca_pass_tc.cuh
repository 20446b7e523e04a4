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

// A region: 2 warpgroups x (hi, lo) operand tiles of 128 rows; after the
// last tile it is the epilogue's reduction scratch.  Then the Gram staging:
// one buffer of 32 rows per warp (up to 24 frames), or of 128 rows per
// warpgroup (32 frames, whose Gram blocks outnumber a warp's lanes).
template <int TB, int KP, bool BF16>
__host__ __device__ constexpr size_t pass_tc_aregion() {
  return 4 * (size_t)TcShape<KP, BF16>::A_BYTES;
}
template <int TB>
__host__ __device__ constexpr size_t pass_tc_zregion() {
  return (size_t)kTile * (TB + 4) * sizeof(float);
}

template <int TB, int KP, bool BF16>
__host__ __device__ constexpr size_t pass_tc_smem() {
  return 4 * (size_t)TcShape<KP, BF16>::B_BYTES + pass_tc_aregion<TB, KP, BF16>() + pass_tc_zregion<TB>();
}

constexpr uint32_t kTcWaitLimit = 1u << 21;  // tries (each may suspend for a bounded, system-dependent time) before a wait gives up

// The fused pass with tensor-core contractions over the tiles of this CTA
// (number lc of nc), on kPassThreads threads.  `tc_smem` holds
// pass_tc_smem<TB, KP, BF16>() bytes (128-byte aligned); `tmem` is a TMEM
// allocation of TcShape<KP, BF16>::TMEM_COLS columns owned by the CTA.
// Returns true in the CTA that wrote the final reduced sums (b.finalize).
//
// The two warpgroups work independently: warpgroup g takes the 128-pixel
// half g of every tile of the CTA, stages its rows of Z (then Z') as the A
// operand, and its first thread issues that half's MMAs into its own TMEM
// columns and commits them to its own mbarrier; the warpgroup syncs on a
// named barrier of its own.  So while one warpgroup waits on its MMAs the
// other computes, and no CTA-wide barrier runs between tiles.  The Gram of
// Z~ is accumulated per warp (a warp's 32 rows, its own lanes' blocks) up to
// 24 frames, per warpgroup at 32 frames.  Tiles inside the window of a window
// with exactly TB frames (after the first iteration) take the exact form:
// no frame or pixel guards, paired f32x2 elementwise arithmetic.
template <int TB, int KP, bool BF16, bool SPLIT>
__device__ bool pass_tc_body(Bufs b, int lc, int nc, unsigned char* tc_smem, uint32_t tmem) {
  using SH = TcShape<KP, BF16>;
  using GM = GramMap<TB>;
  constexpr int ZS = TB + 4;
  static_assert(TB <= KP, "frames exceed the MMA width");
  constexpr bool kWarpGram = TB <= 24;
  using WG = WarpGramMap<(TB <= 24 ? TB : 8)>;
  constexpr int NGRP_WG = GM::NGRP / 2;  // pixel groups of a warpgroup's Gram (32 frames)
  constexpr int kNgrp = kWarpGram ? WG::NGRP : GM::NGRP;
  static_assert(kWarpGram || (NGRP_WG >= 1 && GM::NBLK * NGRP_WG <= 128), "warpgroup Gram map");
  static_assert(pass_tc_aregion<TB, KP, BF16>() >= (size_t)kNgrp * GM::NBLK * 16 * sizeof(float), "scratch");
  unsigned char* sWh = tc_smem;
  unsigned char* sWl = sWh + SH::B_BYTES;
  unsigned char* sVh = sWl + SH::B_BYTES;
  unsigned char* sVl = sVh + SH::B_BYTES;
  unsigned char* sA = sVl + SH::B_BYTES;  // warpgroup g: hi at sA + 2 g A_BYTES, lo after it
  float* sZst = reinterpret_cast<float*>(sA + pass_tc_aregion<TB, KP, BF16>());  // Gram staging
  __shared__ double sRed[2][kPassThreads / 32];
  __shared__ double sScal[2 * kMaxGroups];
  __shared__ int sLast;
  __shared__ __align__(8) uint64_t sMbar[2];

  const Ctrl* ctrl = b.ctrl;
  if (solve_done_uniform(ctrl)) return false;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) atomicMin(&b.red->t_start, gtimer());
  const int T = b.T;
  const int64_t m = b.m;
  const Job job = *b.job;
  const int kc = __ldcg(&ctrl->k);
  const bool first = (kc == 0) && !__ldcg(&ctrl->warm);  // a warm start reads S0, Y0
  const float f_mu = __ldcg(&ctrl->f_mu), inv_mu = __ldcg(&ctrl->f_inv_mu), gamma = __ldcg(&ctrl->f_gamma);
  const float inv_mu_nxt = __ldcg(&ctrl->f_inv_mu_nxt);
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
      w[u] = in ? __ldcg(&b.eig->Wbar[k * kMaxT + n]) : 0.f;
      v[u] = in ? __ldcg(&b.eig->V32[k * kMaxT + n]) : 0.f;
    }
    const uint32_t o = SH::off(n, k4);
    tc_store4<BF16>(sWh, sWl, o, w[0], w[1], w[2], w[3], SPLIT);
    tc_store4<BF16>(sVh, sVl, o, v[0], v[1], v[2], v[3], SPLIT);
  }
  // A operands: the columns from TB to KP stay zero for the whole pass
  for (int i = tid; i < (int)(pass_tc_aregion<TB, KP, BF16>() / 16); i += kPassThreads)
    reinterpret_cast<float4*>(sA)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
  if (tid == 0) {
    mbar_init(&sMbar[0], 1);
    mbar_init(&sMbar[1], 1);
  }
  fence_async_smem();
  __syncthreads();
  tc_fence_after();

  const int wg = warp >> 2;            // warpgroup: half wg of every tile
  const int row = tid & 127;           // M row = TMEM lane
  unsigned char* myAh = sA + (size_t)(2 * wg) * SH::A_BYTES;
  unsigned char* myAl = myAh + SH::A_BYTES;
  uint64_t* mbar = &sMbar[wg];
  const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;
  const uint32_t colQ = (uint32_t)(wg * 2 * KP), colZ = colQ + (uint32_t)KP;
  const bool leader = row == 0;
  const int bar_id = 1 + wg;
  constexpr uint32_t idesc = tc_idesc(BF16 ? 1u : 2u, 128, KP);

  // Gram blocks: per warp (32 rows of the warp's own) or per warpgroup
  const int gtid = kWarpGram ? lane : row;
  const bool gthr = kWarpGram ? lane < GM::NBLK * WG::G : row < GM::NBLK * NGRP_WG;
  const int gblk = gtid % GM::NBLK, glocal = gtid / GM::NBLK;
  const int ggrp = kWarpGram ? warp * WG::G + glocal : wg * NGRP_WG + glocal;
  int bi, bj;
  blk_coords(gblk, GM::NB, bi, bj);
  float* zst = kWarpGram ? sZst + warp * 32 * ZS : sZst + wg * 128 * ZS;

  float acc[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) acc[i] = 0.f;
  float e2 = 0.f;
  uint64_t e2p = 0;
  const uint64_t inv_mu2 = f2_pack(inv_mu, inv_mu), f_mu2 = f2_pack(f_mu, f_mu);
  const uint64_t inv_nxt2 = f2_pack(inv_mu_nxt, inv_mu_nxt);
  uint32_t parity = 0;
  bool ok = true;

  // the warpgroup's leader: the MMAs of one product into TMEM column col0, then
  // commit (the K steps stop at the window's frames, not at the padded width)
  constexpr int KSTEPS = (TB + SH::KSTEP - 1) / SH::KSTEP;
  static_assert(KSTEPS * SH::KSTEP <= KP, "K steps exceed the operand width");
  auto issue = [&](const unsigned char* Bh, const unsigned char* Bl, uint32_t col0) {
    tc_fence_after();
    const uint32_t ah = smem_u32(myAh), al = smem_u32(myAl);
    const uint32_t d = tmem + col0;
#pragma unroll
    for (int kk = 0; kk < KSTEPS; ++kk) {
      const uint32_t ko = (uint32_t)kk * (SH::KSTEP / SH::KC) * kTcLBO;
      const uint64_t dah = tc_desc(ah + ko, kTcLBO, SH::SBO), dbh = tc_desc(smem_u32(Bh) + ko, kTcLBO, SH::SBO);
      tc_mma<BF16>(d, dah, dbh, idesc, kk > 0 ? 1u : 0u);
      if (SPLIT) {
        const uint64_t dal = tc_desc(al + ko, kTcLBO, SH::SBO), dbl = tc_desc(smem_u32(Bl) + ko, kTcLBO, SH::SBO);
        tc_mma<BF16>(d, dal, dbh, idesc, 1u);
        tc_mma<BF16>(d, dah, dbl, idesc, 1u);
      }
    }
    tc_commit(mbar);
  };
  // stage this thread's row (TB values) as the A operand, then the
  // warpgroup's leader issues the product against B into column col
  auto mma_row = [&](const float (&v)[TB], const unsigned char* Bh, const unsigned char* Bl, uint32_t col) {
#pragma unroll
    for (int k4 = 0; k4 < TB; k4 += 4)
      tc_store4<BF16>(myAh, myAl, SH::off(row, k4), v[k4], v[k4 + 1], v[k4 + 2], v[k4 + 3], SPLIT);
    fence_async_smem();
    tc_fence_before();
    named_bar(bar_id, 128);
    if (leader) issue(Bh, Bl, col);
    ok = mbar_wait(mbar, parity, kTcWaitLimit) && ok;
    parity ^= 1u;
    tc_fence_after();
  };

  const int64_t ntiles = (m + kTile - 1) / kTile;
  const bool exact_ok = T == TB && !first;
  auto tile_body = [&](auto exact_c, int64_t tile) {
    constexpr bool EXACT = decltype(exact_c)::value;
    const int TT = EXACT ? TB : T;
    const int64_t p = tile * kTile + wg * 128 + row;
    const bool valid = EXACT || p < m;
    float z[TB];
    float q[KP];
    if constexpr (EXACT) {
      uint64_t s2[TB / 2], d2[TB / 2], z2[TB / 2];
#pragma unroll
      for (int i = 0; i < TB / 2; ++i) {
        const int64_t o0 = (int64_t)(2 * i) * m + p, o1 = o0 + m;
        const uint64_t x2 = f2_pack(job.X[o0], job.X[o1]);
        s2[i] = f2_pack(job.S[o0], job.S[o1]);
        const uint64_t y2 = f2_pack(Yin[o0], Yin[o1]);
        d2[i] = f2_mul(y2, inv_mu2);
        z2[i] = f2_fma(y2, inv_mu2, f2_sub(x2, s2[i]));   // form_z per lane
        const float2 h = f2_unpack(z2[i]);
        z[2 * i] = h.x;
        z[2 * i + 1] = h.y;
      }
      mma_row(z, sWh, sWl, colQ);
      tmem_ld_row<KP>(tmem + lane_base + colQ, q);   // (Z Wbar)_j
#pragma unroll
      for (int i = 0; i < TB / 2; ++i) {
        const uint64_t q2 = f2_pack(q[2 * i], q[2 * i + 1]);
        const uint64_t r2 = f2_add(s2[i], q2);                         // X - L + Y/mu
        const float2 r = f2_unpack(r2);
        const uint64_t c2 = f2_pack(fminf(fmaxf(r.x, -gamma), gamma),  // clip to +-lambda/mu
                                    fminf(fmaxf(r.y, -gamma), gamma));
        const float2 sn = f2_unpack(f2_sub(r2, c2));                   // Eq. 5
        const uint64_t yn2 = f2_mul(f_mu2, c2);                        // Eq. 6
        const float2 yn = f2_unpack(yn2);
        const uint64_t e = f2_sub(c2, d2[i]);                          // X - L - S'
        e2p = f2_fma(e, e, e2p);
        const int64_t o0 = (int64_t)(2 * i) * m + p, o1 = o0 + m;
        job.S[o0] = sn.x;
        job.S[o1] = sn.y;
        Yout[o0] = yn.x;
        Yout[o1] = yn.y;
        // Z' = X - S' + Y'/mu' with X = Z + S - Y/mu and S' = S + Q - clip
        const float2 zn = f2_unpack(f2_fma(yn2, inv_nxt2, f2_add(f2_sub(f2_sub(z2[i], d2[i]), q2), c2)));
        z[2 * i] = zn.x;
        z[2 * i + 1] = zn.y;
      }
    } else {
      const bool frst = first;
      float x[TB], s[TB], d[TB];
#pragma unroll
      for (int t = 0; t < TB; ++t) {
        const bool in = valid && t < TT;
        x[t] = in ? job.X[t * m + p] : 0.f;
        s[t] = (in && !frst) ? job.S[t * m + p] : 0.f;
        const float y = (in && !frst) ? Yin[t * m + p] : 0.f;
        d[t] = y * inv_mu;
        z[t] = form_z(x[t], s[t], y, inv_mu);
      }
      mma_row(z, sWh, sWl, colQ);
      tmem_ld_row<KP>(tmem + lane_base + colQ, q);
#pragma unroll
      for (int t = 0; t < TB; ++t) {
        z[t] = 0.f;
        if (t < TT) {
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
    }
    // the next tile's rows of this warp into L2 while this one finishes
    if (tile + nc < ntiles) {
      const int64_t s0 = (tile + nc) * kTile + wg * 128 + 32 * (warp & 3);
      if (s0 < m)
        for (int t = lane; t < T; t += 32) {
          const int64_t off = (int64_t)t * m + s0;
          prefetch_l2(job.X + off);
          prefetch_l2(job.S + off);
          prefetch_l2(Yin + off);
        }
    }
    mma_row(z, sVh, sVl, colZ);                     // Z~ = Z' V
    float zt[KP];
    tmem_ld_row<KP>(tmem + lane_base + colZ, zt);
    // the Gram of Z~ (pixels outside the window add zero rows)
    if constexpr (kWarpGram) {
      float4* dst = reinterpret_cast<float4*>(&zst[lane * ZS]);
#pragma unroll
      for (int j4 = 0; j4 < TB / 4; ++j4)
        dst[j4] = make_float4(valid ? zt[4 * j4] : 0.f, valid ? zt[4 * j4 + 1] : 0.f, valid ? zt[4 * j4 + 2] : 0.f,
                              valid ? zt[4 * j4 + 3] : 0.f);
      __syncwarp();
      if (gthr) gram_rows<TB, 32, WG::G>(zst, acc, glocal, bi, bj);
      __syncwarp();
    } else {
      float4* dst = reinterpret_cast<float4*>(&zst[row * ZS]);
#pragma unroll
      for (int j4 = 0; j4 < TB / 4; ++j4)
        dst[j4] = make_float4(valid ? zt[4 * j4] : 0.f, valid ? zt[4 * j4 + 1] : 0.f, valid ? zt[4 * j4 + 2] : 0.f,
                              valid ? zt[4 * j4 + 3] : 0.f);
      named_bar(bar_id, 128);
      if (gthr) gram_rows<TB, 128, (NGRP_WG > 0 ? NGRP_WG : 1)>(zst, acc, glocal, bi, bj);
      named_bar(bar_id, 128);
    }
    tc_fence_before();
  };
  for (int64_t tile = lc; tile < ntiles; tile += nc) {
    // (uniform over the warpgroup)
    if (exact_ok && tile * kTile + (wg + 1) * 128 <= m)
      tile_body(BoolC<true>{}, tile);
    else
      tile_body(BoolC<false>{}, tile);
  }
  if (!ok) atomicExch(&b.red->err, 1);
  {
    const float2 h = f2_unpack(e2p);
    e2 += h.x + h.y;
  }
  tc_fence_before();
  __syncthreads();
  if (tid == 0) {
    mbar_inval(&sMbar[0]);
    mbar_inval(&sMbar[1]);
  }
  return pass_epilogue<TB, true, kNgrp>(b, acc, e2, 0.f, reinterpret_cast<float*>(sA), sRed, sScal, &sLast, gthr,
                                         ggrp, gblk, lc, nc);
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
