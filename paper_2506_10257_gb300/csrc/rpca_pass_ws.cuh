// rpca_pass_ws.cuh -- the fused per-iteration pass as a warp-specialised,
// TMA-fed tensor-core pipeline (included inside namespace rpca).
//
// One CTA per SM strides over 128-pixel tiles.  Warp 0 (one lane) streams the
// X, S, Y tiles of the CTA's next tiles into a ring of shared-memory stages
// with TMA (box = 128 pixels x T frames; out-of-range pixels read as zero).
// Two compute warpgroups (warps 4-7 and 8-11) take alternate tiles; thread r
// of a warpgroup owns pixel r of its tile, which is also row r of the MMA
// tiles and lane r of TMEM.  Per tile a warpgroup
//   1. forms z = x - s + y/mu from the stage and writes it (hi/lo split) as the
//      A operand, and its leader issues Q = Z Wbar on the tensor cores;
//   2. reads its row of Q from TMEM, applies Eq. 5-6, accumulates the residual,
//      stores S', Y', hands the stage back to the producer, writes the next
//      iteration's z' as the A operand, and its leader issues Z~ = Z' V;
//   3. reads Z~ from TMEM and adds the tile into its FP32 Gram partial.
// While one warpgroup waits on an MMA the other computes, and the producer
// keeps loads in flight, so the SM keeps HBM busy.  Arithmetic is that of
// pass_tc_kernel; only the data movement differs.
#pragma once

template <int TB, int KP, bool BF16>
struct WsShape {
  using SH = TcShape<KP, BF16>;
  // Gram staging row stride (padded when the warpgroup's A buffers have room)
  static constexpr int ZS = (2 * SH::A_BYTES >= 128 * (TB + 4) * 4) ? TB + 4 : TB;
  static constexpr size_t B_REGION = 4 * (size_t)SH::B_BYTES;        // Wbar, V hi/lo
  static constexpr size_t A_REGION = 2 * 2 * (size_t)SH::A_BYTES;    // 2 warpgroups x hi/lo
  static constexpr size_t FIXED = B_REGION + A_REGION;
  // a warpgroup stages its Z~ tile for the Gram in its own hi/lo A buffers
  static_assert(2 * (size_t)SH::A_BYTES >= (size_t)128 * ZS * 4, "staging does not fit the A buffers");
  static constexpr size_t STAGE_MAX = (size_t)3 * TB * 128 * 4;      // X, S, Y tiles of up to TB frames
  static constexpr int NS = (FIXED + 4 * STAGE_MAX <= 220 * 1024) ? 4 : 2;
  static constexpr size_t SMEM = FIXED + NS * STAGE_MAX;
};

constexpr int kWsThreads = 384;

template <int TB, int KP, bool BF16>
__host__ __device__ constexpr size_t pass_ws_smem() {
  return WsShape<TB, KP, BF16>::SMEM;
}

template <int TB, int KP, bool BF16, bool SPLIT>
__global__ void __launch_bounds__(kWsThreads, 1) pass_ws_kernel(Bufs b) {
  using SH = TcShape<KP, BF16>;
  using WS = WsShape<TB, KP, BF16>;
  constexpr int NS = WS::NS;
  constexpr int ZS = WS::ZS;
  // Gram block map of a 128-thread warpgroup
  constexpr int NB = TB / 4, NBLK = NB * (NB + 1) / 2;
  constexpr int NGRP = (NBLK * 8 <= 128) ? 8 : (NBLK * 4 <= 128) ? 4 : 2;
  static_assert(NBLK * NGRP <= 128, "gram blocks exceed a warpgroup");
  extern __shared__ __align__(1024) unsigned char ws_smem[];
  unsigned char* sWh = ws_smem;
  unsigned char* sWl = sWh + SH::B_BYTES;
  unsigned char* sVh = sWl + SH::B_BYTES;
  unsigned char* sVl = sVh + SH::B_BYTES;
  unsigned char* sA = ws_smem + WS::B_REGION;                       // [wg][hi|lo]
  unsigned char* sStage = ws_smem + WS::FIXED;                      // [NS][X|S|Y][T][128]
  __shared__ __align__(8) uint64_t mb_full[NS], mb_empty[NS], mb_q[2], mb_z[2];
  __shared__ uint32_t sTmem;
  __shared__ double sRed[2][kWsThreads / 32];
  __shared__ double sScal[2 * kMaxGroups];
  __shared__ int sLast;

  const Ctrl* ctrl = b.ctrl;
  if (ctrl->done) return;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) atomicMin(&b.red->t_start, gtimer());
  const int T = b.T;
  const int64_t m = b.m;
  const Job* jobp = b.job;
  const int kc = ctrl->k;
  const bool first = (kc == 0) && !__ldcg(&ctrl->warm);  // a warm start reads S0, Y0
  const float f_mu = ctrl->f_mu, inv_mu = ctrl->f_inv_mu, gamma = ctrl->f_gamma;
  const float inv_mu_nxt = ctrl->f_inv_mu_nxt;
  float* Sp = jobp->S;
  float* Yout = (kc & 1) ? jobp->Y0 : jobp->Y1;
  const CUtensorMap* mapY = (kc & 1) ? &jobp->map_y1 : &jobp->map_y0;
  const uint32_t tile_bytes = (uint32_t)T * 128u * 4u;
  const size_t stage_bytes = 3 * (size_t)tile_bytes;

  // B operands: B[n][k] = Wbar[k][n], V[k][n] (K-major), zero outside T
  for (int i = tid; i < KP * (KP / 4); i += kWsThreads) {
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
  if (warp == 1) tmem_alloc(&sTmem, SH::TMEM_COLS);
  if (tid == 0) {
    for (int i = 0; i < NS; ++i) {
      mbar_init(&mb_full[i], 1);
      mbar_init(&mb_empty[i], 128);
    }
    for (int g = 0; g < 2; ++g) {
      mbar_init(&mb_q[g], 1);
      mbar_init(&mb_z[g], 1);
    }
  }
  fence_async_smem();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = sTmem;

  const int64_t ntiles = (m + 127) / 128;
  // local tiles of this CTA: blockIdx.x + j * gridDim.x, j = 0 .. nloc - 1
  const int64_t nloc = (ntiles > blockIdx.x) ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  bool ok = true;
  float e2 = 0.f;
  float acc[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) acc[i] = 0.f;
  const int wg = (warp >= 4) ? (warp - 4) / 4 : -1;      // compute warpgroup or -1
  const int r = tid & 127;                               // pixel row within a tile
  const int gblk = r % NBLK, ggrp = r / NBLK;
  const bool gthr = (wg >= 0) && (r < NBLK * NGRP);
  int bi, bj;
  blk_coords(gblk, NB, bi, bj);

  if (warp == 0) {
    // ---- producer: TMA loads of the X, S, Y tiles ----
    if (lane == 0) {
      tmap_acquire(&jobp->map_x);
      tmap_acquire(&jobp->map_s);
      tmap_acquire(mapY);
      for (int64_t j = 0; j < nloc; ++j) {
        const int st = (int)(j % NS);
        const uint32_t use = (uint32_t)(j / NS);
        if (j >= NS) ok = mbar_wait(&mb_empty[st], (use - 1) & 1u, kTcWaitLimit) && ok;
        unsigned char* dst = sStage + st * stage_bytes;
        const int x0 = (int)((blockIdx.x + j * gridDim.x) * 128);
        mbar_arrive_expect_tx(&mb_full[st], first ? tile_bytes : 3 * tile_bytes);
        tma_load_2d(dst, &jobp->map_x, x0, 0, &mb_full[st]);
        if (!first) {
          tma_load_2d(dst + tile_bytes, &jobp->map_s, x0, 0, &mb_full[st]);
          tma_load_2d(dst + 2 * tile_bytes, mapY, x0, 0, &mb_full[st]);
        }
      }
    }
  } else if (wg >= 0) {
    // ---- compute warpgroup wg: local tiles j = wg, wg + 2, ... ----
    unsigned char* Ah = sA + (size_t)(2 * wg) * SH::A_BYTES;
    unsigned char* Al = Ah + SH::A_BYTES;
    float* zst = reinterpret_cast<float*>(Ah);  // Gram staging reuses the A buffers once Z~ is in TMEM
    const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;
    const uint32_t colQ = (uint32_t)(wg * 2 * KP), colZ = colQ + (uint32_t)KP;
    const bool leader = (r == 0);
    constexpr uint32_t idesc = tc_idesc(BF16 ? 1u : 2u, 128, KP);
    const int bar_id = 1 + wg;
    uint32_t wuse = 0;  // tiles processed by this warpgroup
    auto issue = [&](const unsigned char* Bh, const unsigned char* Bl, uint32_t col, uint64_t* mb) {
      tc_fence_after();
      const uint32_t ah = smem_u32(Ah), al = smem_u32(Al);
#pragma unroll
      for (int kk = 0; kk < KP / SH::KSTEP; ++kk) {
        const uint32_t ko = (uint32_t)kk * (SH::KSTEP / SH::KC) * kTcLBO;
        const uint64_t dah = tc_desc(ah + ko, kTcLBO, SH::SBO), dbh = tc_desc(smem_u32(Bh) + ko, kTcLBO, SH::SBO);
        tc_mma<BF16>(tmem + col, dah, dbh, idesc, kk > 0 ? 1u : 0u);
        if (SPLIT) {
          const uint64_t dal = tc_desc(al + ko, kTcLBO, SH::SBO), dbl = tc_desc(smem_u32(Bl) + ko, kTcLBO, SH::SBO);
          tc_mma<BF16>(tmem + col, dal, dbh, idesc, 1u);
          tc_mma<BF16>(tmem + col, dah, dbl, idesc, 1u);
        }
      }
      tc_commit(mb);
    };
    for (int64_t j = wg; j < nloc; j += 2, ++wuse) {
      const int st = (int)(j % NS);
      const uint32_t use = (uint32_t)(j / NS);
      const int64_t p = (blockIdx.x + j * gridDim.x) * 128 + r;
      const bool valid = p < m;
      ok = mbar_wait(&mb_full[st], use & 1u, kTcWaitLimit) && ok;
      const float* tx = reinterpret_cast<const float*>(sStage + st * stage_bytes);
      const float* ts = tx + T * 128;
      const float* ty = ts + T * 128;
      float z[KP];
#pragma unroll
      for (int t = 0; t < KP; ++t) {
        z[t] = 0.f;
        if (t < T) z[t] = first ? tx[t * 128 + r] : form_z(tx[t * 128 + r], ts[t * 128 + r], ty[t * 128 + r], inv_mu);
      }
#pragma unroll
      for (int k4 = 0; k4 < KP; k4 += 4)
        tc_store4<BF16>(Ah, Al, SH::off(r, k4), z[k4], z[k4 + 1], z[k4 + 2], z[k4 + 3], SPLIT);
      fence_async_smem();
      named_bar(bar_id, 128);
      if (leader) issue(sWh, sWl, colQ, &mb_q[wg]);
      ok = mbar_wait(&mb_q[wg], wuse & 1u, kTcWaitLimit) && ok;
      tc_fence_after();
      float q[KP];
      tmem_ld_row<KP>(tmem + lane_base + colQ, q);
#pragma unroll
      for (int t = 0; t < KP; ++t) {
        const float qt = q[t];
        z[t] = 0.f;
        if (t < T) {
          const float x = tx[t * 128 + r];
          const float sv = first ? 0.f : ts[t * 128 + r];
          const float y = first ? 0.f : ty[t * 128 + r];
          const float d = y * inv_mu;
          const float rr = sv + qt;                          // X - L + Y/mu
          const float c = fminf(fmaxf(rr, -gamma), gamma);   // clip to +-lambda/mu
          const float sn = rr - c;                           // Eq. 5
          const float yn = f_mu * c;                         // Eq. 6
          const float e = c - d;                             // X - L - S'
          e2 = fmaf(e, e, e2);
          if (valid) {
            Sp[t * m + p] = sn;
            Yout[t * m + p] = yn;
            z[t] = form_z(x, sn, yn, inv_mu_nxt);
          }
        }
      }
      mbar_arrive(&mb_empty[st]);  // this thread is done with the stage
#pragma unroll
      for (int k4 = 0; k4 < KP; k4 += 4)
        tc_store4<BF16>(Ah, Al, SH::off(r, k4), z[k4], z[k4 + 1], z[k4 + 2], z[k4 + 3], SPLIT);
      fence_async_smem();
      tc_fence_before();
      named_bar(bar_id, 128);
      if (leader) issue(sVh, sVl, colZ, &mb_z[wg]);
      ok = mbar_wait(&mb_z[wg], wuse & 1u, kTcWaitLimit) && ok;
      tc_fence_after();
      float zt[KP];
      tmem_ld_row<KP>(tmem + lane_base + colZ, zt);
      float4* dst = reinterpret_cast<float4*>(&zst[r * ZS]);
#pragma unroll
      for (int j4 = 0; j4 < TB / 4; ++j4)
        dst[j4] = make_float4(zt[4 * j4], zt[4 * j4 + 1], zt[4 * j4 + 2], zt[4 * j4 + 3]);
      tc_fence_before();
      named_bar(bar_id, 128);
      if (gthr) {
        for (int pp = ggrp; pp < 128; pp += NGRP) {
          const float4 a = *reinterpret_cast<const float4*>(&zst[pp * ZS + 4 * bi]);
          const float4 c = *reinterpret_cast<const float4*>(&zst[pp * ZS + 4 * bj]);
          const float av[4] = {a.x, a.y, a.z, a.w};
          const float cv[4] = {c.x, c.y, c.z, c.w};
#pragma unroll
          for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[u * 4 + v] = fmaf(av[u], cv[v], acc[u * 4 + v]);
        }
      }
      named_bar(bar_id, 128);
    }
  }
  if (!ok) atomicExch(&b.red->err, 1);
  tc_fence_before();
  __syncthreads();
  if (warp == 1) tmem_dealloc(tmem, SH::TMEM_COLS);

  // ---- CTA partials: both warpgroups' Gram blocks, residual ----
  const int TT = T * T;
  float* red = reinterpret_cast<float*>(sStage);  // [wg][grp][blk][16]
  if (gthr) {
#pragma unroll
    for (int i = 0; i < 16; ++i) red[((wg * NGRP + ggrp) * NBLK + gblk) * 16 + i] = acc[i];
  }
  __syncthreads();
  for (int e = tid; e < NBLK * 16; e += kWsThreads) {
    float sum = 0.f;
    for (int g = 0; g < 2 * NGRP; ++g) sum += red[g * NBLK * 16 + e];
    int ebi, ebj;
    blk_coords(e / 16, NB, ebi, ebj);
    const int a = 4 * ebi + (e % 16) / 4, c = 4 * ebj + (e % 4);
    if (a < T && c < T) {
      b.gram_part[(int64_t)blockIdx.x * TT + a * T + c] = sum;
      b.gram_part[(int64_t)blockIdx.x * TT + c * T + a] = sum;
    }
  }
  {
    const double v0 = warp_sum_d((double)e2);
    if (lane == 0) sRed[0][warp] = v0;
    __syncthreads();
    if (tid == 0) {
      double s0 = 0;
      for (int w = 0; w < kWsThreads / 32; ++w) s0 += sRed[0][w];
      b.scal_part[2 * blockIdx.x] = s0;
      b.scal_part[2 * blockIdx.x + 1] = 0.0;
    }
  }
  cross_cta_reduce(b, true, sScal, &sLast, blockIdx.x, gridDim.x);
}
