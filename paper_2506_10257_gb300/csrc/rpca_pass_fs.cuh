// rpca_pass_fs.cuh -- the FP32 CUDA-core fused pass fed by TMA (included
// inside namespace rpca after rpca_tc.cuh).
//
// Per pixel row the arithmetic is that of pass_body<TB, MODE> (Eq. 4-6 through
// the Gram, the rotated-basis Gram of the next Z); the data movement differs:
//   * the CTA's X, S, Y tiles (128 pixels x T frames each, the TMA box of the
//     plan's tensor maps) stream into a ring of NS shared-memory stages, so
//     several tiles per SM are in flight from HBM at all times;
//   * kFsWG warpgroups take the CTA's tiles in turn (thread r of a warpgroup
//     owns pixel r of its tile) and read their operands from the stage: no
//     global address arithmetic and no register held for a load in flight,
//     so the registers go to the two T x T contractions;
//   * a warpgroup stages its tile's Z~ rows in the same stage for its Gram
//     blocks; once done with tile j it refills the stage with tile j + NS
//     (one elected thread issues the TMA), so no producer warp is needed.
//     The warpgroups are not in lockstep: the one that owns tile j + NS may
//     reach it before tile j is done, when the stage's barrier still waits for
//     tile j and a parity wait would alias with the phase before.  So every
//     stage records the tile whose load was issued last (fs_issued), and a
//     consumer waits for its own tile's issue before the parity wait.
// S' and Y' are written straight to global memory (coalesced rows), and the
// next Z is formed as X - S' + Y'/mu' from the staged X.
// Every wait is bounded: a wait that runs out marks red->err and the pass
// finishes with whatever the stage holds (the host reports the error).
#pragma once

constexpr int kFsWG = 4;                       // warpgroups per CTA
constexpr int kFsThreads = 128 * kFsWG;
constexpr int kFsTile = 128;                   // pixels per tile (one per compute thread)
constexpr size_t kFsSmemCap = 224 * 1024;      // dynamic shared memory budget of a CTA

template <int TB>
struct FsShape {
  static constexpr int ZS = TB + 4;                                   // Gram staging row stride
  static constexpr int NB = TB / 4, NBLK = NB * (NB + 1) / 2;         // 4x4 Gram blocks
  static constexpr int NGRP = (NBLK * 8 <= 128) ? 8 : (NBLK * 4 <= 128) ? 4 : 2;
  static constexpr size_t WV = 2 * (size_t)TB * TB * sizeof(float);   // Wbar, V
  static constexpr size_t STAGE = 3 * (size_t)TB * kFsTile * sizeof(float);
  static constexpr int NS_FIT = (int)((kFsSmemCap - WV) / STAGE);
  static constexpr int NS = NS_FIT > 8 ? 8 : NS_FIT;
  static constexpr size_t SMEM = (size_t)NS * STAGE + WV;
  // NS > kFsWG keeps tiles in flight beyond the ones being computed (all
  // buckets but 32 frames, whose stages hold only one tile per warpgroup)
  static_assert(NS >= kFsWG, "every warpgroup needs a stage");
  static_assert(NS <= 8, "barrier array size");
  static_assert((size_t)kFsTile * ZS * sizeof(float) <= STAGE, "Gram staging must fit a stage");
  static_assert((size_t)kFsWG * NGRP * NBLK * 16 * sizeof(float) <= NS * STAGE, "reduction scratch");
  static_assert(NBLK * NGRP <= 128, "Gram blocks exceed a warpgroup");
};

// Waits (bounded) until the stage's last issued load is local tile j.
__device__ __forceinline__ bool wait_issued(const int* issued, int j, uint32_t limit) {
  const volatile int* v = issued;
  for (uint32_t it = 0; it < limit; ++it) {
    if (*v == j) return true;
    __nanosleep(64);
  }
  return false;
}

// One pass over the pixels of this CTA (number lc of nc) with kFsThreads
// threads; `dsm` holds FsShape<TB>::SMEM bytes (1024-byte aligned).  Needs the
// job's tensor maps (m % 4 == 0).  Returns true in the CTA that wrote the final
// reduced sums (when b.finalize).
template <int TB, int MODE>
__device__ bool pass_fs_body(Bufs b, int lc, int nc, unsigned char* dsm) {
  using FS = FsShape<TB>;
  constexpr bool kGram = (MODE != PM_UPDATE);
  constexpr int NS = FS::NS, ZS = FS::ZS;
  unsigned char* sStage = dsm;                                       // [NS][X | S | Y rows][128]
  float* sW = reinterpret_cast<float*>(dsm + (size_t)NS * FS::STAGE);  // Wbar, row-major TB x TB
  float* sV = sW + TB * TB;                                          // V
  __shared__ __align__(8) uint64_t fs_full[NS];
  __shared__ int fs_issued[NS];  // local tile whose load into the stage was issued last
  __shared__ double sRed[2][kFsThreads / 32];
  __shared__ double sScal[2 * kMaxGroups];
  __shared__ int sLast;

  const Ctrl* ctrl = b.ctrl;
  if (solve_done_uniform(ctrl)) return false;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) atomicMin(&b.red->t_start, gtimer());
  const int T = b.T;
  const int64_t m = b.m;
  const Job* jobp = b.job;
  const int kc = __ldcg(&ctrl->k);
  const bool first = (kc == 0) && !__ldcg(&ctrl->warm);  // a warm start reads S0, Y0
  const bool xonly = (MODE == PM_INIT) || first;
  const float f_mu = __ldcg(&ctrl->f_mu), inv_mu = __ldcg(&ctrl->f_inv_mu), gamma = __ldcg(&ctrl->f_gamma);
  const float inv_mu_nxt = __ldcg(&ctrl->f_inv_mu_nxt);
  float* Sp = jobp->S;
  float* Yout = (kc & 1) ? jobp->Y0 : jobp->Y1;
  const CUtensorMap* mapY = (kc & 1) ? &jobp->map_y1 : &jobp->map_y0;
  const uint32_t rows_bytes = (uint32_t)T * kFsTile * 4u;

  if (MODE != PM_INIT) {
    for (int i = tid; i < TB * TB; i += kFsThreads) {
      const int r = i / TB, c = i % TB;
      const bool in = (r < T && c < T);
      sW[r * TB + c] = in ? __ldcg(&b.eig->Wbar[r * kMaxT + c]) : 0.f;
      sV[r * TB + c] = in ? __ldcg(&b.eig->V32[r * kMaxT + c]) : 0.f;
    }
  }
  const int64_t ntiles = (m + kFsTile - 1) / kFsTile;
  const int64_t nloc = (ntiles > lc) ? (ntiles - 1 - lc) / nc + 1 : 0;  // tiles lc, lc + nc, ...
  // TMA of local tile j into its stage j % NS, completion counted on fs_full;
  // the expected bytes are armed before the stage records tile j as issued
  auto load_tile = [&](int64_t j) {
    const int st = (int)(j % NS);
    unsigned char* dst = sStage + (size_t)st * FS::STAGE;
    const int x0 = (int)((lc + j * nc) * kFsTile);
    mbar_arrive_expect_tx(&fs_full[st], xonly ? rows_bytes : 3 * rows_bytes);
    tma_load_2d(dst, &jobp->map_x, x0, 0, &fs_full[st]);
    if (!xonly) {
      tma_load_2d(dst + rows_bytes, &jobp->map_s, x0, 0, &fs_full[st]);
      tma_load_2d(dst + 2 * rows_bytes, mapY, x0, 0, &fs_full[st]);
    }
    __threadfence_block();
    *reinterpret_cast<volatile int*>(&fs_issued[st]) = (int)j;
  };
  const int wg = tid >> 7;   // warpgroup
  const int r = tid & 127;   // pixel of the tile
  if (r == 0) {
    // each warpgroup leader issues the refills of its own tiles
    tmap_acquire(&jobp->map_x);
    if (!xonly) {
      tmap_acquire(&jobp->map_s);
      tmap_acquire(mapY);
    }
  }
  if (tid == 0) {
    for (int i = 0; i < NS; ++i) {
      mbar_init(&fs_full[i], 1);
      fs_issued[i] = -1;
    }
    for (int64_t j = 0; j < nloc && j < NS; ++j) load_tile(j);
  }
  __syncthreads();

  bool ok = true;
  float acc[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) acc[i] = 0.f;
  float e2 = 0.f, l1 = 0.f;
  const int gblk = r % FS::NBLK, ggrp = r / FS::NBLK;
  const bool gthr = kGram && (r < FS::NBLK * FS::NGRP);
  int bi, bj;
  blk_coords(gblk, FS::NB, bi, bj);

  {
    // ---- warpgroup wg: local tiles wg, wg + kFsWG, ... ----
    for (int64_t j = wg; j < nloc; j += kFsWG) {
      const int st = (int)(j % NS);
      const uint32_t use = (uint32_t)(j / NS);
      const int64_t p = (lc + j * nc) * kFsTile + r;
      const bool valid = p < m;  // pixels past m arrive as zeros
      ok = wait_issued(&fs_issued[st], (int)j, kTcWaitLimit) && ok;
      ok = mbar_wait(&fs_full[st], use & 1u, kTcWaitLimit) && ok;
      float* tx = reinterpret_cast<float*>(sStage + (size_t)st * FS::STAGE);
      const float* ts = tx + T * kFsTile;
      const float* ty = ts + T * kFsTile;
      float zt[TB];
      if (MODE == PM_INIT) {
#pragma unroll
        for (int t = 0; t < TB; ++t) {
          const float x = (t < T) ? tx[t * kFsTile + r] : 0.f;
          zt[t] = x;
          e2 = fmaf(x, x, e2);
          l1 += fabsf(x);
        }
      } else {
        // z = X - S + Y/mu (the argument of Eq. 4); S, Y and X are read again
        // from the stage below instead of being held in registers
        float z[TB];
#pragma unroll
        for (int t = 0; t < TB; ++t) {
          const bool in = t < T;
          const float x = in ? tx[t * kFsTile + r] : 0.f;
          const float sv = (in && !first) ? ts[t * kFsTile + r] : 0.f;
          const float y = (in && !first) ? ty[t * kFsTile + r] : 0.f;
          z[t] = form_z(x, sv, y, inv_mu);
        }
        if (MODE == PM_GRAM) {
          vec_mat<TB>(z, sV, zt);
        } else {
          float q[TB];
          vec_mat<TB>(z, sW, q);   // (Z Wbar)_j
#pragma unroll
          for (int t = 0; t < TB; ++t) {
            float zn = 0.f;
            if (t < T) {
              const float sv = first ? 0.f : ts[t * kFsTile + r];
              const float d = (first ? 0.f : ty[t * kFsTile + r]) * inv_mu;
              const float rr = sv + q[t];                        // X - L + Y/mu
              const float c = fminf(fmaxf(rr, -gamma), gamma);   // clip to +-lambda/mu
              const float sn = rr - c;                           // Eq. 5
              const float yn = f_mu * c;                         // Eq. 6
              const float e = c - d;                             // X - L - S'
              e2 = fmaf(e, e, e2);
              if (valid) {
                Sp[t * m + p] = sn;
                Yout[t * m + p] = yn;
                zn = form_z(tx[t * kFsTile + r], sn, yn, inv_mu_nxt);   // Z' = X - S' + Y'/mu'
              }
            }
            q[t] = zn;
          }
          if (MODE == PM_FUSED) {
            vec_mat<TB>(q, sV, zt);
          }
        }
      }
      if (kGram) {
        // the warpgroup is done reading the stage: its Z~ rows go there
        named_bar(1 + wg, 128);
        float4* dst = reinterpret_cast<float4*>(&tx[r * ZS]);
#pragma unroll
        for (int j4 = 0; j4 < TB / 4; ++j4)
          dst[j4] = make_float4(zt[4 * j4], zt[4 * j4 + 1], zt[4 * j4 + 2], zt[4 * j4 + 3]);
        named_bar(1 + wg, 128);
        if (gthr) gram_rows<TB, kFsTile, FS::NGRP>(tx, acc, ggrp, bi, bj);
      }
      // this thread's stage accesses come before the next TMA write into it
      fence_async_smem();
      named_bar(1 + wg, 128);
      if (r == 0 && j + NS < nloc) load_tile(j + NS);
    }
  }
  if (!ok) atomicExch(&b.red->err, 1);
  __syncthreads();
  if (tid == 0) {
    // every issued load has been waited for; after a wait that ran out, give
    // the copies still in flight (bounded) time to land before the exit
    for (int i = 0; i < NS; ++i) {
      const int jl = fs_issued[i];
      if (jl >= 0 && !mbar_wait(&fs_full[i], (uint32_t)(jl / NS) & 1u, kTcWaitLimit)) atomicExch(&b.red->err, 1);
      mbar_inval(&fs_full[i]);
    }
  }

  // ---- CTA partials: the warpgroups' Gram blocks, residual, ||X|| sums ----
  const int TT = T * T;
  if (kGram) {
    float* red = reinterpret_cast<float*>(sStage);  // [wg][grp][blk][16]
    if (gthr) {
#pragma unroll
      for (int i = 0; i < 16; ++i) red[((wg * FS::NGRP + ggrp) * FS::NBLK + gblk) * 16 + i] = acc[i];
    }
    __syncthreads();
    for (int e = tid; e < FS::NBLK * 16; e += kFsThreads) {
      float sum = 0.f;
      for (int g = 0; g < kFsWG * FS::NGRP; ++g) sum += red[g * FS::NBLK * 16 + e];
      int ebi, ebj;
      blk_coords(e / 16, FS::NB, ebi, ebj);
      const int a = 4 * ebi + (e % 16) / 4, c = 4 * ebj + (e % 4);
      if (a < T && c < T) {
        b.gram_part[(int64_t)lc * TT + a * T + c] = sum;
        b.gram_part[(int64_t)lc * TT + c * T + a] = sum;
      }
    }
  }
  {
    const double v0 = warp_sum_d((double)e2), v1 = warp_sum_d((double)l1);
    if (lane == 0) {
      sRed[0][warp] = v0;
      sRed[1][warp] = v1;
    }
    __syncthreads();
    if (tid == 0) {
      double s0 = 0, s1 = 0;
      for (int w = 0; w < kFsThreads / 32; ++w) {
        s0 += sRed[0][w];
        s1 += sRed[1][w];
      }
      b.scal_part[2 * lc] = s0;
      b.scal_part[2 * lc + 1] = s1;
    }
  }
  return cross_cta_reduce(b, kGram, sScal, &sLast, lc, nc);
}

template <int TB, int MODE>
__global__ void __launch_bounds__(kFsThreads, 1) pass_fs_kernel(Bufs b) {
  extern __shared__ __align__(1024) unsigned char fs_dsm[];
  pass_fs_body<TB, MODE>(b, blockIdx.x, gridDim.x, fs_dsm);
}
