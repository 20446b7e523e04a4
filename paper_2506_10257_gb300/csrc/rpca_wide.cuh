// rpca_wide.cuh -- the iteration for windows of many frames (kMaxT < T <= kMaxTW) and for
// complex windows: device bodies and kernels (host side in rpca_wide.cu).
//
// Same algebra as the register-resident path (see rpca_device.cuh): per
// iteration one fused pass over the pixels (Eq. 4-6 through the Gram of Z, the
// residual of Sec. II-A, and the rotated Gram of the next Z) and one
// eigen-step on one CTA.  With T up to 224 a pixel row no longer fits in one
// thread's registers, so the pass works on tiles of 32 pixels x TP frames
// (TP = T rounded up to a multiple of 32) staged in shared memory:
//   1. X, S, Y of the tile -> shared memory, frame-major [t][p] (coalesced);
//   2. Q = Z Wbar (Z = X - S + Y/mu formed on the fly), Wbar streamed through
//      shared memory 32 rows at a time; lane = pixel, warp = 1/8 of the
//      columns, so every Wbar read is a warp-wide broadcast;
//   3. the Eq. 5-6 update of the lane's pixel for the warp's frames, S' and
//      Y' written straight to HBM (coalesced), Z' kept in shared memory;
//   4. U = Z' V (the next Gram's basis), written pixel-major;
//   5. the partial Gram U^T U accumulated in registers across the CTA's tiles
//      (4 x 4 blocks of the upper triangle spread over the CTA's threads).
// The CTA partials go through the same two-level reduction as the narrow path.
//
// The eigen-step (one CTA of 1024 threads) runs cyclic Jacobi with FP32
// rotations on the rotated Gram held in shared memory: each round of the
// round-robin order rotates T/2 disjoint pairs; every 2 x 2 block of pairs is
// then updated in place by one thread (the four entries of a block depend
// only on each other), and the rotations are applied to the columns of V
// (kept in the workspace) in the same phase.  The decisions (sigma, tau, the
// rank and the first mu) are FP64, and Wbar = V diag(g) V^T is formed with V
// staged in shared memory.
#pragma once
#include <cuda_runtime.h>
#include <math.h>

#include "rpca_kernels.cuh"

namespace rpca {

constexpr int kWP = 32;           // pixels per tile (one per lane)
// Frame rows per warp whose loads the tiled passes' staging issues together:
// the compiler cannot tell the staging's shared-memory stores from the global
// loads that follow them, so a load placed after a store waits for the store's
// operand, i.e. for the previous load.
constexpr int kResLd = 4;
constexpr int kWKC = 32;          // rows of Wbar / V staged per step
constexpr int kWideThreads = 256;
constexpr int kEigWThreads = 1024;
constexpr int kVRows = 16;        // rows of V staged per step of V <- V + V D (stand-alone kernel)

// Upper-triangle block (A, C), A <= C < K, of linear index idx in row order
// (row A holds K - A blocks): closed form with one correction step.
__device__ __forceinline__ void tri_coords(int idx, int K, int& A, int& C) {
  const float k2 = 2.f * K + 1.f;
  int a = (int)floorf(0.5f * (k2 - sqrtf(fmaxf(k2 * k2 - 8.f * (float)idx, 0.f))));
  a = max(0, min(a, K - 1));
  while (a > 0 && a * K - a * (a - 1) / 2 > idx) --a;
  while (a + 1 < K && (a + 1) * K - (a + 1) * a / 2 <= idx) ++a;
  A = a;
  C = a + (idx - (a * K - a * (a - 1) / 2));
}

template <int CW>
struct WideShape {
  static constexpr int TP = 8 * CW;               // padded frames (8 warps x CW columns)
  static constexpr int UP = TP + 4;               // row stride of the pixel-major U
  static constexpr int NB = TP / 4;               // 4-frame blocks
  static constexpr int NBLK = NB * (NB + 1) / 2;  // upper-triangle 4 x 4 blocks of the Gram
  static constexpr int BPT = (NBLK + kWideThreads - 1) / kWideThreads;  // blocks per thread
  static constexpr size_t smem = sizeof(float) * (3 * (size_t)TP * kWP + (size_t)kWKC * TP);
  static_assert(CW % 4 == 0, "columns per warp must be a multiple of 4");
  static_assert((size_t)kWP * UP <= 2 * (size_t)TP * kWP, "U must fit in the S and Y tiles");
};

// Dynamic shared memory of the tiled pass with CW columns per warp.
__host__ __device__ constexpr size_t wide_pass_smem_bytes(int CW) {
  return sizeof(float) * (3 * (size_t)(8 * CW) * kWP + (size_t)kWKC * (8 * CW));
}

// Stages rows [k0, k0 + kWKC) of a T x T row-major matrix into sM[kWKC][TP]
// (zero outside T x T).
template <int TP>
__device__ __forceinline__ void stage_rows(float* sM, const float* M, int k0, int T) {
  for (int i = threadIdx.x; i < kWKC * TP; i += kWideThreads) {
    const int r = i / TP, c = i % TP;
    const int k = k0 + r;
    sM[i] = (k < T && c < T) ? __ldcg(&M[(size_t)k * T + c]) : 0.f;
  }
}

// acc[j] = sum_t z(t) * M[t][w*CW + j], z(t) from zfun(t), M streamed from
// global, in increasing t; column pairs share one paired FMA (fma.rn.f32x2).
template <int CW, typename ZF>
__device__ __forceinline__ void tile_times(float (&acc)[CW], float* sM, const float* M, int T, int w, ZF zfun) {
  constexpr int TP = WideShape<CW>::TP;
  uint64_t a2[CW / 2];  // a2[h] = (acc[2h], acc[2h + 1])
#pragma unroll
  for (int h = 0; h < CW / 2; ++h) a2[h] = 0;  // (+0.f, +0.f)
  for (int k0 = 0; k0 < T; k0 += kWKC) {
    __syncthreads();
    stage_rows<TP>(sM, M, k0, T);
    __syncthreads();
    const int kn = min(kWKC, T - k0);
    for (int kk = 0; kk < kn; ++kk) {
      const float z = zfun(k0 + kk);
      const uint64_t zz = f2_pack(z, z);
      const float4* row = reinterpret_cast<const float4*>(&sM[kk * TP + w * CW]);
#pragma unroll
      for (int j4 = 0; j4 < CW / 4; ++j4) {
        const float4 v = row[j4];
        a2[2 * j4] = f2_fma(zz, f2_pack(v.x, v.y), a2[2 * j4]);
        a2[2 * j4 + 1] = f2_fma(zz, f2_pack(v.z, v.w), a2[2 * j4 + 1]);
      }
    }
  }
#pragma unroll
  for (int h = 0; h < CW / 2; ++h) {
    const float2 v = f2_unpack(a2[h]);
    acc[2 * h] = v.x;
    acc[2 * h + 1] = v.y;
  }
}

// CPLX: complex windows as their interleaved real embedding (column 2t = Re,
// 2t + 1 = Im of frame t; T = 2 x frames).  The Hermitian Gram Z^H Z is the
// real Gram of the 2m rows a = [Re z, Im z] and b = a P = [-Im z, Re z] (the
// row of i z) per pixel, so the pass adds both rows of every pixel to the
// Gram; the shrink of Eq. 5 acts on the magnitude of each complex entry.
template <int CW, int MODE, bool CPLX>
__device__ bool pass_wide_body(Bufs b, int lc, int nc, float* wide_smem) {
  using WS = WideShape<CW>;
  constexpr int TP = WS::TP;
  constexpr int UP = CPLX ? TP : WS::UP;       // U row stride (complex: 64 rows over the S, Y tiles)
  constexpr int NROWS = CPLX ? 2 * kWP : kWP;  // Gram rows per tile
  constexpr bool kGram = (MODE != PM_UPDATE);
  float* sX = wide_smem;               // [TP][kWP]
  float* sS = sX + TP * kWP;           // [TP][kWP]
  float* sY = sS + TP * kWP;           // [TP][kWP]
  float* sM = sY + TP * kWP;           // [kWKC][TP]
  float* sU = sS;                      // [NROWS][UP], over the S and Y tiles once they are used
  __shared__ double sRed[2][kWideThreads / 32];
  __shared__ double sScal[2 * kMaxGroups];
  __shared__ int sLast;

  const Ctrl* ctrl = b.ctrl;
  if (solve_done_uniform(ctrl)) return false;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  if (tid == 0) atomicMin(&b.red->t_start, gtimer());
  const int T = b.T;
  const int64_t m = b.m;
  const Job job = *b.job;
  const int kc = __ldcg(&ctrl->k);
  const bool first = (kc == 0) && !__ldcg(&ctrl->warm);
  const float f_mu = __ldcg(&ctrl->f_mu), inv_mu = __ldcg(&ctrl->f_inv_mu), gamma = __ldcg(&ctrl->f_gamma);
  const float inv_mu_nxt = __ldcg(&ctrl->f_inv_mu_nxt);
  const float* Yin = (kc & 1) ? job.Y1 : job.Y0;
  float* Yout = (kc & 1) ? job.Y0 : job.Y1;

  // Gram blocks owned by this thread
  int gbi[WS::BPT], gbj[WS::BPT];
  float gacc[WS::BPT][16];
#pragma unroll
  for (int u = 0; u < WS::BPT; ++u) {
    const int blk = tid + u * kWideThreads;
    gbi[u] = gbj[u] = -1;
    if (blk < WS::NBLK) blk_coords(blk, WS::NB, gbi[u], gbj[u]);
#pragma unroll
    for (int i = 0; i < 16; ++i) gacc[u][i] = 0.f;
  }
  float e2 = 0.f, l1 = 0.f;

  const int64_t ntiles = (m + kWP - 1) / kWP;
  for (int64_t tile = lc; tile < ntiles; tile += nc) {
    const int64_t p = tile * kWP + lane;
    const bool valid = p < m;
    __syncthreads();  // the previous tile's U is consumed
    // ---- 1. stage the tile (frame-major); the loads of kResLd frame rows
    //      per warp are issued before their shared-memory stores ----
    if constexpr (CPLX) {
      const float2* X2 = reinterpret_cast<const float2*>(job.X);
      const float2* S2 = reinterpret_cast<const float2*>(job.S);
      const float2* Y2 = reinterpret_cast<const float2*>(Yin);
      constexpr int G = kResLd / 2;
      static_assert((TP / 2) % (8 * G) == 0, "whole groups of frame rows");
      for (int f0 = w; f0 < TP / 2; f0 += 8 * G) {
        float2 xg[G], sg[G], yg[G];
#pragma unroll
        for (int i = 0; i < G; ++i) {
          const int f = f0 + 8 * i;
          const bool in = valid && 2 * f < T;
          const int64_t gi = in ? (int64_t)f * m + p : 0;
          xg[i] = in ? X2[gi] : make_float2(0.f, 0.f);
          sg[i] = (MODE != PM_INIT && in && !first) ? S2[gi] : make_float2(0.f, 0.f);
          yg[i] = (MODE != PM_INIT && in && !first) ? Y2[gi] : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int i = 0; i < G; ++i) {
          const int f = f0 + 8 * i;
          const float2 x = xg[i];
          sX[(2 * f) * kWP + lane] = x.x;
          sX[(2 * f + 1) * kWP + lane] = x.y;
          if (MODE == PM_INIT) {
            const float a2 = fmaf(x.x, x.x, x.y * x.y);
            e2 += a2;
            l1 += sqrtf(a2);
          } else {
            sS[(2 * f) * kWP + lane] = sg[i].x;
            sS[(2 * f + 1) * kWP + lane] = sg[i].y;
            sY[(2 * f) * kWP + lane] = yg[i].x;
            sY[(2 * f + 1) * kWP + lane] = yg[i].y;
          }
        }
      }
    } else {
      constexpr int G = kResLd;
      static_assert(TP % (8 * G) == 0, "whole groups of frame rows");
      for (int t0 = w; t0 < TP; t0 += 8 * G) {
        float xg[G], sg[G], yg[G];
#pragma unroll
        for (int i = 0; i < G; ++i) {
          const int t = t0 + 8 * i;
          const bool in = valid && t < T;
          const int64_t gi = in ? (int64_t)t * m + p : 0;
          xg[i] = in ? job.X[gi] : 0.f;
          sg[i] = (MODE != PM_INIT && in && !first) ? job.S[gi] : 0.f;
          yg[i] = (MODE != PM_INIT && in && !first) ? Yin[gi] : 0.f;
        }
#pragma unroll
        for (int i = 0; i < G; ++i) {
          const int t = t0 + 8 * i;
          const float x = xg[i];
          sX[t * kWP + lane] = x;
          if (MODE == PM_INIT) {
            e2 = fmaf(x, x, e2);
            l1 += fabsf(x);
          } else {
            sS[t * kWP + lane] = sg[i];
            sY[t * kWP + lane] = yg[i];
          }
        }
      }
    }
    __syncthreads();
    if (MODE == PM_INIT) {
      // U = X (standard basis), pixel-major; complex: also the rows of i X
      for (int i = tid; i < TP * kWP; i += kWideThreads) {
        const int t = i / kWP, pp = i % kWP;
        sU[pp * UP + t] = sX[t * kWP + pp];
        if (CPLX) sU[(kWP + pp) * UP + t] = (t & 1) ? sX[(t - 1) * kWP + pp] : -sX[(t + 1) * kWP + pp];
      }
    } else {
      if (MODE != PM_GRAM) {
        // ---- 2. Q = Z Wbar ----
        float q[CW];
        tile_times<CW>(q, sM, b.Ww, T, w, [&](int t) {
          return form_z(sX[t * kWP + lane], sS[t * kWP + lane], sY[t * kWP + lane], inv_mu);
        });
        __syncthreads();  // every warp has read the whole tile before Z' overwrites X
        // ---- 3. Eq. 5-6 for (lane's pixel, warp's frames) ----
        if constexpr (CPLX) {
          float2* S2 = reinterpret_cast<float2*>(job.S);
          float2* Yo2 = reinterpret_cast<float2*>(Yout);
#pragma unroll
          for (int j = 0; j < CW; j += 2) {
            const int t = w * CW + j;   // even: (Re, Im) of frame t / 2
            if (t < T) {
              const float xr = sX[t * kWP + lane], xi = sX[(t + 1) * kWP + lane];
              const float sr = sS[t * kWP + lane], si = sS[(t + 1) * kWP + lane];
              const float yr = sY[t * kWP + lane], yi = sY[(t + 1) * kWP + lane];
              const float rr = sr + q[j], ri = si + q[j + 1];
              const float mag = sqrtf(fmaf(rr, rr, ri * ri));
              const float f = (mag > gamma) ? gamma / mag : 1.f;   // clip to the disc of radius gamma
              const float cr = rr * f, ci = ri * f;
              const float snr = rr - cr, sni = ri - ci;           // Eq. 5 (magnitude shrink)
              const float ynr = f_mu * cr, yni = f_mu * ci;       // Eq. 6
              const float er = cr - yr * inv_mu, ei = ci - yi * inv_mu;
              e2 = fmaf(er, er, fmaf(ei, ei, e2));
              if (valid) {
                S2[(int64_t)(t >> 1) * m + p] = make_float2(snr, sni);
                Yo2[(int64_t)(t >> 1) * m + p] = make_float2(ynr, yni);
              }
              sX[t * kWP + lane] = valid ? form_z(xr, snr, ynr, inv_mu_nxt) : 0.f;
              sX[(t + 1) * kWP + lane] = valid ? form_z(xi, sni, yni, inv_mu_nxt) : 0.f;
            }
          }
        } else {
#pragma unroll
          for (int j = 0; j < CW; ++j) {
            const int t = w * CW + j;
            if (t < T) {
              const float x = sX[t * kWP + lane], s = sS[t * kWP + lane], y = sY[t * kWP + lane];
              const float r = s + q[j];
              const float c = fminf(fmaxf(r, -gamma), gamma);
              const float sn = r - c;
              const float yn = f_mu * c;
              const float e = c - y * inv_mu;
              e2 = fmaf(e, e, e2);
              if (valid) {
                job.S[(int64_t)t * m + p] = sn;
                Yout[(int64_t)t * m + p] = yn;
              }
              // Z' of the next iteration replaces X in the tile (only this thread reads it)
              sX[t * kWP + lane] = valid ? form_z(x, sn, yn, inv_mu_nxt) : 0.f;
            }
          }
        }
      } else {
        // Z of the current iterate in place of X
        for (int t = w; t < T; t += 8)
          sX[t * kWP + lane] = form_z(sX[t * kWP + lane], sS[t * kWP + lane], sY[t * kWP + lane], inv_mu);
      }
      if (kGram) {
        // ---- 4. U = Z' V, pixel-major over the dead S, Y tiles ----
        float u[CW];
        tile_times<CW>(u, sM, b.Vw, T, w, [&](int t) { return sX[t * kWP + lane]; });
        __syncthreads();  // every warp is done reading S, Y (aliased by U)
        float4* dst = reinterpret_cast<float4*>(&sU[lane * UP + w * CW]);
#pragma unroll
        for (int j4 = 0; j4 < CW / 4; ++j4) dst[j4] = make_float4(u[4 * j4], u[4 * j4 + 1], u[4 * j4 + 2], u[4 * j4 + 3]);
        if constexpr (CPLX) {
          // rows of i Z': (-Im, Re) per frame, in the same basis
          tile_times<CW>(u, sM, b.Vw, T, w, [&](int t) {
            return (t & 1) ? sX[(t - 1) * kWP + lane] : -sX[(t + 1) * kWP + lane];
          });
          float4* dstb = reinterpret_cast<float4*>(&sU[(kWP + lane) * UP + w * CW]);
#pragma unroll
          for (int j4 = 0; j4 < CW / 4; ++j4)
            dstb[j4] = make_float4(u[4 * j4], u[4 * j4 + 1], u[4 * j4 + 2], u[4 * j4 + 3]);
        }
      }
    }
    if (kGram) {
      __syncthreads();
      // ---- 5. partial Gram U^T U (upper 4 x 4 blocks) ----
#pragma unroll
      for (int uu = 0; uu < WS::BPT; ++uu) {
        if (gbi[uu] < 0) continue;
        const int bi = gbi[uu], bj = gbj[uu];
        uint64_t g2[8];  // g2[2i + h] = (gacc[4i + 2h], gacc[4i + 2h + 1])
#pragma unroll
        for (int i = 0; i < 8; ++i) g2[i] = f2_pack(gacc[uu][2 * i], gacc[uu][2 * i + 1]);
        for (int pp = 0; pp < NROWS; ++pp) {
          const float4 a = *reinterpret_cast<const float4*>(&sU[pp * UP + 4 * bi]);
          const float4 c = *reinterpret_cast<const float4*>(&sU[pp * UP + 4 * bj]);
          const float av[4] = {a.x, a.y, a.z, a.w};
          const uint64_t c01 = f2_pack(c.x, c.y), c23 = f2_pack(c.z, c.w);
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const uint64_t ai = f2_pack(av[i], av[i]);
            g2[2 * i] = f2_fma(ai, c01, g2[2 * i]);
            g2[2 * i + 1] = f2_fma(ai, c23, g2[2 * i + 1]);
          }
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const float2 v = f2_unpack(g2[i]);
          gacc[uu][2 * i] = v.x;
          gacc[uu][2 * i + 1] = v.y;
        }
      }
    }
  }

  // ---- CTA partials ----
  const int TT = T * T;
  if (kGram) {
#pragma unroll
    for (int uu = 0; uu < WS::BPT; ++uu) {
      if (gbi[uu] < 0) continue;
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const int a = 4 * gbi[uu] + i / 4, c = 4 * gbj[uu] + i % 4;
        if (a < T && c < T && a <= c) {
          b.gram_part[(int64_t)lc * TT + a * T + c] = gacc[uu][i];
          b.gram_part[(int64_t)lc * TT + c * T + a] = gacc[uu][i];
        }
      }
    }
  }
  {
    const double v0 = warp_sum_d((double)e2), v1 = warp_sum_d((double)l1);
    if (lane == 0) {
      sRed[0][w] = v0;
      sRed[1][w] = v1;
    }
    __syncthreads();
    if (tid == 0) {
      double s0 = 0, s1 = 0;
      for (int i = 0; i < kWideThreads / 32; ++i) {
        s0 += sRed[0][i];
        s1 += sRed[1][i];
      }
      b.scal_part[2 * lc] = s0;
      b.scal_part[2 * lc + 1] = s1;
    }
  }
  return cross_cta_reduce<4>(b, kGram, sScal, &sLast, lc, nc);
}

template <int CW, int MODE, bool CPLX>
__global__ void __launch_bounds__(kWideThreads, 1) pass_wide_kernel(Bufs b) {
  extern __shared__ __align__(16) float wide_smem[];
  pass_wide_body<CW, MODE, CPLX>(b, blockIdx.x, gridDim.x, wide_smem);
}

// ---------------------------------------------------------------------------
// Tiled pass with Wbar and V resident in shared memory (TP <= 128 columns).
// Tiles of 64 pixels; thread (tx, ty) of a 16 x 16 grid owns 4 pixels x TP/16
// columns of both contractions (register-blocked: per k one 16-byte load of
// Z and TP/16 values of Wbar or V feed 4 TP/16 FMAs).  The tile holds Z (in
// place of X), S and Y/mu; Z' = Z - Y/mu - Q + clip(R) + Y'/mu' needs no X.
// ---------------------------------------------------------------------------
constexpr int kRP = 64;   // pixels per tile

// Shared-memory position of pixel pp of frame row t in the frame-major tiles
// (Z, S, Y/mu): rows of 64 pixels, the pixel index XOR-ed with 4 * ((t / 4) % 8)
// so that the Eq. 5-6 update, whose threads walk down the columns of a tile 4
// rows apart, spreads over eight banks instead of one; groups of 4 pixels stay
// contiguous and 16-byte aligned for the contractions' vector loads.
__device__ __forceinline__ int res_at(int t, int pp) { return t * kRP + (pp ^ (((t >> 2) & 7) << 2)); }

template <int TP, bool CPLX>
struct ResShape {
  static constexpr int CPT = TP / 16;                     // columns per thread
  static constexpr int NR = CPLX ? 2 * kRP : kRP;         // Gram rows per tile
  static constexpr int UP = CPLX ? TP : TP + 4;           // U row stride
  static constexpr int NB = TP / 4;
  static constexpr int NBLK = NB * (NB + 1) / 2;
  static constexpr int BPT = (NBLK + kWideThreads - 1) / kWideThreads;
  static constexpr size_t floats = 2 * (size_t)TP * TP + 3 * (size_t)TP * kRP;
  static constexpr size_t smem = sizeof(float) * floats;
  static_assert(TP % 32 == 0 && TP <= 128, "resident tiles need TP in {32, 64, 96, 128}");
  static_assert((size_t)NR * UP <= 2 * (size_t)TP * kRP, "U must fit over the S and Y/mu tiles");
};

__host__ __device__ constexpr size_t res_pass_smem_bytes(int TP) {
  return sizeof(float) * (2 * (size_t)TP * TP + 3 * (size_t)TP * kRP);
}

// acc[i][j] = sum_k zrow(k)[i] * M[k][c0 + j], 4 pixels i, CPT columns j, in
// increasing k; column pairs (j, j + 1) share one paired FMA (fma.rn.f32x2)
template <int TP, typename ZF>
__device__ __forceinline__ void res_times(float (&acc)[4][TP / 16], const float* sM, int T, int c0, ZF zrow) {
  constexpr int CPT = TP / 16;
  uint64_t a2[4][CPT / 2];  // a2[i][h] = (acc[i][2h], acc[i][2h + 1])
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int h = 0; h < CPT / 2; ++h) a2[i][h] = 0;  // (+0.f, +0.f)
  for (int k = 0; k < T; ++k) {
    const float4 z = zrow(k);
    const float2* wr = reinterpret_cast<const float2*>(&sM[k * TP + c0]);
    const uint64_t zz[4] = {f2_pack(z.x, z.x), f2_pack(z.y, z.y), f2_pack(z.z, z.z), f2_pack(z.w, z.w)};
#pragma unroll
    for (int h = 0; h < CPT / 2; ++h) {
      const float2 v = wr[h];
      const uint64_t w2 = f2_pack(v.x, v.y);
#pragma unroll
      for (int i = 0; i < 4; ++i) a2[i][h] = f2_fma(zz[i], w2, a2[i][h]);
    }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int h = 0; h < CPT / 2; ++h) {
      const float2 v = f2_unpack(a2[i][h]);
      acc[i][2 * h] = v.x;
      acc[i][2 * h + 1] = v.y;
    }
}

template <int TP, int MODE, bool CPLX>
__device__ bool pass_res_body(Bufs b, int lc, int nc, float* smem) {
  using RS = ResShape<TP, CPLX>;
  constexpr int CPT = RS::CPT;
  constexpr int UP = RS::UP;
  constexpr bool kGram = (MODE != PM_UPDATE);
  float* sW = smem;                    // Wbar [TP][TP]
  float* sV = sW + TP * TP;            // V [TP][TP]
  float* sZ = sV + TP * TP;            // [TP][kRP]: X, then Z, then Z'
  float* sS = sZ + TP * kRP;           // [TP][kRP]
  float* sD = sS + TP * kRP;           // [TP][kRP]: Y / mu
  float* sU = sS;                      // [NR][UP], over S and Y/mu once they are used
  __shared__ double sRed[2][kWideThreads / 32];
  __shared__ double sScal[2 * kMaxGroups];
  __shared__ int sLast;

  const Ctrl* ctrl = b.ctrl;
  if (solve_done_uniform(ctrl)) return false;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int tx = tid & 15, ty = tid >> 4;     // column group, pixel group
  const int c0 = tx * CPT, p0 = 4 * ty;
  if (tid == 0) atomicMin(&b.red->t_start, gtimer());
  const int T = b.T;
  const int64_t m = b.m;
  const Job job = *b.job;
  const int kc = __ldcg(&ctrl->k);
  const bool first = (kc == 0) && !__ldcg(&ctrl->warm);
  const float f_mu = __ldcg(&ctrl->f_mu), inv_mu = __ldcg(&ctrl->f_inv_mu), gamma = __ldcg(&ctrl->f_gamma);
  const float inv_mu_nxt = __ldcg(&ctrl->f_inv_mu_nxt);
  const float* Yin = (kc & 1) ? job.Y1 : job.Y0;
  float* Yout = (kc & 1) ? job.Y0 : job.Y1;

  // Wbar and V resident for the whole pass (zero outside T x T)
  if (MODE != PM_INIT) {
    for (int i = tid; i < TP * TP; i += kWideThreads) {
      const int r = i / TP, c = i % TP;
      const bool in = r < T && c < T;
      sW[i] = in ? __ldcg(&b.Ww[r * T + c]) : 0.f;
      sV[i] = in ? __ldcg(&b.Vw[r * T + c]) : 0.f;
    }
  }

  int gbi[RS::BPT], gbj[RS::BPT];
  float gacc[RS::BPT][16];
#pragma unroll
  for (int u = 0; u < RS::BPT; ++u) {
    const int blk = tid + u * kWideThreads;
    gbi[u] = gbj[u] = -1;
    if (blk < RS::NBLK) blk_coords(blk, RS::NB, gbi[u], gbj[u]);
#pragma unroll
    for (int i = 0; i < 16; ++i) gacc[u][i] = 0.f;
  }
  float e2 = 0.f, l1 = 0.f;

  const int64_t ntiles = (m + kRP - 1) / kRP;
  for (int64_t tile = lc; tile < ntiles; tile += nc) {
    const int64_t pb = tile * kRP;
    __syncthreads();  // the previous tile (and the resident matrices) are ready / consumed
    // ---- 1. stage: warp w takes frames w, w + 8, ...; lane l pixels l, l + 32;
    //      the loads of kResLd frame rows per warp are issued before their
    //      shared-memory stores ----
    if constexpr (CPLX) {
      const float2* X2 = reinterpret_cast<const float2*>(job.X);
      const float2* S2 = reinterpret_cast<const float2*>(job.S);
      const float2* Y2 = reinterpret_cast<const float2*>(Yin);
      constexpr int G = kResLd / 2;   // TP / 2 is a multiple of 16
      for (int f0 = w; f0 < TP / 2; f0 += 8 * G) {
        float2 xg[G][2], sg[G][2], yg[G][2];
#pragma unroll
        for (int i = 0; i < G; ++i)
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int f = f0 + 8 * i, pp = lane + 32 * h;
            const bool in = (pb + pp < m) && 2 * f < T;
            const int64_t gi = in ? (int64_t)f * m + pb + pp : 0;
            xg[i][h] = in ? X2[gi] : make_float2(0.f, 0.f);
            sg[i][h] = (MODE != PM_INIT && in && !first) ? S2[gi] : make_float2(0.f, 0.f);
            yg[i][h] = (MODE != PM_INIT && in && !first) ? Y2[gi] : make_float2(0.f, 0.f);
          }
#pragma unroll
        for (int i = 0; i < G; ++i)
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int f = f0 + 8 * i, pp = lane + 32 * h;
            const float2 x = xg[i][h];
            if (MODE == PM_INIT) {
              sZ[res_at(2 * f, pp)] = x.x;
              sZ[res_at(2 * f + 1, pp)] = x.y;
              const float a2 = fmaf(x.x, x.x, x.y * x.y);
              e2 += a2;
              l1 += sqrtf(a2);
            } else {
              const float2 sv = sg[i][h], yv = yg[i][h];
              sZ[res_at(2 * f, pp)] = form_z(x.x, sv.x, yv.x, inv_mu);
              sZ[res_at(2 * f + 1, pp)] = form_z(x.y, sv.y, yv.y, inv_mu);
              sS[res_at(2 * f, pp)] = sv.x;
              sS[res_at(2 * f + 1, pp)] = sv.y;
              sD[res_at(2 * f, pp)] = yv.x * inv_mu;
              sD[res_at(2 * f + 1, pp)] = yv.y * inv_mu;
            }
          }
      }
    } else {
      constexpr int G = kResLd;       // TP is a multiple of 32
      for (int t0 = w; t0 < TP; t0 += 8 * G) {
        float xg[G][2], sg[G][2], yg[G][2];
#pragma unroll
        for (int i = 0; i < G; ++i)
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int t = t0 + 8 * i, pp = lane + 32 * h;
            const bool in = (pb + pp < m) && t < T;
            const int64_t gi = in ? (int64_t)t * m + pb + pp : 0;
            xg[i][h] = in ? job.X[gi] : 0.f;
            sg[i][h] = (MODE != PM_INIT && in && !first) ? job.S[gi] : 0.f;
            yg[i][h] = (MODE != PM_INIT && in && !first) ? Yin[gi] : 0.f;
          }
#pragma unroll
        for (int i = 0; i < G; ++i)
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int t = t0 + 8 * i, pp = lane + 32 * h;
            const float x = xg[i][h];
            if (MODE == PM_INIT) {
              sZ[res_at(t, pp)] = x;
              e2 = fmaf(x, x, e2);
              l1 += fabsf(x);
            } else {
              const float sv = sg[i][h], yv = yg[i][h];
              sZ[res_at(t, pp)] = form_z(x, sv, yv, inv_mu);
              sS[res_at(t, pp)] = sv;
              sD[res_at(t, pp)] = yv * inv_mu;
            }
          }
      }
    }
    __syncthreads();
    auto zrow = [&](int k) { return *reinterpret_cast<const float4*>(&sZ[res_at(k, p0)]); };
    auto zrow_i = [&](int k) {  // rows of i Z (complex): (-Im, Re) per frame
      const float4 v = (k & 1) ? *reinterpret_cast<const float4*>(&sZ[res_at(k - 1, p0)])
                               : *reinterpret_cast<const float4*>(&sZ[res_at(k + 1, p0)]);
      return (k & 1) ? v : make_float4(-v.x, -v.y, -v.z, -v.w);
    };
    if (MODE == PM_INIT) {
      // U = X (standard basis), pixel-major; complex: also the rows of i X
      for (int i = tid; i < TP * kRP; i += kWideThreads) {
        const int t = i / kRP, pp = i % kRP;
        sU[pp * UP + t] = sZ[res_at(t, pp)];
        if (CPLX) sU[(kRP + pp) * UP + t] = (t & 1) ? sZ[res_at(t - 1, pp)] : -sZ[res_at(t + 1, pp)];
      }
    } else {
      if (MODE != PM_GRAM) {
        // ---- 2. Q = Z Wbar ----
        float q[4][CPT];
        res_times<TP>(q, sW, T, c0, zrow);
        __syncthreads();  // every thread has read Z before Z' replaces it
        // ---- 3. Eq. 5-6 for (4 pixels, CPT columns) ----
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int pp = p0 + i;
          const bool valid = pb + pp < m;
          if constexpr (CPLX) {
            float2* S2 = reinterpret_cast<float2*>(job.S);
            float2* Yo2 = reinterpret_cast<float2*>(Yout);
#pragma unroll
            for (int j = 0; j < CPT; j += 2) {
              const int t = c0 + j;
              if (t < T) {
                const float zr = sZ[res_at(t, pp)], zi = sZ[res_at(t + 1, pp)];
                const float sr = sS[res_at(t, pp)], si = sS[res_at(t + 1, pp)];
                const float dr = sD[res_at(t, pp)], di = sD[res_at(t + 1, pp)];
                const float rr = sr + q[i][j], ri = si + q[i][j + 1];
                const float mag = sqrtf(fmaf(rr, rr, ri * ri));
                const float f = (mag > gamma) ? gamma / mag : 1.f;
                const float cr = rr * f, ci = ri * f;
                const float ynr = f_mu * cr, yni = f_mu * ci;
                const float er = cr - dr, ei = ci - di;
                e2 = fmaf(er, er, fmaf(ei, ei, e2));
                if (valid) {
                  S2[(int64_t)(t >> 1) * m + pb + pp] = make_float2(rr - cr, ri - ci);
                  Yo2[(int64_t)(t >> 1) * m + pb + pp] = make_float2(ynr, yni);
                }
                sZ[res_at(t, pp)] = valid ? ((zr - dr) - q[i][j]) + cr + ynr * inv_mu_nxt : 0.f;
                sZ[res_at(t + 1, pp)] = valid ? ((zi - di) - q[i][j + 1]) + ci + yni * inv_mu_nxt : 0.f;
              }
            }
          } else {
#pragma unroll
            for (int j = 0; j < CPT; ++j) {
              const int t = c0 + j;
              if (t < T) {
                const float z = sZ[res_at(t, pp)], sv = sS[res_at(t, pp)], d = sD[res_at(t, pp)];
                const float r = sv + q[i][j];                      // X - L + Y/mu
                const float c = fminf(fmaxf(r, -gamma), gamma);    // clip to +-lambda/mu
                const float yn = f_mu * c;                         // Eq. 6
                const float e = c - d;                             // X - L - S'
                e2 = fmaf(e, e, e2);
                if (valid) {
                  job.S[(int64_t)t * m + pb + pp] = r - c;         // Eq. 5
                  Yout[(int64_t)t * m + pb + pp] = yn;
                }
                // Z' = X - S' + Y'/mu' with X = Z + S - Y/mu and S' = S + Q - clip
                sZ[res_at(t, pp)] = valid ? ((z - d) - q[i][j]) + c + yn * inv_mu_nxt : 0.f;
              }
            }
          }
        }
        __syncthreads();  // Z' complete; S, Y/mu are free for U
      }
      if (kGram) {
        // ---- 4. U = Z' V (complex: and (i Z') V), pixel-major ----
        float u[4][CPT];
        res_times<TP>(u, sV, T, c0, zrow);
        if (MODE == PM_GRAM) __syncthreads();  // (no update phase: S, Y/mu read up to here)
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < CPT; ++j) sU[(p0 + i) * UP + c0 + j] = u[i][j];
        if constexpr (CPLX) {
          res_times<TP>(u, sV, T, c0, zrow_i);
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < CPT; ++j) sU[(kRP + p0 + i) * UP + c0 + j] = u[i][j];
        }
      }
    }
    if (kGram) {
      __syncthreads();
      // ---- 5. partial Gram U^T U (upper 4 x 4 blocks) ----
#pragma unroll
      for (int uu = 0; uu < RS::BPT; ++uu) {
        if (gbi[uu] < 0) continue;
        const int bi = gbi[uu], bj = gbj[uu];
        uint64_t g2[8];  // g2[2i + h] = (gacc[4i + 2h], gacc[4i + 2h + 1])
#pragma unroll
        for (int i = 0; i < 8; ++i) g2[i] = f2_pack(gacc[uu][2 * i], gacc[uu][2 * i + 1]);
        for (int pp = 0; pp < RS::NR; ++pp) {
          const float4 a = *reinterpret_cast<const float4*>(&sU[pp * UP + 4 * bi]);
          const float4 c = *reinterpret_cast<const float4*>(&sU[pp * UP + 4 * bj]);
          const float av[4] = {a.x, a.y, a.z, a.w};
          const uint64_t c01 = f2_pack(c.x, c.y), c23 = f2_pack(c.z, c.w);
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const uint64_t ai = f2_pack(av[i], av[i]);
            g2[2 * i] = f2_fma(ai, c01, g2[2 * i]);
            g2[2 * i + 1] = f2_fma(ai, c23, g2[2 * i + 1]);
          }
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const float2 v = f2_unpack(g2[i]);
          gacc[uu][2 * i] = v.x;
          gacc[uu][2 * i + 1] = v.y;
        }
      }
    }
  }

  // ---- CTA partials ----
  const int TT = T * T;
  if (kGram) {
#pragma unroll
    for (int uu = 0; uu < RS::BPT; ++uu) {
      if (gbi[uu] < 0) continue;
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const int a = 4 * gbi[uu] + i / 4, c = 4 * gbj[uu] + i % 4;
        if (a < T && c < T && a <= c) {
          b.gram_part[(int64_t)lc * TT + a * T + c] = gacc[uu][i];
          b.gram_part[(int64_t)lc * TT + c * T + a] = gacc[uu][i];
        }
      }
    }
  }
  {
    const double v0 = warp_sum_d((double)e2), v1 = warp_sum_d((double)l1);
    if (lane == 0) {
      sRed[0][w] = v0;
      sRed[1][w] = v1;
    }
    __syncthreads();
    if (tid == 0) {
      double s0 = 0, s1 = 0;
      for (int i = 0; i < kWideThreads / 32; ++i) {
        s0 += sRed[0][i];
        s1 += sRed[1][i];
      }
      b.scal_part[2 * lc] = s0;
      b.scal_part[2 * lc + 1] = s1;
    }
  }
  return cross_cta_reduce<4>(b, kGram, sScal, &sLast, lc, nc);
}

// CTAs per SM: two below 64 columns (128 registers a thread), else one.
__host__ __device__ constexpr int res_blocks_per_sm(int TP) { return TP <= 64 ? 2 : 1; }

template <int TP, int MODE, bool CPLX>
__global__ void __launch_bounds__(kWideThreads, res_blocks_per_sm(TP)) pass_res_kernel(Bufs b) {
  extern __shared__ __align__(16) float res_smem[];
  pass_res_body<TP, MODE, CPLX>(b, blockIdx.x, gridDim.x, res_smem);
}

#include "rpca_wide_tc.cuh"

// The B operand images of the tiled tensor-core pass (b.wtc), written by the
// eigen-step once Ww and Vw are final.
__device__ __forceinline__ void wtc_images(const Bufs& b) {
  const int TP = wtc_tp(b.T);
  if (b.wtc == 1) {
    if (TP == 64) wtc_write_images<64, false>(b);
    else if (TP == 96) wtc_write_images<96, false>(b);
    else if (TP == 128) wtc_write_images<128, false>(b);
  } else if (b.wtc == 2) {
    if (TP == 64) wtc_write_images<64, true>(b);
    else if (TP == 96) wtc_write_images<96, true>(b);
    else if (TP == 128) wtc_write_images<128, true>(b);
  }
}

// ---------------------------------------------------------------------------
// Eigen-step for wide windows (one CTA; the stand-alone kernel uses kEigWThreads threads).
// ---------------------------------------------------------------------------
// Windows up to this many frames keep D = Q - I (the product of the step's
// rotations, minus I) in shared memory beside G and update it in every round
// (each round's items are independent, so the CTA shares them); larger ones
// log the rotations and replay them onto D after the sweeps, when G is
// consumed.
constexpr int kWideInlineDMaxT = 144;
__host__ __device__ constexpr bool eig_wide_inline_d(int T) { return T <= kWideInlineDMaxT; }

// The eigen-step on one CTA of any multiple of 32 threads; `eigw_smem` holds
// eig_wide_smem(T, vrows) bytes.
__host__ __device__ constexpr size_t eig_wide_smem(int T, int vrows) {
  return sizeof(float) * ((size_t)(eig_wide_inline_d(T) ? 2 : 1) * (T + (T & 1)) * (T + (T & 1) + 1) +
                          (size_t)vrows * T);
}

static __device__ void eig_wide_body(Bufs b, int flags, cudaGraphConditionalHandle h, int use_cond, float* eigw_smem,
                              int vrows) {
  __shared__ float sC[kMaxTW / 2], sSn[kMaxTW / 2];
  __shared__ float sDp[kMaxTW / 2], sDq[kMaxTW / 2];
  __shared__ float sCm1[kMaxTW / 2];  // c - 1 = -s^2 / (1 + c) of every pair slot of the round
  __shared__ double sEv[kMaxTW];
  __shared__ float sG[kMaxTW];
  __shared__ int sAct[kMaxTW / 2], sPos[kMaxTW / 2];
  __shared__ int4 sPair[kMaxTW / 2];    // (p, q, c, s) of every pair slot of the round
  __shared__ int sWarpCnt[(kMaxTW / 2 + 31) / 32];
  __shared__ int sFlag;
  __shared__ double sTau;

  Ctrl* ctrl = b.ctrl;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int T = b.T;
  const int Te = T + (T & 1);   // even size (a zero row/column pads odd T)
  const int K = Te / 2;
  const int LD = Te + 1;
  float* G = eigw_smem;          // [Te][LD]
  const bool inline_d = eig_wide_inline_d(T);
  float* Dn = eigw_smem + (size_t)Te * LD;  // [Te][LD]: D = Q - I, updated per round (inline_d)
  float* after = eigw_smem + (size_t)(inline_d ? 2 : 1) * Te * LD;  // staging beyond G (and D)
  const unsigned long long t0 = gtimer();
  if (!eig_control(b, flags, h, use_cond, &sFlag)) return;
  const bool cold = (flags & EF_INIT) != 0;

  for (int i = tid; i < Te * LD; i += nthr) {
    const int r = i / LD, c = i % LD;
    G[i] = (r < T && c < T) ? b.Gw[r * T + c] : 0.f;
  }
  if (cold)
    for (int i = tid; i < T * T; i += nthr) b.Vw[i] = (i / T == i % T) ? 1.f : 0.f;
  if (inline_d)
    for (int i = tid; i < Te * LD; i += nthr) Dn[i] = 0.f;
  __syncthreads();  // (global writes of the block are visible to its later reads)
  const unsigned long long t1 = gtimer();

  const float eps = (float)ctrl->jacobi_eps;
  const float eps2 = eps * eps;
  int max_sweeps = (cold || (flags & EF_FULL)) ? ctrl->cold_sweeps : ctrl->warm_sweeps;
  if (max_sweeps > kWideLogSweeps) max_sweeps = kWideLogSweeps;
  int sweeps = 0, rounds_run = 0;
  // Each round's rotated pairs are logged (round number, count, slots and
  // (c, s)) to the workspace and applied to V after the sweeps, with V staged
  // in shared memory.
  float2* log_cs = b.rot_log;   // (c, s) of every rotated pair, round after round
  int* log_k = b.rot_k;          // its columns p | q << 8, bit 16 on the first rotation of a round
  int* log_rnd = b.rot_rnd;      // per logged round: round number, rotated pairs
  const int KW = (K + 31) / 32;  // warps covering the pair slots
  int logged = 0;                // entries logged so far
  while (sweeps < max_sweeps) {
    int need = 0;
    for (int i = tid; i < Te * Te; i += nthr) {
      const int a = i / Te, c = i % Te;
      if (a < c) {
        const float apq = G[a * LD + c];
        if (apq != 0.f && apq * apq > eps2 * fabsf(G[a * LD + a] * G[c * LD + c])) need = 1;
      }
    }
    if (!__syncthreads_or(need)) break;
    for (int rnd = 0; rnd < Te - 1; ++rnd) {
      // ---- phase A: the round's rotations (GVL sym.schur2, FP32) ----
      int act = 0;
      if (tid < K) {
        int pa, pb;
        rr_pair(rnd, tid, Te, pa, pb);
        const int p = min(pa, pb), q = max(pa, pb);
        const float app = G[p * LD + p], aqq = G[q * LD + q], apq = G[p * LD + q];
        float c = 1.f, s = 0.f, dp = app, dq = aqq;
        if (apq != 0.f && apq * apq > eps2 * fabsf(app * aqq)) {
          act = 1;
          const float dd = aqq - app;
          const float r2 = fmaf(dd, dd, 4.f * apq * apq);
          const float den = fabsf(dd) + sqrtf(r2);
          const float t = copysignf(1.f, dd) * (2.f * apq) * __fdividef(1.f, den);
          c = rsqrtf(fmaf(t, t, 1.f));
          s = t * c;
          dp = app - t * apq;
          dq = aqq + t * apq;
        }
        sC[tid] = c;
        sSn[tid] = s;
        sCm1[tid] = -s * s / (1.f + c);
        sDp[tid] = dp;
        sDq[tid] = dq;
        sPair[tid] = make_int4(p, q, __float_as_int(c), __float_as_int(s));
      }
      // compact list of the rotated pairs (ballot per warp, then prefix)
      unsigned bal = 0u;
      if (tid < 32 * KW) {
        bal = __ballot_sync(0xffffffffu, act);
        if ((tid & 31) == 0) sWarpCnt[tid >> 5] = __popc(bal);
      }
      __syncthreads();
      int na = 0, off = 0;
      for (int wq = 0; wq < KW; ++wq) {
        if (wq < (tid >> 5)) off += sWarpCnt[wq];
        na += sWarpCnt[wq];
      }
      if (na == 0) {  // (uniform: every thread read the same counts)
        __syncthreads();  // the counts are read before the next round rewrites them
        continue;
      }
      if (tid < K) {
        // (each slot has one writer, and the previous round's readers passed
        // its closing barrier)
        int pos = -1;
        if (act) {
          pos = off + __popc(bal & ((1u << (tid & 31)) - 1u));
          sAct[pos] = tid;
          if (!inline_d) {
            // the replay needs the pair's columns and where each round starts
            const int4 pr = sPair[tid];
            log_k[logged + pos] = pr.x | (pr.y << 8) | (pos == 0 ? (1 << 16) : 0);
            log_cs[logged + pos] = make_float2(sC[tid], sSn[tid]);
          }
        }
        sPos[tid] = pos;
      }
      if (tid == 0 && !inline_d) {
        log_rnd[2 * rounds_run] = rnd;
        log_rnd[2 * rounds_run + 1] = na;
      }
      logged += na;
      ++rounds_run;
      __syncthreads();
      // ---- phase B: G <- J^T G J on every 2 x 2 block of pairs that holds a
      //      rotated pair (a block of two rotated pairs once), in place ----
      // warp w takes rotated pairs w, w + 32, ...; lane l takes partner pairs
      // l, l + 32, ... (the rotated pair's values are read once per warp row;
      // a partner's (p, q, c, s) is one 16-byte load)
      for (int ai = tid >> 5; ai < na; ai += nthr / 32) {
        const int A = sAct[ai];
        const int4 pa4 = sPair[A];
        const int pA = pa4.x, qA = pa4.y;
        const float cA = __int_as_float(pa4.z), sA = __int_as_float(pa4.w);
        for (int C = tid & 31; C < K; C += 32) {
        if (C == A) {
          G[pA * LD + pA] = sDp[A];
          G[qA * LD + qA] = sDq[A];
          G[pA * LD + qA] = 0.f;
          G[qA * LD + pA] = 0.f;
          continue;
        }
        const int pc = sPos[C];
        if (pc >= 0 && pc < ai) continue;  // the block of two rotated pairs belongs to the earlier one
        const int4 pc4 = sPair[C];
        const int pC = pc4.x, qC = pc4.y;
        const float cC = __int_as_float(pc4.z), sC_ = __int_as_float(pc4.w);
        const float g00 = G[pA * LD + pC], g01 = G[pA * LD + qC];
        const float g10 = G[qA * LD + pC], g11 = G[qA * LD + qC];
        // columns of J for the pair: p -> (c, -s), q -> (s, c)
        const float h00 = cC * g00 - sC_ * g01, h01 = sC_ * g00 + cC * g01;  // G J (rows pA)
        const float h10 = cC * g10 - sC_ * g11, h11 = sC_ * g10 + cC * g11;  // G J (rows qA)
        const float n00 = cA * h00 - sA * h10, n01 = cA * h01 - sA * h11;    // J^T (G J)
        const float n10 = sA * h00 + cA * h10, n11 = sA * h01 + cA * h11;
        G[pA * LD + pC] = n00;
        G[pC * LD + pA] = n00;
        G[pA * LD + qC] = n01;
        G[qC * LD + pA] = n01;
        G[qA * LD + pC] = n10;
        G[pC * LD + qA] = n10;
        G[qA * LD + qC] = n11;
        G[qC * LD + qA] = n11;
        }
      }
      if (inline_d) {
        // D' = D J + (J - I) on the round's rotated pairs: (row r, rotated
        // pair) touches D[r][p] and D[r][q] only; lane = rotated pair, warp =
        // rows
        const int warp = tid >> 5, lane = tid & 31, nwarps = nthr >> 5;
        for (int ai = lane; ai < na; ai += 32) {
          const int A = sAct[ai];
          const int4 pr = sPair[A];
          const int p = pr.x, q = pr.y;
          const float c = __int_as_float(pr.z), sn = __int_as_float(pr.w), cm1 = sCm1[A];
          for (int r = warp; r < T; r += nwarps) {
            float* dr = &Dn[r * LD];
            const float dp = dr[p], dq = dr[q];
            float np = fmaf(c, dp, -sn * dq), nq = fmaf(sn, dp, c * dq);
            if (r == p) {
              np += cm1;
              nq += sn;
            } else if (r == q) {
              np -= sn;
              nq += cm1;
            }
            dr[p] = np;
            dr[q] = nq;
          }
        }
      }
      __syncthreads();
    }
    ++sweeps;
  }
  const unsigned long long t2 = gtimer();
  if (tid < T) sEv[tid] = (double)G[tid * LD + tid];
  __syncthreads();

  // ---- Q = J_1 J_2 ... kept as D = Q - I: near the identity D is small, so
  //      its rounding errors are relative to small entries; then V <- V + V D.
  //      Inline: D is already complete; else replay the logged rounds onto D
  //      over the consumed G ----
  float* D = inline_d ? Dn : G;  // [T][LD]
  if (!inline_d)
    for (int i = tid; i < T * LD; i += nthr) D[i] = 0.f;
  // The rows of D are independent (D' = D J + (J - I) mixes columns p and q
  // of each row) and warp w owns rows w, w + nwarps, ..., so between rounds
  // only a warp has to wait for itself.  The CTA stages the log a chunk at a
  // time into shared memory (over the V staging rows, free until the update
  // below; one barrier per chunk); each warp walks the chunk 32 entries at a
  // time, lane = rotation, and applies the rotations of one round (a run of
  // entries starting at a flagged one) before those of the next.
  if (!inline_d) {
    const int nwarps = nthr >> 5, warp = tid >> 5, lane = tid & 31;
    float2* stc = reinterpret_cast<float2*>(after);
    const int E = max(1, (vrows * T * (int)sizeof(float)) / (int)(sizeof(float2) + sizeof(int)));
    int* stp = reinterpret_cast<int*>(stc + E);
    for (int c0 = 0; c0 < logged; c0 += E) {
      const int ne = min(E, logged - c0);
      __syncthreads();  // (D zeroed; the previous chunk consumed)
      for (int i = tid; i < ne; i += nthr) {
        stc[i] = __ldcg(&log_cs[c0 + i]);
        stp[i] = __ldcg(&log_k[c0 + i]);
      }
      __syncthreads();
      for (int w0 = 0; w0 < ne; w0 += 32) {
        const int i = w0 + lane;
        const bool have = i < ne;
        const int pk = have ? stp[i] : 0;
        const float2 cs = have ? stc[i] : make_float2(1.f, 0.f);
        const unsigned starts = __ballot_sync(0xffffffffu, have && (pk >> 16) != 0);
        const int p = pk & 255, q = (pk >> 8) & 255;
        // Q' = Q J  <=>  D' = D J + (J - I); c - 1 = -s^2 / (1 + c)
        const float c = cs.x, sn = cs.y, cm1 = -sn * sn / (1.f + c);
        const int nlive = min(32, ne - w0);
        for (int lo = 0; lo < nlive;) {
          const unsigned later = lo < 31 ? (starts & ~((2u << lo) - 1u)) : 0u;
          const int hi = later ? __ffs(later) - 1 : 32;
          if (lane >= lo && lane < hi && have && q < T) {
            for (int r = warp; r < T; r += nwarps) {
              float* dr = &D[r * LD];
              const float dp = dr[p], dq = dr[q];
              float np = fmaf(c, dp, -sn * dq), nq = fmaf(sn, dp, c * dq);
              if (r == p) {
                np += cm1;
                nq += sn;
              } else if (r == q) {
                np -= sn;
                nq += cm1;
              }
              dr[p] = np;
              dr[q] = nq;
            }
          }
          __syncwarp();
          lo = hi;
        }
      }
    }
  }
  __syncthreads();
  // V <- V + V D, vrows rows of V at a time staged after D
  float* sVo = after;  // [vrows][T]
  for (int r0 = 0; r0 < T; r0 += vrows) {
    const int nr = min(vrows, T - r0);
    for (int i = tid; i < nr * T; i += nthr) sVo[i] = __ldcg(&b.Vw[(size_t)r0 * T + i]);
    __syncthreads();
    const int ncg = (T + 3) / 4;
    for (int item = tid; item < nr * ncg; item += nthr) {
      const int rr = item / ncg, c0 = 4 * (item % ncg);
      float acc[4] = {0.f, 0.f, 0.f, 0.f};
      int cc[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) cc[k] = min(c0 + k, T - 1);
      for (int j = 0; j < T; ++j) {
        const float v = sVo[rr * T + j];
#pragma unroll
        for (int k = 0; k < 4; ++k) acc[k] = fmaf(v, D[j * LD + cc[k]], acc[k]);
      }
#pragma unroll
      for (int k = 0; k < 4; ++k)
        if (c0 + k < T) b.Vw[(size_t)(r0 + rr) * T + c0 + k] = sVo[rr * T + c0 + k] + acc[k];
    }
    __syncthreads();
  }
  // V (new) staged over D for the orthonormalisation and Wbar
  float* sV = G;  // [T][T + 1]
  const int LV = T + 1;
  for (int i = tid; i < T * T; i += nthr) sV[(i / T) * LV + i % T] = __ldcg(&b.Vw[i]);
  __syncthreads();

  // ---- FP64 decisions ----
  if (tid == 0) {
    if (flags & EF_INIT) {
      double lmax = 0.0;
      for (int a = 0; a < T; ++a) lmax = fmax(lmax, sEv[a]);
      init_mu(b, lmax);
    }
    sTau = 1.0 / ctrl->mu_cur;
  }
  __syncthreads();
  int keep = 0;
  if (tid < T) {
    const double sig = sqrt(fmax(sEv[tid], 0.0));
    keep = sig > sTau;
    sG[tid] = keep ? (float)(sTau / sig) : 1.f;
  }
  const int rank = __syncthreads_count(keep);
  // ---- re-orthonormalise V (one Newton-Schulz step, V <- V (3 I - V^T V) / 2),
  //      then Wbar = V diag(g) V^T; V is staged over G ----
  const int NB4 = (T + 3) / 4;
  const int nb2 = NB4 * (NB4 + 1) / 2;
  const unsigned long long t3 = gtimer();
  // A = V^T V into the (consumed) Gram array, and its largest deviation from I
  float dev = 0.f;
  for (int bidx = tid; bidx < nb2; bidx += nthr) {
    int bi, bj;
    blk_coords(bidx, NB4, bi, bj);
    float acc[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) acc[i] = 0.f;
    int ca[4], cc[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      ca[i] = min(4 * bi + i, T - 1);
      cc[i] = min(4 * bj + i, T - 1);
    }
    for (int r = 0; r < T; ++r) {
      float va[4], vc[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        va[i] = sV[r * LV + ca[i]];
        vc[i] = sV[r * LV + cc[i]];
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int k = 0; k < 4; ++k) acc[i * 4 + k] = fmaf(va[i], vc[k], acc[i * 4 + k]);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int a = 4 * bi + i, c = 4 * bj + k;
        if (a < T && c < T) {
          b.Gw[a * T + c] = acc[i * 4 + k];
          b.Gw[c * T + a] = acc[i * 4 + k];
          dev = fmaxf(dev, fabsf(acc[i * 4 + k] - (a == c ? 1.f : 0.f)));
        }
      }
  }
  // skip the correction once V is orthonormal to FP32 rounding
  const int correct = __syncthreads_or(dev > 4e-7f);
  if (correct) {
    // V_new = 1.5 V - 0.5 V A  (rows of V from shared memory, A from the workspace)
    const int nbf = NB4 * NB4;
    for (int bidx = tid; bidx < nbf; bidx += nthr) {
      const int bi = bidx / NB4, bj = bidx % NB4;
      float acc[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) acc[i] = 0.f;
      int ra[4], cc[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        ra[i] = min(4 * bi + i, T - 1);
        cc[i] = min(4 * bj + i, T - 1);
      }
      for (int j = 0; j < T; ++j) {
        float va[4], ac[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          va[i] = sV[ra[i] * LV + j];
          ac[i] = __ldcg(&b.Gw[j * T + cc[i]]);
        }
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int k = 0; k < 4; ++k) acc[i * 4 + k] = fmaf(va[i], ac[k], acc[i * 4 + k]);
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int r = 4 * bi + i, c = 4 * bj + k;
          if (r < T && c < T) b.Vw[r * T + c] = 1.5f * sV[r * LV + c] - 0.5f * acc[i * 4 + k];
        }
    }
    __syncthreads();
    for (int i = tid; i < T * T; i += nthr) sV[(i / T) * LV + i % T] = __ldcg(&b.Vw[i]);
    __syncthreads();
  }
  for (int bidx = tid; bidx < nb2; bidx += nthr) {
    int bi, bj;
    blk_coords(bidx, NB4, bi, bj);
    float acc[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) acc[i] = 0.f;
    int ra[4], rc[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      ra[i] = min(4 * bi + i, T - 1);
      rc[i] = min(4 * bj + i, T - 1);
    }
    for (int j = 0; j < T; ++j) {
      const float gj = sG[j];
      float va[4], vc[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        va[i] = sV[ra[i] * LV + j] * gj;
        vc[i] = sV[rc[i] * LV + j];
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int k = 0; k < 4; ++k) acc[i * 4 + k] = fmaf(va[i], vc[k], acc[i * 4 + k]);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int a = 4 * bi + i, c = 4 * bj + k;
        if (a < T && c < T) {
          b.Ww[a * T + c] = acc[i * 4 + k];
          b.Ww[c * T + a] = acc[i * 4 + k];
        }
      }
  }
  if (b.wtc) {
    __syncthreads();  // Ww written by the whole CTA
    wtc_images(b);
  }
  if (tid < T) b.evw[tid] = sEv[tid];
  if (tid == 0) {
    ctrl->rank = rank;
    ctrl->sweeps = sweeps;
    ctrl->total_sweeps += sweeps;
    const unsigned long long t4 = gtimer();
    ctrl->eig_ns += t4 - t0;
    ctrl->eig_cnt += 1;
    ctrl->eig_phase_ns[0] += t1 - t0;
    ctrl->eig_phase_ns[1] += t2 - t1;
    ctrl->eig_phase_ns[2] += t3 - t2;
    ctrl->eig_phase_ns[3] += t4 - t3;
    ctrl->eig_rounds += rounds_run;
    set_cond(h, use_cond, 1u);
  }
}

static __global__ void __launch_bounds__(kEigWThreads, 1) eig_wide_kernel(Bufs b, int flags,
                                                                          cudaGraphConditionalHandle h, int use_cond) {
  extern __shared__ __align__(16) float eigw_smem[];
  eig_wide_body(b, flags, h, use_cond, eigw_smem, kVRows);
}

}  // namespace rpca
