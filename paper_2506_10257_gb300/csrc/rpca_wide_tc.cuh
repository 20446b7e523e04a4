// rpca_wide_tc.cuh -- the fused per-iteration pass of windows of 33..128 frames
// with all three dense contractions on the 5th-generation tensor cores
// (included inside namespace rpca by rpca_wide.cuh).
//
// Same iteration as pass_res_body (Eq. 4-6 through the Gram of Z, the residual
// of Sec. II-A and the rotated Gram of the next Z), arranged for tcgen05:
//   Q  = Z Wbar       (128-pixel tile x TP columns, K = TP frames)
//   Z~ = Z' V         (the next iteration's Z in the current eigenbasis)
//   G += Z~^T Z~      (the CTA's partial of the next rotated Gram, K = pixels)
// as TF32x3 or BF16x3 split products (A B ~ Ahi Bhi + Alo Bhi + Ahi Blo),
// accumulated in FP32 in TMEM: Q in columns [0, TP), Z~ in [TP, 2 TP), and
// the Gram, which accumulates over all of the CTA's tiles, in [2 TP, 3 TP)
// (lane = row t of the Gram).  TP = frames rounded up to 32, at most 128.
//
// One CTA per SM, 8 warps; thread (warpgroup wg, row r) owns pixel r of the
// tile (TMEM lane r) for the frame chunks of 32 that wg owns (chunk c belongs
// to warpgroup c % 2).  Per tile:
//   1. chunk pairs (2j, 2j+1): each warpgroup loads X, S, Y of its chunk from
//      HBM, forms Z = X - S + Y/mu and writes it (hi/lo split) as an A
//      operand chunk; thread 0 issues the chunks' MMAs against the Wbar chunks
//      (B operand images split and laid out by the eigen-step, brought in by
//      bulk copies one pair ahead);
//   2. chunk pairs again: each warpgroup reads its Q columns from TMEM,
//      reloads X, S, Y (now in L2), applies Eq. 5-6, stores S', Y', forms
//      Z' = X - S' + Y'/mu' and writes it as an A chunk; thread 0 issues the
//      MMAs against the V chunks;
//   3. every warp reads Z~ for its 32 pixels and its half of the columns,
//      and writes Z~^T (rows t, K = pixels) as the A and B operand of the
//      Gram; thread 0 issues the Gram MMAs.
// A pair's loads and arithmetic overlap the previous pair's MMAs; a buffer is
// rewritten only after the MMAs that read it have completed (commit ->
// mbarrier, waited by every thread, so no thread falls a phase behind).  Every
// wait is bounded: a wait that runs out sets the pass's error flag and the
// CTA leaves its tile loop (the solve then ends with RPCA_ERR_TIMEOUT).
//
// Complex windows (CPLX) run as their interleaved real embedding (columns
// 2f, 2f+1 = Re, Im of frame f; up to 64 frames): step 2 applies the complex
// shrink of Eq. 5 to each (Re, Im) pair, and after each pair's Z~ chunks the
// rows of i Z' (per frame (-Im, Re)) are staged and multiplied by V as well
// (columns [3 TP, 4 TP)); step 3 adds both row sets to the Gram (the real
// embedding of the Hermitian Gram is the real Gram of the rows of Z and i Z).
//
// Shared-memory layouts: the canonical K-major no-swizzle layout of rpca_tc.cuh.
// A and B chunks keep K-adjacent core matrices contiguous (LBO 128 B); the
// Gram operand spaces them 144 B apart, so that the 32 lanes of a warp, which
// write 32 consecutive pixels (K) of one row t, hit 32 different banks.
#pragma once

constexpr int kWtcThreads = 256;
constexpr int kWtcKCh = 32;            // frames per K-chunk
// Step 2 reads X, S, Y of a chunk in groups of kWtcLd columns, every load of
// a group issued before the group's stores of S', Y': the compiler cannot
// tell those stores from the loads (for all it knows the arrays overlap), so
// a load placed after a store waits until the store's operands are ready,
// and one load per column would cost one L2 round trip per column.
constexpr int kWtcLd = 16;
constexpr uint32_t kWtcGLbo = 144;     // Gram operand: K-adjacent core matrices 144 B apart

template <int TP, bool BF16>
struct WtcShape {
  static constexpr int EB = BF16 ? 2 : 4;
  static constexpr int KC = 16 / EB;                         // elements per 16-byte core row
  static constexpr int NCH = TP / kWtcKCh;                   // frame chunks
  static constexpr int NPAIR = (NCH + 1) / 2;
  static constexpr uint32_t LBO = 128;
  static constexpr uint32_t SBO = (kWtcKCh / KC) * 128;      // next 8 rows of an A / B chunk
  static constexpr uint32_t A_BYTES = 16 * SBO;              // 128 pixel rows x 32 frames
  static constexpr uint32_t B_BYTES = (TP / 8) * SBO;        // TP rows (n) x 32 frames (k)
  static constexpr uint32_t G_SBO = (32 / KC) * kWtcGLbo;    // next 8 rows t of a Gram chunk
  static constexpr uint32_t G_BYTES = 16 * G_SBO;            // 128 rows t x 32 pixels
  static constexpr int KSTEP = BF16 ? 16 : 8;                // K of one tcgen05.mma
  static constexpr uint32_t TMEM_COLS = 512;
  static constexpr size_t A_REGION = 2 * 2 * (size_t)A_BYTES;   // 2 buffers x (hi, lo)
  static constexpr size_t B_REGION = 4 * 2 * (size_t)B_BYTES;   // 4 slots x (hi, lo)
  static constexpr size_t G_REGION = 4 * 2 * (size_t)G_BYTES;   // 4 pixel chunks x (hi, lo)
  static constexpr size_t OPS = (A_REGION + B_REGION > G_REGION) ? A_REGION + B_REGION : G_REGION;
  // at least 116 KB so that one CTA holds an SM (it allocates all of TMEM)
  static constexpr size_t SMEM = OPS > 118784 ? OPS : 118784;
  static_assert(TP % kWtcKCh == 0 && TP >= 64 && TP <= 128, "TP in {64, 96, 128}");
  static_assert(3 * TP <= (int)TMEM_COLS, "TMEM columns");
  __host__ __device__ static constexpr uint32_t off(int r, int k) {
    return (uint32_t)((r / 8) * SBO + (k / KC) * LBO + (r % 8) * 16 + (k % KC) * EB);
  }
  __host__ __device__ static constexpr uint32_t goff(int t, int p) {
    return (uint32_t)((t / 8) * G_SBO + (p / KC) * kWtcGLbo + (t % 8) * 16 + (p % KC) * EB);
  }
  // bytes of the B operand images a plan keeps: [Wbar, V][chunk][hi, lo]
  static constexpr size_t IMG_BYTES = 2 * (size_t)NCH * 2 * B_BYTES;
};

// Columns the tiled tensor-core pass pads a window of T real columns to: T
// rounded up to 32, at least 64 (complex windows of up to 16 frames).
__host__ __device__ constexpr int wtc_tp(int T) { return ((T + 31) / 32 * 32) < 64 ? 64 : (T + 31) / 32 * 32; }

__host__ __device__ constexpr size_t wtc_img_bytes(int TP, bool bf16) {
  return 2 * (size_t)(TP / kWtcKCh) * 2 * (size_t)((TP / 8) * ((kWtcKCh / (bf16 ? 8 : 4)) * 128));
}

// Stores one value into an operand (hi at base_hi + o, lo at base_lo + o).
template <bool BF16>
__device__ __forceinline__ void tc_store1(unsigned char* hi, unsigned char* lo, uint32_t o, float v) {
  if (BF16) {
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    *reinterpret_cast<__nv_bfloat16*>(hi + o) = h;
    *reinterpret_cast<__nv_bfloat16*>(lo + o) = __float2bfloat16_rn(v - __bfloat162float(h));
  } else {
    const float h = to_tf32(v);
    *reinterpret_cast<float*>(hi + o) = h;
    *reinterpret_cast<float*>(lo + o) = to_tf32(v - h);
  }
}

// The B operand images of Wbar and V for the pass (called by the eigen-step
// CTA after it has written Ww and Vw): image [m][c] holds rows n < TP and
// frames k of chunk c of B[n][k] = M[k][n] (M = Wbar or V), zero outside T.
template <int TP, bool BF16>
__device__ void wtc_write_images(const Bufs& b) {
  using SH = WtcShape<TP, BF16>;
  const int T = b.T;
  for (int i = threadIdx.x; i < 2 * TP * TP; i += blockDim.x) {
    const int mat = i / (TP * TP), e = i % (TP * TP);
    const int n = e / TP, k = e % TP;
    const float* M = mat ? b.Vw : b.Ww;
    const float v = (n < T && k < T) ? __ldcg(&M[k * T + n]) : 0.f;
    const int c = k / kWtcKCh;
    unsigned char* hi = b.wtc_img + ((size_t)(mat * SH::NCH + c) * 2) * SH::B_BYTES;
    tc_store1<BF16>(hi, hi + SH::B_BYTES, SH::off(n, k % kWtcKCh), v);
  }
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* mbar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(mbar))
               : "memory");
}

template <int TP, bool BF16, bool CPLX>
__global__ void __launch_bounds__(kWtcThreads, 1) pass_wtc_kernel(Bufs b) {
  using SH = WtcShape<TP, BF16>;
  static_assert(!CPLX || 4 * TP <= (int)SH::TMEM_COLS, "TMEM columns of the complex form");
  constexpr int NCH = SH::NCH, NPAIR = SH::NPAIR;
  extern __shared__ __align__(1024) unsigned char wtc_smem[];
  unsigned char* sA = wtc_smem;                       // [2][hi, lo]
  unsigned char* sB = wtc_smem + SH::A_REGION;        // [4][hi, lo]
  unsigned char* sG = wtc_smem;                       // [4][hi, lo], over A and B in step 3
  __shared__ __align__(8) uint64_t mb_mma, mb_b[4];
  __shared__ uint32_t sTmem;
  __shared__ int sFail;
  __shared__ double sRed[kWtcThreads / 32];
  __shared__ double sScal[2 * kMaxGroups];
  __shared__ int sLast;

  const Ctrl* ctrl = b.ctrl;
  if (solve_done_uniform(ctrl)) return;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int wg = tid >> 7, r = tid & 127;
  if (tid == 0) atomicMin(&b.red->t_start, gtimer());
  const int T = b.T;
  const int64_t m = b.m;
  const Job* jobp = b.job;
  const float* X = jobp->X;
  float* Sp = jobp->S;
  const int kc0 = __ldcg(&ctrl->k);
  const bool first = (kc0 == 0) && !__ldcg(&ctrl->warm);
  const float f_mu = __ldcg(&ctrl->f_mu), inv_mu = __ldcg(&ctrl->f_inv_mu), gamma = __ldcg(&ctrl->f_gamma);
  const float inv_mu_nxt = __ldcg(&ctrl->f_inv_mu_nxt);
  const float* Yin = (kc0 & 1) ? jobp->Y1 : jobp->Y0;
  float* Yout = (kc0 & 1) ? jobp->Y0 : jobp->Y1;
  const unsigned char* img = b.wtc_img;

  if (warp == 0) tmem_alloc(&sTmem, SH::TMEM_COLS);
  if (tid == 0) {
    mbar_init(&mb_mma, 1);
    for (int i = 0; i < 4; ++i) mbar_init(&mb_b[i], 1);
    sFail = 0;
  }
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = sTmem;
  const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;
  const uint32_t colQ = 0, colZ = TP, colG = 2 * TP, colZi = 3 * TP;
  // float index of real column t of pixel p in a frame-major X, S or Y
  // (complex: interleaved (Re, Im) of frame t / 2)
  auto gidx = [&](int t, int64_t px) -> int64_t {
    return CPLX ? ((int64_t)(t >> 1) * m + px) * 2 + (t & 1) : (int64_t)t * m + px;
  };
  constexpr uint32_t idesc = tc_idesc(BF16 ? 1u : 2u, 128, TP);

  uint32_t ncommit = 0;      // MMA groups committed (uniform across the CTA)
  uint32_t ub[4] = {0, 0, 0, 0};   // uses of each B slot (thread 0)
  uint32_t ib[4] = {0, 0, 0, 0};   // copies issued into each B slot (thread 0)
  bool gram_started = false;
  float e2 = 0.f;

  auto wait_mma = [&]() {
    // the latest committed group has completed (no thread is more than one
    // phase behind: a group is committed after every thread passed the
    // barrier that follows its wait for the group before)
    if (ncommit > 0 && !mbar_wait(&mb_mma, (ncommit - 1) & 1u, kTcWaitLimit)) atomicOr(&sFail, 1);
  };
  // thread 0: bulk copies of chunk c of matrix mat (0 Wbar, 1 V) into B slot s
  auto load_b = [&](int mat, int c, int s) {
    const unsigned char* src = img + ((size_t)(mat * NCH + c) * 2) * SH::B_BYTES;
    mbar_arrive_expect_tx(&mb_b[s], 2 * SH::B_BYTES);
    bulk_g2s(sB + (size_t)s * 2 * SH::B_BYTES, src, 2 * SH::B_BYTES, &mb_b[s]);
    ++ib[s];
  };
  // thread 0: the MMAs of chunk c (A buffer c % 2, B slot s) into TMEM column col
  auto issue_chunk = [&](int c, int s, uint32_t col, bool b_resident = false) {
    if (!b_resident) {
      if (!mbar_wait(&mb_b[s], ub[s] & 1u, kTcWaitLimit)) atomicOr(&sFail, 1);
      ++ub[s];
    }
    tc_fence_after();
    const uint32_t ah = smem_u32(sA + (size_t)(c & 1) * 2 * SH::A_BYTES), al = ah + SH::A_BYTES;
    const uint32_t bh = smem_u32(sB + (size_t)s * 2 * SH::B_BYTES), bl = bh + SH::B_BYTES;
#pragma unroll
    for (int kk = 0; kk < kWtcKCh / SH::KSTEP; ++kk) {
      const uint32_t ko = (uint32_t)kk * (SH::KSTEP / SH::KC) * SH::LBO;
      const uint64_t dah = tc_desc(ah + ko, SH::LBO, SH::SBO), dbh = tc_desc(bh + ko, SH::LBO, SH::SBO);
      const uint64_t dal = tc_desc(al + ko, SH::LBO, SH::SBO), dbl = tc_desc(bl + ko, SH::LBO, SH::SBO);
      tc_mma<BF16>(tmem + col, dah, dbh, idesc, (c > 0 || kk > 0) ? 1u : 0u);
      tc_mma<BF16>(tmem + col, dal, dbh, idesc, 1u);
      tc_mma<BF16>(tmem + col, dah, dbl, idesc, 1u);
    }
  };

  const int64_t ntiles = (m + 127) / 128;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t p = tile * 128 + r;
    const bool valid = p < m;
    // pull the CTA's next tile (X, and S, Y after the first iteration) from HBM
    // into L2 while this one is computed: one prefetch per 128-byte piece
    if (tile + gridDim.x < ntiles) {
      const int64_t pn = (tile + gridDim.x) * 128;
      const int pieces = T * 4;   // frame rows x 128-byte pieces (32 real or 16 complex pixels)
      for (int k = tid; k < (first ? 1 : 3) * pieces; k += kWtcThreads) {
        const int a = k / pieces, q = k % pieces;
        const float* base = a == 0 ? X : (a == 1 ? Sp : Yin);
        if (CPLX) {
          const int f = q / 8;
          const int64_t px = pn + 16 * (q % 8);
          if (px >= m) continue;
          prefetch_l2(base + ((int64_t)f * m + px) * 2);
        } else {
          const int t = q / 4;
          const int64_t px = pn + 32 * (q % 4);
          if (px >= m) continue;
          prefetch_l2(base + (int64_t)t * m + px);
        }
      }
    }
    // the previous tile's Gram MMAs read the operand region the B slots use
    wait_mma();
    if (tid == 0) {
      load_b(0, 0, 0);
      if (NCH > 1) load_b(0, 1, 1);
    }
    // ---- 1. Q = Z Wbar, chunk pairs ----
    for (int j = 0; j < NPAIR; ++j) {
      const int c = 2 * j + wg;
      const bool has = c < NCH;
      float z[kWtcKCh];
#pragma unroll
      for (int u = 0; u < kWtcKCh; ++u) {
        const int t = c * kWtcKCh + u;
        const bool in = has && valid && t < T;
        const int64_t gi = in ? gidx(t, p) : 0;
        const float x = in ? X[gi] : 0.f;
        const float s = (in && !first) ? Sp[gi] : 0.f;
        const float y = (in && !first) ? Yin[gi] : 0.f;
        z[u] = form_z(x, s, y, inv_mu);
      }
      wait_mma();   // A buffers free (the group before has completed)
      if (has) {
        unsigned char* ah = sA + (size_t)wg * 2 * SH::A_BYTES;
#pragma unroll
        for (int k4 = 0; k4 < kWtcKCh; k4 += 4)
          tc_store4<BF16>(ah, ah + SH::A_BYTES, SH::off(r, k4), z[k4], z[k4 + 1], z[k4 + 2], z[k4 + 3], true);
      }
      fence_async_smem();
      tc_fence_before();
      __syncthreads();
      if (sFail) break;
      if (tid == 0) {
        const int sb = 2 * (j & 1);
        issue_chunk(2 * j, sb, colQ);
        if (2 * j + 1 < NCH) issue_chunk(2 * j + 1, sb + 1, colQ);
        tc_commit(&mb_mma);
        // the next pair's B chunks: Wbar chunks, or V chunks 0, 1 after the last pair
        const int sn = 2 * ((j + 1) & 1);
        if (j + 1 < NPAIR) {
          load_b(0, 2 * j + 2, sn);
          if (2 * j + 3 < NCH) load_b(0, 2 * j + 3, sn + 1);
        }
      }
      ++ncommit;
    }
    if (sFail) break;
    // V chunks of the first pair of step 2 go to the slot pair after the last Q pair
    const int sv0 = 2 * (NPAIR & 1);
    wait_mma();   // Q complete; the B slots of the last Q pair are free
    if (tid == 0) {
      load_b(1, 0, sv0);
      if (NCH > 1) load_b(1, 1, sv0 + 1);
    }
    tc_fence_after();
    // ---- 2. Eq. 5-6, Z' and Z~ = Z' V, chunk pairs ----
    for (int j = 0; j < NPAIR; ++j) {
      const int c = 2 * j + wg;
      const bool has = c < NCH;
      float zn[kWtcKCh];
      if (has) {
        float q[kWtcKCh];
        tmem_ld32(tmem + lane_base + colQ + (uint32_t)(c * kWtcKCh), q);
        if constexpr (CPLX) {
          // Eq. 5-6 on each complex value: the shrink scales R by
          // max(|R| - gamma, 0) / |R| (phase kept), Y' = mu R min(1, gamma / |R|)
          float2* S2 = reinterpret_cast<float2*>(Sp);
          float2* Yo2 = reinterpret_cast<float2*>(Yout);
#pragma unroll
          for (int u0 = 0; u0 < kWtcKCh; u0 += kWtcLd) {
            float2 xg[kWtcLd / 2], sg[kWtcLd / 2], yg[kWtcLd / 2];
#pragma unroll
            for (int v = 0; v < kWtcLd / 2; ++v) {
              const int t = c * kWtcKCh + u0 + 2 * v;
              const bool in = valid && t < T;
              const int64_t gf = in ? (int64_t)(t >> 1) * m + p : 0;
              xg[v] = in ? reinterpret_cast<const float2*>(X)[gf] : make_float2(0.f, 0.f);
              sg[v] = (in && !first) ? S2[gf] : make_float2(0.f, 0.f);
              yg[v] = (in && !first) ? reinterpret_cast<const float2*>(Yin)[gf] : make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int v = 0; v < kWtcLd / 2; ++v) {
              const int u = u0 + 2 * v;
              const int t = c * kWtcKCh + u;
              zn[u] = 0.f;
              zn[u + 1] = 0.f;
              if (valid && t < T) {
                const int64_t gf = (int64_t)(t >> 1) * m + p;
                const float2 x = xg[v], sv = sg[v], y = yg[v];
                const float dr = y.x * inv_mu, di = y.y * inv_mu;
                const float rr = sv.x + q[u], ri = sv.y + q[u + 1];    // X - L + Y/mu
                const float mag = sqrtf(fmaf(rr, rr, ri * ri));
                const float f = (mag > gamma) ? gamma / mag : 1.f;
                const float cr = rr * f, ci = ri * f;
                const float ynr = f_mu * cr, yni = f_mu * ci;          // Eq. 6
                const float er = cr - dr, ei = ci - di;                // X - L - S'
                e2 = fmaf(er, er, fmaf(ei, ei, e2));
                const float snr = rr - cr, sni = ri - ci;              // Eq. 5
                S2[gf] = make_float2(snr, sni);
                Yo2[gf] = make_float2(ynr, yni);
                zn[u] = form_z(x.x, snr, ynr, inv_mu_nxt);
                zn[u + 1] = form_z(x.y, sni, yni, inv_mu_nxt);
              }
            }
          }
        } else {
#pragma unroll
          for (int u0 = 0; u0 < kWtcKCh; u0 += kWtcLd) {
            float xg[kWtcLd], sg[kWtcLd], yg[kWtcLd];
#pragma unroll
            for (int v = 0; v < kWtcLd; ++v) {
              const int t = c * kWtcKCh + u0 + v;
              const bool in = valid && t < T;
              const int64_t gi = in ? (int64_t)t * m + p : 0;
              xg[v] = in ? X[gi] : 0.f;
              sg[v] = (in && !first) ? Sp[gi] : 0.f;
              yg[v] = (in && !first) ? Yin[gi] : 0.f;
            }
#pragma unroll
            for (int v = 0; v < kWtcLd; ++v) {
              const int u = u0 + v;
              const int t = c * kWtcKCh + u;
              zn[u] = 0.f;
              if (valid && t < T) {
                const int64_t gi = (int64_t)t * m + p;
                const float d = yg[v] * inv_mu;
                const float rr = sg[v] + q[u];                      // X - L + Y/mu
                const float cl = fminf(fmaxf(rr, -gamma), gamma);   // clip to +-lambda/mu
                const float sn = rr - cl;                           // Eq. 5
                const float yn = f_mu * cl;                         // Eq. 6
                const float e = cl - d;                             // X - L - S'
                e2 = fmaf(e, e, e2);
                Sp[gi] = sn;
                Yout[gi] = yn;
                zn[u] = form_z(xg[v], sn, yn, inv_mu_nxt);
              }
            }
          }
        }
      }
      if (j > 0) wait_mma();   // the previous Z~ pair has read its A buffers
      if (has) {
        unsigned char* ah = sA + (size_t)wg * 2 * SH::A_BYTES;
#pragma unroll
        for (int k4 = 0; k4 < kWtcKCh; k4 += 4)
          tc_store4<BF16>(ah, ah + SH::A_BYTES, SH::off(r, k4), zn[k4], zn[k4 + 1], zn[k4 + 2], zn[k4 + 3], true);
      }
      fence_async_smem();
      tc_fence_before();
      __syncthreads();
      if (sFail) break;
      if (tid == 0) {
        const int sb = 2 * ((NPAIR + j) & 1);
        issue_chunk(2 * j, sb, colZ);
        if (2 * j + 1 < NCH) issue_chunk(2 * j + 1, sb + 1, colZ);
        tc_commit(&mb_mma);
        const int sn = 2 * ((NPAIR + j + 1) & 1);
        if (j + 1 < NPAIR) {
          load_b(1, 2 * j + 2, sn);
          if (2 * j + 3 < NCH) load_b(1, 2 * j + 3, sn + 1);
        }
      }
      ++ncommit;
      if constexpr (CPLX) {
        // the rows of i Z' (per frame (-Im, Re)) times the same V chunks, which
        // stay in their slots until the next pair's MMAs have been issued
        wait_mma();   // the Z' chunks have been read
        if (has) {
          unsigned char* ah = sA + (size_t)wg * 2 * SH::A_BYTES;
#pragma unroll
          for (int k4 = 0; k4 < kWtcKCh; k4 += 4)
            tc_store4<BF16>(ah, ah + SH::A_BYTES, SH::off(r, k4), -zn[k4 + 1], zn[k4], -zn[k4 + 3], zn[k4 + 2], true);
        }
        fence_async_smem();
        tc_fence_before();
        __syncthreads();
        if (sFail) break;
        if (tid == 0) {
          const int sb = 2 * ((NPAIR + j) & 1);
          issue_chunk(2 * j, sb, colZi, true);
          if (2 * j + 1 < NCH) issue_chunk(2 * j + 1, sb + 1, colZi, true);
          tc_commit(&mb_mma);
        }
        ++ncommit;
      }
    }
    if (sFail) break;
    // ---- 3. G += Z~^T Z~ (complex: then the rows of (i Z') V) ----
    for (int round = 0; round < (CPLX ? 2 : 1); ++round) {
    const uint32_t colU = round == 0 ? colZ : colZi;
    wait_mma();   // Z~ complete (or the round before has read the operands); A and B regions free
    tc_fence_after();
    {
      const int kq = warp & 3;              // pixel chunk of this warp: pixels 32 kq .. 32 kq + 31
      unsigned char* gh = sG + (size_t)kq * 2 * SH::G_BYTES;
      unsigned char* gl = gh + SH::G_BYTES;
      const int t0 = wg * (TP / 2), t1 = t0 + TP / 2;
      for (int tb = t0; tb < t1; tb += 16) {
        float v[16];
        tmem_ld16(tmem + lane_base + colU + (uint32_t)tb, v);
#pragma unroll
        for (int u = 0; u < 16; ++u) tc_store1<BF16>(gh, gl, SH::goff(tb + u, lane), valid ? v[u] : 0.f);
      }
      // rows t >= TP of the 128-row operand are zero
      if (TP < 128 && wg == 1)
        for (int t = TP; t < 128; ++t) tc_store1<BF16>(gh, gl, SH::goff(t, lane), 0.f);
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    if (sFail) break;
    if (tid == 0) {
      tc_fence_after();
#pragma unroll
      for (int kq = 0; kq < 4; ++kq) {
        const uint32_t gh = smem_u32(sG + (size_t)kq * 2 * SH::G_BYTES), gl = gh + SH::G_BYTES;
#pragma unroll
        for (int kk = 0; kk < 32 / SH::KSTEP; ++kk) {
          const uint32_t ko = (uint32_t)kk * (SH::KSTEP / SH::KC) * kWtcGLbo;
          const uint64_t dh = tc_desc(gh + ko, kWtcGLbo, SH::G_SBO), dl = tc_desc(gl + ko, kWtcGLbo, SH::G_SBO);
          tc_mma<BF16>(tmem + colG, dh, dh, idesc, (gram_started || round > 0 || kq > 0 || kk > 0) ? 1u : 0u);
          tc_mma<BF16>(tmem + colG, dl, dh, idesc, 1u);
          tc_mma<BF16>(tmem + colG, dh, dl, idesc, 1u);
        }
      }
      tc_commit(&mb_mma);
    }
    ++ncommit;
    }
    if (sFail) break;
    gram_started = true;
  }
  wait_mma();
  if (tid == 0) {
    // copies issued but not consumed (only after a wait ran out) land before the CTA exits
    for (int s = 0; s < 4; ++s)
      if (ib[s] > ub[s] && !mbar_wait(&mb_b[s], (ib[s] - 1) & 1u, kTcWaitLimit)) atomicOr(&sFail, 1);
  }
  tc_fence_after();
  __syncthreads();
  const bool failed = sFail != 0;

  // ---- CTA partials: the Gram from TMEM (row t = lane), the residual ----
  const int TT = T * T;
  {
    const int t = 32 * (warp & 3) + lane;
    const int c0 = wg * (TP / 2), c1 = c0 + TP / 2;
    for (int cb = c0; cb < c1; cb += 16) {
      float v[16];
      if (gram_started) tmem_ld16(tmem + lane_base + colG + (uint32_t)cb, v);
#pragma unroll
      for (int u = 0; u < 16; ++u)
        if (t < T && cb + u < T) b.gram_part[(int64_t)blockIdx.x * TT + t * T + cb + u] = gram_started ? v[u] : 0.f;
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, SH::TMEM_COLS);
  if (failed && tid == 0) atomicExch(&b.red->err, 1);
  {
    const double v0 = warp_sum_d((double)e2);
    if (lane == 0) sRed[warp] = v0;
    __syncthreads();
    if (tid == 0) {
      double s0 = 0;
      for (int w = 0; w < kWtcThreads / 32; ++w) s0 += sRed[w];
      b.scal_part[2 * blockIdx.x] = s0;
      b.scal_part[2 * blockIdx.x + 1] = 0.0;
    }
  }
  cross_cta_reduce<4>(b, true, sScal, &sLast, blockIdx.x, gridDim.x);
}
