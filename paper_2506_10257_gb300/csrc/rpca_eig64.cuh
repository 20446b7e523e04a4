// rpca_eig64.cuh -- the narrow eigen-step (T <= 32) with FP64 Jacobi
// rotations and FP64 basis arithmetic (included inside namespace rpca by
// rpca_kernels.cuh).  This is the plans' default eigen-step.
//
// Same iteration as eig_fast_body (cyclic Jacobi in round-robin order on the
// rotated Gram G~ = V^T Z^T Z V, which arrives as FP64 sums of the CTAs' FP32
// partials and nearly diagonal), arranged for GB300's FP64 pipe, where one
// FP64 warp instruction occupies an SM sub-partition for tens of cycles: the
// number of dependent FP64 instructions per round, not the flops, sets the
// time.  So
//   * a rotation's tangent t (GVL sym.schur2) is found in FP32, and (c, s) are
//     then made orthonormal in FP64 (c^2 + s^2 = 1 + d, |d| ~ 1e-7, scaled by
//     1 - d/2 + 3d^2/8): every rotation applied to G and V is an exact FP64
//     orthogonal transform; the pair it targets is left with an off-diagonal
//     entry ~1e-7 of its old value (computed, not assumed zero), which the
//     next sweep removes;
//   * every entry of J^T G J is computed from four entries of G in FP64 by one
//     thread per upper-triangle entry, diagonal and targeted pair included
//     (entries of two unrotated pairs are copied);
//   * the rotations are applied to the columns of V (in shared memory, FP64,
//     starting from the FP32 basis the pass used, exact in FP64) in the same
//     round by the same threads, so no rotation log is replayed afterwards;
//   * the entries a round's successor needs ((p,p), (q,q), (p,q) of each of
//     its pairs) are computed from the current G by three lanes per pair of
//     the last warp(s) while the other warps update the round, and one lane
//     per pair forms the next rotation, so a round costs one CTA barrier.
// After the sweeps V <- V (3I - V^T V)/2 (Newton-Schulz, FP64; to first order
// it also removes the departure of the FP32-rounded old basis from
// orthonormality), sigma = sqrt(lambda), the sigma > tau = 1/mu decision,
// g = min(1, tau/sigma) and Wbar = V diag(g) V^T are FP64; Wbar and V are
// rounded to FP32 once for the passes (Eq. 4 through the Gram).
#pragma once

// Thread roles (8 warps; warp w runs on SM sub-partition w % 4): warp 7 forms
// the rotations and is the only warp of its sub-partition with FP64 work, so
// its dependent chain does not queue behind the updates; warps 0-2 and 4-6
// update G and V; warp 3 waits at the barriers.
template <int TB>
struct Eig64Shape {
  static constexpr int K = TB / 2;                          // pairs per round
  static constexpr int NR = TB - 1;                         // rounds per sweep
  static constexpr int NE = TB * (TB + 1) / 2;              // upper-triangle entries
  static constexpr int LPP = K <= 10 ? 3 : 2;               // rotation lanes per pair
  static constexpr int NW = 192;                            // threads updating G and V
  static constexpr int EPT = (NE + NW - 1) / NW;            // entries per updating thread
  static constexpr int VPT = (TB * K + NW - 1) / NW;        // (row, pair) items of V per updating thread
  static_assert(LPP * K <= 32, "the rotation lanes exceed a warp");
  static_assert(kEigThreads == 256, "eight warps");
};

template <int TB>
struct Eig64Smem {
  double G[2][TB * (TB + 1)];
  double V[TB * (TB + 1)];
  double A[TB * (TB + 1)];
  double2 cs[2][TB / 2];       // (c, s) of the current round and of the next (by round parity)
  int2 pq[TB - 1][TB / 2];    // (p, q), p < q, of every pair of every round
  int2 pinfo[TB - 1][TB];     // (pair index, slot) of every index in every round
  double ev[TB];
  double g[TB];
};

template <int TB>
__device__ void eig64_body(Bufs b, int flags, cudaGraphConditionalHandle h, int use_cond, unsigned char* dsm) {
  using SH = Eig64Shape<TB>;
  constexpr int K = SH::K, NR = SH::NR, NE = SH::NE, NW = SH::NW, LPP = SH::LPP;
  constexpr int LD = TB + 1;
  Eig64Smem<TB>& S = *reinterpret_cast<Eig64Smem<TB>*>(dsm);
  __shared__ int sFlag;
  __shared__ double sTau;

  Ctrl* ctrl = b.ctrl;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int T = b.T;
  const unsigned long long t0 = gtimer();
  if (!eig_control(b, flags, h, use_cond, &sFlag)) return;
  const bool cold = (flags & EF_INIT) != 0;

  for (int i = tid; i < TB * TB; i += nthr) {
    const int r = i / TB, c = i % TB;
    const bool in = r < T && c < T;
    S.G[0][r * LD + c] = in ? b.red->G[r * kMaxT + c] : 0.0;
    double v = (r == c) ? 1.0 : 0.0;
    if (!cold && in) v = (double)b.eig->V32[r * kMaxT + c];
    S.V[r * LD + c] = v;
  }
  for (int i = tid; i < NR * K; i += nthr) {
    const int r = i / K, k = i % K;
    int pa, pb;
    rr_pair(r, k, TB, pa, pb);
    const int p = min(pa, pb), q = max(pa, pb);
    S.pq[r][k] = make_int2(p, q);
    S.pinfo[r][p] = make_int2(k, 0);
    S.pinfo[r][q] = make_int2(k, 1);
  }
  __syncthreads();
  const unsigned long long t1 = gtimer();

  const double eps = ctrl->jacobi_eps;
  const double eps2 = eps * eps;
  const float epsf2 = (float)eps2;
  int max_sweeps = (cold || (flags & EF_FULL)) ? ctrl->cold_sweeps : ctrl->warm_sweeps;
  if (max_sweeps > 30) max_sweeps = 30;
  // roles (Eig64Shape): updating thread index wi in [0, NW) for warps 0-2 and
  // 4-6; warp 7 forms the rotations, LPP lanes per pair
  const int warp = tid >> 5;
  const int wi = warp < 3 ? tid : (warp >= 4 && warp < 7 ? tid - 32 : -1);
  const bool worker = wi >= 0;
  const bool rwarp = warp == 7;
  const int rl = tid & 31;                                          // lane
  const int rk = (rwarp && rl < LPP * K) ? rl / LPP : K;            // pair of a rotation lane (K: none)
  const int rj = rl % LPP;                                          // its part: 0 (p,p) [and (p,q) if LPP = 2],
                                                                    // 1 (q,q), 2 (p,q)
  const bool rlead = rwarp && rj == 0 && rk < K;
  // The entries beyond the first NW (and the V items beyond the first NW) go
  // to workers whose warps run on other sub-partitions than warp 0's, so
  // the FP64 pipes of sub-partitions 0-2 carry about equal shares of a round.
  int ea[SH::EPT], ec[SH::EPT];
#pragma unroll
  for (int u = 0; u < SH::EPT; ++u) {
    int e = (u == 0 ? wi : (wi + NW - 128) % NW) + u * NW, a = 0;
    ea[u] = -1;
    ec[u] = -1;
    if (worker && e < NE) {
      while (e >= TB - a) {
        e -= TB - a;
        ++a;
      }
      ea[u] = a;
      ec[u] = a + e;
    }
  }

  // Entry (a, c) of J^T G J for round rnd's rotations in cs[cb] (G = S.G[cur]).
  auto rot_entry = [&](int rnd, int cb, int cur, int a, int c) -> double {
    const int2 ia = S.pinfo[rnd][a], ic = S.pinfo[rnd][c];
    const double2 ra = S.cs[cb][ia.x], rc = S.cs[cb][ic.x];
    if (ra.y == 0.0 && rc.y == 0.0) return S.G[cur][a * LD + c];
    const int2 pa2 = S.pq[rnd][ia.x], pc2 = S.pq[rnd][ic.x];
    // column a of J: slot 0 (c, -s) at (p, q); slot 1 (s, c)
    const double wa0 = ia.y ? ra.y : ra.x, wa1 = ia.y ? ra.x : -ra.y;
    const double wc0 = ic.y ? rc.y : rc.x, wc1 = ic.y ? rc.x : -rc.y;
    const double* g0 = &S.G[cur][pa2.x * LD];
    const double* g1 = &S.G[cur][pa2.y * LD];
    const double u0 = fma(wc1, g0[pc2.y], wc0 * g0[pc2.x]);
    const double u1 = fma(wc1, g1[pc2.y], wc0 * g1[pc2.x]);
    return fma(wa1, u1, wa0 * u0);
  };
  // Rotation of a pair from (app, aqq, apq) into cs[cb][k]; returns whether it rotates.
  // The threshold test and the tangent run on FP32 copies of the three
  // entries (the test's outcome only decides whether the pair rotates this
  // sweep; rotating or not, G stays an exact FP64 similarity transform of the
  // Gram), so the FP64 part of the chain is the conversions and the
  // normalisation.
  auto make_rotation = [&](int cb, int k, double app, double aqq, double apq) -> int {
    double c = 1.0, s = 0.0;
    int act = 0;
    const float apf = (float)apq, ppf = (float)app, qqf = (float)aqq;
    if (apf != 0.f && apf * apf > epsf2 * fabsf(ppf * qqf)) {
      act = 1;
      const float ddf = qqf - ppf;
      const float r2 = fmaf(ddf, ddf, 4.f * apf * apf);
      const float tf = copysignf(1.f, ddf) * (2.f * apf) / (fabsf(ddf) + sqrtf(r2));
      if (isfinite(tf) && isfinite(r2) && fabsf(apf) > 1e-30f) {
        const float cf = rsqrtf(fmaf(tf, tf, 1.f));
        c = (double)cf;
        s = (double)(tf * cf);
      } else {
        // outside FP32 range: the same rotation in FP64
        const double dd = aqq - app;
        const double t = copysign(1.0, dd) * (2.0 * apq) / (fabs(dd) + sqrt(fma(dd, dd, 4.0 * apq * apq)));
        c = 1.0 / sqrt(fma(t, t, 1.0));
        s = t * c;
      }
      // exact FP64 orthonormality: scale by (c^2 + s^2)^(-1/2) to third order
      const double d = fma(c, c, s * s) - 1.0;
      const double r = fma(fma(0.375, d, -0.5), d, 1.0);
      c *= r;
      s *= r;
    }
    S.cs[cb][k] = make_double2(c, s);
    return act;
  };

  int cur = 0, sweeps = 0, rounds_run = 0;
  while (sweeps < max_sweeps) {
    int need = 0;
#pragma unroll
    for (int u = 0; u < SH::EPT; ++u) {
      const int a = ea[u], c = ec[u];
      if (a >= 0 && a < c) {
        const double apq = S.G[cur][a * LD + c];
        if (apq != 0.0 && apq * apq > eps2 * fabs(S.G[cur][a * LD + a] * S.G[cur][c * LD + c])) need = 1;
      }
    }
    if (!__syncthreads_or(need)) break;
    int act = 0;
    if (rlead) {
      const int2 pq = S.pq[0][rk];
      act = make_rotation(0, rk, S.G[cur][pq.x * LD + pq.x], S.G[cur][pq.y * LD + pq.y], S.G[cur][pq.x * LD + pq.y]);
    }
    int any = __syncthreads_or(act);
    for (int rnd = 0; rnd < NR; ++rnd) {
      const int cb = rnd & 1;
      const int nxt = any ? (cur ^ 1) : cur;
      if (any && worker) {
        ++rounds_run;
#pragma unroll
        for (int u = 0; u < SH::EPT; ++u) {
          const int a = ea[u], c = ec[u];
          if (a < 0) continue;
          const double v = rot_entry(rnd, cb, cur, a, c);
          S.G[nxt][a * LD + c] = v;
          S.G[nxt][c * LD + a] = v;
        }
        // V <- V J on the round's pairs (each (row, pair) item touches only its two entries)
#pragma unroll
        for (int u = 0; u < SH::VPT; ++u) {
          const int item = (u == 0 ? wi : (wi + NW - 64) % NW) + u * NW;
          if (item >= T * K) continue;
          const int r = item / K, k = item % K;
          const double2 r2 = S.cs[cb][k];
          if (r2.y == 0.0) continue;
          const int2 pq = S.pq[rnd][k];
          const double vp = S.V[r * LD + pq.x], vq = S.V[r * LD + pq.y];
          S.V[r * LD + pq.x] = fma(r2.x, vp, -r2.y * vq);
          S.V[r * LD + pq.y] = fma(r2.y, vp, r2.x * vq);
        }
      }
      int act_next = 0;
      if (rwarp && rnd + 1 < NR) {
        // the entries (p,p), (q,q), (p,q) of the next round's pair rk after this
        // round, LPP lanes per pair
        double v = 0.0, w = 0.0;
        if (rk < K) {
          const int2 pq = S.pq[rnd + 1][rk];
          const int a = rj == 1 ? pq.y : pq.x, c = rj == 0 ? pq.x : pq.y;
          v = any ? rot_entry(rnd, cb, cur, a, c) : S.G[cur][a * LD + c];
          if (LPP == 2 && rj == 0) w = any ? rot_entry(rnd, cb, cur, pq.x, pq.y) : S.G[cur][pq.x * LD + pq.y];
        }
        const unsigned full = 0xffffffffu;
        const double aqq = __shfl_sync(full, v, rl + 1 < 32 ? rl + 1 : rl);
        const double apq = LPP == 2 ? w : __shfl_sync(full, v, rl + 2 < 32 ? rl + 2 : rl);
        if (rlead) act_next = make_rotation(cb ^ 1, rk, v, aqq, apq);
      }
      if (any) cur = nxt;
      any = __syncthreads_or(act_next);
    }
    ++sweeps;
  }

  const unsigned long long t2 = gtimer();
  if (tid < TB) S.ev[tid] = S.G[cur][tid * LD + tid];
  const int qb = cur ^ 1;  // free buffer
  // Newton-Schulz: A = 1.5 I - 0.5 V^T V (symmetric), then V <- V A -> S.G[qb]
  for (int i = tid; i < TB * TB; i += nthr) {
    const int a = i / TB, c = i % TB;
    if (a > c) continue;
    double acc = 0.0;
    if (c < T)
      for (int r = 0; r < T; ++r) acc = fma(S.V[r * LD + a], S.V[r * LD + c], acc);
    const double v = (a == c ? 1.5 : 0.0) - 0.5 * acc;
    S.A[a * LD + c] = v;
    S.A[c * LD + a] = v;
  }
  __syncthreads();
  for (int i = tid; i < TB * TB; i += nthr) {
    const int r = i / TB, c = i % TB;
    double acc = 0.0;
    if (r < T && c < T)
      for (int a = 0; a < T; ++a) acc = fma(S.V[r * LD + a], S.A[a * LD + c], acc);
    S.G[qb][r * LD + c] = acc;
  }
  const unsigned long long t3 = gtimer();

  // ---- FP64 decisions: mu (first call), tau, sigma > tau, g ----
  if (tid == 0) {
    if (flags & EF_INIT) {
      double lmax = 0.0;
      for (int a = 0; a < T; ++a) lmax = fmax(lmax, S.ev[a]);
      init_mu(b, lmax);
    }
    sTau = 1.0 / ctrl->mu_cur;
  }
  __syncthreads();
  int keep = 0;
  if (tid < TB) {
    const double sig = sqrt(fmax(S.ev[tid], 0.0));
    keep = (tid < T) && (sig > sTau);
    S.g[tid] = keep ? sTau / sig : 1.0;
  }
  const int rank = __syncthreads_count(keep);

  // Wbar = V diag(g) V^T in FP64 (upper triangle, mirrored), rounded to FP32
  // once; V rounded to FP32 for the next pass
  const double* Vn = S.G[qb];
  for (int i = tid; i < T * T; i += nthr) {
    const int a = i / T, c = i % T;
    b.eig->V32[a * kMaxT + c] = (float)Vn[a * LD + c];
    if (a > c) continue;
    double acc = 0.0;
    for (int j = 0; j < T; ++j) acc = fma(Vn[a * LD + j] * S.g[j], Vn[c * LD + j], acc);
    b.eig->Wbar[a * kMaxT + c] = (float)acc;
    b.eig->Wbar[c * kMaxT + a] = (float)acc;
  }
  if (tid < T) b.eig->evals[tid] = S.ev[tid];
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

template <int TB>
__global__ void __launch_bounds__(kEigThreads) eig64_kernel(Bufs b, int flags, cudaGraphConditionalHandle h,
                                                            int use_cond) {
  extern __shared__ __align__(16) unsigned char eig64_smem_raw[];
  eig64_body<TB>(b, flags, h, use_cond, eig64_smem_raw);
}
