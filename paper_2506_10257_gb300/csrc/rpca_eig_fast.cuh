// rpca_eig_fast.cuh -- eigen-step with FP32 Jacobi rotations (included inside
// namespace rpca by rpca_kernels.cuh).
//
// The rotated Gram G~ = V^T Z^T Z V of the next iteration arrives nearly
// diagonal, so a few cyclic Jacobi sweeps in FP32 diagonalise it to the
// accuracy of its FP32 entries.  Each round of a sweep annihilates T/2
// disjoint (p, q) pairs (round-robin order):
//   phase A  T/2 threads compute the rotations (GVL sym.schur2) and the exact
//            new diagonal entries, and log them;
//   phase B  one thread per upper-triangle entry forms (J^T G J)_ab from four
//            entries of G (pairs not rotated this round have c = 1, s = 0).
// The eigenvector update is not done per round: after the sweeps every row of
// Q (the product of the logged rotations) is accumulated in registers by one
// thread, with the (p, q) indices of each round known at compile time.  Then
// V_new = V_old Q, one Newton-Schulz step keeps it orthonormal, and the FP64
// part follows: sigma = sqrt(lambda), the sigma > tau = 1/mu decision and
// g = min(1, tau/sigma), with Wbar = V diag(g) V^T (Eq. 4 through the Gram).
#pragma once

constexpr int kEigLogSweeps = 10;  // sweeps one eigen-step may take (and log)
constexpr int kEigThreads = 256;   // threads of the eigen-step CTA

template <int TB>
struct EigFastSmem {
  float G[2][TB * (TB + 1)];
  float2 log[kEigLogSweeps][TB - 1][TB / 2];
  int ran[kEigLogSweeps][TB - 1];
  float2 cs[2][TB / 2];       // rotations of the current round and of the next (by round parity)
  int2 pq[TB - 1][TB / 2];   // (p, q), p < q, of every pair of every round (fixed order)
  int2 pinfo[TB - 1][TB];    // (pair index, slot) of every index in every round
  float dnew[2][TB];          // new diagonal entries, same double buffering
  float A[TB * (TB + 1)];
  double ev[TB];
  float g[TB];
};

// The eigen-step on one CTA of kEigThreads threads; `dsm` holds
// sizeof(EigFastSmem<TB>) bytes of shared memory.
template <int TB>
__device__ void eig_fast_body(Bufs b, int flags, cudaGraphConditionalHandle h, int use_cond, unsigned char* dsm) {
  constexpr int K = TB / 2;
  constexpr int NR = TB - 1;
  constexpr int LD = TB + 1;
  constexpr int NE = TB * (TB + 1) / 2;
  constexpr int EPT = (NE + kEigThreads - 1) / kEigThreads;  // upper-triangle entries per thread
  EigFastSmem<TB>& S = *reinterpret_cast<EigFastSmem<TB>*>(dsm);
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
    S.G[0][r * LD + c] = (r < T && c < T) ? b.red->G[r * kMaxT + c] : 0.f;
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
  int rounds_run = 0;

  const float eps = (float)ctrl->jacobi_eps;
  const float eps2 = eps * eps;
  int max_sweeps = (cold || (flags & EF_FULL)) ? ctrl->cold_sweeps : ctrl->warm_sweeps;
  if (max_sweeps > kEigLogSweeps) max_sweeps = kEigLogSweeps;
  // upper-triangle entries owned by this thread
  int ea[EPT], ec[EPT];
#pragma unroll
  for (int u = 0; u < EPT; ++u) {
    int e = tid + u * nthr, a = 0;
    ea[u] = -1;
    ec[u] = -1;
    if (e < NE) {
      while (e >= TB - a) {
        e -= TB - a;
        ++a;
      }
      ea[u] = a;
      ec[u] = a + e;
    }
  }
  // Entry (a, c), a <= c, of J^T G J for round rnd's rotations (buffers cb):
  // pairs not rotated have c = 1, s = 0; a rotated pair's own entry is 0.
  auto rotated_entry = [&](int rnd, int cb, int cur, int a, int c) -> float {
    if (a == c) return S.dnew[cb][a];
    const int2 ia = S.pinfo[rnd][a], ic = S.pinfo[rnd][c];
    if (ia.x == ic.x) {
      const float2 r = S.cs[cb][ia.x];
      return (r.y != 0.f) ? 0.f : S.G[cur][a * LD + c];  // annihilated when rotated
    }
    const int2 pa2 = S.pq[rnd][ia.x], pc2 = S.pq[rnd][ic.x];
    const float2 ra = S.cs[cb][ia.x], rc = S.cs[cb][ic.x];
    // column a of J: slot 0 (c, -s) at (p, q); slot 1 (s, c)
    const float wa0 = ia.y ? ra.y : ra.x, wa1 = ia.y ? ra.x : -ra.y;
    const float wc0 = ic.y ? rc.y : rc.x, wc1 = ic.y ? rc.x : -rc.y;
    const float* g0 = &S.G[cur][pa2.x * LD];
    const float* g1 = &S.G[cur][pa2.y * LD];
    return wa0 * (wc0 * g0[pc2.x] + wc1 * g0[pc2.y]) + wa1 * (wc0 * g1[pc2.x] + wc1 * g1[pc2.y]);
  };
  // Rotation of pair k of round rnd from (app, aqq, apq) into buffers cb (GVL
  // sym.schur2: t = 2 apq sgn(d) / (|d| + sqrt(d^2 + 4 apq^2)), d = aqq - app);
  // returns whether the pair rotates.
  auto make_rotation = [&](int rnd, int cb, int sw, int k, float app, float aqq, float apq) -> int {
    const int2 pq = S.pq[rnd][k];
    float c = 1.f, s = 0.f, dp = app, dq = aqq;
    int act = 0;
    if (apq != 0.f && apq * apq > eps2 * fabsf(app * aqq)) {
      act = 1;
      const float dd = aqq - app;
      const float r2 = fmaf(dd, dd, 4.f * apq * apq);
      const float den = fabsf(dd) + r2 * rsqrtf(r2);
      const float t = copysignf(1.f, dd) * (2.f * apq) * __fdividef(1.f, den);
      c = rsqrtf(fmaf(t, t, 1.f));
      s = t * c;
      dp = app - t * apq;
      dq = aqq + t * apq;
    }
    S.cs[cb][k] = make_float2(c, s);
    S.log[sw][rnd][k] = make_float2(c, s);
    S.dnew[cb][pq.x] = dp;
    S.dnew[cb][pq.y] = dq;
    return act;
  };
  // The next round's rotations are formed by the last K threads of the CTA
  // (the ones with the fewest upper-triangle entries) while every thread
  // updates its entries for the current round, so a round needs one barrier.
  const int pk = tid - (nthr - K);  // pair of this thread, or < 0

  int cur = 0, sweeps = 0;
  while (sweeps < max_sweeps) {
    int need = 0;
#pragma unroll
    for (int u = 0; u < EPT; ++u) {
      const int a = ea[u], c = ec[u];
      if (a >= 0 && a < c) {
        const float apq = S.G[cur][a * LD + c];
        if (apq != 0.f && apq * apq > eps2 * fabsf(S.G[cur][a * LD + a] * S.G[cur][c * LD + c])) need = 1;
      }
    }
    if (!__syncthreads_or(need)) break;
    int act = 0;
    if (pk >= 0) {
      const int2 pq = S.pq[0][pk];
      act = make_rotation(0, 0, sweeps, pk, S.G[cur][pq.x * LD + pq.x], S.G[cur][pq.y * LD + pq.y],
                          S.G[cur][pq.x * LD + pq.y]);
    }
    int any = __syncthreads_or(act);
    for (int rnd = 0; rnd < NR; ++rnd) {
      const int cb = rnd & 1;
      if (tid == 0) S.ran[sweeps][rnd] = any;
      const int nxt = any ? (cur ^ 1) : cur;
      if (any) {
        ++rounds_run;
#pragma unroll
        for (int u = 0; u < EPT; ++u) {
          const int a = ea[u], c = ec[u];
          if (a < 0) continue;
          const float v = rotated_entry(rnd, cb, cur, a, c);
          S.G[nxt][a * LD + c] = v;
          S.G[nxt][c * LD + a] = v;
        }
      }
      int act_next = 0;
      if (pk >= 0 && rnd + 1 < NR) {
        // the entries (p, p), (q, q), (p, q) of the next round's pair after this round
        const int2 pq = S.pq[rnd + 1][pk];
        float app, aqq, apq;
        if (any) {
          app = S.dnew[cb][pq.x];
          aqq = S.dnew[cb][pq.y];
          apq = rotated_entry(rnd, cb, cur, pq.x, pq.y);
        } else {
          app = S.G[cur][pq.x * LD + pq.x];
          aqq = S.G[cur][pq.y * LD + pq.y];
          apq = S.G[cur][pq.x * LD + pq.y];
        }
        act_next = make_rotation(rnd + 1, cb ^ 1, sweeps, pk, app, aqq, apq);
      }
      cur = nxt;
      any = __syncthreads_or(act_next);
    }
    ++sweeps;
  }

  const unsigned long long t2 = gtimer();
  // ---- eigenvalues; rows of Q = product of the logged rotations ----
  if (tid < TB) S.ev[tid] = (double)S.G[cur][tid * LD + tid];
  const int qb = cur ^ 1;  // Q goes to the other G buffer
  if (tid < TB) {
    float qr[TB];
#pragma unroll
    for (int j = 0; j < TB; ++j) qr[j] = (j == tid) ? 1.f : 0.f;
    for (int sw = 0; sw < sweeps; ++sw) {
#pragma unroll
      for (int rnd = 0; rnd < NR; ++rnd) {
        if (!S.ran[sw][rnd]) continue;
#pragma unroll
        for (int k = 0; k < K; ++k) {
          int pa, pb;
          rr_pair(rnd, k, TB, pa, pb);
          const int p = pa < pb ? pa : pb, q = pa < pb ? pb : pa;
          const float2 r = S.log[sw][rnd][k];
          const float xp = qr[p], xq = qr[q];
          qr[p] = r.x * xp - r.y * xq;
          qr[q] = r.y * xp + r.x * xq;
        }
      }
    }
#pragma unroll
    for (int j = 0; j < TB; ++j) S.G[qb][tid * LD + j] = qr[j];
  }
  __syncthreads();
  const unsigned long long t3 = gtimer();
  // old basis -> S.A
  for (int i = tid; i < TB * TB; i += nthr) {
    const int r = i / TB, c = i % TB;
    float v = (r == c) ? 1.f : 0.f;
    if (!cold && r < T && c < T) v = b.eig->V32[r * kMaxT + c];
    S.A[r * LD + c] = v;
  }
  __syncthreads();
  // V_new = V_old Q  -> S.G[cur]
  for (int i = tid; i < TB * TB; i += nthr) {
    const int r = i / TB, c = i % TB;
    float acc = 0.f;
#pragma unroll 4
    for (int j = 0; j < TB; ++j) acc = fmaf(S.A[r * LD + j], S.G[qb][j * LD + c], acc);
    S.G[cur][r * LD + c] = acc;
  }
  __syncthreads();
  // Newton-Schulz: P = 1.5 I - 0.5 V^T V -> S.A ; V <- V P -> S.G[qb]
  for (int i = tid; i < TB * TB; i += nthr) {
    const int a = i / TB, c = i % TB;
    float acc = 0.f;
#pragma unroll 4
    for (int r = 0; r < TB; ++r) acc = fmaf(S.G[cur][r * LD + a], S.G[cur][r * LD + c], acc);
    S.A[a * LD + c] = (a == c ? 1.5f : 0.f) - 0.5f * acc;
  }
  __syncthreads();
  for (int i = tid; i < TB * TB; i += nthr) {
    const int r = i / TB, c = i % TB;
    float acc = 0.f;
#pragma unroll 4
    for (int a = 0; a < TB; ++a) acc = fmaf(S.G[cur][r * LD + a], S.A[a * LD + c], acc);
    S.G[qb][r * LD + c] = acc;
  }

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
    S.g[tid] = keep ? (float)(sTau / sig) : 1.f;
  }
  const int rank = __syncthreads_count(keep);

  const float* Vn = S.G[qb];
  for (int i = tid; i < T * T; i += nthr) {
    const int a = i / T, c = i % T;
    float acc = 0.f;
    for (int j = 0; j < T; ++j) acc = fmaf(Vn[a * LD + j] * S.g[j], Vn[c * LD + j], acc);
    b.eig->Wbar[a * kMaxT + c] = acc;
    b.eig->V32[a * kMaxT + c] = Vn[a * LD + c];
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
__global__ void __launch_bounds__(kEigThreads) eig_fast_kernel(Bufs b, int flags, cudaGraphConditionalHandle h,
                                                               int use_cond) {
  extern __shared__ __align__(16) unsigned char eig_smem_raw[];
  eig_fast_body<TB>(b, flags, h, use_cond, eig_smem_raw);
}
