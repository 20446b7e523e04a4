// rpca_eig_fast.cuh -- the narrow eigen-step (T <= 32): cyclic Jacobi on the
// rotated Gram, in FP64 (default) or FP32 rotations (included inside
// namespace rpca by rpca_kernels.cuh).
//
// The rotated Gram G~ = V^T Z^T Z V of the next iteration arrives nearly
// diagonal (V is the basis the pass rotated Z into), so a few cyclic Jacobi
// sweeps diagonalise it.  Each round of a sweep annihilates T/2 disjoint
// (p, q) pairs (round-robin order):
//   phase A  T/2 threads compute the rotations (GVL sym.schur2) and the exact
//            new diagonal entries, and log them;
//   phase B  one thread per upper-triangle entry forms (J^T G J)_ab from four
//            entries of G (pairs not rotated this round have c = 1, s = 0).
// The eigenvector update is not done per round: after the sweeps every row of
// Q (the product of the logged rotations) is accumulated in registers by one
// thread, with the (p, q) indices of each round known at compile time.  Then
// V_new = V Q with V the basis the pass used, one Newton-Schulz step
// V <- V (3I - V^T V)/2 makes it orthonormal (to first order this also
// removes the departure of the FP32-rounded V from orthonormality), and the
// decisions follow in FP64: sigma = sqrt(lambda), sigma > tau = 1/mu and
// g = min(1, tau/sigma), with Wbar = V diag(g) V^T (Eq. 4 through the Gram).
// Real = double does all of that in FP64 (the Gram arrives as FP64 sums) and
// rounds Wbar and V to FP32 once for the passes; Real = float is the faster
// opt-in with FP32 rotations and basis arithmetic.
#pragma once

constexpr int kEigLogSweeps = 10;  // sweeps one eigen-step may take (and log)
constexpr int kEigThreads = 256;   // threads of the eigen-step CTA

template <typename Real>
struct Pair2 {
  Real x, y;
};

template <int TB, typename Real>
struct EigFastSmem {
  Real G[2][TB * (TB + 1)];
  Pair2<Real> log[kEigLogSweeps][TB - 1][TB / 2];
  int ran[kEigLogSweeps][TB - 1];
  Pair2<Real> cs[2][TB / 2];  // rotations of the current round and of the next (by round parity)
  int2 pq[TB - 1][TB / 2];   // (p, q), p < q, of every pair of every round (fixed order)
  int2 pinfo[TB - 1][TB];    // (pair index, slot) of every index in every round
  Real dnew[2][TB];           // new diagonal entries, same double buffering
  Real A[TB * (TB + 1)];
  double ev[TB];
  Real g[TB];
};

__device__ __forceinline__ float rsqrt_r(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsqrt_r(double x) { return 1.0 / sqrt(x); }
__device__ __forceinline__ float recip_r(float x) { return __fdividef(1.f, x); }
__device__ __forceinline__ double recip_r(double x) { return 1.0 / x; }

// The eigen-step on one CTA of kEigThreads threads; `dsm` holds
// sizeof(EigFastSmem<TB>) bytes of shared memory.
template <int TB, typename Real>
__device__ void eig_fast_body(Bufs b, int flags, cudaGraphConditionalHandle h, int use_cond, unsigned char* dsm) {
  constexpr int K = TB / 2;
  constexpr int NR = TB - 1;
  constexpr int LD = TB + 1;
  constexpr int NE = TB * (TB + 1) / 2;
  constexpr int EPT = (NE + kEigThreads - 1) / kEigThreads;  // upper-triangle entries per thread
  using P2 = Pair2<Real>;
  EigFastSmem<TB, Real>& S = *reinterpret_cast<EigFastSmem<TB, Real>*>(dsm);
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
    S.G[0][r * LD + c] = (r < T && c < T) ? (Real)b.red->G[r * kMaxT + c] : (Real)0;
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

  const Real eps = (Real)ctrl->jacobi_eps;
  const Real eps2 = eps * eps;
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
  auto rotated_entry = [&](int rnd, int cb, int cur, int a, int c) -> Real {
    if (a == c) return S.dnew[cb][a];
    const int2 ia = S.pinfo[rnd][a], ic = S.pinfo[rnd][c];
    if (ia.x == ic.x) {
      const P2 r = S.cs[cb][ia.x];
      return (r.y != (Real)0) ? (Real)0 : S.G[cur][a * LD + c];  // annihilated when rotated
    }
    const int2 pa2 = S.pq[rnd][ia.x], pc2 = S.pq[rnd][ic.x];
    const P2 ra = S.cs[cb][ia.x], rc = S.cs[cb][ic.x];
    // pairs not rotated this round keep their entries (c = 1, s = 0)
    if (ra.y == (Real)0 && rc.y == (Real)0) return S.G[cur][a * LD + c];
    // column a of J: slot 0 (c, -s) at (p, q); slot 1 (s, c)
    const Real wa0 = ia.y ? ra.y : ra.x, wa1 = ia.y ? ra.x : -ra.y;
    const Real wc0 = ic.y ? rc.y : rc.x, wc1 = ic.y ? rc.x : -rc.y;
    const Real* g0 = &S.G[cur][pa2.x * LD];
    const Real* g1 = &S.G[cur][pa2.y * LD];
    return wa0 * (wc0 * g0[pc2.x] + wc1 * g0[pc2.y]) + wa1 * (wc0 * g1[pc2.x] + wc1 * g1[pc2.y]);
  };
  // Rotation of pair k of round rnd from (app, aqq, apq) into buffers cb (GVL
  // sym.schur2: t = 2 apq sgn(d) / (|d| + sqrt(d^2 + 4 apq^2)), d = aqq - app);
  // returns whether the pair rotates.
  auto make_rotation = [&](int rnd, int cb, int sw, int k, Real app, Real aqq, Real apq) -> int {
    const int2 pq = S.pq[rnd][k];
    Real c = 1, s = 0, dp = app, dq = aqq;
    int act = 0;
    if (apq != (Real)0 && apq * apq > eps2 * fabs(app * aqq)) {
      act = 1;
      const Real dd = aqq - app;
      const Real r2 = fma(dd, dd, (Real)4 * apq * apq);
      const Real den = fabs(dd) + sqrt(r2);
      const Real t = copysign((Real)1, dd) * ((Real)2 * apq) * recip_r(den);
      c = rsqrt_r(fma(t, t, (Real)1));
      s = t * c;
      dp = app - t * apq;
      dq = aqq + t * apq;
    }
    S.cs[cb][k] = P2{c, s};
    S.log[sw][rnd][k] = P2{c, s};
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
        const Real apq = S.G[cur][a * LD + c];
        if (apq != (Real)0 && apq * apq > eps2 * fabs(S.G[cur][a * LD + a] * S.G[cur][c * LD + c])) need = 1;
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
          const Real v = rotated_entry(rnd, cb, cur, a, c);
          S.G[nxt][a * LD + c] = v;
          S.G[nxt][c * LD + a] = v;
        }
      }
      int act_next = 0;
      if (pk >= 0 && rnd + 1 < NR) {
        // the entries (p, p), (q, q), (p, q) of the next round's pair after this round
        const int2 pq = S.pq[rnd + 1][pk];
        Real app, aqq, apq;
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
    Real qr[TB];
#pragma unroll
    for (int j = 0; j < TB; ++j) qr[j] = (j == tid) ? (Real)1 : (Real)0;
    for (int sw = 0; sw < sweeps; ++sw) {
#pragma unroll
      for (int rnd = 0; rnd < NR; ++rnd) {
        if (!S.ran[sw][rnd]) continue;
#pragma unroll
        for (int k = 0; k < K; ++k) {
          int pa, pb;
          rr_pair(rnd, k, TB, pa, pb);
          const int p = pa < pb ? pa : pb, q = pa < pb ? pb : pa;
          const P2 r = S.log[sw][rnd][k];
          if (r.y == (Real)0) continue;  // not rotated
          const Real xp = qr[p], xq = qr[q];
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
  // the basis the pass used (V32, exact in FP64) -> S.A
  for (int i = tid; i < TB * TB; i += nthr) {
    const int r = i / TB, c = i % TB;
    Real v = (r == c) ? (Real)1 : (Real)0;
    if (!cold && r < T && c < T) v = (Real)b.eig->V32[r * kMaxT + c];
    S.A[r * LD + c] = v;
  }
  __syncthreads();
  // V_new = V_old Q  -> S.G[cur] (rows and columns past T stay zero)
  for (int i = tid; i < TB * TB; i += nthr) {
    const int r = i / TB, c = i % TB;
    Real acc = 0;
    if (r < T && c < T) {
#pragma unroll 4
      for (int j = 0; j < T; ++j) acc = fma(S.A[r * LD + j], S.G[qb][j * LD + c], acc);
    }
    S.G[cur][r * LD + c] = acc;
  }
  __syncthreads();
  // Newton-Schulz: P = 1.5 I - 0.5 V^T V -> S.A (symmetric: upper triangle
  // computed, mirrored); V <- V P -> S.G[qb]
  for (int i = tid; i < TB * TB; i += nthr) {
    const int a = i / TB, c = i % TB;
    if (a > c) continue;
    Real acc = 0;
    if (c < T) {
#pragma unroll 4
      for (int r = 0; r < T; ++r) acc = fma(S.G[cur][r * LD + a], S.G[cur][r * LD + c], acc);
    }
    const Real v = (a == c ? (Real)1.5 : (Real)0) - (Real)0.5 * acc;
    S.A[a * LD + c] = v;
    S.A[c * LD + a] = v;
  }
  __syncthreads();
  for (int i = tid; i < TB * TB; i += nthr) {
    const int r = i / TB, c = i % TB;
    Real acc = 0;
    if (r < T && c < T) {
#pragma unroll 4
      for (int a = 0; a < T; ++a) acc = fma(S.G[cur][r * LD + a], S.A[a * LD + c], acc);
    }
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
    S.g[tid] = keep ? (Real)(sTau / sig) : (Real)1;
  }
  const int rank = __syncthreads_count(keep);

  // Wbar = V diag(g) V^T (symmetric: upper triangle, mirrored), rounded to
  // FP32 once; V rounded to FP32 for the next pass
  const Real* Vn = S.G[qb];
  for (int i = tid; i < T * T; i += nthr) {
    const int a = i / T, c = i % T;
    b.eig->V32[a * kMaxT + c] = (float)Vn[a * LD + c];
    if (a > c) continue;
    Real acc = 0;
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

template <int TB, typename Real>
__global__ void __launch_bounds__(kEigThreads) eig_fast_kernel(Bufs b, int flags, cudaGraphConditionalHandle h,
                                                               int use_cond) {
  extern __shared__ __align__(16) unsigned char eig_smem_raw[];
  eig_fast_body<TB, Real>(b, flags, h, use_cond, eig_smem_raw);
}
