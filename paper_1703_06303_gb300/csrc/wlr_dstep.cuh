// Step a3 of Algorithm 1 (Dutta & Li, arXiv 1703.06303): one step of the subspace
// iteration for the top r - k eigenpairs of G2 = (P_perp A2)^T (P_perp A2) = K - B^T B
// (Theorem 2 / Eckart-Young through the Gram matrix), the Ritz vectors V_s that define
// D = U_s Sigma_s V_s^T, and the two small products of step a5 that depend on them
// (G = C C^T and C V_s).
//
// Z = G2 V is formed without G2: kv_pair takes K V in double-float on all SMs (K = Kh + Kl
// is stored as a float pair), and the cluster kernels subtract B^T (B V) before rounding
// to T (K and B^T B nearly cancel on the subspace).  Two cluster kernels (NC = 16 CTAs
// where the device allows it, else 8):
//   dstep_front, the steady-state step for k <= 32: also steps a1 (the second CholeskyQR
//     factor, on CTA 0) and a2 (B, C), arranged so that the other CTAs work on their basis
//     rows while CTA 0 factors (see the comment above the kernel);
//   dstep_cluster, the further steps of a cold start and every step for k > 32 (B and C
//     come from coef_kernel3): CTA r owns rows [r R, r R + R), R = ceil(n2 / NC):
//     1. partial B V over the CTA's rows, summed by every CTA through distributed shared
//        memory; Z(rows) = K V - B^T (B V);
//     2. partial H = V^T Z and P = Z^T Z, summed by CTA 0, which runs the Rayleigh-Ritz
//        step (ritz_step) on the b x b problem;
//     3. every CTA reads Y, Mv, Mz from CTA 0 and forms its rows of the next basis
//        V Mv + Z Mz and of V_s = (V Y)(:, :s); then the partials of C C^T and C V_s are
//        summed by CTA 0.
// All waits are cluster barriers reached unconditionally by every CTA.
#pragma once

#include <cooperative_groups.h>

#include "wlr_kernels.cuh"

namespace wlr {

namespace cgrp = cooperative_groups;

constexpr int DS_THREADS = 512;
constexpr int DS_BM = EIG_BMAX;   // largest b
constexpr int DS_P = DS_BM + 1;   // row pitch of the b x b work arrays

// Reciprocal and square root for the short serial chains of the small factorizations:
// hardware estimate plus one Newton step (float; within a few ulp, about a third of the
// latency of the correctly rounded operations), exact operations for double.
__device__ __forceinline__ float qrcp(float x) {
  const float r = __fdividef(1.0f, x);
  return fmaf(r, fmaf(-x, r, 1.0f), r);
}
__device__ __forceinline__ double qrcp(double x) { return 1.0 / x; }
__device__ __forceinline__ float qsqrt(float x) { return x > 0.f ? x * wrsqrt(x) : 0.f; }
__device__ __forceinline__ double qsqrt(double x) { return sqrt(x); }

// Sum of products in double-float (float) or plain double: hi + lo.
template <typename T>
struct DfAcc;
template <>
struct DfAcc<float> {
  float hi = 0.f, lo = 0.f;
  // += (xh + xl) y, the product xh y kept exactly (TwoProduct by FMA)
  __device__ __forceinline__ void add(float xh, float xl, float y) {
    const float p = xh * y;
    const float pe = fmaf(xh, y, -p);
    const float x = fmaf(xl, y, pe);
    float s, e;
    two_sum(hi, p, s, e);
    hi = s;
    lo += e + x;
  }
  // -= (xh + xl)(yh + yl)
  __device__ __forceinline__ void sub2(float xh, float xl, float yh, float yl) {
    const float p = xh * yh;
    const float pe = fmaf(xh, yh, -p);
    const float x = fmaf(xh, yl, fmaf(xl, yh, pe));
    float s, e;
    two_sum(hi, -p, s, e);
    hi = s;
    lo += e - x;
  }
  __device__ __forceinline__ void add_pair(float h, float l) {
    float s, e;
    two_sum(hi, h, s, e);
    hi = s;
    lo = (lo + l) + e;
  }
  __device__ __forceinline__ void warp_reduce() {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float h2 = __shfl_xor_sync(0xffffffffu, hi, o);
      const float l2 = __shfl_xor_sync(0xffffffffu, lo, o);
      add_pair(h2, l2);
    }
  }
};
template <>
struct DfAcc<double> {
  double hi = 0.0, lo = 0.0;
  __device__ __forceinline__ void add(double xh, double, double y) { hi = fma(xh, y, hi); }
  __device__ __forceinline__ void sub2(double xh, double, double yh, double) { hi = fma(-xh, yh, hi); }
  __device__ __forceinline__ void add_pair(double h, double) { hi += h; }
  __device__ __forceinline__ void warp_reduce() { hi = warp_sum(hi); }
};

template <typename T>
struct DstepArgs {
  const T* ZKh;  // K V (n2 x b) from kv_pair: high part (the whole product for double)
  const T* ZKl;  // low part (nullptr: none)
  const T* Bh;   // B = Q^T A2 (k x n2, column j at B + j*k): high part
  const T* Bl;   // low part (nullptr: none)
  T* Z2;         // n2 x NP row-major: C^T in columns < k (read); V_s into columns k..k+s-1
  T* V;          // n2 x b basis: in, the current one; out, the next one
  T* Vs;         // n2 x s Ritz vectors
  T* theta;      // b Ritz values, descending
  T* resid;      // b residual estimates (Y^T P Y)_cc - theta_c^2
  T* G;          // k x k, C C^T
  T* CV;         // k x s, C V_s
  int* err;
  int n2, k, b, s, NP;
  int sweeps;    // Jacobi sweeps of the Rayleigh-Ritz step
  // Steps a1 (second CholeskyQR factor) and a2 first, when `front` is set (k <= 32, the
  // kernel dstep_front): CTA 0 forms the second factor of Q1^T Q1 = I + F, and the other
  // CTAs form B and C for their columns.
  int front;
  const double* S2T;   // Q1^T [Q1 A2] summed over the Gram chunks: k x (k + n2) column-major
  const T* F2;         // S2 - I (k x k, column-major) = leading block of S2T minus I
  const T* R1inv;      // inverse of the first factor (k x k; upper triangular after a
                       // Cholesky first factor, full after chol2_series)
  T* Nout;             // N = R2^{-T} - I (lower triangular, or full after chol2_series)
  T* Rinv;             // R^{-1} = R1inv (I + N)^T
  T* Cout;             // C = R^{-1} B (k x n2)
  double* B64;         // B (k x n2), FP64 path
  float* Bho;          // B = Bho + Blo, float path
  float* Blo;
  double* bpart;       // ||B||^2 over each CTA's columns (nc entries)
  int series;          // float front stage: the second factor may be (I + F)^{1/2} (chol2_series)
};

// Element offsets of the dynamic shared memory (every CTA has the same layout; the b x b
// work arrays are used by CTA 0 only).
struct DsLayout {
  size_t Vt, Bs, Cs, Zh, Zl, Zr, Vsr, BVp, BV, HPp, Gp, CVp, Ml, Wk, total;
  template <typename T>
  __host__ __device__ static DsLayout make(int n2, int k, int b, int s, int R) {
    return DsLayout(n2, k, b, s, R);
  }
  __host__ __device__ DsLayout(int n2, int k, int b, int s, int R) {
    const size_t ss = s > 0 ? s : 1;
    size_t o = 0;
    Vt = o;  o += (size_t)b * n2;           // basis, V(j, c) at Vt[c*n2 + j]
    Bs = o;  o += 2 * (size_t)k * R;        // B(:, rows): high, low
    Cs = o;  o += (size_t)R * k;            // C(:, rows), C(x, j) at Cs[(j - l0)*k + x]
    Zh = o;  o += (size_t)R * b;            // (K V)(rows), high, Zh[c*R + rr]
    Zl = o;  o += (size_t)R * b;            // low
    Zr = o;  o += (size_t)R * b;            // Z(rows), Zr[rr*b + c]
    Vsr = o; o += (size_t)R * ss;           // V_s(rows)
    BVp = o; o += 2 * (size_t)k * b;        // partial B V (high, low)
    BV = o;  o += 2 * (size_t)k * b;        // B V
    HPp = o; o += 2 * (size_t)b * b;        // partial H, P
    Gp = o;  o += (size_t)k * k;            // partial C C^T
    CVp = o; o += (size_t)k * ss;           // partial C V_s
    Ml = o;  o += 3 * (size_t)b * b;        // local copies of Y, Mv, Mz
    Wk = o;  o += 10 * (size_t)DS_BM * DS_P;    // Rayleigh-Ritz work arrays
    total = o;
  }
};

// Rayleigh-Ritz step of the subspace iteration on one CTA (DS_THREADS threads), b <= 32.
// In: H (=V^T G2 V) and P (=Z^T Z) in wk[0] and wk[4]; out: the sorted eigenvectors Y,
// Mv and Mz (b x b, column-major, at wk + 7*DS_BM*DS_P, + 8*, + 9*), theta and resid.
//  - H = Y Theta Y^T by the parallel cyclic Jacobi method (round-robin ordering): a round
//    applies its b/2 rotations, H <- J^T H J and Y <- Y J element by element into the
//    other buffer of a pair, while threads tid < b/2 take the next round's angles from the
//    rotated entries they need (one barrier per round).
//  - Next basis W = [V Y F_v + Z Y F_z], F_z = diag(1/||Z y_c||) for the columns with a
//    non-negligible Ritz value, F_v = 1 for the others; W^T W = L L^T (Cholesky of the
//    Gram formed from I, Y^T P Y and Theta); Mv = Y F_v L^{-T}, Mz = Y F_z L^{-T}.
// Each thread owns the elements e = tid + q DS_THREADS, q < NE, of a b x b array (row
// e % b, column e / b; NE DS_THREADS >= b^2), indexed once.
template <typename T, int NE>
__device__ void ritz_step(T* wk, int b, int max_sweeps, T* __restrict__ theta,
                          T* __restrict__ resid, int* __restrict__ err) {
  using Row = T[DS_P];
  Row* Hc = reinterpret_cast<Row*>(wk);                      // current / next buffers
  Row* Hn = reinterpret_cast<Row*>(wk + DS_BM * DS_P);
  Row* Yc = reinterpret_cast<Row*>(wk + 2 * DS_BM * DS_P);
  Row* Yn = reinterpret_cast<Row*>(wk + 3 * DS_BM * DS_P);
  Row* Pm = reinterpret_cast<Row*>(wk + 4 * DS_BM * DS_P);
  Row* Wm = reinterpret_cast<Row*>(wk + 5 * DS_BM * DS_P);   // sorted eigenvectors
  Row* Gm = reinterpret_cast<Row*>(wk + 6 * DS_BM * DS_P);   // Gram, then its elimination
  T* Yo = wk + 7 * DS_BM * DS_P;                             // outputs, b x b col-major
  T* Mvo = wk + 8 * DS_BM * DS_P;
  T* Mzo = wk + 9 * DS_BM * DS_P;
  // rotation of index x in a round: J(x,x) = c, J(partner, x) = s (one 16-byte load for float)
  struct alignas(2 * sizeof(T)) Rot {
    T c, s;
    int partner, pad;
  };
  __shared__ Rot rot[2][DS_BM];
  __shared__ T th[DS_BM], fz[DS_BM], rdg[DS_BM];
  __shared__ int perm[DS_BM], usev[DS_BM];
  __shared__ T red[2][DS_THREADS / 32];
  __shared__ int bad_s;
  const int tid = threadIdx.x;
  const int bb = b * b;
  int er[NE], ec[NE];
#pragma unroll
  for (int q = 0; q < NE; ++q) {
    const int e = tid + q * DS_THREADS;
    er[q] = e % b;
    ec[q] = e / b;
  }
  // f(e, r, c) for each of this thread's elements
  auto each = [&](auto&& f) {
#pragma unroll
    for (int q = 0; q < NE; ++q) {
      const int e = tid + q * DS_THREADS;
      if (e < bb) f(e, er[q], ec[q]);
    }
  };

  // symmetric H, Y = I, zero padding of both buffers (the dummy index b of an odd b is
  // read with a zero coefficient)
  for (int e = tid; e < DS_BM * DS_P; e += DS_THREADS) {
    const int r = e / DS_P, c = e % DS_P;
    const bool in = r < b && c < b;
    Hn[r][c] = T(0);
    Yc[r][c] = (r == c && r < b) ? T(1) : T(0);
    Yn[r][c] = T(0);
    if (!in) {
      Hc[r][c] = T(0);
      Pm[r][c] = T(0);
    }
  }
  if (tid == 0) bad_s = 0;
  __syncthreads();
  each([&](int, int r, int c) {
    if (r < c) {
      const T v = T(0.5) * (Hc[r][c] + Hc[c][r]);
      Hc[r][c] = v;
      Hc[c][r] = v;
    }
  });
  __syncthreads();

  const int N = (b + 1) & ~1, half = N / 2;
  const T eps = T(4 * b) * (sizeof(T) == 4 ? T(5.96e-8) : T(1.11e-16));
  // pair i of a round of the round-robin order (N even): index N - 1 meets `round`, and
  // i, j < N - 1 meet when i + j = 2 round (mod N - 1)
  auto pair_of = [&](int round, int i, int& p, int& q) {
    p = i == 0 ? N - 1 : round + i;
    if (i != 0 && p >= N - 1) p -= N - 1;
    q = round + N - 1 - i;
    if (q >= N - 1) q -= N - 1;
    if (p > q) { const int t = p; p = q; q = t; }
  };

  // the partner of index x in round `round` (the inverse of pair_of: N - 1 meets `round`,
  // the others meet when their sum is 2 round mod N - 1)
  auto partner_of = [&](int round, int x) -> int {
    if (x == N - 1) return round;
    if (x == round) return N - 1;
    int y = 2 * round - x;
    if (y < 0) y += N - 1;
    if (y >= N - 1) y -= N - 1;
    return y;
  };
  // rotation annihilating (p, q): t = sign(tau) / (|tau| + sqrt(1 + tau^2)),
  // c = 1 / sqrt(1 + t^2), s = t c (square roots as x rsqrt(x); t ~ 1/(2 tau) once tau^2
  // would overflow).  An off-diagonal entry below 1e-30 in magnitude counts as zero.
  auto set_rot = [&](int cb, int p, int q, T app, T aqq, T apq) {
    T c = T(1), sn = T(0);
    if (q < b && fabs(apq) >= T(5e-31)) {
      const T dq = aqq - app;
      const T a2 = T(2) * apq;
      const T tau = dq == T(0) ? T(0) : dq * qrcp(a2);
      const T at = fabs(tau), tt = T(1) + tau * tau;
      T ta;
      if (at > T(1e15)) ta = at < T(1e30) ? T(0.5) * qrcp(at) : T(0);
      else ta = qrcp(at + tt * wrsqrt(tt));
      const T t = tau >= T(0) ? ta : -ta;
      c = wrsqrt(T(1) + t * t);
      sn = t * c;
    }
    rot[cb][p] = Rot{c, -sn, q, 0};
    rot[cb][q] = Rot{c, sn, p, 0};
  };
  // pair i's angle is taken by lane 0 of warp DS_THREADS / 32 - 1 - i (one per warp,
  // spreading the shared-memory traffic of the angle computations over the schedulers;
  // counted from the last warp, which holds no elements while b^2 <= DS_THREADS - 32 i, so
  // that a round's angles for the next round are computed alongside its element updates,
  // from the same inputs, instead of after them)
  const int ai = DS_THREADS / 32 - 1 - (tid >> 5);
  const bool angler = (tid & 31) == 0 && ai < half;
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    T off = T(0), tot = T(0);
    each([&](int, int r, int c) {
      const T v = Hc[r][c];
      tot += v * v;
      if (r != c) off += v * v;
    });
    off = warp_sum(off);
    tot = warp_sum(tot);
    if ((tid & 31) == 0) {
      red[0][tid >> 5] = off;
      red[1][tid >> 5] = tot;
    }
    __syncthreads();
    off = T(0);
    tot = T(0);
#pragma unroll
    for (int w = 0; w < DS_THREADS / 32; ++w) {
      off += red[0][w];
      tot += red[1][w];
    }
    if (off <= eps * eps * tot) break;
    if (angler) {
      int p, q;
      pair_of(0, ai, p, q);
      set_rot(0, p, q, Hc[p][p], Hc[q][q], Hc[p][q]);
    }
    __syncthreads();
    int cb = 0;
    for (int round = 0; round < N - 1; ++round) {
      each([&](int, int r, int c) {
        const Rot R = rot[cb][r], C = rot[cb][c];
        Hn[r][c] = R.c * (C.c * Hc[r][c] + C.s * Hc[r][C.partner]) +
                   R.s * (C.c * Hc[R.partner][c] + C.s * Hc[R.partner][C.partner]);
        Yn[r][c] = C.c * Yc[r][c] + C.s * Yc[r][C.partner];
      });
      if (round + 1 < N - 1 && angler) {
        // the next round's pair (p, q) from the entries (p,p), (q,q), (p,q) of this round's
        // J^T H J; this round's partners P, Q of p, q follow from the order, so the loads
        // of H do not wait for those of the rotations
        int p, q;
        pair_of(round + 1, ai, p, q);
        if (q < b) {
          const int P = partner_of(round, p), Q = partner_of(round, q);
          const Rot Rp = rot[cb][p], Rq = rot[cb][q];
          const T hpp = Hc[p][p], hpP = Hc[p][P], hPp = Hc[P][p], hPP = Hc[P][P];
          const T hqq = Hc[q][q], hqQ = Hc[q][Q], hQq = Hc[Q][q], hQQ = Hc[Q][Q];
          const T hpq = Hc[p][q], hpQ = Hc[p][Q], hPq = Hc[P][q], hPQ = Hc[P][Q];
          const T app = Rp.c * (Rp.c * hpp + Rp.s * hpP) + Rp.s * (Rp.c * hPp + Rp.s * hPP);
          const T aqq = Rq.c * (Rq.c * hqq + Rq.s * hqQ) + Rq.s * (Rq.c * hQq + Rq.s * hQQ);
          const T apq = Rp.c * (Rq.c * hpq + Rq.s * hpQ) + Rp.s * (Rq.c * hPq + Rq.s * hPQ);
          set_rot(cb ^ 1, p, q, app, aqq, apq);
        } else {
          set_rot(cb ^ 1, p, q, T(0), T(0), T(0));
        }
      }
      __syncthreads();
      Row* t0 = Hc; Hc = Hn; Hn = t0;
      Row* t1 = Yc; Yc = Yn; Yn = t1;
      cb ^= 1;
    }
  }
  Row* H = Hc;
  Row* Y = Yc;
  Row* S = Hn;   // scratch: P Y, then L^{-1}
  // ---- sort descending: c's rank = #{d : theta_d > theta_c, or equal with d < c}
  if (tid < b) {
    const T tc = H[tid][tid];
    int rank = 0;
    for (int d = 0; d < b; ++d) {
      const T td = H[d][d];
      rank += (td > tc) || (td == tc && d < tid);
    }
    perm[rank] = tid;
    if (!wfinite(tc)) atomicOr(err, ERRBIT_EIG);
  }
  __syncthreads();
  if (tid < b) th[tid] = H[perm[tid]][perm[tid]];
  each([&](int, int r, int c) { Wm[r][c] = Y[r][perm[c]]; });
  __syncthreads();
  // S = P W, then Pm <- W^T P W
  each([&](int, int r, int c) {
    T v = T(0);
    for (int l = 0; l < b; ++l) v = fma(Pm[r][l], Wm[l][c], v);
    S[r][c] = v;
  });
  __syncthreads();
  each([&](int, int r, int c) {
    T v = T(0);
    for (int l = 0; l < b; ++l) v = fma(Wm[l][r], S[l][c], v);
    Pm[r][c] = v;
  });
  __syncthreads();
  if (tid < b) {
    const int c = tid;
    const T tmax = fabs(th[0]);
    const T small = sizeof(T) == 4 ? T(1e-6) : T(1e-13);
    const T nz2 = Pm[c][c];
    const bool use_v = !(th[c] > small * tmax) || !(nz2 > T(0));
    usev[c] = use_v ? 1 : 0;
    fz[c] = use_v ? T(0) : wrsqrt(nz2);
    resid[c] = nz2 - th[c] * th[c];
    theta[c] = th[c];
  }
  __syncthreads();
  // Gram of W: <Vy_a, Vy_b> = delta_ab, <Zy_a, Zy_b> = fz_a fz_b (Y^T P Y)_ab, mixed 0;
  // S <- I
  each([&](int, int r, int c) {
    T g;
    if (usev[r] && usev[c]) g = r == c ? T(1) : T(0);
    else if (!usev[r] && !usev[c]) g = fz[r] * fz[c] * Pm[r][c];
    else g = T(0);
    Gm[r][c] = g;
    S[r][c] = r == c ? T(1) : T(0);
  });
  __syncthreads();
  // W^T W = L D L^T by symmetric elimination, with L^{-1} formed alongside (Gauss-Jordan
  // on [W^T W | I]): step t takes, for rows i > t with m = G(i,t) / G(t,t),
  // G(i,j) -= m G(j,t) on the trailing lower triangle (j > t) and X(i,j) -= m X(t,j) for
  // j <= t.  The Cholesky factor is L D^{1/2}, so its inverse is D^{-1/2} L^{-1}.
  for (int t = 0; t < b; ++t) {
    T d = Gm[t][t];
    if (!(d > T(0)) || !wfinite(d)) {
      if (tid == 0) bad_s = 1;
      d = T(1);
    }
    const T rd = qrcp(d);
    each([&](int, int i, int j) {
      if (i > t) {
        const T m = Gm[i][t] * rd;
        if (j > t) {
          if (j <= i) Gm[i][j] = fma(-m, Gm[j][t], Gm[i][j]);
        } else {
          S[i][j] = fma(-m, S[t][j], S[i][j]);
        }
      }
    });
    __syncthreads();
  }
  if (tid < b) {
    T d = Gm[tid][tid];
    if (!(d > T(0)) || !wfinite(d)) d = T(1);
    rdg[tid] = wrsqrt(d);
  }
  __syncthreads();
  if (tid == 0 && bad_s) atomicOr(err, ERRBIT_EIG);
  // Mv(r, c) = sum_l W(r, l) [use_v(l)] X(c, l), Mz(r, c) = sum_l W(r, l) fz(l) X(c, l),
  // X = D^{-1/2} L^{-1}
  each([&](int e, int r, int c) {
    T mv = T(0), mz = T(0);
    for (int l = 0; l <= c; ++l) {
      const T x = S[c][l] * rdg[c];
      const T y = Wm[r][l] * x;
      if (usev[l]) mv += y;
      else mz += y * fz[l];
    }
    Yo[e] = Wm[r][c];
    Mvo[e] = mv;
    Mzo[e] = mz;
  });
  __syncthreads();
}

// Second CholeskyQR factor on one CTA (k <= 32), the difference form of chol2_warp with
// the steps spread over the CTA: Q1^T Q1 = I + F = (I + Lambda)(I + Lambda)^T by
// right-looking elimination (step t: Lambda_tt = F_tt / (1 + sqrt(1 + F_tt)), and the
// trailing lower triangle takes F_ij -= F_it F_jt / (1 + Lambda_tt)^2, so that
// Lambda_it = F_it / (1 + Lambda_tt) uses column t as it stands after step t - 1); the
// forward elimination for (I + Lambda) N = -Lambda runs alongside (its step t needs only
// column t of Lambda), and R^{-1} = R1inv (I + N)^T.  F arrives as F(i, j) = get(i + j k)
// (lower part used).
// Work arrays in wk: F, R1inv, N (row-major, pitch k), R^{-1} (row-major).
template <typename T, int NE, typename Get>
__device__ void chol2_block(T* wk, int k, Get get, const T* __restrict__ R1inv,
                            T* __restrict__ Nout, T* __restrict__ Rinv, int* __restrict__ err) {
  T* F = wk;
  T* Rm = wk + DS_BM * DS_BM;
  T* Nm = wk + 2 * DS_BM * DS_BM;
  T* Ri = wk + 3 * DS_BM * DS_BM;
  __shared__ T lam_s[DS_BM], rdg_s[DS_BM];
  __shared__ int flag_s;
  const int tid = threadIdx.x;
  const int kk = k * k;
  // this thread's elements (i, j) = (e / k, e % k), e = tid + q DS_THREADS, q < NE, of a
  // k x k array (NE DS_THREADS >= k^2)
  int ei[NE], ej[NE];
#pragma unroll
  for (int q = 0; q < NE; ++q) {
    const int e = tid + q * DS_THREADS;
    ei[q] = e / k;
    ej[q] = e % k;
  }
  auto each = [&](auto&& f) {
#pragma unroll
    for (int q = 0; q < NE; ++q)
      if (tid + q * DS_THREADS < kk) f(ei[q], ej[q]);
  };
  each([&](int i, int j) {
    F[i * k + j] = get(i + j * k);
    Rm[i * k + j] = R1inv[i + j * k];
  });
  if (tid == 0) flag_s = 0;
  __syncthreads();
  // rhs of (I + Lambda) N = -Lambda, filled column by column as Lambda's columns appear
  each([&](int i, int c) { Nm[i * k + c] = T(0); });
  __syncthreads();
  for (int t = 0; t < k; ++t) {
    const T ftt = F[t * k + t];
    T lam = T(0);
    const bool bad = !(T(1) + ftt > T(0)) || !wfinite(ftt);
    if (!bad) lam = ftt * qrcp(T(1) + qsqrt(T(1) + ftt));
    const T rden = qrcp(T(1) + lam);
    if (tid == 0) {
      lam_s[t] = lam;
      rdg_s[t] = rden;
      if (bad) flag_s = 1;
    }
    const T r2 = rden * rden;
    // one phase: the trailing update of the factorization, and step t of the forward
    // elimination for N (row t of the rhs is final up to 1 / (1 + Lambda_tt); its entry t
    // is -Lambda_tt, the rows below take their entry t = -Lambda_it first)
    each([&](int i, int j) {
      if (i >= j && j > t) F[i * k + j] = fma(-F[i * k + t] * r2, F[j * k + t], F[i * k + j]);
      if (i > t && j <= t) {
        const T lit = F[i * k + t] * rden;                 // Lambda_it
        const T rtj = j == t ? -lam : Nm[t * k + j];       // raw row t of the rhs
        const T base = j == t ? -lit : Nm[i * k + j];
        Nm[i * k + j] = fma(-lit * rden, rtj, base);
      }
      if (i == t && j == t) Nm[t * k + t] = -lam;
    });
    __syncthreads();
  }
  each([&](int i, int c) {
    const T v = Nm[i * k + c] * rdg_s[i];
    Nm[i * k + c] = v;
    Nout[i + c * k] = v;
  });
  __syncthreads();
  // full sums: R1inv is upper triangular after a Cholesky first factor but a full matrix
  // after chol2_series (the terms outside the triangles are exact zeros otherwise)
  each([&](int a, int b) {
    T v = Rm[a * k + b];
    for (int l = 0; l < k; ++l) v = fma(Rm[a * k + l], Nm[b * k + l], v);
    Ri[a * k + b] = v;
    Rinv[a + b * k] = v;
  });
  __syncthreads();
  if (tid == 0 && flag_s) atomicOr(err, ERRBIT_RANK_DEFICIENT);
}

// Second factor as an inverse square root (float path, small F).  With Q1^T Q1 = I + F,
// any R2 with R2^T R2 = I + F completes X1 = Q1 R1 to X1 = (Q1 R2^{-1}) (R2 R1) with an
// orthonormal first factor; the symmetric R2 = (I + F)^{1/2} serves as well as the
// triangular Cholesky factor, because what the step uses (C = (X1^T X1)^{-1} X1^T A2,
// B^T B and ||B||^2) does not depend on which orthonormal basis of range(X1) is taken.
// Its inverse is the binomial series (I + F)^{-1/2} = I + sum_{j>=1} c_j F^j,
// c_j = c_{j-1} (1 - 2j) / (2j), summed by Horner's rule with the fewest terms whose
// remainder (about 0.3 ||F||_F^{m+1}) is below float precision: m products of k x k
// matrices instead of k serial elimination steps.  Writes N = (I + F)^{-1/2} - I (full,
// symmetric up to rounding) and R^{-1} = R1inv (I + N)^T in the places chol2_block uses.
// Returns false, having written nothing outside wk, when ||F||_F > 0.06 (or is not finite).
template <typename Get>
__device__ bool chol2_series(float* wk, int k, Get get, const float* __restrict__ R1inv,
                             float* __restrict__ Nout, float* __restrict__ Rinv) {
  float* F = wk;                          // row-major k x k
  float* Rm = wk + DS_BM * DS_BM;         // R1inv, row-major
  float* Nm = wk + 2 * DS_BM * DS_BM;     // N, row-major
  float* Ri = wk + 3 * DS_BM * DS_BM;     // R^{-1}, row-major
  float* P = wk + 4 * DS_BM * DS_BM;      // Horner partial sums (two buffers)
  float* Pn = wk + 5 * DS_BM * DS_BM;
  constexpr int MMAX = 8;
  __shared__ float red_s[DS_THREADS / 32];
  __shared__ float cj[MMAX + 1];
  __shared__ int m_s;
  const int tid = threadIdx.x, kk = k * k;
  float f2 = 0.f;
  for (int e = tid; e < kk; e += DS_THREADS) {
    const int i = e / k, j = e % k;
    const float v = i >= j ? get(i + j * k) : get(j + i * k);   // the lower triangle of F
    F[e] = v;
    Rm[e] = R1inv[i + j * k];
    f2 = fmaf(v, v, f2);
  }
  f2 = warp_sum(f2);
  if ((tid & 31) == 0) red_s[tid >> 5] = f2;
  __syncthreads();
  if (tid == 0) {
    float t = 0.f;
    for (int w = 0; w < DS_THREADS / 32; ++w) t += red_s[w];
    const float nf = sqrtf(t);
    int m = 0;
    if (nf <= 0.06f) {
      float pw = nf;   // nf^m
      m = 1;
      while (m < MMAX && 0.3f * pw * nf > 3e-8f) {
        pw *= nf;
        ++m;
      }
    }
    m_s = m;
    cj[0] = 1.f;
    for (int j = 1; j <= MMAX; ++j) cj[j] = cj[j - 1] * (float)(1 - 2 * j) / (float)(2 * j);
  }
  __syncthreads();
  const int m = m_s;
  if (m == 0) return false;
  // P = c_m I, then P <- c_j I + F P for j = m - 1 .. 1, and N = F P
  for (int e = tid; e < kk; e += DS_THREADS) P[e] = (e / k == e % k) ? cj[m] : 0.f;
  __syncthreads();
  for (int j = m - 1; j >= 0; --j) {
    float* out = j == 0 ? Nm : Pn;
    for (int e = tid; e < kk; e += DS_THREADS) {
      const int r = e / k, c = e % k;
      float v = (j > 0 && r == c) ? cj[j] : 0.f;
      for (int l = 0; l < k; ++l) v = fmaf(F[r * k + l], P[l * k + c], v);
      out[e] = v;
      if (j == 0) Nout[r + c * k] = v;
    }
    __syncthreads();
    float* t = P;
    P = Pn;
    Pn = t;
  }
  // R^{-1} = R1inv (I + N)^T
  for (int e = tid; e < kk; e += DS_THREADS) {
    const int r = e / k, c = e % k;
    float v = Rm[e];
    for (int l = 0; l < k; ++l) v = fmaf(Rm[r * k + l], Nm[c * k + l], v);
    Ri[e] = v;
    Rinv[r + c * k] = v;
  }
  __syncthreads();
  return true;
}

// Sum over the cluster's CTAs, in rank order, of element e of a shared array (the remote
// loads are issued together; float sums are compensated).
template <typename T>
__device__ __forceinline__ T cluster_sum(cgrp::cluster_group& cl, T* base, int e, int nc) {
  T v[16];
#pragma unroll
  for (int u = 0; u < 16; ++u) v[u] = u < nc ? cl.map_shared_rank(base, u)[e] : T(0);
  WideAcc<T> acc;
#pragma unroll
  for (int u = 0; u < 16; ++u)
    if (u < nc) acc.add(v[u]);
  return (T)acc.value();
}

// (K V)(l, c) for all rows in double-float: one warp per (row l, group of KV_CG columns),
// the lanes splitting the sum over j (K is symmetric, so row l of K is the contiguous
// column l).  Each lane loads the K and V entries of KV_JM values of j before using them
// (one memory round trip per chunk), then the partial sums meet by warp shuffles.
constexpr int KV_CG = 4;
constexpr int KV_JM = 8;
template <typename T>
__global__ void __launch_bounds__(256)
kv_pair(const T* __restrict__ Kh, const T* __restrict__ Kl, const T* __restrict__ V, int n2, int b,
        T* __restrict__ ZKh, T* __restrict__ ZKl) {
  const int lane = threadIdx.x & 31;
  const int ncg = (b + KV_CG - 1) / KV_CG;
  const int w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int l = w / ncg, c0 = (w % ncg) * KV_CG;
  if (l >= n2) return;   // whole warp
  DfAcc<T> acc[KV_CG];
  for (int j0 = 0; j0 < n2; j0 += 32 * KV_JM) {
    T kh[KV_JM], kl[KV_JM], vv[KV_JM][KV_CG];
#pragma unroll
    for (int q = 0; q < KV_JM; ++q) {
      const int j = j0 + lane + 32 * q;
      const bool ok = j < n2;
      const int64_t o = j + (int64_t)l * n2;
      kh[q] = ok ? Kh[o] : T(0);
      kl[q] = (ok && Kl) ? Kl[o] : T(0);
#pragma unroll
      for (int u = 0; u < KV_CG; ++u)
        vv[q][u] = (ok && c0 + u < b) ? V[j + (int64_t)(c0 + u) * n2] : T(0);
    }
#pragma unroll
    for (int q = 0; q < KV_JM; ++q)
#pragma unroll
      for (int u = 0; u < KV_CG; ++u) acc[u].add(kh[q], kl[q], vv[q][u]);
  }
#pragma unroll
  for (int u = 0; u < KV_CG; ++u) {
    acc[u].warp_reduce();
    if (lane == 0 && c0 + u < b) {
      ZKh[l + (int64_t)(c0 + u) * n2] = acc[u].hi;
      if (ZKl) ZKl[l + (int64_t)(c0 + u) * n2] = acc[u].lo;
    }
  }
}

// The cluster kernel (grid = one cluster of NC CTAs, DS_THREADS threads each).
// NE: elements of a b x b (and k x k) array per thread, 1 when both fit in one pass (a
// second pass doubles the straight-line code of the serial phases on CTA 0).
template <typename T, int NE>
__global__ void __launch_bounds__(DS_THREADS, 1)
dstep_cluster(DstepArgs<T> a) {
  extern __shared__ unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  cgrp::cluster_group cluster = cgrp::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int nc = (int)cluster.num_blocks();
  const int tid = threadIdx.x;
  const int n2 = a.n2, k = a.k, b = a.b, s = a.s, NP = a.NP;
  const int R = (n2 + nc - 1) / nc;
  const int l0 = min(n2, rank * R), l1 = min(n2, l0 + R), nr = l1 - l0;
  const DsLayout L = DsLayout::make<T>(n2, k, b, s, R);
  T* Vt = sm + L.Vt;
  T* Bs = sm + L.Bs;
  T* Cs = sm + L.Cs;
  T* Zh = sm + L.Zh;
  T* Zl = sm + L.Zl;
  T* Zr = sm + L.Zr;
  T* Vsr = sm + L.Vsr;
  T* BVp = sm + L.BVp;
  T* BV = sm + L.BV;
  T* HPp = sm + L.HPp;
  T* Gp = sm + L.Gp;
  T* CVp = sm + L.CVp;
  T* Ml = sm + L.Ml;
  T* Wk = sm + L.Wk;
  const int kb = k * b;

  // ---- inputs into shared memory (asynchronous copies, one group): the whole basis,
  // and for the CTA's rows: K V, B's columns and C (from Z2)
  for (int e = tid; e < b * n2; e += DS_THREADS) cp_async_elem(Vt + e, a.V + e, true);
  for (int e = tid; e < k * nr; e += DS_THREADS) {
    cp_async_elem(Bs + e, a.Bh + (int64_t)l0 * k + e, true);
    if (a.Bl) cp_async_elem(Bs + k * R + e, a.Bl + (int64_t)l0 * k + e, true);
    const int rr = e / k, x = e % k;
    cp_async_elem(Cs + e, a.Z2 + (int64_t)(l0 + rr) * NP + x, true);
  }
  for (int e = tid; e < b * nr; e += DS_THREADS) {
    const int c = e / nr, rr = e % nr;
    cp_async_elem(Zh + c * R + rr, a.ZKh + l0 + rr + (int64_t)c * n2, true);
    if (a.ZKl) cp_async_elem(Zl + c * R + rr, a.ZKl + l0 + rr + (int64_t)c * n2, true);
  }
  cp_async_commit();

  cp_async_wait<0>();
  __syncthreads();

  // ---- partial C C^T and B V over the CTA's rows
  for (int e = tid; e < k * k; e += DS_THREADS) {
    const int x = e % k, y = e / k;
    T v = T(0);
    for (int rr = 0; rr < nr; ++rr) v = fma(Cs[rr * k + x], Cs[rr * k + y], v);
    Gp[e] = v;
  }
  for (int e = tid; e < kb; e += DS_THREADS) {
    const int x = e % k, c = e / k;
    DfAcc<T> acc;
    for (int rr = 0; rr < nr; ++rr)
      acc.add(Bs[rr * k + x], a.Bl ? Bs[k * R + rr * k + x] : T(0), Vt[c * n2 + l0 + rr]);
    BVp[e] = acc.hi;
    BVp[kb + e] = acc.lo;
  }
  cluster.sync();
  // ---- B V: the CTAs' partials in rank order
  for (int e = tid; e < kb; e += DS_THREADS) {
    T ph[16], pl[16];
    DfAcc<T> acc;
    for (int r0 = 0; r0 < nc; r0 += 16) {
#pragma unroll
      for (int u = 0; u < 16; ++u) {
        if (r0 + u < nc) {
          const T* rp = cluster.map_shared_rank(BVp, r0 + u);
          ph[u] = rp[e];
          pl[u] = rp[kb + e];
        }
      }
#pragma unroll
      for (int u = 0; u < 16; ++u)
        if (r0 + u < nc) acc.add_pair(ph[u], pl[u]);
    }
    BV[e] = acc.hi;
    BV[kb + e] = acc.lo;
  }
  __syncthreads();
  // ---- Z(rows) = K V - B^T (B V), rounded to T after the subtraction
  for (int e = tid; e < nr * b; e += DS_THREADS) {
    const int rr = e % nr, c = e / nr;
    DfAcc<T> acc;
    acc.hi = Zh[c * R + rr];
    acc.lo = a.ZKl ? Zl[c * R + rr] : T(0);
    for (int x = 0; x < k; ++x)
      acc.sub2(Bs[rr * k + x], a.Bl ? Bs[k * R + rr * k + x] : T(0), BV[x + c * k], BV[kb + x + c * k]);
    Zr[rr * b + c] = acc.hi + acc.lo;
  }
  __syncthreads();
  // ---- partial H = V^T Z and P = Z^T Z over the CTA's rows
  for (int e = tid; e < b * b; e += DS_THREADS) {
    const int c1 = e % b, c2 = e / b;
    T h = T(0), p = T(0);
    for (int rr = 0; rr < nr; ++rr) {
      const T z2 = Zr[rr * b + c2];
      h = fma(Vt[c1 * n2 + l0 + rr], z2, h);
      p = fma(Zr[rr * b + c1], z2, p);
    }
    HPp[e] = h;
    HPp[b * b + e] = p;
  }
  cluster.sync();
  // ---- Rayleigh-Ritz on CTA 0
  if (rank == 0) {
    for (int e = tid; e < 2 * b * b; e += DS_THREADS) {
      const T v = cluster_sum(cluster, HPp, e, nc);
      const int f = e % (b * b), r_ = f % b, c_ = f / b;
      // H into work array 0, P into work array 4
      Wk[(e < b * b ? 0 : 4 * DS_BM * DS_P) + r_ * DS_P + c_] = v;
    }
    __syncthreads();
    ritz_step<T, NE>(Wk, b, a.sweeps, a.theta, a.resid, a.err);
  }
  cluster.sync();
  // ---- next basis rows and Ritz vectors (Y, Mv, Mz from CTA 0)
  {
    const T* w0 = cluster.map_shared_rank(Wk, 0);
    T* Yl = Ml;
    T* Mvl = Ml + b * b;
    T* Mzl = Ml + 2 * b * b;
    for (int e = tid; e < b * b; e += DS_THREADS) {
      Yl[e] = w0[7 * DS_BM * DS_P + e];
      Mvl[e] = w0[8 * DS_BM * DS_P + e];
      Mzl[e] = w0[9 * DS_BM * DS_P + e];
    }
    __syncthreads();
    for (int e = tid; e < nr * b; e += DS_THREADS) {
      const int rr = e % nr, c = e / nr;
      const int l = l0 + rr;
      T vr = T(0), vn = T(0);
      for (int x = 0; x < b; ++x) {
        const T v = Vt[x * n2 + l], z = Zr[rr * b + x];
        vr = fma(v, Yl[x + c * b], vr);
        vn = fma(v, Mvl[x + c * b], vn);
        vn = fma(z, Mzl[x + c * b], vn);
      }
      a.V[l + (int64_t)c * n2] = vn;
      if (c < s) {
        a.Vs[l + (int64_t)c * n2] = vr;
        a.Z2[(int64_t)l * NP + k + c] = vr;
        Vsr[rr * s + c] = vr;
      }
    }
  }
  __syncthreads();
  // ---- partial C V_s over the CTA's rows, then CTA 0 sums C C^T and C V_s
  for (int e = tid; e < k * s; e += DS_THREADS) {
    const int x = e % k, c = e / k;
    T v = T(0);
    for (int rr = 0; rr < nr; ++rr) v = fma(Cs[rr * k + x], Vsr[rr * s + c], v);
    CVp[e] = v;
  }
  cluster.sync();
  // outputs e = rank, rank + nc, ... of G (then of C V_s) summed by this CTA
  for (int e = rank + nc * tid; e < k * k + k * s; e += nc * DS_THREADS) {
    if (e < k * k) a.G[e] = cluster_sum(cluster, Gp, e, nc);
    else a.CV[e - k * k] = cluster_sum(cluster, CVp, e - k * k, nc);
  }
  // every CTA keeps its shared memory until the others have read it
  cluster.sync();
}

// ------------------------------------------------------------------------------------
// The steady-state step with the front stage (k <= 32), arranged so that the second
// CholeskyQR factor does not hold up the products over the basis rows.  With
// t = Q1^T A2 (the Gram's sums), B = (I + N) t and C = R^{-1} B:
//   B V = (I + N) (t V)   and   B^T (B V) = t^T X,  X = (I + N)^T (B V),
// so the partials of t V need only t.  CTA 0 owns no basis rows: it forms the second
// factor of Q1^T Q1 = I + F (chol2_series while ||F|| is small, else the elimination
// chol2_block) while CTAs 1 .. nc-1 form t V over their rows; after one cluster barrier
// they form (I + N) t V and X from the summed t V and their rows of Z = K V - t^T X, H
// and P.  CTA 0 then runs the Rayleigh-Ritz step while the others form their columns of
// B, C (and ||B||^2, C C^T) in its shadow.  N and R^{-1} are full matrices after the
// series, triangular after the elimination; the loops below run over full rows.
// Partial sums travel by remote stores from their producers into slot rank - 1 of the
// consumer's exchange region (PUSH, where one slot per worker fits), which the consumer
// adds in rank order after the next cluster barrier: the stores are posted, and each
// consumer then reads its own shared memory.  What CTA 0 hands to every worker (N,
// R^{-1}, then Y, Mv, Mz) the workers load from it: fifteen SMs loading in parallel
// beat one SM storing fifteen copies.  Without PUSH every partial is loaded remotely.
struct DfLayout {
  size_t Tq, Th, Tl, Vr, Zh, Zl, Zr, Bs, Cs, Vsr, TV, BVx, Xs, Ml, NR, Wk, Xch, total;
  // Exchange region Xch.  push: on a worker, the t V partials of every worker (slot
  // u = rank - 1, 2 k b values); on CTA 0, the workers' partials of H and P (2 b^2 each), of
  // C C^T (k^2) and of C V_s (k s), all written by their owners with remote stores.
  // Otherwise (pull, when those slots do not fit): each CTA's own partials at the same
  // offsets with one slot, read by their consumers with remote loads.
  size_t xtv, xhp, xg, xcv;   // offsets inside Xch
  template <typename T>
  __host__ __device__ static DfLayout make(int k, int b, int s, int RL, int nw, bool push) {
    return DfLayout(k, b, s, RL, nw, (int)(sizeof(double) / sizeof(T)), push);
  }
  __host__ __device__ DfLayout(int k, int b, int s, int RL, int nw, int dw, bool push) {
    const size_t ss = s > 0 ? s : 1;
    size_t o = 0;
    Tq = o;  o += (size_t)dw * k * RL;     // t(:, rows) in double, t(x, j) at Tq[(j - l0) k + x]
    Th = o;  o += (size_t)k * RL;          // t(:, rows) as a T pair: high
    Tl = o;  o += (size_t)k * RL;          // low
    Vr = o;  o += (size_t)b * RL;          // V(rows), V(j, c) at Vr[c RL + j - l0]
    Zh = o;  o += (size_t)b * RL;          // (K V)(rows), high
    Zl = o;  o += (size_t)b * RL;          // low
    Zr = o;  o += (size_t)RL * b;          // Z(rows), Zr[(j - l0) b + c]
    Bs = o;  o += 2 * (size_t)k * RL;      // B(:, rows): high, low
    Cs = o;  o += (size_t)RL * k;          // C(:, rows)
    Vsr = o; o += (size_t)RL * ss;         // V_s(rows)
    TV = o;  o += 2 * (size_t)k * b;       // t V
    BVx = o; o += 2 * (size_t)k * b;       // B V = (I + N) t V
    Xs = o;  o += 2 * (size_t)k * b;       // X = (I + N)^T B V
    Ml = o;  o += 3 * (size_t)b * b;       // local copies of Y, Mv, Mz (from CTA 0)
    NR = o;  o += 2 * (size_t)k * k;       // local copies of N and R^{-1} (from CTA 0)
    Wk = o;  o += 10 * (size_t)DS_BM * DS_P;   // second factor, then Rayleigh-Ritz (CTA 0)
    const size_t slots = push ? (size_t)nw : 1;
    xhp = 0;
    xg = xhp + slots * 2 * b * b;
    xcv = xg + slots * k * k;
    const size_t x0 = xcv + slots * k * ss;
    xtv = push ? 0 : x0;                   // push: the t V slots share the space with the above
    const size_t x1 = xtv + slots * 2 * k * b;
    Xch = o; o += x0 > x1 ? x0 : x1;
    total = o;
  }
};
__host__ __device__ inline int df_rows(int n2, int nc) { return (n2 + nc - 2) / (nc - 1); }

// Sum over ranks 1 .. nc - 1, in rank order, of element e of a shared array (the remote
// loads issued together; float sums compensated): the exchange of dstep_front without
// room for one slot per worker.
template <typename T>
__device__ __forceinline__ T pull_sum(cgrp::cluster_group& cl, T* base, int e, int nc) {
  T v[15];
#pragma unroll
  for (int u = 0; u < 15; ++u) v[u] = u + 1 < nc ? cl.map_shared_rank(base, u + 1)[e] : T(0);
  WideAcc<T> acc;
#pragma unroll
  for (int u = 0; u < 15; ++u)
    if (u + 1 < nc) acc.add(v[u]);
  return (T)acc.value();
}

template <typename T, int NE, bool PUSH>
__global__ void __launch_bounds__(DS_THREADS, 1)
dstep_front(DstepArgs<T> a) {
  extern __shared__ unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  cgrp::cluster_group cluster = cgrp::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int nc = (int)cluster.num_blocks();
  const int nw = nc - 1;
  const int tid = threadIdx.x;
  const int n2 = a.n2, k = a.k, b = a.b, s = a.s, NP = a.NP;
  const int RL = df_rows(n2, nc);
  const int l0 = rank == 0 ? 0 : min(n2, (rank - 1) * RL);
  const int l1 = rank == 0 ? 0 : min(n2, l0 + RL);
  const int nr = l1 - l0;
  const DfLayout L = DfLayout::make<T>(k, b, s, RL, nw, PUSH);
  double* Tq = reinterpret_cast<double*>(sm + L.Tq);
  T* Th = sm + L.Th;
  T* Tl = sm + L.Tl;
  T* Vr = sm + L.Vr;
  T* Zh = sm + L.Zh;
  T* Zl = sm + L.Zl;
  T* Zr = sm + L.Zr;
  T* Bs = sm + L.Bs;
  T* Cs = sm + L.Cs;
  T* Vsr = sm + L.Vsr;
  T* TV = sm + L.TV;
  T* BVx = sm + L.BVx;
  T* Xs = sm + L.Xs;
  T* Ml = sm + L.Ml;
  T* Nl = sm + L.NR;
  T* Rl = Nl + k * k;
  T* Wk = sm + L.Wk;
  T* Xch = sm + L.Xch;
  const int kb = k * b, bb = b * b, ss = s > 0 ? s : 1;
  constexpr bool kF = sizeof(T) == 4;
  __shared__ double bsh[32];

  // ---- inputs of the CTA's rows (one asynchronous group): t in double, V, K V
  for (int e = tid; e < k * nr; e += DS_THREADS) cp_async_elem(Tq + e, a.S2T + (int64_t)(k + l0) * k + e, true);
  for (int e = tid; e < b * nr; e += DS_THREADS) {
    const int c = e / nr, rr = e % nr;
    const int64_t g = l0 + rr + (int64_t)c * n2;
    cp_async_elem(Vr + c * RL + rr, a.V + g, true);
    cp_async_elem(Zh + c * RL + rr, a.ZKh + g, true);
    if (a.ZKl) cp_async_elem(Zl + c * RL + rr, a.ZKl + g, true);
  }
  cp_async_commit();
  if (rank == 0) {
    // ---- (1) the second factor (into Wk and global memory) by the inverse square root
    // series when F is small enough, else by elimination
    auto getF = [&](int e) { return a.F2[e]; };
    bool done = false;
    if constexpr (kF) done = a.series && chol2_series(Wk, k, getF, a.R1inv, a.Nout, a.Rinv);
    if (!done) chol2_block<T, NE>(Wk, k, getF, a.R1inv, a.Nout, a.Rinv, a.err);
    if (tid == 0) a.bpart[0] = 0.0;
    cp_async_wait<0>();
  } else {
    cp_async_wait<0>();
    __syncthreads();
    for (int v = tid; v < k * nr; v += DS_THREADS) {
      const double t = Tq[v];
      const T h = (T)t;
      Th[v] = h;
      Tl[v] = kF ? (T)(t - (double)h) : T(0);
    }
    __syncthreads();
    // ---- (2) partial t V over the CTA's rows (double-float): with PUSH into slot
    // rank - 1 of every worker's exchange region, else into the CTA's own
    for (int e = tid; e < kb; e += DS_THREADS) {
      const int x = e % k, c = e / k;
      DfAcc<T> acc;
      for (int rr = 0; rr < nr; ++rr) acc.add(Th[rr * k + x], Tl[rr * k + x], Vr[c * RL + rr]);
      if constexpr (PUSH) {
        const size_t o = L.xtv + (size_t)(rank - 1) * 2 * kb + e;
        for (int w = 1; w < nc; ++w) {
          T* dst = cluster.map_shared_rank(Xch, w);
          dst[o] = acc.hi;
          dst[o + kb] = acc.lo;
        }
      } else {
        Xch[L.xtv + e] = acc.hi;
        Xch[L.xtv + kb + e] = acc.lo;
      }
    }
  }
  cluster.sync();
  if (rank > 0) {
    // ---- (3) N and R^{-1} from CTA 0; t V summed in rank order; B V = t V + N t V and
    // X = B V + N^T B V (the N products in T, added to the double-float sums)
    {
      const T* w0 = cluster.map_shared_rank(Wk, 0);
      for (int e = tid; e < k * k; e += DS_THREADS) {
        Nl[e] = w0[2 * DS_BM * DS_BM + e];
        Rl[e] = w0[3 * DS_BM * DS_BM + e];
      }
    }
    for (int e = tid; e < kb; e += DS_THREADS) {
      DfAcc<T> acc;
      if constexpr (PUSH) {
        const T* tv = Xch + L.xtv;
        for (int u = 0; u < nw; ++u) acc.add_pair(tv[(size_t)u * 2 * kb + e], tv[(size_t)u * 2 * kb + kb + e]);
      } else {
        T ph[15], pl[15];
#pragma unroll
        for (int u = 0; u < 15; ++u) {
          if (u + 1 < nc) {
            const T* rp = cluster.map_shared_rank(Xch, u + 1) + L.xtv;
            ph[u] = rp[e];
            pl[u] = rp[kb + e];
          }
        }
#pragma unroll
        for (int u = 0; u < 15; ++u)
          if (u + 1 < nc) acc.add_pair(ph[u], pl[u]);
      }
      TV[e] = acc.hi;
      TV[kb + e] = acc.lo;
    }
    __syncthreads();
    for (int e = tid; e < kb; e += DS_THREADS) {
      const int x = e % k, c = e / k;
      T corr = T(0);
      for (int l = 0; l < k; ++l) corr = fma(Nl[x * k + l], TV[l + c * k], corr);
      DfAcc<T> acc;
      acc.hi = TV[e];
      acc.lo = TV[kb + e];
      acc.add_pair(corr, T(0));
      BVx[e] = acc.hi;
      BVx[kb + e] = acc.lo;
    }
    __syncthreads();
    for (int e = tid; e < kb; e += DS_THREADS) {
      const int x = e % k, c = e / k;
      T corr = T(0);
      for (int l = 0; l < k; ++l) corr = fma(Nl[l * k + x], BVx[l + c * k], corr);
      DfAcc<T> acc;
      acc.hi = BVx[e];
      acc.lo = BVx[kb + e];
      acc.add_pair(corr, T(0));
      Xs[e] = acc.hi;
      Xs[kb + e] = acc.lo;
    }
    __syncthreads();
    // ---- Z(rows) = K V - t^T X, rounded to T after the subtraction
    for (int e = tid; e < nr * b; e += DS_THREADS) {
      const int rr = e % nr, c = e / nr;
      DfAcc<T> acc;
      acc.hi = Zh[c * RL + rr];
      acc.lo = a.ZKl ? Zl[c * RL + rr] : T(0);
      for (int x = 0; x < k; ++x) acc.sub2(Th[rr * k + x], Tl[rr * k + x], Xs[x + c * k], Xs[kb + x + c * k]);
      Zr[rr * b + c] = acc.hi + acc.lo;
    }
    __syncthreads();
    // ---- partial H = V^T Z and P = Z^T Z over the CTA's rows
    {
      T* dst = (PUSH ? cluster.map_shared_rank(Xch, 0) + (size_t)(rank - 1) * 2 * bb : Xch) + L.xhp;
      for (int e = tid; e < bb; e += DS_THREADS) {
        const int c1 = e % b, c2 = e / b;
        T h = T(0), p = T(0);
        for (int rr = 0; rr < nr; ++rr) {
          const T z2 = Zr[rr * b + c2];
          h = fma(Vr[c1 * RL + rr], z2, h);
          p = fma(Zr[rr * b + c1], z2, p);
        }
        dst[e] = h;
        dst[bb + e] = p;
      }
    }
  }
  cluster.sync();
  if (rank == 0) {
    // ---- (4) Rayleigh-Ritz on CTA 0 (H into work array 0, P into work array 4, summed over
    // the workers in rank order)
    for (int e = tid; e < 2 * bb; e += DS_THREADS) {
      const int part = e / bb, f = e % bb;
      T v;
      if constexpr (PUSH) {
        const T* hp = Xch + L.xhp;
        WideAcc<T> acc;
        for (int u = 0; u < nw; ++u) acc.add(hp[(size_t)u * 2 * bb + e]);
        v = (T)acc.value();
      } else {
        v = pull_sum(cluster, Xch + L.xhp, e, nc);
      }
      const int r_ = f % b, c_ = f / b;
      Wk[(part == 0 ? 0 : 4 * DS_BM * DS_P) + r_ * DS_P + c_] = v;
    }
    __syncthreads();
    ritz_step<T, NE>(Wk, b, a.sweeps, a.theta, a.resid, a.err);
  } else {
    // ---- meanwhile B = t + N t and C = R^{-1} B for the CTA's columns, ||B||^2 and the
    // partial C C^T
    double bn = 0.0;
    for (int v = tid; v < k * nr; v += DS_THREADS) {
      const int x = v % k, jj = v / k;
      T corr = T(0);
      for (int l = 0; l < k; ++l) corr = fma(Nl[x * k + l], Th[jj * k + l], corr);
      const double bv = Tq[v] + (double)corr;
      const int64_t o = (int64_t)(l0 + jj) * k + x;
      if (a.B64) a.B64[o] = bv;
      if constexpr (kF) {
        const float hi = (float)bv, lo = (float)(bv - (double)hi);
        a.Bho[o] = hi;
        a.Blo[o] = lo;
        Bs[v] = hi;
        Bs[k * RL + v] = lo;
      } else {
        Bs[v] = (T)bv;
      }
      bn += bv * bv;
    }
    __syncthreads();
    for (int v = tid; v < k * nr; v += DS_THREADS) {
      const int x = v % k, jj = v / k;
      T cv = T(0);
      for (int l = 0; l < k; ++l) {
        const T bl = kF ? Bs[jj * k + l] + Bs[k * RL + jj * k + l] : Bs[jj * k + l];
        cv = fma(Rl[x * k + l], bl, cv);
      }
      Cs[v] = cv;
      const int64_t o = (int64_t)(l0 + jj) * k + x;
      a.Cout[o] = cv;
      a.Z2[(int64_t)(l0 + jj) * NP + x] = cv;
    }
    bn = block_sum_double(bn, bsh);
    if (tid == 0) a.bpart[rank] = bn;
    __syncthreads();
    {
      T* dst = (PUSH ? cluster.map_shared_rank(Xch, 0) + (size_t)(rank - 1) * k * k : Xch) + L.xg;
      for (int e = tid; e < k * k; e += DS_THREADS) {
        const int x = e % k, y = e / k;
        T v = T(0);
        for (int rr = 0; rr < nr; ++rr) v = fma(Cs[rr * k + x], Cs[rr * k + y], v);
        dst[e] = v;
      }
    }
  }
  cluster.sync();
  if (rank == 0) {
    // ---- (5) G = C C^T over the workers' partials
    for (int e = tid; e < k * k; e += DS_THREADS) {
      if constexpr (PUSH) {
        const T* gp = Xch + L.xg;
        WideAcc<T> acc;
        for (int u = 0; u < nw; ++u) acc.add(gp[(size_t)u * k * k + e]);
        a.G[e] = (T)acc.value();
      } else {
        a.G[e] = pull_sum(cluster, Xch + L.xg, e, nc);
      }
    }
  } else {
    // ---- next basis rows and Ritz vectors (Y, Mv, Mz from CTA 0), then the partial C V_s
    {
      const T* w0 = cluster.map_shared_rank(Wk, 0);
      for (int e = tid; e < 3 * bb; e += DS_THREADS) Ml[e] = w0[(7 + e / bb) * DS_BM * DS_P + e % bb];
      __syncthreads();
    }
    const T* Yl = Ml;
    const T* Mvl = Ml + bb;
    const T* Mzl = Ml + 2 * bb;
    for (int e = tid; e < nr * b; e += DS_THREADS) {
      const int rr = e % nr, c = e / nr;
      const int l = l0 + rr;
      T vr = T(0), vn = T(0);
      for (int x = 0; x < b; ++x) {
        const T v = Vr[x * RL + rr], z = Zr[rr * b + x];
        vr = fma(v, Yl[x + c * b], vr);
        vn = fma(v, Mvl[x + c * b], vn);
        vn = fma(z, Mzl[x + c * b], vn);
      }
      a.V[l + (int64_t)c * n2] = vn;
      if (c < s) {
        a.Vs[l + (int64_t)c * n2] = vr;
        a.Z2[(int64_t)l * NP + k + c] = vr;
        Vsr[rr * s + c] = vr;
      }
    }
    __syncthreads();
    T* dst = (PUSH ? cluster.map_shared_rank(Xch, 0) + (size_t)(rank - 1) * k * ss : Xch) + L.xcv;
    for (int e = tid; e < k * s; e += DS_THREADS) {
      const int x = e % k, c = e / k;
      T v = T(0);
      for (int rr = 0; rr < nr; ++rr) v = fma(Cs[rr * k + x], Vsr[rr * s + c], v);
      dst[e] = v;
    }
  }
  cluster.sync();
  if constexpr (PUSH) {
    // after the last exchange no CTA reads another's shared memory
    if (rank == 0) {
      const T* cvp = Xch + L.xcv;
      for (int e = tid; e < k * s; e += DS_THREADS) {
        WideAcc<T> acc;
        for (int u = 0; u < nw; ++u) acc.add(cvp[(size_t)u * k * ss + e]);
        a.CV[e] = (T)acc.value();
      }
    }
  } else {
    // C V_s over the workers' partials, spread over every CTA; each CTA keeps its shared
    // memory until the others have read it
    for (int e = rank + nc * tid; e < k * s; e += nc * DS_THREADS) a.CV[e] = pull_sum(cluster, Xch + L.xcv, e, nc);
    cluster.sync();
  }
}

// K = Kh + Kl as a float pair (once per problem).
static __global__ void split_pair(const double* __restrict__ K, int64_t n, float* __restrict__ Kh,
                           float* __restrict__ Kl) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const double v = K[e];
    const float h = (float)v;
    Kh[e] = h;
    Kl[e] = (float)(v - (double)h);
  }
}

}  // namespace wlr
