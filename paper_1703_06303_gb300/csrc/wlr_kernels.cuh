// Device kernels of the sWLR iteration (Dutta & Li, arXiv 1703.06303, Algorithm 1).
//
// Every kernel is templated on the storage/arithmetic type T (float or double).
// Matrices are column-major with leading dimensions; A2 = A + k*lda.
//
// Step map (Section 3 / Algorithm 1):
//   a1  X1 = Q R by CholeskyQR2:  S1 = X1^T X1 -> R1;  Q1 = X1 R1^{-1};
//       S2 = Q1^T Q1 -> R2;  R = R2 R1                    gram_tn, chol1_kernel, form_q,
//                                                         chol2_kernel
//   a2  B = Q^T A2 = R2^{-T} Q1^T A2,  C = R^{-1} B        gram_tn, coef_kernel2
//   a3  D = H_{r-k}((I - Q Q^T) A2) through the Gram (P_perp A2)^T (P_perp A2) = K - B^T B,
//       K = A2^T A2 formed once; top-(r-k) eigenpairs by subspace iteration with
//       Rayleigh-Ritz (parallel Jacobi on the b x b projection)
//                                                         form_g2_df, eig_mult, eig_small,
//                                                         eig_update
//   a4  E = A1 o W1 o W1 + A2 C^T - U_s (V_s^T C^T), U_s = A2 V_s - X1 (C V_s)  = (A2 - D) C^T
//   a5  X1(i,:) = E(i,:) (diag(W1(i,:)^2) + C C^T)^{-1}   prep_gram, row_pass
//   a6  F_p = ||(A1-X1) o W1||^2 + ||A2||^2 - ||B||^2 - sum_{j<=r-k} sigma_j^2
//                                                         row_pass (last block), x2_pass (exact)
#pragma once

#include <type_traits>

#include "wlr_common.cuh"

namespace wlr {

constexpr int EIG_BMAX = 32;   // largest subspace block (Jacobi size)

// --------------------------------------------------------------------------------
// Asynchronous global -> shared copies of one element (zero-filled when !ok).
template <typename T>
__device__ __forceinline__ void cp_async_elem(T* dst_smem, const T* src, bool ok) {
  const unsigned dst = (unsigned)__cvta_generic_to_shared(dst_smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;\n" ::"r"(dst), "l"(src),
               "n"(sizeof(T)), "r"(ok ? (int)sizeof(T) : 0));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

// Four consecutive shared-memory elements (one 16-byte load for float).
__device__ __forceinline__ void load4(float (&a)[4], const float* p) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  a[0] = v.x; a[1] = v.y; a[2] = v.z; a[3] = v.w;
}
__device__ __forceinline__ void load4(double (&a)[4], const double* p) {
  a[0] = p[0]; a[1] = p[1]; a[2] = p[2]; a[3] = p[3];
}

// 1/sqrt(x): hardware estimate plus one Newton step (float); IEEE for double.
__device__ __forceinline__ float wrsqrt(float x) {
  float r = rsqrtf(x);
  return r * (1.5f - 0.5f * x * r * r);
}
__device__ __forceinline__ double wrsqrt(double x) { return 1.0 / sqrt(x); }

// Error-free transformations (Dekker 1971; Knuth TAOCP vol. 2, 4.2.2):
// a + b = s + e exactly (TwoSum).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bp = s - a;
  const float ap = s - bp;
  e = (a - ap) + (b - bp);
}

// Running sum that keeps about twice the working precision: float hi + lo pairs
// (TwoSum) for T = float, a plain double for T = double.
template <typename T>
struct WideAcc;
template <>
struct WideAcc<float> {
  float hi = 0.f, lo = 0.f;
  __device__ __forceinline__ void add(float x) {
    float s, e;
    two_sum(hi, x, s, e);
    hi = s;
    lo += e;
  }
  __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};
template <>
struct WideAcc<double> {
  double v = 0.0;
  __device__ __forceinline__ void add(double x) { v += x; }
  __device__ __forceinline__ double value() const { return v; }
};

// Block-wide sum of WideAcc partials, valid in thread 0.  Float pairs are combined with
// TwoSum inside each warp; only the per-warp results are added in FP64 (FP64 arithmetic
// runs at a small fraction of the FP32 rate, so it stays off the per-element path).
__device__ __forceinline__ double block_sum_wide(const WideAcc<float>& a, double* sh) {
  float hi = a.hi, lo = a.lo;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float h2 = __shfl_xor_sync(0xffffffffu, hi, o);
    const float l2 = __shfl_xor_sync(0xffffffffu, lo, o);
    float s, e;
    two_sum(hi, h2, s, e);
    hi = s;
    lo = (lo + l2) + e;
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[wid] = (double)hi + (double)lo;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)((blockDim.x + 31) >> 5); ++w) r += sh[w];
  return r;
}
__device__ __forceinline__ double block_sum_wide(const WideAcc<double>& a, double* sh) {
  return block_sum_double(a.v, sh);
}

// Split-m Gram product with hierarchical accumulation:
//   part[off + c*stride + a + b*P] = sum_{i in rows of chunk c} X[i, a] * Y[i, b]
// for a < P, b < Q, where column b of Y is Y1[:, b] for b < q1 and Y2[:, b - q1] after
// (a virtual concatenation [Y1 Y2]).  With Rq != nullptr the X operand and Y1 are
// Q1 = X R^{-1} formed on the fly per 32-row slab (Rq: upper P x P, so q1 = P).
// Each 32-row slab is summed in T, then added to a WideAcc, so the cross-slab sum keeps
// about FP64 accuracy while the inner products run at the T rate.  The next slab is
// prefetched into registers.  One (PT x QT) output tile per block; thread (tx, ty) owns
// rows ty + (PT/4) u and columns tx + (QT/4) v (conflict-free shared reads).
template <typename T, int PT, int QT, bool FUSE>
__global__ void __launch_bounds__((PT / 4) * (QT / 4))
gram_tn(const T* __restrict__ X, int64_t ldx, const T* __restrict__ Y1, int64_t ldy1, int q1,
        const T* __restrict__ Y2, int64_t ldy2, const T* __restrict__ Rq, int m, int P, int Q,
        int chunk_rows, double* __restrict__ part, int64_t part_stride, int64_t part_offset) {
  constexpr int BK = 32;
  constexpr int NTX = QT / 4, NTY = PT / 4, NT = NTX * NTY;
  constexpr int XQ = BK * PT / NT, YQ = BK * QT / NT;
  __shared__ T Xs[BK][PT + 1];
  __shared__ T Ys[BK][QT + 1];
  __shared__ T Xraw[FUSE ? BK : 1][FUSE ? PT + 1 : 1];   // raw X1 slab (FUSE)
  __shared__ T Rs[FUSE ? PT : 1][FUSE ? PT + 1 : 1];     // R^{-1} (FUSE)
  constexpr bool fuse_q = FUSE;
  const int a0 = blockIdx.x * PT, b0 = blockIdx.y * QT, c = blockIdx.z;
  const int i_begin = c * chunk_rows;
  const int i_end = min(m, i_begin + chunk_rows);
  const int tx = threadIdx.x % NTX, ty = threadIdx.x / NTX;
  // in the fused form every block needs the whole Q1 slab (a0 must be 0: P <= PT)
  if (fuse_q)
    for (int e = threadIdx.x; e < PT * PT; e += NT) {
      const int r = e % PT, q = e / PT;
      Rs[FUSE ? r : 0][FUSE ? q : 0] = (r < P && q < P) ? Rq[r + q * P] : T(0);
    }
  WideAcc<T> acc[4][4];
  T rx[XQ], ry[YQ];
  auto fetch = [&](int i0) {
#pragma unroll
    for (int q = 0; q < XQ; ++q) {
      const int e = threadIdx.x + NT * q;
      const int kk = e % BK, a = e / BK;
      const int i = i0 + kk, ga = a0 + a;
      rx[q] = (i < i_end && ga < P) ? X[i + (int64_t)ga * ldx] : T(0);
    }
#pragma unroll
    for (int q = 0; q < YQ; ++q) {
      const int e = threadIdx.x + NT * q;
      const int kk = e % BK, b = e / BK;
      const int i = i0 + kk, gb = b0 + b;
      T v = T(0);
      if (i < i_end && gb < Q && !(fuse_q && gb < q1))
        v = gb < q1 ? Y1[i + (int64_t)gb * ldy1] : Y2[i + (int64_t)(gb - q1) * ldy2];
      ry[q] = v;
    }
  };
  if (i_begin < i_end) fetch(i_begin);
  for (int i0 = i_begin; i0 < i_end; i0 += BK) {
    __syncthreads();
#pragma unroll
    for (int q = 0; q < XQ; ++q) {
      const int e = threadIdx.x + NT * q;
      if (fuse_q) Xraw[FUSE ? e % BK : 0][FUSE ? e / BK : 0] = rx[q];
      else Xs[e % BK][e / BK] = rx[q];
    }
#pragma unroll
    for (int q = 0; q < YQ; ++q) {
      const int e = threadIdx.x + NT * q;
      Ys[e % BK][e / BK] = ry[q];
    }
    __syncthreads();
    if (i0 + BK < i_end) fetch(i0 + BK);
    if (fuse_q) {
      // Q1 slab = X1 slab * R^{-1} (upper), written to Xs and to the Q1 columns of Ys;
      // each thread carries XQ independent dot products through the l loop
      T qv[XQ];
#pragma unroll
      for (int q = 0; q < XQ; ++q) qv[q] = T(0);
      for (int l = 0; l < P; ++l) {
#pragma unroll
        for (int q = 0; q < XQ; ++q) {
          const int e = threadIdx.x + NT * q;
          const int kk = e % BK, a = e / BK;
          if (l <= a) qv[q] = fma(Xraw[FUSE ? kk : 0][FUSE ? l : 0], Rs[FUSE ? l : 0][FUSE ? a : 0], qv[q]);
        }
      }
#pragma unroll
      for (int q = 0; q < XQ; ++q) {
        const int e = threadIdx.x + NT * q;
        const int kk = e % BK, a = e / BK;
        Xs[kk][a] = qv[q];
        const int gb = a - b0;
        if (gb >= 0 && gb < QT && a < q1) Ys[kk][gb] = qv[q];
      }
      __syncthreads();
    }
    T sl[4][4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) sl[u][v] = T(0);
#pragma unroll 8
    for (int kk = 0; kk < BK; ++kk) {
      T xa[4], yb[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) xa[u] = Xs[kk][ty + NTY * u];
#pragma unroll
      for (int v = 0; v < 4; ++v) yb[v] = Ys[kk][tx + NTX * v];
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) sl[u][v] = fma(xa[u], yb[v], sl[u][v]);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) acc[u][v].add(sl[u][v]);
  }
  double* out = part + part_offset + (int64_t)c * part_stride;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int a = a0 + ty + NTY * u;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int b = b0 + tx + NTX * v;
      if (a < P && b < Q) out[a + (int64_t)b * P] = acc[u][v].value();
    }
  }
}

// out64[e] = sum_c part[c*stride + e] (in double, fixed order); outT the same rounded.
template <typename T>
__global__ void reduce_partials(const T* __restrict__ part, int64_t stride, int nchunks,
                                int64_t len, double* __restrict__ out64, T* __restrict__ outT) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < len;
       e += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int c = 0; c < nchunks; ++c) s += (double)part[(int64_t)c * stride + e];
    if (out64) out64[e] = s;
    if (outT) outT[e] = (T)s;
  }
}

// out[e] = sum_c part[c*stride + e], e < len, c < nchunks: block = 32 outputs, warp w adds
// the chunks c = w, w + 8, ... in order, then the 8 warp sums are added in warp order
// (deterministic, and each thread has only about nchunks / 8 loads in flight).  With Fout,
// also Fout[e] = out[e] - [e is a diagonal entry] for the leading kf x kf block (the
// shifted copy S2 - I that the second Cholesky factor reads, formed here in FP64).
template <typename T, typename TF = T>
__global__ void __launch_bounds__(256)
reduce_partials_split(const T* __restrict__ part, int64_t stride, int nchunks, int64_t len,
                      double* __restrict__ out64, T* __restrict__ outT, int kf = 0,
                      TF* __restrict__ Fout = nullptr) {
  __shared__ double sh[8][33];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t e = (int64_t)blockIdx.x * 32 + lane;
  double s = 0.0;
  if (e < len)
#pragma unroll 4
    for (int c = w; c < nchunks; c += 8) s += (double)part[(int64_t)c * stride + e];
  sh[w][lane] = s;
  __syncthreads();
  if (w == 0 && e < len) {
    double t = 0.0;
#pragma unroll
    for (int q = 0; q < 8; ++q) t += sh[q][lane];
    if (out64) out64[e] = t;
    if (outT) outT[e] = (T)t;
    if (Fout && e < (int64_t)kf * kf) Fout[e] = (TF)(t - (e % (kf + 1) == 0 ? 1.0 : 0.0));
  }
}

// The same reduction for chunk partials stored as float pairs (hi, lo) in 8-byte slots
// (tc::gram_tf32x3_t): each warp adds its chunks c = w, w + 8, ... in double-float
// (TwoSum), warp 0 adds the eight pairs in warp order, and the sum is converted to double
// once.
template <typename TF>
__global__ void __launch_bounds__(256)
reduce_pairs_split(const double* __restrict__ part, int64_t stride, int nchunks, int64_t len,
                   double* __restrict__ out64, int kf = 0, TF* __restrict__ Fout = nullptr) {
  __shared__ float2 sh[8][33];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t e = (int64_t)blockIdx.x * 32 + lane;
  float hs = 0.f, ls = 0.f;
  if (e < len) {
    const float2* p2 = reinterpret_cast<const float2*>(part);
#pragma unroll 4
    for (int c = w; c < nchunks; c += 8) {
      const float2 v = p2[(int64_t)c * stride + e];
      float s, er;
      two_sum(hs, v.x, s, er);
      hs = s;
      ls = (ls + v.y) + er;
    }
  }
  sh[w][lane] = make_float2(hs, ls);
  __syncthreads();
  if (w == 0 && e < len) {
    float h = 0.f, l = 0.f;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const float2 v = sh[q][lane];
      float s, er;
      two_sum(h, v.x, s, er);
      h = s;
      l = (l + v.y) + er;
    }
    const double t = (double)h + (double)l;
    if (out64) out64[e] = t;
    if (Fout && e < (int64_t)kf * kf) Fout[e] = (TF)(t - (e % (kf + 1) == 0 ? 1.0 : 0.0));
  }
}

// Sum of squares of an m x ncols column-major block, partial per block (double).
template <typename T>
__global__ void sumsq_partial(const T* __restrict__ A, int64_t lda, int m, int ncols,
                              double* __restrict__ part) {
  __shared__ double sh[32];
  const int64_t total = (int64_t)m * ncols;
  double s = 0.0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = e / m, i = e - j * m;
    const double v = (double)A[i + j * lda];
    s += v * v;
  }
  s = block_sum_double(s, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// W1 > 0 and finite everywhere, else set the error bit.
template <typename T>
__global__ void check_weights(const T* __restrict__ W1, int64_t ldw, int m, int k,
                              int* __restrict__ err) {
  const int64_t total = (int64_t)m * k;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = e / m, i = e - j * m;
    const T w = W1[i + j * ldw];
    if (!(w > T(0)) || !wfinite(w)) atomicOr(err, ERRBIT_BAD_WEIGHT);
  }
}

// dst (m x ncols, ld_dst) <- src (m x ncols, ld_src) with type conversion.
template <typename TD, typename TS>
__global__ void convert_copy(TD* __restrict__ dst, int64_t ld_dst, const TS* __restrict__ src,
                             int64_t ld_src, int m, int ncols) {
  const int64_t total = (int64_t)m * ncols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = e / m, i = e - j * m;
    dst[i + j * ld_dst] = (TD)src[i + j * ld_src];
  }
}

// X1_0 i.i.d. N(0,1) from the counter-based SplitMix64 + Box-Muller stream.
template <typename T>
__global__ void random_normal_fill(T* __restrict__ X, int64_t ldx, int m, int k, uint64_t seed) {
  const int64_t total = (int64_t)m * k;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = t / m, i = t - j * m;
    X[i + j * ldx] = (T)normal_at(seed, (uint64_t)t);
  }
}

// --------------------------------------------------------------------------------
// First CholeskyQR factor (one block): S1 = sum of the nch partial Grams (double, in a
// fixed order), S1 = R1^T R1 in double, and R1^{-1} (upper) written in T.  A pivot
// below 1e-13 of its column's original diagonal means X1 is numerically of rank < k.
template <typename T>
__global__ void __launch_bounds__(256)
chol1_kernel(const double* __restrict__ part, int nch, int k, T* __restrict__ R1inv,
             int* __restrict__ err) {
  extern __shared__ unsigned char smem_raw[];
  double* L = reinterpret_cast<double*>(smem_raw);  // k*k
  double* Ri = L + k * k;                            // k*k
  double* dg = Ri + k * k;                           // k: original diagonal
  __shared__ int flag;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int kk = k * k;
  for (int e = tid; e < kk; e += nt) {
    double v = 0.0;
    for (int c = 0; c < nch; ++c) v += part[(int64_t)c * kk + e];
    const int i = e % k, j = e / k;
    L[e] = i >= j ? v : 0.0;
    if (i == j) dg[i] = v;
  }
  if (tid == 0) flag = 0;
  __syncthreads();
  __shared__ double rpiv;
  for (int t = 0; t < k; ++t) {
    if (tid == 0) {
      double d = L[t + t * k];
      if (!(d > 1e-13 * dg[t]) || !isfinite(d)) { flag = 1; d = 1.0; }
      // 1/sqrt(d): float estimate, two Newton steps in double (error ~1e-16)
      double r = (double)rsqrtf((float)d);
      r = r * (1.5 - 0.5 * d * r * r);
      r = r * (1.5 - 0.5 * d * r * r);
      L[t + t * k] = d * r;
      rpiv = r;
    }
    __syncthreads();
    const double rp = rpiv;
    for (int i = t + 1 + tid; i < k; i += nt) L[i + t * k] *= rp;
    __syncthreads();
    const int w = k - t - 1;
    for (int e = tid; e < w * w; e += nt) {
      const int i = t + 1 + e % w, j = t + 1 + e / w;
      if (i >= j) L[i + j * k] -= L[i + t * k] * L[j + t * k];
    }
    __syncthreads();
  }
  if (flag && tid == 0) atomicOr(err, ERRBIT_RANK_DEFICIENT);
  // reciprocals of the diagonal: float estimate + two Newton steps in double
  for (int a = tid; a < k; a += nt) {
    const double d = L[a + a * k];
    double r = (double)(1.0f / (float)d);
    r = r * (2.0 - d * r);
    r = r * (2.0 - d * r);
    dg[a] = r;
  }
  __syncthreads();
  // R1^{-1}: column c solves R1 x = e_c (R1(a,l) = L(l,a)), one thread per column.
  for (int c = tid; c < k; c += nt) {
    for (int a = k - 1; a >= 0; --a) {
      double v = a == c ? 1.0 : 0.0;
      for (int l = a + 1; l <= c; ++l) v -= L[l + a * k] * Ri[l + c * k];
      Ri[a + c * k] = a <= c ? v * dg[a] : 0.0;
    }
  }
  __syncthreads();
  for (int e = tid; e < kk; e += nt) R1inv[e] = (T)Ri[e];
}

// Second CholeskyQR factor (one block).  S2 = Q1^T Q1 is close to I, so it is factored
// in "difference form": S2 = (I + F)(I + F)^T with F lower triangular, computed from
// Delta = S2 - I so that the small F keeps full relative precision in T:
//   F_tt = delta / (1 + sqrt(1 + delta)),  delta = Delta_tt - sum_{j<t} F_tj^2
//   F_it = (Delta_it - sum_{j<t} F_ij F_tj) / (1 + F_tt)               (i > t)
// Outputs (T): N = (I + F)^{-1} - I = R2^{-T} - I (lower), and
// Rinv = R1^{-1} (I + N)^T = (R2 R1)^{-1}, the inverse of the full triangular factor.
template <typename T>
__global__ void __launch_bounds__(256)
chol2_kernel(const double* __restrict__ part, int nch, int64_t pstride, int k,
             const T* __restrict__ R1inv, T* __restrict__ Nout, T* __restrict__ Rinv,
             int* __restrict__ err) {
  extern __shared__ unsigned char smem_raw[];
  T* F = reinterpret_cast<T*>(smem_raw);  // k*k lower (col-major)
  T* Nm = F + k * k;                       // k*k lower
  T* Ri1 = Nm + k * k;                     // k*k upper
  __shared__ int flag;
  const int tid = threadIdx.x, nt = blockDim.x;
  // S2 = Q1^T Q1: the leading k x k block of the nch chunk partials (fixed order)
  for (int e = tid; e < k * k; e += nt) {
    const int i = e % k, j = e / k;
    double v = 0.0;
    if (i >= j)
      for (int c = 0; c < nch; ++c) v += part[(int64_t)c * pstride + e];
    F[e] = i >= j ? (T)(v - (i == j ? 1.0 : 0.0)) : T(0);
    Ri1[e] = R1inv[e];
  }
  if (tid == 0) flag = 0;
  __syncthreads();
  for (int t = 0; t < k; ++t) {
    if (tid == 0) {
      T d = F[t + t * k];
      for (int j = 0; j < t; ++j) d -= F[t + j * k] * F[t + j * k];
      if (!(T(1) + d > T(0)) || !wfinite(d)) { flag = 1; d = T(0); }
      F[t + t * k] = d / (T(1) + wsqrt(T(1) + d));
    }
    __syncthreads();
    const T den = T(1) + F[t + t * k];
    for (int i = t + 1 + tid; i < k; i += nt) {
      T v = F[i + t * k];
      for (int j = 0; j < t; ++j) v -= F[i + j * k] * F[t + j * k];
      F[i + t * k] = v / den;
    }
    __syncthreads();
  }
  if (flag && tid == 0) atomicOr(err, ERRBIT_RANK_DEFICIENT);
  __shared__ T rdiag[64];
  for (int a = tid; a < k; a += nt) rdiag[a] = T(1) / (T(1) + F[a + a * k]);
  __syncthreads();
  // (I + F) N = -F, column c by forward substitution (N lower)
  for (int c = tid; c < k; c += nt) {
    for (int a = 0; a < k; ++a) {
      T v = T(0);
      if (a >= c) {
        v = -F[a + c * k];
        for (int l = c; l < a; ++l) v -= F[a + l * k] * Nm[l + c * k];
        v *= rdiag[a];
      }
      Nm[a + c * k] = v;
    }
  }
  __syncthreads();
  // Rinv(a, b) = R1inv(a, b) + sum_{l=a..b} R1inv(a, l) N(b, l)
  for (int e = tid; e < k * k; e += nt) {
    const int a = e % k, b = e / k;
    T v = T(0);
    if (a <= b) {
      v = Ri1[a + b * k];
      for (int l = a; l <= b; ++l) v += Ri1[a + l * k] * Nm[b + l * k];
    }
    Rinv[e] = v;
    Nout[e] = Nm[e];
  }
}

// The same second factor for k <= 32 with one warp; F = S2 - I arrives as T (k x k,
// column-major, formed where S2 is summed).  Right-looking Cholesky of I + F in difference
// form: at step t the pivot F_tt (after the updates of steps < t) gives
// Lambda_tt = F_tt / (1 + sqrt(1 + F_tt)), the rows below take Lambda_it = F_it / (1 +
// Lambda_tt), and every row i > t updates F(i,j) -= Lambda_it Lambda_jt for j > t with
// Lambda_jt broadcast from lane j.  Lane i keeps its row of F in registers shifted left by
// one entry per step (so the pivot column is always entry 0 and every register index is a
// compile-time constant while the step loop stays rolled: a single warp runs this once, so
// compact code matters more than unrolling).  Then (I + Lambda) N = -Lambda by forward
// substitution over the rows, and Rinv = R1inv (I + N)^T.
template <typename T>
__global__ void __launch_bounds__(32)
chol2_warp(const T* __restrict__ Fin, int k, const T* __restrict__ R1inv,
           T* __restrict__ Nout, T* __restrict__ Rinv, int* __restrict__ err) {
  constexpr int KP = 32;
  constexpr unsigned FULL = 0xffffffffu;
  __shared__ T Ls[KP][KP + 1];   // Lambda, lower with the diagonal, row-major
  __shared__ T Ns[KP][KP + 1];   // N, lower, row-major
  __shared__ T rdg_s[KP];        // 1 / (1 + Lambda_tt)
  const int i = threadIdx.x;
  const bool live = i < k;
  T M[KP];
#pragma unroll
  for (int j = 0; j < KP; ++j) {
    const int hi = i > j ? i : j, lo = i > j ? j : i;
    M[j] = (live && j < k) ? Fin[hi + lo * k] : T(0);
  }
  bool flag = false;
#pragma unroll 1
  for (int t = 0; t < k; ++t) {
    const T ftt = __shfl_sync(FULL, M[0], t);
    T lam = T(0);
    if (!(T(1) + ftt > T(0)) || !wfinite(ftt)) flag = true;
    else lam = ftt / (T(1) + wsqrt(T(1) + ftt));
    const T rden = T(1) / (T(1) + lam);
    const T lit = i > t ? M[0] * rden : T(0);
    if (i == t) {
      Ls[t][t] = lam;
      rdg_s[t] = rden;
    }
    if (i > t) Ls[i][t] = lit;
#pragma unroll
    for (int j = 1; j < KP; ++j) {
      // lane (t + j) mod 32: rows past the end and rows <= t broadcast 0
      const T ljt = __shfl_sync(FULL, lit, (t + j) & (KP - 1));
      M[j - 1] = fma(-lit, ljt, M[j]);
    }
    M[KP - 1] = T(0);
  }
  __syncwarp();
  // rows of N: rhs = -Lambda (lower, with the diagonal); row l is final at step l and its
  // entries beyond l are zero, so broadcasting the whole row needs no mask
  T Nr[KP];
#pragma unroll
  for (int c = 0; c < KP; ++c) Nr[c] = (live && c <= i) ? -Ls[i][c] : T(0);
#pragma unroll 1
  for (int l = 0; l < k; ++l) {
    const T f = i > l && live ? Ls[i][l] * rdg_s[l] : T(0);
#pragma unroll
    for (int c = 0; c < KP; ++c) {
      const T v = __shfl_sync(FULL, Nr[c], l);
      Nr[c] = fma(-f, v, Nr[c]);
    }
  }
  const T rdg = live ? rdg_s[i] : T(1);
#pragma unroll
  for (int c = 0; c < KP; ++c) {
    Nr[c] *= rdg;
    Ns[i][c] = Nr[c];
  }
  __syncwarp();
  // Rinv(a, b) = R1inv(a, b) + sum_l R1inv(a, l) N(b, l), lane a = row a (R1inv upper and
  // N lower make the sum run over a <= l <= b by itself)
  T V[KP];
#pragma unroll
  for (int b = 0; b < KP; ++b) V[b] = (live && b < k && b >= i) ? R1inv[i + b * k] : T(0);
#pragma unroll
  for (int b = 0; b < KP; ++b) Ls[i][b] = V[b];   // Lambda is no longer needed
  __syncwarp();
#pragma unroll 1
  for (int l = 0; l < k; ++l) {
    const T ral = Ls[i][l];
#pragma unroll
    for (int b = 0; b < KP; ++b) V[b] = fma(ral, Ns[b][l], V[b]);
  }
#pragma unroll
  for (int b = 0; b < KP; ++b)
    if (live && b < k) {
      Rinv[i + b * k] = i <= b ? V[b] : T(0);
      Nout[i + b * k] = Nr[b];
    }
  if (flag && i == 0) atomicOr(err, ERRBIT_RANK_DEFICIENT);
}

// Q1 = X1 R1^{-1} (m x k); R1^{-1} upper triangular.
template <typename T>
__global__ void form_q(const T* __restrict__ X1, int64_t ldx, const T* __restrict__ Rinv,
                       int m, int k, T* __restrict__ Q1) {
  extern __shared__ unsigned char smem_raw[];
  T* Ri = reinterpret_cast<T*>(smem_raw);
  for (int e = threadIdx.x; e < k * k; e += blockDim.x) Ri[e] = Rinv[e];
  __syncthreads();
  const int64_t total = (int64_t)m * k;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int a = (int)(e / m);
    const int64_t i = e - (int64_t)a * m;
    T v = T(0);
    for (int b = 0; b <= a; ++b) v = fma(X1[i + b * ldx], Ri[b + a * k], v);
    Q1[i + (int64_t)a * m] = v;
  }
}

// Coefficient step, one thread per column j of A2:
//   B(:,j) = R2^{-T} (Q1^T A2)(:,j) = t + N t  (t kept in double, the small N t in T)
//   C(:,j) = R^{-1} B(:,j)
// Writes C (k x n2, T), B in double, B split as float hi + lo (for the double-float
// Gram), the C^T part of Z2 (row j: Z2[j*NP + a] = C(a,j)), and the block's ||B||^2.
template <typename T>
__global__ void __launch_bounds__(128)
coef_kernel2(const double* __restrict__ QtA2, const T* __restrict__ Nm, const T* __restrict__ Rinv,
             int k, int n2, int NP, T* __restrict__ Cout, double* __restrict__ B64,
             float* __restrict__ Bh, float* __restrict__ Bl, T* __restrict__ Z2,
             double* __restrict__ bnorm_part) {
  extern __shared__ unsigned char smem_raw[];
  T* Ns = reinterpret_cast<T*>(smem_raw);
  T* Rs = Ns + k * k;
  __shared__ double sh[32];
  for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
    Ns[e] = Nm[e];
    Rs[e] = Rinv[e];
  }
  __syncthreads();
  double bn = 0.0;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n2) {
    T tv[64];
    T bv[64];
    for (int a = 0; a < k; ++a) tv[a] = (T)QtA2[a + (int64_t)j * k];
    for (int a = 0; a < k; ++a) {
      T corr = T(0);
      for (int l = 0; l <= a; ++l) corr = fma(Ns[a + l * k], tv[l], corr);
      const double b = QtA2[a + (int64_t)j * k] + (double)corr;
      B64[a + (int64_t)j * k] = b;
      const float hi = (float)b;
      Bh[a + (int64_t)j * k] = hi;
      Bl[a + (int64_t)j * k] = (float)(b - (double)hi);
      bv[a] = (T)b;
      bn += b * b;
    }
    for (int a = 0; a < k; ++a) {
      T c = T(0);
      for (int l = a; l < k; ++l) c = fma(Rs[a + l * k], bv[l], c);
      Cout[a + (int64_t)j * k] = c;
      Z2[(int64_t)j * NP + a] = c;
    }
  }
  bn = block_sum_double(bn, sh);
  if (threadIdx.x == 0) bnorm_part[blockIdx.x] = bn;
}

// Coefficient step, one warp per column j of A2 (lanes over the k coefficients):
//   t = (Q1^T A2)(:,j) summed from the chunk partials in double,
//   B(:,j) = R2^{-T} t = t + N t  (t kept in double, the small N t in T)
//   C(:,j) = R^{-1} B(:,j)
// Writes C (k x n2, T), B in double and as float hi + lo (for the double-float Gram),
// the C^T part of Z2 (row j: Z2[j*NP + a] = C(a,j)) and the block's ||B||_F^2.
template <typename T>
__global__ void __launch_bounds__(256)
coef_kernel3(const double* __restrict__ part, int nch, int64_t pstride,
             const T* __restrict__ Nm, const T* __restrict__ Rinv,
             int k, int n2, int NP, T* __restrict__ Cout, double* __restrict__ B64,
             float* __restrict__ Bh, float* __restrict__ Bl, T* __restrict__ Z2,
             double* __restrict__ bnorm_part) {
  extern __shared__ unsigned char smem_raw[];
  T* Ns = reinterpret_cast<T*>(smem_raw);   // k*k
  T* Rs = Ns + k * k;                       // k*k
  T* tw = Rs + k * k;                       // [8][64] per-warp t
  T* bw = tw + 8 * 64;                      // [8][64] per-warp B
  __shared__ double sh[32];
  for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
    Ns[e] = Nm[e];
    Rs[e] = Rinv[e];
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int j = blockIdx.x * 8 + w;
  double bn = 0.0;
  if (j < n2) {
    double t64[2] = {0.0, 0.0};
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int a = lane + 32 * h;
      if (a < k) {
        // (Q1^T A2)(a, j): column k + j of the k x (k + n2) chunk partials
        const int64_t o = a + (int64_t)(k + j) * k;
        double v = 0.0;
        for (int c = 0; c < nch; ++c) v += part[(int64_t)c * pstride + o];
        t64[h] = v;
        tw[w * 64 + a] = (T)v;
      }
    }
    __syncwarp();
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int a = lane + 32 * h;
      if (a < k) {
        T corr = T(0);
        for (int l = 0; l <= a; ++l) corr = fma(Ns[a + l * k], tw[w * 64 + l], corr);
        const double b = t64[h] + (double)corr;
        B64[a + (int64_t)j * k] = b;
        const float hi = (float)b;
        Bh[a + (int64_t)j * k] = hi;
        Bl[a + (int64_t)j * k] = (float)(b - (double)hi);
        bw[w * 64 + a] = (T)b;
        bn += b * b;
      }
    }
    __syncwarp();
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int a = lane + 32 * h;
      if (a < k) {
        T cv = T(0);
        for (int l = a; l < k; ++l) cv = fma(Rs[a + l * k], bw[w * 64 + l], cv);
        Cout[a + (int64_t)j * k] = cv;
        Z2[(int64_t)j * NP + a] = cv;
      }
    }
  }
  bn = block_sum_double(bn, sh);
  if (threadIdx.x == 0) bnorm_part[blockIdx.x] = bn;
}

// a * b = p + e exactly (TwoProduct via fma, Dekker 1971).
// G2 = K - B^T B (n2 x n2), 32x32 tile per block, 256 threads (4 entries each).
// FP32 path: sum_a B_ai B_aj in double-float arithmetic from B = hi + lo (the dropped
// lo*lo term is below 2^-48 relative), then K (double) minus it in double, rounded
// to T.  FP64 path: plain double.
template <typename T>
__global__ void __launch_bounds__(256)
form_g2_df(const double* __restrict__ K64, const double* __restrict__ B64,
           const float* __restrict__ Bh, const float* __restrict__ Bl, int k, int n2,
           T* __restrict__ G2) {
  constexpr bool kDouble = std::is_same<T, double>::value;
  constexpr int FR = kDouble ? 1 : 64, DR = kDouble ? 64 : 1;
  __shared__ float Hi[FR][33], Li[FR][33], Hj[FR][33], Lj[FR][33];
  __shared__ double Di[DR][33], Dj[DR][33];
  const int i0 = blockIdx.x * 32, j0 = blockIdx.y * 32;
  for (int e = threadIdx.x; e < k * 32; e += blockDim.x) {
    const int a = e % k, c = e / k;
    const bool vi = i0 + c < n2, vj = j0 + c < n2;
    const int64_t oi = a + (int64_t)(i0 + c) * k, oj = a + (int64_t)(j0 + c) * k;
    if (kDouble) {
      Di[a][c] = vi ? B64[oi] : 0.0;
      Dj[a][c] = vj ? B64[oj] : 0.0;
    } else {
      Hi[a][c] = vi ? Bh[oi] : 0.f;
      Li[a][c] = vi ? Bl[oi] : 0.f;
      Hj[a][c] = vj ? Bh[oj] : 0.f;
      Lj[a][c] = vj ? Bl[oj] : 0.f;
    }
  }
  __syncthreads();
  const int ti = threadIdx.x % 32, tj = threadIdx.x / 32;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int jj = tj + 8 * u;
    double sum;
    if (kDouble) {
      double v = 0.0;
      for (int a = 0; a < k; ++a) v = fma(Di[a][ti], Dj[a][jj], v);
      sum = v;
    } else {
      float sh_ = 0.f, sl_ = 0.f;
      for (int a = 0; a < k; ++a) {
        const float hi = Hi[a][ti], hj = Hj[a][jj];
        const float p = hi * hj;
        const float pe = fmaf(hi, hj, -p);
        const float x = fmaf(hi, Lj[a][jj], fmaf(Li[a][ti], hj, pe));
        float s, e;
        two_sum(sh_, p, s, e);
        sh_ = s;
        sl_ += e + x;
      }
      sum = (double)sh_ + (double)sl_;
    }
    const int i = i0 + ti, j = j0 + jj;
    if (i < n2 && j < n2) G2[i + (int64_t)j * n2] = (T)(K64[i + (int64_t)j * n2] - sum);
  }
}

// --------------------------------------------------------------------------------
// Subspace iteration, multiply: Z = G2 V (n2 x b), one warp per row of Z (G2 is
// symmetric, so row j of Z uses the contiguous column j of G2).  Per block partials
// H = V^T Z and P = Z^T Z over its rows: part[blk][0][b][b], part[blk][1][b][b].
// VSMEM: V is staged in shared memory transposed (Vt[c][l]) once per block.
template <typename T, bool VSMEM>
__global__ void __launch_bounds__(256)
eig_mult(const T* __restrict__ G2, const T* __restrict__ V, int n2, int b, T* __restrict__ Z,
         T* __restrict__ part, unsigned int* __restrict__ ticket, T* __restrict__ HP) {
  constexpr int RB = 8;   // one row of Z per warp
  extern __shared__ unsigned char smem_raw[];
  T* Vt = reinterpret_cast<T*>(smem_raw);  // [b][n2] when VSMEM
  __shared__ T Zs[RB][EIG_BMAX + 1];
  __shared__ T Vr[RB][EIG_BMAX + 1];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int j0 = blockIdx.x * RB;
  if (VSMEM) {
    for (int e = threadIdx.x; e < b * n2; e += blockDim.x) Vt[e] = V[e];
    __syncthreads();
  }
  const T* Vsrc = VSMEM ? Vt : V;
  for (int rr = w; rr < RB; rr += 8) {
    const int j = j0 + rr;
    T acc[EIG_BMAX];
#pragma unroll
    for (int c = 0; c < EIG_BMAX; ++c) acc[c] = T(0);
    if (j < n2) {
#pragma unroll 4
      for (int l = lane; l < n2; l += 32) {
        const T g = G2[l + (int64_t)j * n2];
#pragma unroll
        for (int c = 0; c < EIG_BMAX; ++c)
          if (c < b) acc[c] = fma(g, Vsrc[l + (int64_t)c * n2], acc[c]);
      }
    }
    T mine = T(0);
#pragma unroll
    for (int c = 0; c < EIG_BMAX; ++c) {
      if (c < b) {
        const T sum = warp_sum(acc[c]);
        if (lane == c) mine = sum;
      }
    }
    if (lane < b) {
      Zs[rr][lane] = j < n2 ? mine : T(0);
      Vr[rr][lane] = j < n2 ? Vsrc[j + (int64_t)lane * n2] : T(0);
      if (j < n2) Z[j + (int64_t)lane * n2] = mine;
    }
  }
  __syncthreads();
  T* out = part + (int64_t)blockIdx.x * 2 * b * b;
  for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
    const int c1 = e % b, c2 = e / b;
    T h = T(0), p = T(0);
#pragma unroll
    for (int rr = 0; rr < RB; ++rr) {
      h = fma(Vr[rr][c1], Zs[rr][c2], h);
      p = fma(Zs[rr][c1], Zs[rr][c2], p);
    }
    out[e] = h;
    out[b * b + e] = p;
  }
  // the last block to finish adds the partials in block order (no block waits)
  __shared__ bool is_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) is_last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  // summed in T: the Ritz problem is solved in T anyway (and FP64 adds are slow here)
  for (int e = threadIdx.x; e < 2 * b * b; e += blockDim.x) {
    T v0 = T(0), v1 = T(0), v2 = T(0), v3 = T(0);
    const int nb = (int)gridDim.x;
    int c = 0;
    for (; c + 4 <= nb; c += 4) {
      v0 += __ldcg(&part[(int64_t)c * 2 * b * b + e]);
      v1 += __ldcg(&part[(int64_t)(c + 1) * 2 * b * b + e]);
      v2 += __ldcg(&part[(int64_t)(c + 2) * 2 * b * b + e]);
      v3 += __ldcg(&part[(int64_t)(c + 3) * 2 * b * b + e]);
    }
    for (; c < nb; ++c) v0 += __ldcg(&part[(int64_t)c * 2 * b * b + e]);
    HP[e] = (v0 + v1) + (v2 + v3);
  }
  if (threadIdx.x == 0) *ticket = 0u;
}

// Subspace iteration, small step (one warp, b <= 32):
//  1. H = V^T G2 V and P = Z^T Z (b x b, summed by the last eig_mult block).
//  2. Rayleigh-Ritz: H = Y Theta Y^T by the parallel cyclic Jacobi method (round-robin
//     ordering, b/2 disjoint rotations per round), sorted descending.
//  3. Next basis W = [V Y F_v + Z Y F_z], F_z = diag(1/||Z y_c||) for the columns with a
//     non-negligible Ritz value and F_v = diag(1) for the others (which keeps an
//     orthonormal Ritz vector where G2 V has no component); W^T W is formed from
//     I, Y^T P Y and Theta, factored W^T W = L L^T, and Mv = Y F_v L^{-T},
//     Mz = Y F_z L^{-T}, so that V_next = V Mv + Z Mz has orthonormal columns.
// Outputs (T, b x b col-major): Y, Mv, Mz; theta (b, descending); resid (b): estimate of
// ||G2 v_c - theta_c v_c||^2 = (Y^T P Y)_cc - theta_c^2.
// One warp, no block barriers: a Jacobi round is three warp-synchronous phases (angles by
// lanes < b/2; row rotations with lane l taking column l; column rotations of H and Y
// with lane r taking row r).  The Cholesky factor of W^T W and L^{-1} use register rows
// (lane = row) with per-step broadcasts by shuffle; loops over steps stay rolled, since a
// single warp runs this code once and compact code matters more than unrolling.
template <typename T>
__global__ void __launch_bounds__(32)
eig_small(const T* __restrict__ HP, int b, int max_sweeps, T* __restrict__ Yout,
          T* __restrict__ Mv, T* __restrict__ Mz, T* __restrict__ theta,
          T* __restrict__ resid, int* __restrict__ err) {
  constexpr int BM = EIG_BMAX;
  constexpr unsigned FULL = 0xffffffffu;
  __shared__ T Hs[BM][BM + 1];   // H; later P Y; later L (lower)
  __shared__ T Ps[BM][BM + 1];   // P; later Y^T P Y
  __shared__ T Ys[BM][BM + 1];   // eigenvectors; later L^{-1} (lower)
  __shared__ T Ws[BM][BM + 1];   // sorted eigenvectors
  __shared__ T cs[BM / 2][2];
  __shared__ int pq[BM / 2][2];
  __shared__ int perm[BM];
  __shared__ int usev_s[BM];
  __shared__ T fz_s[BM];
  const int lane = threadIdx.x;
  const int bb = b * b;
  for (int e = lane; e < BM * BM; e += 32) {
    const int r = e / BM, q = e % BM;
    Hs[r][q] = T(0);
    Ps[r][q] = T(0);
    Ys[r][q] = r == q ? T(1) : T(0);
    Ws[r][q] = T(0);
  }
  __syncwarp();
  for (int e = lane; e < bb; e += 32) {
    const int r = e % b, q = e / b;
    Hs[r][q] = T(0.5) * (HP[e] + HP[q + r * b]);
    Ps[r][q] = HP[bb + e];
  }
  __syncwarp();

  // ---- parallel Jacobi; stop once ||offdiag|| <= 4 b u ||H||
  const int N = (b + 1) & ~1, half = N / 2;
  const T eps = T(4 * b) * (sizeof(T) == 4 ? T(5.96e-8) : T(1.11e-16));
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    T off = T(0), tot = T(0);
    for (int e = lane; e < bb; e += 32) {
      const int r = e % b, q = e / b;
      const T v = Hs[r][q];
      tot += v * v;
      if (r != q) off += v * v;
    }
    off = warp_sum(off);
    tot = warp_sum(tot);
    if (off <= eps * eps * tot) break;
    for (int round = 0; round < N - 1; ++round) {
      if (lane < half) {
        int p = lane == 0 ? N - 1 : round + lane;
        if (p >= N - 1 && lane != 0) p -= N - 1;
        int q = round + N - 1 - lane;
        if (q >= N - 1) q -= N - 1;
        if (p > q) { const int t = p; p = q; q = t; }
        T c = T(1), sn = T(0);
        if (q < b) {
          const T apq = Hs[p][q];
          if (apq != T(0)) {
            const T tau = (Hs[q][q] - Hs[p][p]) / (T(2) * apq);
            const T t = (tau >= T(0) ? T(1) : T(-1)) / (fabs(tau) + wsqrt(T(1) + tau * tau));
            c = T(1) / wsqrt(T(1) + t * t);
            sn = t * c;
          }
        }
        pq[lane][0] = p;
        pq[lane][1] = q;
        cs[lane][0] = c;
        cs[lane][1] = sn;
      }
      __syncwarp();
      // H <- J^T H: lane l rotates rows p, q of column l for every pair
      if (lane < b) {
        for (int i0 = 0; i0 < half; i0 += 4) {
          T hp[4], hq[4], cc[4], ss[4];
          int pp[4], qq[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int i = i0 + u < half ? i0 + u : half - 1;
            pp[u] = pq[i][0];
            qq[u] = pq[i][1];
            cc[u] = cs[i][0];
            ss[u] = cs[i][1];
            const bool ok = i0 + u < half && qq[u] < b;
            hp[u] = ok ? Hs[pp[u]][lane] : T(0);
            hq[u] = ok ? Hs[qq[u]][lane] : T(0);
          }
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            if (i0 + u < half && qq[u] < b) {
              Hs[pp[u]][lane] = cc[u] * hp[u] - ss[u] * hq[u];
              Hs[qq[u]][lane] = ss[u] * hp[u] + cc[u] * hq[u];
            }
          }
        }
      }
      __syncwarp();
      // H <- H J, Y <- Y J: lane r rotates columns p, q of row r for every pair
      if (lane < b) {
        for (int i0 = 0; i0 < half; i0 += 4) {
          T hp[4], hq[4], yp[4], yq[4], cc[4], ss[4];
          int pp[4], qq[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int i = i0 + u < half ? i0 + u : half - 1;
            pp[u] = pq[i][0];
            qq[u] = pq[i][1];
            cc[u] = cs[i][0];
            ss[u] = cs[i][1];
            const bool ok = i0 + u < half && qq[u] < b;
            hp[u] = ok ? Hs[lane][pp[u]] : T(0);
            hq[u] = ok ? Hs[lane][qq[u]] : T(0);
            yp[u] = ok ? Ys[lane][pp[u]] : T(0);
            yq[u] = ok ? Ys[lane][qq[u]] : T(0);
          }
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            if (i0 + u < half && qq[u] < b) {
              Hs[lane][pp[u]] = cc[u] * hp[u] - ss[u] * hq[u];
              Hs[lane][qq[u]] = ss[u] * hp[u] + cc[u] * hq[u];
              Ys[lane][pp[u]] = cc[u] * yp[u] - ss[u] * yq[u];
              Ys[lane][qq[u]] = ss[u] * yp[u] + cc[u] * yq[u];
            }
          }
        }
      }
      __syncwarp();
    }
  }
  // ---- sort descending: lane c's rank = #{d : theta_d > theta_c, or equal with d < c}
  if (lane < b) {
    const T tc = Hs[lane][lane];
    int rank = 0;
    for (int d = 0; d < b; ++d) {
      const T td = Hs[d][d];
      rank += (td > tc) || (td == tc && d < lane);
    }
    perm[rank] = lane;
    if (!wfinite(tc)) atomicOr(err, ERRBIT_EIG);
  }
  __syncwarp();
  const T thl = lane < b ? Hs[perm[lane]][perm[lane]] : T(0);   // sorted Ritz value
  if (lane < b)
    for (int c = 0; c < b; ++c) Ws[lane][c] = Ys[lane][perm[c]];
  // P Y into Hs (lane r: row r of P in registers)
  T pr[BM];
#pragma unroll
  for (int l = 0; l < BM; ++l) pr[l] = Ps[lane][l];
  __syncwarp();
  for (int c = 0; c < b; ++c) {
    T v0 = T(0), v1 = T(0);
#pragma unroll
    for (int l = 0; l < BM; l += 2) {
      v0 = fma(pr[l], Ws[l][c], v0);
      v1 = fma(pr[l + 1], Ws[l + 1][c], v1);
    }
    Hs[lane][c] = v0 + v1;
  }
  // Y^T P Y into Ps (lane r: column r of Y in registers)
#pragma unroll
  for (int l = 0; l < BM; ++l) pr[l] = Ws[l][lane];
  __syncwarp();
  for (int c = 0; c < b; ++c) {
    T v0 = T(0), v1 = T(0);
#pragma unroll
    for (int l = 0; l < BM; l += 2) {
      v0 = fma(pr[l], Hs[l][c], v0);
      v1 = fma(pr[l + 1], Hs[l + 1][c], v1);
    }
    Ps[lane][c] = v0 + v1;
  }
  __syncwarp();
  const T tmax = fabs(__shfl_sync(FULL, thl, 0));
  const T small = sizeof(T) == 4 ? T(1e-6) : T(1e-13);
  const T nz2 = lane < b ? Ps[lane][lane] : T(1);
  const bool use_v = !(thl > small * tmax) || !(nz2 > T(0));
  const T fzl = use_v ? T(0) : T(1) / wsqrt(nz2);
  if (lane < b) {
    resid[lane] = nz2 - thl * thl;
    theta[lane] = thl;
  }
  usev_s[lane] = (use_v || lane >= b) ? 1 : 0;
  fz_s[lane] = lane < b ? fzl : T(0);
  __syncwarp();
  // Gram of W (lane i: row i): <Vy_a, Vy_b> = delta_ab, <Zy_a, Zy_b> = fz_a fz_b (Y^T P Y)_ab,
  // mixed pairs 0; rows and columns past b are the identity
  T G[BM];
#pragma unroll
  for (int j = 0; j < BM; ++j) {
    const bool uj = usev_s[j] != 0;
    T g;
    if (use_v || lane >= b || j >= b) g = (uj && (use_v || lane >= b)) && j == lane ? T(1) : T(0);
    else g = uj ? T(0) : fzl * fz_s[j] * Ps[lane][j];
    G[j] = g;
  }
  // Cholesky W^T W = L L^T (lower L into Hs), rows shifted left by one entry per step
  bool bad = false;
  for (int t = 0; t < b; ++t) {
    T d = __shfl_sync(FULL, G[0], t);
    if (!(d > T(0)) || !wfinite(d)) {
      bad = true;
      d = T(1);
    }
    const T rl = wrsqrt(d);
    const T lit = lane > t ? G[0] * rl : T(0);
    if (lane == t) Hs[t][t] = d * rl;
    if (lane > t) Hs[lane][t] = lit;
#pragma unroll
    for (int j = 1; j < BM; ++j) {
      const T ljt = __shfl_sync(FULL, lit, (t + j) & (BM - 1));
      G[j - 1] = fma(-lit, ljt, G[j]);
    }
    G[BM - 1] = T(0);
  }
  if (lane == 0 && bad) atomicOr(err, ERRBIT_EIG);
  __syncwarp();
  // X = L^{-1} (lower, lane = row): row l is final at step l (up to the factor 1 / L_ll)
  const T rdi = lane < b ? T(1) / Hs[lane][lane] : T(1);
  T X[BM];
#pragma unroll
  for (int c = 0; c < BM; ++c) X[c] = c == lane ? T(1) : T(0);
  for (int l = 0; l < b; ++l) {
    const T rdl = __shfl_sync(FULL, rdi, l);
    const T f = lane > l && lane < b ? Hs[lane][l] * rdl : T(0);
#pragma unroll
    for (int c = 0; c < BM; ++c) {
      const T v = __shfl_sync(FULL, X[c], l);
      X[c] = fma(-f, v, X[c]);
    }
  }
#pragma unroll
  for (int c = 0; c < BM; ++c) Ys[lane][c] = X[c] * rdi;
  __syncwarp();
  // Mv(r, c) = sum_l Y(r, l) [use_v(l)] X(c, l), Mz(r, c) = sum_l Y(r, l) fz(l) X(c, l)
  if (lane < b) {
    T ya[BM], yz[BM];
#pragma unroll
    for (int l = 0; l < BM; ++l) {
      const T y = Ws[lane][l];
      ya[l] = usev_s[l] ? y : T(0);
      yz[l] = usev_s[l] ? T(0) : y * fz_s[l];
    }
    for (int c = 0; c < b; ++c) {
      T mv0 = T(0), mv1 = T(0), mz0 = T(0), mz1 = T(0);
#pragma unroll
      for (int l = 0; l < BM; l += 2) {
        const T x0 = Ys[c][l], x1 = Ys[c][l + 1];
        mv0 = fma(ya[l], x0, mv0);
        mv1 = fma(ya[l + 1], x1, mv1);
        mz0 = fma(yz[l], x0, mz0);
        mz1 = fma(yz[l + 1], x1, mz1);
      }
      const int e = lane + c * b;
      Yout[e] = Ws[lane][c];
      Mv[e] = mv0 + mv1;
      Mz[e] = mz0 + mz1;
    }
  }
}

// Subspace iteration, update (rows of V in place): Vs = (V Y)(:, :s) (the Ritz vectors
// kept for D, also written into the V_s part of Z2) and V <- V Mv + Z Mz.
template <typename T>
__global__ void __launch_bounds__(256)
eig_update(T* __restrict__ V, const T* __restrict__ Z, const T* __restrict__ Y,
           const T* __restrict__ Mv, const T* __restrict__ Mz, int n2, int b, int s, int k,
           int NP, T* __restrict__ Vs, T* __restrict__ Z2) {
  constexpr int RB = 8;
  __shared__ T Vr[RB][EIG_BMAX];
  __shared__ T Zr[RB][EIG_BMAX];
  const int j0 = blockIdx.x * RB;
  for (int e = threadIdx.x; e < RB * b; e += blockDim.x) {
    const int rr = e % RB, c = e / RB, j = j0 + rr;
    Vr[rr][c] = j < n2 ? V[j + (int64_t)c * n2] : T(0);
    Zr[rr][c] = j < n2 ? Z[j + (int64_t)c * n2] : T(0);
  }
  __syncthreads();
  for (int e = threadIdx.x; e < RB * b; e += blockDim.x) {
    const int rr = e % RB, c = e / RB, j = j0 + rr;
    if (j >= n2) continue;
    T vr = T(0), vn = T(0);
    for (int l = 0; l < b; ++l) {
      vr = fma(Vr[rr][l], Y[l + c * b], vr);
      vn = fma(Vr[rr][l], Mv[l + c * b], vn);
      vn = fma(Zr[rr][l], Mz[l + c * b], vn);
    }
    V[j + (int64_t)c * n2] = vn;
    if (c < s) {
      Vs[j + (int64_t)c * n2] = vr;
      Z2[(int64_t)j * NP + k + c] = vr;
    }
  }
}

// Random start for the subspace basis (orthonormalised by the first eig_small).
template <typename T>
__global__ void eig_random_start(T* __restrict__ V, int n2, int b, uint64_t seed) {
  const int total = n2 * b;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x)
    V[t] = (T)normal_at(seed ^ 0x5DEECE66Dull, (uint64_t)t);
}

// Copy the first s Ritz vectors (b >= n2 case, or s = 0 bookkeeping) is done by eig_update.

// G = C C^T (k x k) and CV = C V_s (k x s); block a computes row a.
template <typename T>
__global__ void prep_rowpass(const T* __restrict__ C, const T* __restrict__ Vs, int k, int n2,
                             int s, T* __restrict__ G, T* __restrict__ CV) {
  const int a = blockIdx.x;
  for (int t = threadIdx.x; t < k + s; t += blockDim.x) {
    T v = T(0);
    if (t < k) {
      for (int j = 0; j < n2; ++j) v = fma(C[a + (int64_t)j * k], C[t + (int64_t)j * k], v);
      G[a + t * k] = v;
    } else {
      const int c = t - k;
      for (int j = 0; j < n2; ++j) v = fma(C[a + (int64_t)j * k], Vs[j + (int64_t)c * n2], v);
      CV[a + c * k] = v;
    }
  }
}

// G = C C^T (k x k) and CV = C V_s (k x s) from Z2 = [C^T | V_s] (row-major n2 x NP):
// G(a,t) = sum_j Z2[j][a] Z2[j][t], CV(a,c) = sum_j Z2[j][a] Z2[j][k+c].  Each block
// sums 64 rows into a double partial; the last block to finish (counted with an atomic
// ticket after a memory fence, so it sees every partial) adds the partials in block
// order and resets the ticket for the next launch.  No block ever waits on another.
template <typename T>
__global__ void __launch_bounds__(256)
prep_gram(const T* __restrict__ Z2, int n2, int k, int s, int NP, double* __restrict__ part,
          unsigned int* __restrict__ ticket, T* __restrict__ G, T* __restrict__ CV) {
  constexpr int RB = 64;
  extern __shared__ unsigned char smem_raw[];
  T* Zr = reinterpret_cast<T*>(smem_raw);  // [RB][NP + 1]
  __shared__ bool is_last;
  const int tid = threadIdx.x;
  const int j0 = blockIdx.x * RB;
  const int ks = k + s, L = k * ks;
  for (int e = tid; e < RB * NP; e += blockDim.x) {
    const int r = e / NP, c = e % NP;
    Zr[r * (NP + 1) + c] = j0 + r < n2 ? Z2[(int64_t)(j0 + r) * NP + c] : T(0);
  }
  __syncthreads();
  for (int o = tid; o < L; o += blockDim.x) {
    const int a = o % k, t = o / k;
    T v = T(0);
#pragma unroll 8
    for (int r = 0; r < RB; ++r) v = fma(Zr[r * (NP + 1) + a], Zr[r * (NP + 1) + t], v);
    part[(int64_t)blockIdx.x * L + o] = (double)v;
  }
  __threadfence();
  __syncthreads();
  if (tid == 0) is_last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  for (int o = tid; o < L; o += blockDim.x) {
    double v = 0.0;
    for (int c = 0; c < (int)gridDim.x; ++c) v += __ldcg(&part[(int64_t)c * L + o]);
    const int a = o % k, t = o / k;
    if (t < k) G[a + t * k] = (T)v;
    else CV[a + (t - k) * k] = (T)v;
  }
  if (tid == 0) *ticket = 0u;
}

// --------------------------------------------------------------------------------
// Fused row pass (steps a4 + a5), BM = 64 rows per block, 256 threads.
//   Y = A2(rows,:) [C^T | V_s]                     (GEMM over n2, Z2 row-major n2 x NP)
//   U = Y_V - X1old(rows,:) (C V_s)                (= rows of U_s Sigma_s = P_perp A2 V_s)
//   E = A1 o W1^2 + Y_C - U (C V_s)^T              (= A1 o W1 o W1 + (A2 - D) C^T)
//   X1new(i,:) solves (diag(W1(i,:)^2) + C C^T) x = E(i,:)^T
// Also the block's partial of ||(A1 - X1old) o W1||_F^2.
constexpr int RP_BM = 64;
constexpr int RP_BK = 32;

// Compile-time size KP of the row systems: the smallest of 8, 16, 20, 24, 32, 64 that
// holds k (k <= 64).
inline int row_kp(int k) {
  return k <= 8 ? 8 : k <= 16 ? 16 : k <= 20 ? 20 : k <= 24 ? 24 : k <= 32 ? 32 : 64;
}

// Register row solve (phase 3 of row_pass) for a system padded to KP x KP: LG lanes
// share one row system, lane g holding the NS = KP / LG matrix rows q = g + LG*s in
// registers (KP = 64: a whole warp per system, two rows per lane).  Off for double beyond
// KP = 16 (register budget), where the shared-memory solve below runs instead.
template <typename T, int KP>
struct RegSolve {
  static constexpr bool on = sizeof(T) == 4 ? true : KP <= 16;
  static constexpr int LG = (KP <= 8 || (sizeof(T) == 4 && KP <= 20)) ? 4 : (KP <= 32 ? 8 : 32);
  static constexpr int NS = KP / LG;
};

// Shared-memory row-solve layout (phase 3 of row_pass when the register solve is off).
// LG lanes factor one row's k x k system, held in shared memory as a square
// column-major block with an even leading dimension ld (so the diagonal walk
// j*ld + j + i of the trailing update has odd stride ld + 1 across lanes) and a per-row
// pitch P = LG*(ld + 1) (mod 32), which puts the 32 lanes of a warp on 32 distinct banks.
// R rows are solved per pass, R limited by a 96 KB budget and rounded to whole warps.
template <typename T, int KMAX>
struct RowSolveLayout {
  static constexpr int LG = KMAX <= 8 ? 4 : (KMAX <= 32 ? 8 : 32);
  __host__ __device__ static int ld(int k) { return k + (k & 1); }
  __host__ __device__ static int pitch(int k) {
    const int l = ld(k), want = (LG * (l + 1)) & 31;
    int p = k * l;
    while ((p & 31) != want) ++p;
    return p;
  }
  __host__ __device__ static int rows(int k) {
    const int per_warp = 32 / LG;
    int r = (int)((96 * 1024) / ((size_t)pitch(k) * sizeof(T)));
    r = r < 256 / LG ? r : 256 / LG;
    r = (r / per_warp) * per_warp;
    return r < per_warp ? per_warp : r;
  }
};

// Shared memory of row_pass.  Region 0 holds the phase-1 staging (A2 and Z2 slabs), then
// U (phase 2), then, for the shared-memory solve, the row systems (phase 3); the rows of
// X1old, A1 and W1 are staged for float only (double reads them from global memory to
// keep within 227 KB).
template <typename T>
struct RowPassSmem {
  static constexpr bool kStage = sizeof(T) == 4;
  static constexpr int kStages = sizeof(T) == 4 ? 4 : 2;   // phase-1 pipeline depth
  template <int KP>
  __host__ __device__ static size_t region0(int NP, int k) {
    const size_t stage = (size_t)kStages * ((size_t)RP_BK * RP_BM + (size_t)RP_BK * NP);
    const size_t us = (size_t)RP_BM * (EIG_BMAX + 1);
    const size_t rs = RegSolve<T, KP>::on ? 0
                      : (size_t)RowSolveLayout<T, KP>::rows(k) * RowSolveLayout<T, KP>::pitch(k);
    size_t r0 = stage > us ? stage : us;
    return r0 > rs ? r0 : rs;
  }
  template <int KP>
  static size_t bytes_k(int NP, int k, int s) {
    return sizeof(T) * (region0<KP>(NP, k) + (size_t)RP_BM * (NP + 1) + (size_t)k * k +
                        (size_t)k * (s > 0 ? s : 1) + (kStage ? 3 * (size_t)RP_BM * (k + 1) : 0) +
                        (size_t)k * k);
  }
  static size_t bytes(int NP, int k, int s) {
    switch (row_kp(k)) {
      case 8: return bytes_k<8>(NP, k, s);
      case 16: return bytes_k<16>(NP, k, s);
      case 20: return bytes_k<20>(NP, k, s);
      case 24: return bytes_k<24>(NP, k, s);
      case 32: return bytes_k<32>(NP, k, s);
      default: return bytes_k<64>(NP, k, s);
    }
  }
};

// Optional output of row_pass (float, steady state of the tensor-core path): the rows of
// Q1 = X1new R^{-1} for the next CholeskyQR (R^{-1}: k x k upper triangular, column-major,
// the previous iteration's factor) as a TF32 pair h + l (h = round_tf32(q),
// l = round_tf32(q - h)), leading dimension ld.  h == nullptr: not formed.
struct QSplitOut {
  float* h;
  float* l;
  int64_t ld;
  const float* R;
};

// Objective finalisation done by the last row_pass block (ticket != nullptr):
// F_p = sum(wpart) + ||A2||^2 - sum(bpart) - sum_{c<s} theta_c into Fhist[*iter], *iter += 1.
template <typename T>
struct FinalizeArgs {
  const double* bpart;
  int nb;
  const double* normA2;
  const T* theta;
  double* Fhist;
  int hist_cap;
  int* iter;
  double* Fcur;
  unsigned int* ticket;
};

// 16-byte asynchronous copy global -> shared (zero-filled beyond src_bytes).
__device__ __forceinline__ void cp_async16(void* dst_smem, const void* src, int src_bytes) {
  const unsigned dst = (unsigned)__cvta_generic_to_shared(dst_smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src),
               "r"(src_bytes));
}

// N consecutive shared-memory elements, in the widest aligned vector loads.
template <int N>
__device__ __forceinline__ void load_n(float (&z)[N], const float* p) {
  if constexpr (N % 4 == 0) {
#pragma unroll
    for (int v = 0; v < N; v += 4) {
      const float4 t = *reinterpret_cast<const float4*>(p + v);
      z[v] = t.x; z[v + 1] = t.y; z[v + 2] = t.z; z[v + 3] = t.w;
    }
  } else if constexpr (N % 2 == 0) {
#pragma unroll
    for (int v = 0; v < N; v += 2) {
      const float2 t = *reinterpret_cast<const float2*>(p + v);
      z[v] = t.x; z[v + 1] = t.y;
    }
  } else {
#pragma unroll
    for (int v = 0; v < N; ++v) z[v] = p[v];
  }
}
template <int N>
__device__ __forceinline__ void load_n(double (&z)[N], const double* p) {
  if constexpr (N % 2 == 0) {
#pragma unroll
    for (int v = 0; v < N; v += 2) {
      const double2 t = *reinterpret_cast<const double2*>(p + v);
      z[v] = t.x; z[v + 1] = t.y;
    }
  } else {
#pragma unroll
    for (int v = 0; v < N; ++v) z[v] = p[v];
  }
}

__device__ __forceinline__ float wrcp(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double wrcp(double x) { return 1.0 / x; }

// Phase 1 of row_pass: Ys[r][c] = sum_j A2(i0 + r, j) Z2(j, c) for the block's 64 rows and
// the NP = 16 * NPU columns, with A2 and Z2 streamed through shared memory in slabs of 32
// columns by an S-stage cp.async pipeline (S - 1 slabs in flight while one is consumed).
// Thread (rg, cg) = (tid / 16, tid % 16) owns rows 4 rg .. 4 rg + 3 and columns
// cg NPU .. cg NPU + NPU - 1: one 4-row vector of A2 and one NPU-vector of Z2 per step.
// vec: A2 and lda allow 16-byte copies (rows of a slab column move 16 bytes at a time).
template <typename T, int NPU>
__device__ __forceinline__ void rp_phase1(const T* __restrict__ A2, int64_t lda,
                                          const T* __restrict__ Z2, int m, int n2, int i0,
                                          bool vec, T* __restrict__ As, T* __restrict__ Ys) {
  constexpr int NP = 16 * NPU;
  constexpr int S = RowPassSmem<T>::kStages;
  constexpr int CH = 16 / sizeof(T);                 // elements per 16-byte chunk
  constexpr int slab = RP_BK * RP_BM + RP_BK * NP;   // elements per stage
  const int tid = threadIdx.x;
  const int cg = tid & 15, rg = tid >> 4;
  T acc[4][NPU];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < NPU; ++v) acc[u][v] = T(0);
  const int nsl = (n2 + RP_BK - 1) / RP_BK;
  auto issue = [&](int sl) {
    if (sl < nsl) {
      T* As_ = As + (size_t)(sl % S) * slab;
      T* Zs_ = As_ + RP_BK * RP_BM;
      const int j0 = sl * RP_BK;
      if (vec) {
        for (int e = tid; e < RP_BK * RP_BM / CH; e += 256) {
          const int rc = e % (RP_BM / CH), kk = e / (RP_BM / CH);
          const int i = i0 + CH * rc, j = j0 + kk;
          T* dst = As_ + kk * RP_BM + CH * rc;
          if (j >= n2 || i >= m) {
            cp_async16(dst, A2, 0);
          } else if (i + CH <= m) {
            cp_async16(dst, A2 + i + (int64_t)j * lda, 16);
          } else {
#pragma unroll
            for (int c = 0; c < CH; ++c) {
              const bool ok = i + c < m;
              cp_async_elem(dst + c, ok ? A2 + i + c + (int64_t)j * lda : A2, ok);
            }
          }
        }
      } else {
        for (int e = tid; e < RP_BK * RP_BM; e += 256) {
          const int r = e % RP_BM, kk = e / RP_BM;
          const int i = i0 + r, j = j0 + kk;
          const bool ok = i < m && j < n2;
          cp_async_elem(As_ + kk * RP_BM + r, ok ? A2 + i + (int64_t)j * lda : A2, ok);
        }
      }
      for (int e = tid; e < RP_BK * NP / CH; e += 256) {
        const bool ok = j0 + (CH * e) / NP < n2;
        cp_async16(Zs_ + CH * e, ok ? Z2 + (int64_t)j0 * NP + CH * e : Z2, ok ? 16 : 0);
      }
    }
    cp_async_commit();
  };
#pragma unroll 1
  for (int sl = 0; sl < S - 1; ++sl) issue(sl);
#pragma unroll 1
  for (int sl = 0; sl < nsl; ++sl) {
    cp_async_wait<S - 2>();
    __syncthreads();
    issue(sl + S - 1);
    const T* As_ = As + (size_t)(sl % S) * slab + 4 * rg;
    const T* Zs_ = As + (size_t)(sl % S) * slab + RP_BK * RP_BM + cg * NPU;
#pragma unroll 8
    for (int kk = 0; kk < RP_BK; ++kk) {
      T a[4], z[NPU];
      load4(a, As_ + kk * RP_BM);
      load_n<NPU>(z, Zs_ + kk * NP);
#pragma unroll
      for (int v = 0; v < NPU; ++v)
#pragma unroll
        for (int u = 0; u < 4; ++u) acc[u][v] = fma(a[u], z[v], acc[u][v]);
    }
  }
  cp_async_wait<0>();
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < NPU; ++v) Ys[(4 * rg + u) * (NP + 1) + cg * NPU + v] = acc[u][v];
}

// Phase 1 with each slab split over four groups of 64 threads (float, NP <= 64): group kg
// takes the steps kk = 8 kg .. 8 kg + 7 of every slab, and its thread (rg, cg) =
// (t / 8, t % 8) owns rows 8 rg .. 8 rg + 7 and columns cg CB .. cg CB + CB - 1 (CB = NP / 8):
// two 4-row vectors of A2 and one CB-vector of Z2 per step for 8 CB products (four times
// the products per shared-memory load of rp_phase1, and 8 CB independent sums per thread).
// After the last slab the groups' sums go to the stage buffers and Ys takes them in group
// order.
template <int NPU>
__device__ __forceinline__ void rp_phase1_ks(const float* __restrict__ A2, int64_t lda,
                                             const float* __restrict__ Z2, int m, int n2, int i0,
                                             bool vec, float* __restrict__ As, float* __restrict__ Ys) {
  using T = float;
  constexpr int NP = 16 * NPU, CB = NP / 8;
  constexpr int S = RowPassSmem<T>::kStages;
  constexpr int CH = 16 / sizeof(T);
  constexpr int slab = RP_BK * RP_BM + RP_BK * NP;
  static_assert(4 * RP_BM * NP <= S * slab, "the group sums fit in the stage buffers");
  const int tid = threadIdx.x;
  const int kg = tid >> 6, rg = (tid & 63) >> 3, cg = tid & 7;
  T acc[8][CB];
#pragma unroll
  for (int u = 0; u < 8; ++u)
#pragma unroll
    for (int v = 0; v < CB; ++v) acc[u][v] = T(0);
  const int nsl = (n2 + RP_BK - 1) / RP_BK;
  auto issue = [&](int sl) {
    if (sl < nsl) {
      T* As_ = As + (size_t)(sl % S) * slab;
      T* Zs_ = As_ + RP_BK * RP_BM;
      const int j0 = sl * RP_BK;
      if (vec) {
        for (int e = tid; e < RP_BK * RP_BM / CH; e += 256) {
          const int rc = e % (RP_BM / CH), kk = e / (RP_BM / CH);
          const int i = i0 + CH * rc, j = j0 + kk;
          T* dst = As_ + kk * RP_BM + CH * rc;
          if (j >= n2 || i >= m) {
            cp_async16(dst, A2, 0);
          } else if (i + CH <= m) {
            cp_async16(dst, A2 + i + (int64_t)j * lda, 16);
          } else {
#pragma unroll
            for (int c = 0; c < CH; ++c) {
              const bool ok = i + c < m;
              cp_async_elem(dst + c, ok ? A2 + i + c + (int64_t)j * lda : A2, ok);
            }
          }
        }
      } else {
        for (int e = tid; e < RP_BK * RP_BM; e += 256) {
          const int r = e % RP_BM, kk = e / RP_BM;
          const int i = i0 + r, j = j0 + kk;
          const bool ok = i < m && j < n2;
          cp_async_elem(As_ + kk * RP_BM + r, ok ? A2 + i + (int64_t)j * lda : A2, ok);
        }
      }
      for (int e = tid; e < RP_BK * NP / CH; e += 256) {
        const bool ok = j0 + (CH * e) / NP < n2;
        cp_async16(Zs_ + CH * e, ok ? Z2 + (int64_t)j0 * NP + CH * e : Z2, ok ? 16 : 0);
      }
    }
    cp_async_commit();
  };
#pragma unroll 1
  for (int sl = 0; sl < S - 1; ++sl) issue(sl);
#pragma unroll 1
  for (int sl = 0; sl < nsl; ++sl) {
    cp_async_wait<S - 2>();
    __syncthreads();
    issue(sl + S - 1);
    const T* As_ = As + (size_t)(sl % S) * slab + 8 * rg + (size_t)(8 * kg) * RP_BM;
    const T* Zs_ = As + (size_t)(sl % S) * slab + RP_BK * RP_BM + cg * CB + (size_t)(8 * kg) * NP;
#pragma unroll
    for (int kk = 0; kk < 8; ++kk) {
      T a[4], b4[4], z[CB];
      load4(a, As_ + kk * RP_BM);
      load4(b4, As_ + kk * RP_BM + 4);
      load_n<CB>(z, Zs_ + kk * NP);
#pragma unroll
      for (int v = 0; v < CB; ++v) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          acc[u][v] = fma(a[u], z[v], acc[u][v]);
          acc[4 + u][v] = fma(b4[u], z[v], acc[4 + u][v]);
        }
      }
    }
  }
  cp_async_wait<0>();
  __syncthreads();
  T* Pk = As;   // group kg's sums: Pk[(kg RP_BM + r) NP + c]
#pragma unroll
  for (int u = 0; u < 8; ++u)
#pragma unroll
    for (int v = 0; v < CB; ++v) Pk[(size_t)(kg * RP_BM + 8 * rg + u) * NP + cg * CB + v] = acc[u][v];
  __syncthreads();
  for (int e = tid; e < RP_BM * NP; e += 256) {
    const int r = e / NP, c = e % NP;
    T v = Pk[e];
    v += Pk[RP_BM * NP + e];
    v += Pk[2 * RP_BM * NP + e];
    v += Pk[3 * RP_BM * NP + e];
    Ys[r * (NP + 1) + c] = v;
  }
}

// Row i of Q1 = X1new R^{-1} (QSplitOut) from the row's solution, held by a group of LG
// lanes (lane g: x[sl] = X1new(i, g + LG sl)): q_a = sum_b x_b R^{-1}(b, a), summed in the
// order b = 0, 1, ..., then split into TF32 h + l.  R^{-1} may be a full matrix (after the
// series form of the second factor); when it is upper triangular the terms below the
// diagonal are exact zeros.
template <typename T, int KP, int LG, int NS>
__device__ __forceinline__ void q_split_row(const T (&x)[NS], const T* __restrict__ Rqs, int k, int g,
                                            bool active, int i, const QSplitOut& qo) {
  constexpr unsigned FULL = 0xffffffffu;
  T qa[NS];
#pragma unroll
  for (int sl = 0; sl < NS; ++sl) qa[sl] = T(0);
#pragma unroll
  for (int bq = 0; bq < KP; ++bq) {
    if (bq < k) {
      const T xb = __shfl_sync(FULL, x[bq / LG], bq % LG, LG);
#pragma unroll
      for (int sl = 0; sl < NS; ++sl) {
        const int a = g + LG * sl;
        if (a < k) qa[sl] = fma(xb, Rqs[bq + a * k], qa[sl]);
      }
    }
  }
  if (active) {
#pragma unroll
    for (int sl = 0; sl < NS; ++sl) {
      const int a = g + LG * sl;
      if (a < k) {
        const float v = (float)qa[sl];
        const float h = round_tf32(v);
        qo.h[i + (int64_t)a * qo.ld] = h;
        qo.l[i + (int64_t)a * qo.ld] = round_tf32(v - h);
      }
    }
  }
}

// Gauss-Jordan steps t0 <= t < t1 of a row system held by a group of LG lanes (phase 3 of
// row_pass): lane g holds rows q = g + LG sl (sl < NS) shifted so that R[sl][jj] =
// M(q, t + jj) at step t, i.e. the pivot column is always R[sl][0] and the loop body does
// not depend on t (a rolled loop: the code stays small enough for the instruction cache).
// The pivot rows of these steps sit in slot ST (lane t - LG ST).  Step t: d_t = M(t,t), and
// every row q != t (above the pivot too) takes M(q, j) -= M(q,t) M(t,j) / d_t for j > t and
// e_q -= M(q,t) e_t / d_t, while all rows shift one place left.  After the last step M is
// diagonal with the pivots d_q of the steps, so x_q = e_q / d_q (rd holds 1 / d_q); no factor
// has to be kept for a back substitution.
template <typename T, int KP, int LG, int NS, int ST>
__device__ __forceinline__ void gj_steps(T (&R)[NS][KP], T (&e)[NS], T (&rd)[NS], int t0, int t1, int k,
                                         int g, bool active, bool& bad) {
  constexpr unsigned FULL = 0xffffffffu;
#pragma unroll 1
  for (int t = t0; t < t1; ++t) {
    const int ot = t - LG * ST;
    T d = __shfl_sync(FULL, R[ST][0], ot, LG);
    if (!(d > T(0)) || !wfinite(d)) {
      bad = bad || active;
      d = T(1);
    }
    const T rdt = wrcp(d);
    if (g == ot) rd[ST] = rdt;
    const T et = __shfl_sync(FULL, e[ST], ot, LG);
    T f[NS];
#pragma unroll
    for (int sl = 0; sl < NS; ++sl) {
      f[sl] = (g + LG * sl != t) ? R[sl][0] * rdt : T(0);
      e[sl] = fma(-f[sl], et, e[sl]);
    }
    // columns t .. k - 1 remain (positions 0 .. rem - 1).  Groups of 8 positions: the 8
    // shuffles of a group are in flight together; positions of the last group beyond rem
    // take values that no later step reads.
    const int rem = k - t;
#pragma unroll
    for (int j0 = 1; j0 < KP; j0 += 8) {
      if (j0 < rem) {
        T mj[8];
#pragma unroll
        for (int u = 0; u < 8; ++u)
          if (j0 + u < KP) mj[u] = __shfl_sync(FULL, R[ST][j0 + u], ot, LG);
#pragma unroll
        for (int u = 0; u < 8; ++u)
          if (j0 + u < KP) {
#pragma unroll
            for (int sl = 0; sl < NS; ++sl) R[sl][j0 + u - 1] = fma(-f[sl], mj[u], R[sl][j0 + u]);
          }
      }
    }
  }
}
// All k steps: the pivots of steps LG ST .. LG ST + LG - 1 are in slot ST.
template <typename T, int KP, int LG, int NS, int ST = 0>
__device__ __forceinline__ void gj_all(T (&R)[NS][KP], T (&e)[NS], T (&rd)[NS], int k, int g, bool active,
                                       bool& bad) {
  if constexpr (ST < NS) {
    gj_steps<T, KP, LG, NS, ST>(R, e, rd, LG * ST, min(k, LG * (ST + 1)), k, g, active, bad);
    gj_all<T, KP, LG, NS, ST + 1>(R, e, rd, k, g, active, bad);
  }
}

template <typename T, int KP>
__global__ void __launch_bounds__(256)
row_pass(const T* __restrict__ A, int64_t lda, const T* __restrict__ W1, int64_t ldw,
         const T* __restrict__ X1old, const T* __restrict__ Z2, const T* __restrict__ Gm,
         const T* __restrict__ CV, int m, int n2, int k, int s, int NP, T* __restrict__ X1new,
         double* __restrict__ wpart, int* __restrict__ err, FinalizeArgs<T> fin, QSplitOut qo) {
  extern __shared__ unsigned char smem_raw[];
  constexpr bool kStage = RowPassSmem<T>::kStage;
  T* As = reinterpret_cast<T*>(smem_raw);   // phase-1 stages               (phase 1)
  T* Us = As;                               // [RP_BM][EIG_BMAX+1]          (phase 2)
  T* Ms = As;                               // shared-memory row systems    (phase 3)
  T* Ys = As + RowPassSmem<T>::template region0<KP>(NP, k);  // [RP_BM][NP+1]
  T* Gs = Ys + RP_BM * (NP + 1);            // [k][k]
  T* CVs = Gs + k * k;                      // [k][s]
  T* Xo = CVs + k * (s > 0 ? s : 1);        // [RP_BM][k+1]  X1old rows (float)
  T* A1s = Xo + RP_BM * (k + 1);            // [RP_BM][k+1]  A1 rows    (float)
  T* W1s = A1s + RP_BM * (k + 1);           // [RP_BM][k+1]  W1 rows    (float)
  T* Rqs = W1s + RP_BM * (k + 1);           // [k][k]        R^{-1} for Q1 (float)
  __shared__ double sh[32];
  // the Q1 output exists in the float row passes with KP <= 32 (for 32 < k <= 64 the one-warp
  // elimination needs its registers, and a separate split kernel is cheaper)
  constexpr bool kQ = sizeof(T) == 4 && KP <= 32;
  const bool qon = kQ && qo.h != nullptr;

  const int tid = threadIdx.x;
  const int i0 = blockIdx.x * RP_BM;
  const T* A2 = A + (int64_t)k * lda;
  const int kp = k + 1;
  // row r of the block, column a, of X1old / A1 / W1 (zero / one outside the matrix)
  auto xo_at = [&](int r, int a) -> T {
    if (kStage) return Xo[r * kp + a];
    return i0 + r < m ? X1old[(i0 + r) + (int64_t)a * m] : T(0);
  };
  auto a1_at = [&](int r, int a) -> T {
    if (kStage) return A1s[r * kp + a];
    return i0 + r < m ? A[(i0 + r) + (int64_t)a * lda] : T(0);
  };
  auto w1_at = [&](int r, int a) -> T {
    if (kStage) return W1s[r * kp + a];
    return i0 + r < m ? W1[(i0 + r) + (int64_t)a * ldw] : T(1);
  };

  // G, C V_s and (float) the block's rows of X1old, A1 and W1, copied asynchronously in
  // the first phase-1 copy group (rows outside the matrix read as zero; phases 2 and 3
  // never use them).
  for (int e = tid; e < k * k; e += 256) cp_async_elem(Gs + e, Gm + e, true);
  for (int e = tid; e < k * s; e += 256) cp_async_elem(CVs + e, CV + e, true);
  if (qon)
    for (int e = tid; e < k * k; e += 256) cp_async_elem(Rqs + e, reinterpret_cast<const T*>(qo.R) + e, true);
  if (kStage) {
    for (int e = tid; e < RP_BM * k; e += 256) {
      const int r = e % RP_BM, a = e / RP_BM;
      const int i = i0 + r;
      const bool ok = i < m;
      cp_async_elem(Xo + r * kp + a, ok ? X1old + i + (int64_t)a * m : X1old, ok);
      cp_async_elem(A1s + r * kp + a, ok ? A + i + (int64_t)a * lda : A, ok);
      cp_async_elem(W1s + r * kp + a, ok ? W1 + i + (int64_t)a * ldw : W1, ok);
    }
  }

  // ---- phase 1: Y = A2 rows * Z2
  {
    const bool vec = ((reinterpret_cast<uintptr_t>(A2) & 15) == 0) &&
                     (((uint64_t)lda * sizeof(T)) % 16 == 0);
    if constexpr (sizeof(T) == 4) {
      switch (NP / 16) {
        case 1: rp_phase1_ks<1>(A2, lda, Z2, m, n2, i0, vec, As, Ys); break;
        case 2: rp_phase1_ks<2>(A2, lda, Z2, m, n2, i0, vec, As, Ys); break;
        case 3: rp_phase1_ks<3>(A2, lda, Z2, m, n2, i0, vec, As, Ys); break;
        case 4: rp_phase1_ks<4>(A2, lda, Z2, m, n2, i0, vec, As, Ys); break;
        case 5: rp_phase1<T, 5>(A2, lda, Z2, m, n2, i0, vec, As, Ys); break;
        default: rp_phase1<T, 6>(A2, lda, Z2, m, n2, i0, vec, As, Ys); break;
      }
    } else {
      switch (NP / 16) {
        case 1: rp_phase1<T, 1>(A2, lda, Z2, m, n2, i0, vec, As, Ys); break;
        case 2: rp_phase1<T, 2>(A2, lda, Z2, m, n2, i0, vec, As, Ys); break;
        case 3: rp_phase1<T, 3>(A2, lda, Z2, m, n2, i0, vec, As, Ys); break;
        case 4: rp_phase1<T, 4>(A2, lda, Z2, m, n2, i0, vec, As, Ys); break;
        case 5: rp_phase1<T, 5>(A2, lda, Z2, m, n2, i0, vec, As, Ys); break;
        default: rp_phase1<T, 6>(A2, lda, Z2, m, n2, i0, vec, As, Ys); break;
      }
    }
  }
  __syncthreads();

  // ---- phase 2a: U = Y_V - X1old C V_s
  for (int e = tid; e < RP_BM * s; e += 256) {
    const int r = e % RP_BM, c = e / RP_BM;
    T v = Ys[r * (NP + 1) + k + c];
    for (int a = 0; a < k; ++a) v -= xo_at(r, a) * CVs[a + c * k];
    Us[r * (EIG_BMAX + 1) + c] = v;
  }
  __syncthreads();

  // ---- phase 2b: E (into Ys[:, :k]) and the weighted objective term
  WideAcc<T> wacc;
  for (int e = tid; e < RP_BM * k; e += 256) {
    const int r = e % RP_BM, a = e / RP_BM;
    if (i0 + r >= m) continue;
    const T w = w1_at(r, a);
    const T a1 = a1_at(r, a);
    const T xo = xo_at(r, a);
    T v = a1 * w * w + Ys[r * (NP + 1) + a];
    for (int c = 0; c < s; ++c) v -= Us[r * (EIG_BMAX + 1) + c] * CVs[a + c * k];
    Ys[r * (NP + 1) + a] = v;
    const T d = (a1 - xo) * w;
    wacc.add(d * d);
  }
  const double wsum = block_sum_wide(wacc, sh);
  if (tid == 0) wpart[blockIdx.x] = wsum;
  __syncthreads();

  // ---- phase 3: row solves M x = e, M = diag(W1(i,:)^2) + C C^T (symmetric positive
  // definite), e = E(i,:)^T.
  bool bad = false;
  if constexpr (RegSolve<T, KP>::on) {
    // Gauss-Jordan in registers (gj_all): LG lanes per row system, 256 / LG systems per pass
    constexpr int LG = RegSolve<T, KP>::LG, NS = RegSolve<T, KP>::NS;
    constexpr int GPB = 256 / LG;
    const int g = tid % LG, grp = tid / LG;
#pragma unroll 1
    for (int base = 0; base < RP_BM; base += GPB) {
      const int r = base + grp;                    // GPB divides RP_BM: r < RP_BM
      const bool active = i0 + r < m;
      T R[NS][KP], e[NS], rd[NS];
#pragma unroll
      for (int sl = 0; sl < NS; ++sl) {
        const int q = g + LG * sl;
        const bool qk = q < k;
        const T w = (active && qk) ? w1_at(r, q) : T(1);
#pragma unroll
        for (int j = 0; j < KP; ++j) {
          const T gv = (qk && j < k) ? Gs[q + j * k] : T(0);
          R[sl][j] = q == j ? gv + w * w : gv;
        }
        e[sl] = (active && qk) ? Ys[r * (NP + 1) + q] : T(0);
        rd[sl] = T(1);
      }
      gj_all<T, KP, LG, NS>(R, e, rd, k, g, active, bad);
      T x[NS];
#pragma unroll
      for (int sl = 0; sl < NS; ++sl) x[sl] = e[sl] * rd[sl];
      if (active) {
#pragma unroll
        for (int sl = 0; sl < NS; ++sl) {
          const int q = g + LG * sl;
          if (q < k) X1new[(i0 + r) + (int64_t)q * m] = x[sl];
        }
      }
      if constexpr (kQ) {
        if (qon) q_split_row<T, KP, LG, NS>(x, Rqs, k, g, active, i0 + r, qo);
      }
    }
  } else {
    // A group of LG lanes factors one row's system in shared memory (lower triangle,
    // right-looking Cholesky: at step t the lanes scale column t, then each lane updates
    // its own columns j > t down from the diagonal), then runs the two triangular solves
    // on E(i,:) in place.
    using Lay = RowSolveLayout<T, KP>;
    constexpr int LG = Lay::LG;
    const int ld = Lay::ld(k), P = Lay::pitch(k), R = Lay::rows(k);
    const int grp = tid / LG, g = tid % LG;
    T* M = Ms + (size_t)grp * P;
    for (int base = 0; base < RP_BM; base += R) {
      const int r = base + grp;
      const bool in = grp < R && r < RP_BM;
      const bool active = in && i0 + r < m;
      if (in) {
        for (int j = g; j < k; j += LG) {
          const T w = w1_at(r, j);
          for (int q = j; q < k; ++q) M[j * ld + q] = Gs[q + j * k] + (q == j ? w * w : T(0));
        }
      }
      __syncwarp();
      T* e = Ys + (size_t)(in ? r : 0) * (NP + 1);
      // Cholesky with the forward solve L y = e folded in: at step t column t of L is
      // final, so y_t = e_t / L_tt and e_q -= L_qt y_t (q > t) join the trailing update.
      // The diagonal is left holding 1 / L_tt for the backward solve.
      for (int t = 0; t < k; ++t) {
        T piv = in ? M[t * ld + t] : T(1);
        if (!(piv > T(0)) || !wfinite(piv)) {
          bad = bad || active;
          piv = T(1);
        }
        const T rl = wrsqrt(piv);
        const T yt = in ? e[t] * rl : T(0);
        __syncwarp();
        if (in) {
          for (int q = t + 1 + g; q < k; q += LG) M[t * ld + q] *= rl;
          if (g == 0) {
            M[t * ld + t] = rl;
            e[t] = yt;
          }
        }
        __syncwarp();
        if (in) {
          const T* __restrict__ Mt = M + t * ld;
          for (int q = t + 1 + g; q < k; q += LG) e[q] = fma(-Mt[q], yt, e[q]);
          for (int j = t + 1 + g; j < k; j += LG) {
            const T ljt = Mt[j];
            T* __restrict__ Mj = M + j * ld;
            int q = j;
            for (; q + 4 <= k; q += 4) {
              const T a0 = Mt[q], a1 = Mt[q + 1], a2 = Mt[q + 2], a3 = Mt[q + 3];
              const T b0 = Mj[q], b1 = Mj[q + 1], b2 = Mj[q + 2], b3 = Mj[q + 3];
              Mj[q] = fma(-a0, ljt, b0);
              Mj[q + 1] = fma(-a1, ljt, b1);
              Mj[q + 2] = fma(-a2, ljt, b2);
              Mj[q + 3] = fma(-a3, ljt, b3);
            }
            for (; q < k; ++q) Mj[q] = fma(-Mt[q], ljt, Mj[q]);
          }
        }
        __syncwarp();
      }
      // backward: L^T x = y (column-oriented; L(t,q) for t > q is M[q*ld + t];
      // the diagonal holds 1 / L_tt)
      for (int t = k - 1; t >= 0; --t) {
        if (in && g == 0) e[t] = e[t] * M[t * ld + t];
        __syncwarp();
        if (in) {
          const T xt = e[t];
          for (int q = g; q < t; q += LG) e[q] = fma(-M[q * ld + t], xt, e[q]);
        }
        __syncwarp();
      }
      if (active)
        for (int a = g; a < k; a += LG) X1new[(i0 + r) + (int64_t)a * m] = e[a];
      __syncwarp();
    }
  }
  if (bad) atomicOr(err, ERRBIT_NOT_SPD);
  if (fin.ticket != nullptr) {
    // the last block to finish adds the block partials (in block order) into F_p
    __shared__ bool is_last;
    __threadfence();
    __syncthreads();
    if (tid == 0) is_last = atomicAdd(fin.ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    if (is_last) {
      __threadfence();
      double w = 0.0, bn = 0.0;
      for (int e = tid; e < (int)gridDim.x; e += 256) w += __ldcg(&wpart[e]);
      for (int e = tid; e < fin.nb; e += 256) bn += __ldcg(&fin.bpart[e]);
      w = block_sum_double(w, sh);
      __syncthreads();
      bn = block_sum_double(bn, sh);
      if (tid == 0) {
        double t = 0.0;
        for (int c = 0; c < s; ++c) t += (double)fin.theta[c];
        const double F = w + (*fin.normA2 - bn - t);
        const int p = *fin.iter;
        if (p < fin.hist_cap) fin.Fhist[p] = F;
        *fin.Fcur = F;
        *fin.iter = p + 1;
        *fin.ticket = 0u;
      }
    }
  }
}

// Host-side: the row_pass instantiation for k (see row_kp).
template <typename T>
using RowPassFn = void (*)(const T*, int64_t, const T*, int64_t, const T*, const T*, const T*,
                           const T*, int, int, int, int, int, T*, double*, int*, FinalizeArgs<T>, QSplitOut);
template <typename T>
RowPassFn<T> row_pass_fn(int k) {
  switch (row_kp(k)) {
    case 8: return row_pass<T, 8>;
    case 16: return row_pass<T, 16>;
    case 20: return row_pass<T, 20>;
    case 24: return row_pass<T, 24>;
    case 32: return row_pass<T, 32>;
    default: return row_pass<T, 64>;
  }
}

// --------------------------------------------------------------------------------
// X2 pass (exact evaluation).  For the current factors (X1, Z2 = [C^T | V_s], CV) and,
// optionally, a previous set (X1p, Z2p, CVp), per block of 64 rows:
//   u = A2 V_s - X1 (C V_s),  X2 = X1 C + u V_s^T   (= X1 C + D)
//   acc[0] += ||A2 - X2||^2, acc[1] += ||X2 - X2p||^2, acc[2] += ||X2p||^2,
//   acc[3] += ||X1 - X1p||^2, acc[4] += ||X1p||^2, acc[5] += ||(A1 - X1) o W1||^2
// and writes X2 (m x n2, ldo) when out != nullptr.  Partials: part[blk*8 + q] (double).
template <typename T>
__device__ void x2_rows_uv(const T* __restrict__ A2, int64_t lda, const T* __restrict__ X1,
                           const T* __restrict__ Z2, const T* __restrict__ CV, int m, int n2,
                           int k, int s, int NP, int i0, T* As, T* Zs, T* Ws) {
  // Ws[r][0..k) = X1 rows, Ws[r][k..k+s) = u rows.  Uses As/Zs as GEMM staging.
  const int tid = threadIdx.x;
  // GEMM for y_V = A2 rows * V_s (columns k..k+s of Z2)
  T acc[8];
  const int r = tid % RP_BM, cg = tid / RP_BM;  // 4 column groups
#pragma unroll
  for (int v = 0; v < 8; ++v) acc[v] = T(0);
  for (int j0 = 0; j0 < n2 && s > 0; j0 += RP_BK) {
    __syncthreads();
    for (int e = tid; e < RP_BK * RP_BM; e += 256) {
      const int rr = e % RP_BM, kk = e / RP_BM;
      const int i = i0 + rr, j = j0 + kk;
      As[kk * RP_BM + rr] = (i < m && j < n2) ? A2[i + (int64_t)j * lda] : T(0);
    }
    for (int e = tid; e < RP_BK * EIG_BMAX; e += 256) {
      const int kk = e / EIG_BMAX, c = e % EIG_BMAX;
      const int j = j0 + kk;
      Zs[kk * EIG_BMAX + c] = (j < n2 && c < s) ? Z2[(int64_t)j * NP + k + c] : T(0);
    }
    __syncthreads();
    for (int kk = 0; kk < RP_BK; ++kk) {
      const T a = As[kk * RP_BM + r];
#pragma unroll
      for (int v = 0; v < 8; ++v) acc[v] = fma(a, Zs[kk * EIG_BMAX + cg + 4 * v], acc[v]);
    }
  }
  __syncthreads();
  const int i = i0 + r;
#pragma unroll
  for (int v = 0; v < 8; ++v) {
    const int c = cg + 4 * v;
    if (c < s) {
      T u = acc[v];
      if (i < m)
        for (int a = 0; a < k; ++a) u -= X1[i + (int64_t)a * m] * CV[a + c * k];
      Ws[r * (NP + 1) + k + c] = u;
    }
  }
  for (int e = tid; e < RP_BM * k; e += 256) {
    const int rr = e % RP_BM, a = e / RP_BM;
    const int ii = i0 + rr;
    Ws[rr * (NP + 1) + a] = ii < m ? X1[ii + (int64_t)a * m] : T(0);
  }
  __syncthreads();
}

template <typename T>
__global__ void __launch_bounds__(256)
x2_pass(const T* __restrict__ A, int64_t lda, const T* __restrict__ W1, int64_t ldw,
        const T* __restrict__ X1, const T* __restrict__ Z2, const T* __restrict__ CV,
        const T* __restrict__ X1p, const T* __restrict__ Z2p, const T* __restrict__ CVp,
        int m, int n2, int k, int s, int NP, T* __restrict__ out, int64_t ldo,
        double* __restrict__ part) {
  extern __shared__ unsigned char smem_raw[];
  T* As = reinterpret_cast<T*>(smem_raw);          // [RP_BK][RP_BM]
  T* Zs = As + RP_BK * RP_BM;                      // [RP_BK][max(NP, EIG_BMAX)]
  const int ZW = NP > EIG_BMAX ? NP : EIG_BMAX;
  T* Ws = Zs + RP_BK * ZW;                         // [RP_BM][NP+1]
  T* Wp = Ws + RP_BM * (NP + 1);                   // [RP_BM][NP+1]
  __shared__ double sh[32];
  const int tid = threadIdx.x;
  const int i0 = blockIdx.x * RP_BM;
  const T* A2 = A + (int64_t)k * lda;
  const bool prev = X1p != nullptr;
  x2_rows_uv(A2, lda, X1, Z2, CV, m, n2, k, s, NP, i0, As, Zs, Ws);
  if (prev) x2_rows_uv(A2, lda, X1p, Z2p, CVp, m, n2, k, s, NP, i0, As, Zs, Wp);
  double acc[6] = {0, 0, 0, 0, 0, 0};
  const int ks = k + s;
  for (int j0 = 0; j0 < n2; j0 += RP_BK) {
    __syncthreads();
    // Zs[jj][e] = Z2[(j0+jj)*NP + e] for e < ks
    for (int e = tid; e < RP_BK * ks; e += 256) {
      const int jj = e / ks, c = e % ks;
      const int j = j0 + jj;
      Zs[jj * ZW + c] = j < n2 ? Z2[(int64_t)j * NP + c] : T(0);
    }
    __syncthreads();
    // each thread: row r = tid % 64, columns jj = tid/64 + 4q
    const int r = tid % RP_BM, i = i0 + r;
    T x2v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int jj = tid / RP_BM + 4 * q;
      T v = T(0);
      for (int c = 0; c < ks; ++c) v = fma(Ws[r * (NP + 1) + c], Zs[jj * ZW + c], v);
      x2v[q] = v;
    }
    if (prev) {
      __syncthreads();
      for (int e = tid; e < RP_BK * ks; e += 256) {
        const int jj = e / ks, c = e % ks;
        const int j = j0 + jj;
        Zs[jj * ZW + c] = j < n2 ? Z2p[(int64_t)j * NP + c] : T(0);
      }
      __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int jj = tid / RP_BM + 4 * q;
      const int j = j0 + jj;
      if (i < m && j < n2) {
        const double a2 = (double)A2[i + (int64_t)j * lda];
        const double d = a2 - (double)x2v[q];
        acc[0] += d * d;
        if (out) out[i + (int64_t)j * ldo] = x2v[q];
        if (prev) {
          T v = T(0);
          for (int c = 0; c < ks; ++c) v = fma(Wp[r * (NP + 1) + c], Zs[jj * ZW + c], v);
          const double dd = (double)x2v[q] - (double)v;
          acc[1] += dd * dd;
          acc[2] += (double)v * (double)v;
        }
      }
    }
  }
  for (int e = tid; e < RP_BM * k; e += 256) {
    const int r = e % RP_BM, a = e / RP_BM;
    const int i = i0 + r;
    if (i >= m) continue;
    const double x = (double)X1[i + (int64_t)a * m];
    const double w = (double)W1[i + (int64_t)a * ldw];
    const double a1 = (double)A[i + (int64_t)a * lda];
    acc[5] += (a1 - x) * (a1 - x) * w * w;
    if (prev) {
      const double xp = (double)X1p[i + (int64_t)a * m];
      acc[3] += (x - xp) * (x - xp);
      acc[4] += xp * xp;
    }
  }
  for (int q = 0; q < 6; ++q) {
    const double v = block_sum_double(acc[q], sh);
    if (tid == 0) part[(int64_t)blockIdx.x * 8 + q] = v;
    __syncthreads();
  }
}

}  // namespace wlr
