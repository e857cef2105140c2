// Learned warm start of the sWLR iteration (declared in include/wlr.h): a small conv + MLP
// network that maps a downsampled clip and its weights to frame-mixing weights Omega, whose
// basis U = [A1 | 0] + A Omega(:, 1:r) / n starts Algorithm 1 ("Initialize (X1)_0") from the
// weighted projection of A1 onto span(U).  Everything here runs in this file's kernels: input
// preparation, the two stride-2 convolutions, the clip-context pooling, the two
// fully-connected layers (a tiled float GEMM reading bfloat16 weights), their backward
// passes, Adam, the projector-distance loss with its gradient, the basis of a solution
// (Theorem 1: span of X1 and of the kept left singular vectors) and the learned X1_0.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/wlr.h"
#include "wlr_common.cuh"
#include "wlr_solver.cuh"

using bf16 = __nv_bfloat16;

namespace wlr {
namespace ws {

struct Shape {
  int h, w, c1, c2, hidden, rmax;
  int h1, w1, h2, w2, D;   // conv1 output h1 x w1, conv2 output h2 x w2, D = c2 h2 w2
};

// offsets of the flat parameter vector (Wc1, b1, Wc2, b2, W3, b3, W4, b4)
struct Layout {
  int64_t off[9];
};

Layout layout_of(const Shape& s) {
  const int64_t sz[8] = {(int64_t)s.c1 * 2 * 9, s.c1, (int64_t)s.c2 * s.c1 * 9, s.c2,
                         (int64_t)s.hidden * 2 * s.D, s.hidden, (int64_t)s.rmax * s.hidden, s.rmax};
  Layout L;
  L.off[0] = 0;
  for (int q = 0; q < 8; ++q) L.off[q + 1] = L.off[q] + sz[q];
  return L;
}

int grid_for(int64_t n, int per = 256) {
  const int64_t g = (n + per - 1) / per;
  return (int)std::max<int64_t>(1, std::min<int64_t>(g, 65535LL * 16));
}

// ------------------------------------------------------------------ initialisation, Adam
__global__ void init_normal(float* __restrict__ P, int64_t n, int64_t base, uint64_t seed,
                            float scale) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x)
    P[t] = (float)(normal_at(seed, (uint64_t)(base + t)) * (double)scale);
}

__global__ void to_bf16(const float* __restrict__ P, bf16* __restrict__ Pb, int64_t n) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x)
    Pb[t] = __float2bfloat16_rn(P[t]);
}

// Kingma & Ba (2015), Algorithm 1, on g = grad_scale * G; refreshes the bfloat16 copy.
__global__ void adam_kernel(float* __restrict__ P, bf16* __restrict__ Pb, const float* __restrict__ G,
                            float* __restrict__ M, float* __restrict__ V, int64_t n, float lr,
                            float b1, float b2, float eps, float gs, float c1, float c2) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x) {
    const float g = gs * G[t];
    const float m = b1 * M[t] + (1.f - b1) * g;
    const float v = b2 * V[t] + (1.f - b2) * g * g;
    M[t] = m;
    V[t] = v;
    const float p = P[t] - lr * (m / c1) / (sqrtf(v / c2) + eps);
    P[t] = p;
    Pb[t] = __float2bfloat16_rn(p);
  }
}

// ------------------------------------------------------------------ input preparation
// X[j][0][y][x] = mean of the f x f block (y, x) of frame j (pixel index Y W + X), and the
// sum of squares of all of them into acc[0].
__global__ void prep_frames(const float* __restrict__ A, int64_t lda, int W, int f, int h, int w,
                            int n, float* __restrict__ X, double* __restrict__ acc) {
  __shared__ double sh[32];
  double ss = 0.0;
  const int64_t total = (int64_t)n * h * w;
  const float inv = 1.f / (float)(f * f);
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(t / (h * w));
    const int p = (int)(t - (int64_t)j * h * w);
    const int y = p / w, x = p - (p / w) * w;
    const float* col = A + (int64_t)j * lda;
    float s = 0.f;
    for (int dy = 0; dy < f; ++dy) {
      const float* row = col + (int64_t)(f * y + dy) * W + f * x;
      for (int dx = 0; dx < f; ++dx) s += row[dx];
    }
    s *= inv;
    X[((int64_t)j * 2) * h * w + p] = s;
    ss += (double)s * s;
  }
  ss = block_sum_double(ss, sh);
  if (threadIdx.x == 0) atomicAdd(acc, ss);
}

// wmap[y][x] = mean over the f x f block and the k columns of W1; the sum into acc[1].
__global__ void prep_wmap(const float* __restrict__ W1, int64_t ldw, int W, int f, int h, int w,
                          int k, float* __restrict__ wmap, double* __restrict__ acc) {
  __shared__ double sh[32];
  double sum = 0.0;
  const float inv = 1.f / (float)(f * f * k);
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < h * w; p += gridDim.x * blockDim.x) {
    const int y = p / w, x = p % w;
    float s = 0.f;
    for (int a = 0; a < k; ++a)
      for (int dy = 0; dy < f; ++dy) {
        const float* row = W1 + (int64_t)a * ldw + (int64_t)(f * y + dy) * W + f * x;
        for (int dx = 0; dx < f; ++dx) s += row[dx];
      }
    s *= inv;
    wmap[p] = s;
    sum += s;
  }
  sum = block_sum_double(sum, sh);
  if (threadIdx.x == 0) atomicAdd(acc + 1, sum);
}

__global__ void prep_finish(float* __restrict__ X, const float* __restrict__ wmap, int h, int w,
                            int n, const double* __restrict__ acc) {
  const int hw = h * w;
  const float s0 = (float)(1.0 / sqrt(acc[0] / ((double)n * hw)));
  const float s1 = (float)((double)hw / acc[1]);
  const int64_t total = (int64_t)n * hw;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(t / hw), p = (int)(t - (int64_t)j * hw);
    float* Xj = X + (int64_t)j * 2 * hw;
    Xj[p] *= s0;
    Xj[hw + p] = wmap[p] * s1;
  }
}

// ------------------------------------------------------------------ convolutions
// out[f][o][y][x] = relu(b[o] + sum_{c,u,v} Wt[o][c][u][v] in[f][c][2y+u-1][2x+v-1])
__global__ void conv_fwd(const float* __restrict__ in, int F, int C, int h, int w,
                         const bf16* __restrict__ Wt, const bf16* __restrict__ b, int O,
                         float* __restrict__ out) {
  const int ho = (h + 1) / 2, wo = (w + 1) / 2;
  const int64_t total = (int64_t)F * O * ho * wo;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int x = (int)(t % wo);
    const int y = (int)((t / wo) % ho);
    const int o = (int)((t / ((int64_t)wo * ho)) % O);
    const int64_t f = t / ((int64_t)wo * ho * O);
    float acc = __bfloat162float(b[o]);
    for (int c = 0; c < C; ++c) {
      const float* inc = in + ((f * C + c) * h) * (int64_t)w;
      const bf16* wc = Wt + ((int64_t)o * C + c) * 9;
#pragma unroll
      for (int u = 0; u < 3; ++u) {
        const int iy = 2 * y + u - 1;
        if (iy < 0 || iy >= h) continue;
#pragma unroll
        for (int v = 0; v < 3; ++v) {
          const int ix = 2 * x + v - 1;
          if (ix < 0 || ix >= w) continue;
          acc = fmaf(__bfloat162float(wc[u * 3 + v]), inc[iy * w + ix], acc);
        }
      }
    }
    out[t] = fmaxf(acc, 0.f);
  }
}

// dIn[f][c][iy][ix] = sum over (o, u, v) with 2y + u - 1 = iy, 2x + v - 1 = ix of
// Wt[o][c][u][v] dZ[f][o][y][x]; masked by act > 0 when act is given (the relu of the
// layer that produced `in`).
__global__ void conv_bwd_data(const float* __restrict__ dZ, int F, int O, int C, int h, int w,
                              const bf16* __restrict__ Wt, const float* __restrict__ act,
                              float* __restrict__ dIn) {
  const int ho = (h + 1) / 2, wo = (w + 1) / 2;
  const int64_t total = (int64_t)F * C * h * w;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    if (act != nullptr && !(act[t] > 0.f)) {
      dIn[t] = 0.f;
      continue;
    }
    const int ix = (int)(t % w);
    const int iy = (int)((t / w) % h);
    const int c = (int)((t / ((int64_t)w * h)) % C);
    const int64_t f = t / ((int64_t)w * h * C);
    float acc = 0.f;
#pragma unroll
    for (int u = 0; u < 3; ++u) {
      const int ty = iy + 1 - u;
      if (ty < 0 || (ty & 1) || (ty >> 1) >= ho) continue;
      const int y = ty >> 1;
#pragma unroll
      for (int v = 0; v < 3; ++v) {
        const int tx = ix + 1 - v;
        if (tx < 0 || (tx & 1) || (tx >> 1) >= wo) continue;
        const int x = tx >> 1;
        for (int o = 0; o < O; ++o)
          acc = fmaf(__bfloat162float(Wt[((int64_t)o * C + c) * 9 + u * 3 + v]),
                     dZ[((f * O + o) * ho + y) * (int64_t)wo + x], acc);
      }
    }
    dIn[t] = acc;
  }
}

// dW[o][c][u][v] = sum_{f,y,x} dZ[f][o][y][x] in[f][c][2y+u-1][2x+v-1] (block per weight),
// db[o] = sum_{f,y,x} dZ[f][o][y][x] (blocks O*C*9 .. O*C*9 + O - 1); double sums.
__global__ void conv_bwd_weight(const float* __restrict__ dZ, const float* __restrict__ in, int F,
                                int O, int C, int h, int w, float* __restrict__ dW,
                                float* __restrict__ db) {
  __shared__ double sh[32];
  const int ho = (h + 1) / 2, wo = (w + 1) / 2;
  const int nw = O * C * 9;
  const int q = blockIdx.x;
  const int64_t per = (int64_t)ho * wo;
  const int64_t total = (int64_t)F * per;
  double acc = 0.0;
  if (q < nw) {
    const int o = q / (C * 9), c = (q / 9) % C, u = (q % 9) / 3, v = q % 3;
    for (int64_t t = threadIdx.x; t < total; t += blockDim.x) {
      const int64_t f = t / per;
      const int p = (int)(t - f * per);
      const int y = p / wo, x = p - (p / wo) * wo;
      const int iy = 2 * y + u - 1, ix = 2 * x + v - 1;
      if (iy < 0 || iy >= h || ix < 0 || ix >= w) continue;
      acc += (double)dZ[(f * O + o) * per + p] * in[((f * C + c) * h + iy) * (int64_t)w + ix];
    }
  } else {
    const int o = q - nw;
    for (int64_t t = threadIdx.x; t < total; t += blockDim.x) {
      const int64_t f = t / per;
      const int p = (int)(t - f * per);
      acc += (double)dZ[(f * O + o) * per + p];
    }
  }
  acc = block_sum_double(acc, sh);
  if (threadIdx.x == 0) {
    if (q < nw) dW[q] = (float)acc;
    else db[q - nw] = (float)acc;
  }
}

// ------------------------------------------------------------------ clip context
// z[f] = [a2[f] | mean of a2 over the frames of f's clip]  (block per clip)
__global__ void ctx_forward(const float* __restrict__ a2, const int* __restrict__ start, int D,
                            float* __restrict__ z) {
  const int c = blockIdx.x;
  const int f0 = start[c], f1 = start[c + 1];
  const float inv = 1.f / (float)max(f1 - f0, 1);
  for (int d = threadIdx.x; d < D; d += blockDim.x) {
    float s = 0.f;
    for (int f = f0; f < f1; ++f) s += a2[(int64_t)f * D + d];
    s *= inv;
    for (int f = f0; f < f1; ++f) {
      z[(int64_t)f * 2 * D + d] = a2[(int64_t)f * D + d];
      z[(int64_t)f * 2 * D + D + d] = s;
    }
  }
}

// dz2[f][d] = (dz[f][d] + mean over f's clip of dz[.][D + d]) * (a2[f][d] > 0)
__global__ void ctx_backward(const float* __restrict__ dz, const float* __restrict__ a2,
                             const int* __restrict__ start, int D, float* __restrict__ dz2) {
  const int c = blockIdx.x;
  const int f0 = start[c], f1 = start[c + 1];
  const float inv = 1.f / (float)max(f1 - f0, 1);
  for (int d = threadIdx.x; d < D; d += blockDim.x) {
    float s = 0.f;
    for (int f = f0; f < f1; ++f) s += dz[(int64_t)f * 2 * D + D + d];
    s *= inv;
    for (int f = f0; f < f1; ++f) {
      const int64_t e = (int64_t)f * D + d;
      dz2[e] = a2[e] > 0.f ? dz[(int64_t)f * 2 * D + d] + s : 0.f;
    }
  }
}

// db[j] = sum_f dY[f][j] (double sums; block per column group of 32)
__global__ void col_sum(const float* __restrict__ dY, int F, int N, float* __restrict__ db) {
  __shared__ double sh[8][33];
  const int j = blockIdx.x * 32 + (threadIdx.x & 31);
  const int g = threadIdx.x >> 5;   // 8 row groups
  double s = 0.0;
  if (j < N)
    for (int f = g; f < F; f += 8) s += dY[(int64_t)f * N + j];
  sh[g][threadIdx.x & 31] = s;
  __syncthreads();
  if (g == 0 && j < N) {
    double t = 0.0;
    for (int q = 0; q < 8; ++q) t += sh[q][threadIdx.x & 31];
    db[j] = (float)t;
  }
}

// ------------------------------------------------------------------ tiled GEMM
// float accumulation, 64 x 64 tiles, 16-deep k slabs, 256 threads with 4 x 4 outputs.
//   MODE_NT: C (M x N) = A (M x K) B^T, B N x K      (fc forward; B = weights)
//   MODE_NN: C (M x N) = A (M x K) B,   B K x N      (fc backward, data; B = weights)
//   MODE_TN: C (M x N) = A^T B, A K x M, B K x N     (fc backward, weights)
// All row-major.  Epilogue: + bias[n], relu, or * (mask[m][n] > 0).
enum { MODE_NT = 0, MODE_NN = 1, MODE_TN = 2 };

__device__ __forceinline__ float ldf(const float* p) { return *p; }
__device__ __forceinline__ float ldf(const bf16* p) { return __bfloat162float(*p); }

template <int MODE, typename TB>
__global__ void __launch_bounds__(256)
gemm_kernel(const float* __restrict__ A, int64_t lda, const TB* __restrict__ B, int64_t ldb,
            int M, int N, int K, const TB* __restrict__ bias, int relu,
            const float* __restrict__ mask, int64_t ldm, float* __restrict__ C, int64_t ldc) {
  __shared__ float As[16][64 + 4];
  __shared__ float Bs[16][64 + 4];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
  for (int k0 = 0; k0 < K; k0 += 16) {
    for (int e = threadIdx.x; e < 1024; e += 256) {
      if (MODE == MODE_TN) {
        const int kk = e >> 6, r = e & 63;
        const int gk = k0 + kk, gm = m0 + r;
        As[kk][r] = (gk < K && gm < M) ? A[(int64_t)gk * lda + gm] : 0.f;
      } else {
        const int r = e >> 4, kk = e & 15;
        const int gm = m0 + r, gk = k0 + kk;
        As[kk][r] = (gm < M && gk < K) ? A[(int64_t)gm * lda + gk] : 0.f;
      }
      if (MODE == MODE_NT) {
        const int r = e >> 4, kk = e & 15;
        const int gn = n0 + r, gk = k0 + kk;
        Bs[kk][r] = (gn < N && gk < K) ? ldf(B + (int64_t)gn * ldb + gk) : 0.f;
      } else {
        const int kk = e >> 6, c = e & 63;
        const int gk = k0 + kk, gn = n0 + c;
        Bs[kk][c] = (gk < K && gn < N) ? ldf(B + (int64_t)gk * ldb + gn) : 0.f;
      }
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int gm = m0 + ty + 16 * i;
    if (gm >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gn = n0 + tx + 16 * j;
      if (gn >= N) continue;
      float v = acc[i][j];
      if (bias) v += ldf(bias + gn);
      if (relu) v = fmaxf(v, 0.f);
      if (mask && !(mask[(int64_t)gm * ldm + gn] > 0.f)) v = 0.f;
      C[(int64_t)gm * ldc + gn] = v;
    }
  }
}

template <int MODE, typename TB>
void gemm(cudaStream_t st, const float* A, int64_t lda, const TB* B, int64_t ldb, int M, int N, int K,
          const TB* bias, bool relu, const float* mask, int64_t ldm, float* C, int64_t ldc) {
  dim3 grid((N + 63) / 64, (M + 63) / 64);
  gemm_kernel<MODE, TB><<<grid, 256, 0, st>>>(A, lda, B, ldb, M, N, K, bias, relu ? 1 : 0, mask, ldm, C, ldc);
}

// ------------------------------------------------------------------ tall-skinny algebra
// Y (m x r, column-major, ldy) = [A1 | 0] + A (m x n, lda) Om(:, 0:r) / n, Om row-major
// n x ldo: the k weighted frames plus frame mixtures
template <typename TO>
__global__ void basis_from_omega(const float* __restrict__ A, int64_t lda, int m, int n, int k,
                                 const float* __restrict__ Om, int ldo, int r, TO* __restrict__ Y,
                                 int64_t ldy) {
  const int64_t total = (int64_t)m * r;
  const double inv_n = 1.0 / n;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(t / m);
    const int i = (int)(t - (int64_t)c * m);
    double s = 0.0;
    for (int j = 0; j < n; ++j) s += (double)A[i + (int64_t)j * lda] * Om[(int64_t)j * ldo + c];
    s *= inv_n;
    if (c < k) s += (double)A[i + (int64_t)c * lda];
    Y[i + (int64_t)c * ldy] = (TO)s;
  }
}

constexpr int GR = 128;   // rows per block of the split-m Gram

// part[blk][a + p*b] = sum over the block's rows i of d(i) X[i][a] Y[i][b] (double), with
// X (m x p, ldx), Y (m x q, ldy) column-major; d = weights (NULL: 1), one weight vector
// per grid row y (stride ldd), and likewise X/Y offsets per y (xs, ys columns).
template <typename TX, typename TY>
__global__ void __launch_bounds__(256)
gram_partial(const TX* __restrict__ X, int64_t ldx, int64_t xs, int p, const TY* __restrict__ Y,
             int64_t ldy, int64_t ys, int q, const float* __restrict__ d, int64_t ldd, int m,
             double* __restrict__ part, int64_t pstride) {
  extern __shared__ double gsm[];
  double* Xs = gsm;                  // [GR][p]
  double* Ys = gsm + GR * p;         // [GR][q]
  const int i0 = blockIdx.x * GR;
  const int yb = blockIdx.y;
  const TX* Xb = X + yb * xs;
  const TY* Yb = Y + yb * ys;
  const float* db = d ? d + yb * ldd : nullptr;
  for (int e = threadIdx.x; e < GR * p; e += 256) {
    const int rr = e % GR, a = e / GR;
    const int i = i0 + rr;
    double v = 0.0;
    if (i < m) {
      v = (double)Xb[i + (int64_t)a * ldx];
      if (db) {
        const double w = db[i];
        v *= w * w;
      }
    }
    Xs[rr * p + a] = v;
  }
  for (int e = threadIdx.x; e < GR * q; e += 256) {
    const int rr = e % GR, b = e / GR;
    const int i = i0 + rr;
    Ys[rr * q + b] = i < m ? (double)Yb[i + (int64_t)b * ldy] : 0.0;
  }
  __syncthreads();
  double* out = part + ((int64_t)yb * gridDim.x + blockIdx.x) * pstride;
  for (int e = threadIdx.x; e < p * q; e += 256) {
    const int a = e % p, b = e / p;
    double s = 0.0;
    for (int rr = 0; rr < GR; ++rr) s += Xs[rr * p + a] * Ys[rr * q + b];
    out[e] = s;
  }
}

// out[y][e] = sum over blocks of part[y][blk][e] (fixed order)
__global__ void gram_reduce(const double* __restrict__ part, int nblk, int64_t pstride, int ne,
                            double* __restrict__ out) {
  const int yb = blockIdx.y;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < ne; e += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int b = 0; b < nblk; ++b) s += part[((int64_t)yb * nblk + b) * pstride + e];
    out[(int64_t)yb * ne + e] = s;
  }
}

// In-place Cholesky S = L L^T of an r x r matrix in shared memory (lower part), one block;
// a pivot below floor * (original diagonal) is replaced by that floor.  Returns nothing:
// the ridge added by the callers keeps S positive definite.
__device__ void chol_block(double* S, int r, double* diag0) {
  for (int i = threadIdx.x; i < r; i += blockDim.x) diag0[i] = S[i * r + i];
  __syncthreads();
  for (int t = 0; t < r; ++t) {
    if (threadIdx.x == 0) {
      double pv = S[t * r + t];
      const double fl = 1e-30 + 1e-14 * fabs(diag0[t]);
      S[t * r + t] = sqrt(pv > fl ? pv : fl);
    }
    __syncthreads();
    const double lt = S[t * r + t];
    for (int i = t + 1 + threadIdx.x; i < r; i += blockDim.x) S[i * r + t] /= lt;
    __syncthreads();
    for (int e = threadIdx.x; e < (r - t - 1) * (r - t - 1); e += blockDim.x) {
      const int i = t + 1 + e % (r - t - 1), j = t + 1 + e / (r - t - 1);
      if (j <= i) S[i * r + j] -= S[i * r + t] * S[j * r + t];
    }
    __syncthreads();
  }
}

// Solve L L^T X = B in place for the r x nc matrix B (shared, row-major r x nc).
__device__ void chol_solve_block(const double* L, int r, double* B, int nc) {
  for (int c = threadIdx.x; c < nc; c += blockDim.x) {
    for (int i = 0; i < r; ++i) {
      double s = B[i * nc + c];
      for (int j = 0; j < i; ++j) s -= L[i * r + j] * B[j * nc + c];
      B[i * nc + c] = s / L[i * r + i];
    }
    for (int i = r - 1; i >= 0; --i) {
      double s = B[i * nc + c];
      for (int j = i + 1; j < r; ++j) s -= L[j * r + i] * B[j * nc + c];
      B[i * nc + c] = s / L[i * r + i];
    }
  }
}

// Loss factors of one clip (one block): from G = Y^T Y and T = V^T Y (r x r, column-major
// G[a + r b]), with M = G^{-1} T^T T: loss += (2r - 2 tr M) / (2r); the gradient is
// dY = -(2/r) (V T - Y M) G^{-1} = V P1 + Y P2 with P1 = -(2/r) T G^{-1}, P2 = (2/r) M G^{-1}.
__global__ void loss_small(const double* __restrict__ GT, int r, double* __restrict__ loss,
                           float* __restrict__ P1, float* __restrict__ P2) {
  extern __shared__ double lsm[];
  double* L = lsm;               // r x r   Cholesky of G (row-major, lower)
  double* Tm = L + r * r;        // r x r   T (row-major)
  double* B = Tm + r * r;        // r x 2r  [T^T | ...] workspace
  double* d0 = B + 2 * r * r;    // r
  __shared__ double sh[32];
  const double* G = GT;
  const double* T = GT + r * r;
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
    const int a = e % r, b = e / r;
    L[a * r + b] = G[a + r * b];
    Tm[a * r + b] = T[a + r * b];
  }
  __syncthreads();
  chol_block(L, r, d0);
  // B = [T^T T | T^T] (r x 2r): solving G X = B gives [M | G^{-1} T^T]
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
    const int a = e / r, b = e % r;
    double s = 0.0;
    for (int q = 0; q < r; ++q) s += Tm[q * r + a] * Tm[q * r + b];
    B[a * 2 * r + b] = s;
    B[a * 2 * r + r + b] = Tm[b * r + a];
  }
  __syncthreads();
  chol_solve_block(L, r, B, 2 * r);
  __syncthreads();
  double tr = 0.0;
  for (int a = threadIdx.x; a < r; a += blockDim.x) tr += B[a * 2 * r + a];
  tr = block_sum_double(tr, sh);
  if (threadIdx.x == 0) *loss += (2.0 * r - 2.0 * tr) / (2.0 * r);
  __syncthreads();
  // With X2 = G^{-1} T^T (the right half of B): T G^{-1} = X2^T (G is symmetric) and
  // M G^{-1} = G^{-1} T^T T G^{-1} = X2 X2^T, so P1(a, b) = -(2/r) X2(b, a) and
  // P2(a, b) = (2/r) sum_q X2(a, q) X2(b, q).
  const double sc = 2.0 / r;
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
    const int a = e % r, b = e / r;   // column-major (a, b)
    P1[a + r * b] = (float)(-sc * B[b * 2 * r + r + a]);
    double s = 0.0;
    for (int q = 0; q < r; ++q) s += B[a * 2 * r + r + q] * B[b * 2 * r + r + q];
    P2[a + r * b] = (float)(sc * s);
  }
}

// dY (m x r) = V P1 + Y P2 (column-major; P1, P2 r x r column-major)
__global__ void form_dy(const float* __restrict__ V, int64_t ldv, const float* __restrict__ Y,
                        int m, int r, const float* __restrict__ P1, const float* __restrict__ P2,
                        float* __restrict__ dY) {
  const int64_t total = (int64_t)m * r;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(t / m), i = (int)(t - (int64_t)c * m);
    float s = 0.f;
    for (int q = 0; q < r; ++q)
      s = fmaf(V[i + (int64_t)q * ldv], P1[q + r * c], fmaf(Y[i + (int64_t)q * m], P2[q + r * c], s));
    dY[t] = s;
  }
}

// dOm (n x rmax row-major): dOm[j][c] = scale sum_i A[i][j] dY[i][c] for c < r, else 0.
// Block per frame j; each thread sums rows for 8 columns at a time.
__global__ void omega_grad(const float* __restrict__ A, int64_t lda, int m, const float* __restrict__ dY,
                           int r, int rmax, double scale, float* __restrict__ dOm) {
  __shared__ double sh[32];
  const int j = blockIdx.x;
  const float* Aj = A + (int64_t)j * lda;
  for (int c0 = 0; c0 < rmax; c0 += 8) {
    double acc[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) acc[u] = 0.0;
    if (c0 < r) {
      for (int i = threadIdx.x; i < m; i += blockDim.x) {
        const double a = Aj[i];
#pragma unroll
        for (int u = 0; u < 8; ++u)
          if (c0 + u < r) acc[u] += a * dY[i + (int64_t)(c0 + u) * m];
      }
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const double v = block_sum_double(acc[u], sh);
      if (threadIdx.x == 0 && c0 + u < rmax) dOm[(int64_t)j * rmax + c0 + u] = c0 + u < r ? (float)(scale * v) : 0.f;
      __syncthreads();
    }
  }
}

// ------------------------------------------------------------------ solution basis
// CV (k x s) = C (k x n2) Vs (n2 x s), all column-major, element type T; result double.
template <typename T>
__global__ void cv_product(const T* __restrict__ C, const T* __restrict__ Vs, int k, int n2, int s,
                           double* __restrict__ CV) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < k * s; e += gridDim.x * blockDim.x) {
    const int a = e % k, c = e / k;
    double v = 0.0;
    for (int j = 0; j < n2; ++j) v += (double)C[a + (int64_t)j * k] * (double)Vs[j + (int64_t)c * n2];
    CV[e] = v;
  }
}

// Z (m x r, double, ld m) = [X1 | A2 Vs - X1 CV]: the columns spanning X = (X1, X1 C + D)
// (D = (P_perp A2) Vs Vs^T, P_perp A2 = A2 - X1 C).
template <typename T>
__global__ void basis_columns(const T* __restrict__ A, int64_t lda, const T* __restrict__ X1, int m,
                              int k, int n2, int s, const T* __restrict__ Vs,
                              const double* __restrict__ CV, double* __restrict__ Z) {
  const int r = k + s;
  const int64_t total = (int64_t)m * r;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(t / m), i = (int)(t - (int64_t)c * m);
    double v;
    if (c < k) {
      v = (double)X1[i + (int64_t)c * m];
    } else {
      const int cs = c - k;
      v = 0.0;
      const T* A2 = A + (int64_t)k * lda;
      for (int j = 0; j < n2; ++j) v += (double)A2[i + (int64_t)j * lda] * (double)Vs[j + (int64_t)cs * n2];
      for (int a = 0; a < k; ++a) v -= (double)X1[i + (int64_t)a * m] * CV[a + (int64_t)cs * k];
    }
    Z[t] = v;
  }
}

// Rinv (r x r, column-major, upper) = R^{-1} for S = R^T R (one block)
__global__ void chol_inverse(const double* __restrict__ S, int r, double* __restrict__ Rinv) {
  extern __shared__ double csm[];
  double* L = csm;            // r x r (row-major lower = R^T)
  double* B = L + r * r;      // r x r identity -> L^{-1}
  double* d0 = B + r * r;
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
    const int a = e % r, b = e / r;
    L[a * r + b] = S[a + r * b];
    B[a * r + b] = a == b ? 1.0 : 0.0;
  }
  __syncthreads();
  chol_block(L, r, d0);
  // B <- L^{-1} (forward substitution per column)
  for (int c = threadIdx.x; c < r; c += blockDim.x)
    for (int i = 0; i < r; ++i) {
      double s = B[i * r + c];
      for (int j = 0; j < i; ++j) s -= L[i * r + j] * B[j * r + c];
      B[i * r + c] = s / L[i * r + i];
    }
  __syncthreads();
  // R^{-1} = (L^T)^{-1} = (L^{-1})^T: Rinv(a, b) = Linv(b, a)
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
    const int a = e % r, b = e / r;
    Rinv[a + r * b] = B[b * r + a];
  }
}

// Z <- Z Rinv (m x r, in place through registers of one row)
__global__ void right_mul_upper(double* __restrict__ Z, int m, int r, const double* __restrict__ Rinv) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
    double row[64];
    for (int c = 0; c < r; ++c) row[c] = Z[i + (int64_t)c * m];
    for (int c = 0; c < r; ++c) {
      double s = 0.0;
      for (int q = 0; q <= c; ++q) s += row[q] * Rinv[q + r * c];
      Z[i + (int64_t)c * m] = s;
    }
  }
}

template <typename TD>
__global__ void copy_cols(const double* __restrict__ Z, int m, int r, TD* __restrict__ out, int64_t ldo) {
  const int64_t total = (int64_t)m * r;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(t / m), i = (int)(t - (int64_t)c * m);
    out[i + (int64_t)c * ldo] = (TD)Z[t];
  }
}

// ------------------------------------------------------------------ learned X1_0
// For each weighted frame a (block a): solve (G_a + ridge I) y = b_a with G_a = U^T D_a U,
// b_a = U^T D_a A1(:, a) (Gram part: gram_reduce output, G_a then b_a per a), ridge = 1e-12
// trace(G_a) / r; Yc[:, a] = y.
__global__ void wproj_solve(const double* __restrict__ Gb, int r, double* __restrict__ Yc) {
  extern __shared__ double wsm[];
  double* L = wsm;
  double* B = L + r * r;
  double* d0 = B + r;
  __shared__ double sh[32];
  const int a = blockIdx.x;
  const double* G = Gb + (int64_t)a * (r * r + r);
  const double* bv = G + r * r;
  double tr = 0.0;
  for (int i = threadIdx.x; i < r; i += blockDim.x) tr += G[i + r * i];
  tr = block_sum_double(tr, sh);
  __shared__ double ridge;
  if (threadIdx.x == 0) ridge = 1e-12 * tr / r;
  __syncthreads();
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
    const int i = e % r, j = e / r;
    L[i * r + j] = G[i + r * j] + (i == j ? ridge : 0.0);
  }
  for (int i = threadIdx.x; i < r; i += blockDim.x) B[i] = bv[i];
  __syncthreads();
  chol_block(L, r, d0);
  if (threadIdx.x == 0) {
    for (int i = 0; i < r; ++i) {
      double s = B[i];
      for (int j = 0; j < i; ++j) s -= L[i * r + j] * B[j];
      B[i] = s / L[i * r + i];
    }
    for (int i = r - 1; i >= 0; --i) {
      double s = B[i];
      for (int j = i + 1; j < r; ++j) s -= L[j * r + i] * B[j];
      B[i] = s / L[i * r + i];
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < r; i += blockDim.x) Yc[i + (int64_t)a * r] = B[i];
}

// X1 (m x k, ld m) = U (m x r, double) Yc (r x k)
__global__ void wproj_apply(const double* __restrict__ U, int m, int r, const double* __restrict__ Yc,
                            int k, float* __restrict__ X1) {
  const int64_t total = (int64_t)m * k;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int a = (int)(t / m), i = (int)(t - (int64_t)a * m);
    double s = 0.0;
    for (int q = 0; q < r; ++q) s += U[i + (int64_t)q * m] * Yc[q + (int64_t)a * r];
    X1[t] = (float)s;
  }
}

}  // namespace ws
}  // namespace wlr

// ====================================================================== the network object
using namespace wlr;
using namespace wlr::ws;

struct wlr_ws_net_s {
  Shape sh{};
  Layout lay{};
  int max_frames = 0;
  int64_t np = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  float *P = nullptr, *G = nullptr, *M1 = nullptr, *M2 = nullptr;
  bf16* Pb = nullptr;
  // activations of the last forward (frames x ...)
  float *a1 = nullptr, *a2 = nullptr, *z = nullptr, *a3 = nullptr;
  float *da3 = nullptr, *dz = nullptr, *dz2 = nullptr, *da1 = nullptr;
  const float* Xin = nullptr;
  int frames = 0, nclips = 0;
  int* dstart = nullptr;
  double* dacc = nullptr;     // 2 doubles (input preparation sums)
  float* wmap = nullptr;
  int adam_t = 0;
  int64_t launches = 0;
  // growable scratch for the loss, the basis and the learned init
  void* scratch = nullptr;
  size_t scratch_bytes = 0;
  std::string last_error;
  std::vector<void*> allocs;

  template <typename T>
  T* alloc(size_t n) {
    void* p = nullptr;
    WLR_CUDA(cudaMalloc(&p, std::max<size_t>(n, 1) * sizeof(T)));
    allocs.push_back(p);
    return (T*)p;
  }
  void* scratch_at_least(size_t bytes) {
    if (bytes > scratch_bytes) {
      if (scratch) {
        WLR_CUDA(cudaStreamSynchronize(stream));
        cudaFree(scratch);
        scratch = nullptr;
        scratch_bytes = 0;
      }
      WLR_CUDA(cudaMalloc(&scratch, bytes));
      scratch_bytes = bytes;
    }
    return scratch;
  }
  ~wlr_ws_net_s() {
    if (stream) cudaStreamSynchronize(stream);
    for (void* p : allocs) cudaFree(p);
    if (scratch) cudaFree(scratch);
    if (own_stream && stream) cudaStreamDestroy(stream);
  }
};

namespace {

template <typename F>
wlr_status net_guard(wlr_ws_net net, F&& f) {
  if (!net) {
    wlr::set_global_error("NULL network");
    return WLR_ERR_INVALID_ARG;
  }
  try {
    const wlr_status st = f();
    if (st == WLR_OK) net->last_error.clear();
    return st;
  } catch (const Fail& e) {
    net->last_error = e.msg;
    wlr::set_global_error(e.msg.c_str());
    return e.st;
  } catch (const std::bad_alloc&) {
    wlr::set_global_error("host allocation failed");
    return WLR_ERR_OOM;
  }
}

template <typename F>
wlr_status handle_guard(wlr_handle h, F&& f) {
  if (!h || !h->impl) {
    wlr::set_global_error("NULL handle");
    return WLR_ERR_INVALID_ARG;
  }
  try {
    const wlr_status st = f();
    if (st == WLR_OK) h->last_error.clear();
    return st;
  } catch (const Fail& e) {
    h->last_error = e.msg;
    return e.st;
  } catch (const std::bad_alloc&) {
    h->last_error = "host allocation failed";
    return WLR_ERR_OOM;
  }
}

void check_launch(wlr_ws_net net, int n) {
  net->launches += n;
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) throw Fail{WLR_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e)};
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Gram partials of X^T diag(d^2) Y over m rows into `out` (ny groups of p x q); scratch
// from `base`.  Returns the bytes used at base.
void gram(wlr_ws_net net, cudaStream_t st, const void* X, bool Xd, int64_t ldx, int64_t xs, int p,
          const void* Y, bool Yd, int64_t ldy, int64_t ys, int q, const float* d, int64_t ldd,
          int m, int ny, double* part, double* out) {
  const int nblk = (m + GR - 1) / GR;
  const size_t smem = sizeof(double) * GR * (p + q);
  const int64_t ps = (int64_t)p * q;
  dim3 grid(nblk, ny);
  if (Xd && Yd)
    gram_partial<double, double><<<grid, 256, smem, st>>>((const double*)X, ldx, xs, p, (const double*)Y, ldy, ys, q, d, ldd, m, part, ps);
  else if (!Xd && !Yd)
    gram_partial<float, float><<<grid, 256, smem, st>>>((const float*)X, ldx, xs, p, (const float*)Y, ldy, ys, q, d, ldd, m, part, ps);
  else if (Xd && !Yd)
    gram_partial<double, float><<<grid, 256, smem, st>>>((const double*)X, ldx, xs, p, (const float*)Y, ldy, ys, q, d, ldd, m, part, ps);
  else
    gram_partial<float, double><<<grid, 256, smem, st>>>((const float*)X, ldx, xs, p, (const double*)Y, ldy, ys, q, d, ldd, m, part, ps);
  gram_reduce<<<dim3((unsigned)((ps + 255) / 256), ny), 256, 0, st>>>(part, nblk, ps, (int)ps, out);
  check_launch(net, 2);
}

bool smem_ok(const void* fn, size_t bytes) {
  if (bytes <= 48 * 1024) return true;
  return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) == cudaSuccess;
}

void setup_smem_limits() {
  static bool done = false;
  if (done) return;
  const size_t g = sizeof(double) * GR * (64 + 64);
  bool ok = smem_ok((const void*)gram_partial<double, double>, g) &&
            smem_ok((const void*)gram_partial<float, float>, g) &&
            smem_ok((const void*)gram_partial<double, float>, g) &&
            smem_ok((const void*)gram_partial<float, double>, g) &&
            smem_ok((const void*)loss_small, sizeof(double) * (4 * 64 * 64 + 64)) &&
            smem_ok((const void*)chol_inverse, sizeof(double) * (2 * 64 * 64 + 64)) &&
            smem_ok((const void*)wproj_solve, sizeof(double) * (64 * 64 + 2 * 64));
  if (!ok) throw Fail{WLR_ERR_CUDA, "cudaFuncSetAttribute failed for the warm-start kernels"};
  done = true;
}

}  // namespace

extern "C" {

wlr_status wlr_ws_create(wlr_ws_net* out, const wlr_ws_shape* shape, int32_t max_frames,
                         uint64_t seed, void* stream) {
  if (out) *out = nullptr;
  if (!out || !shape) {
    wlr::set_global_error("out and shape must be non-NULL");
    return WLR_ERR_INVALID_ARG;
  }
  const wlr_ws_shape& s = *shape;
  if (s.h < 1 || s.w < 1 || s.c1 < 1 || s.c2 < 1 || s.hidden < 1 || s.r_max < 1 || s.r_max > 64 ||
      max_frames < 1 || s.h > 4096 || s.w > 4096) {
    wlr::set_global_error("need h, w, c1, c2, hidden >= 1, 1 <= r_max <= 64, max_frames >= 1");
    return WLR_ERR_INVALID_ARG;
  }
  wlr_ws_net net = new (std::nothrow) wlr_ws_net_s;
  if (!net) return WLR_ERR_OOM;
  const wlr_status st = net_guard(net, [&]() -> wlr_status {
    Shape& S = net->sh;
    S.h = s.h; S.w = s.w; S.c1 = s.c1; S.c2 = s.c2; S.hidden = s.hidden; S.rmax = s.r_max;
    S.h1 = (S.h + 1) / 2; S.w1 = (S.w + 1) / 2;
    S.h2 = (S.h1 + 1) / 2; S.w2 = (S.w1 + 1) / 2;
    S.D = S.c2 * S.h2 * S.w2;
    net->lay = layout_of(S);
    net->np = net->lay.off[8];
    net->max_frames = max_frames;
    // NULL: the legacy default stream, so that the network's work is ordered with the
    // caller's default-stream work (as the solver handles order theirs)
    net->stream = (cudaStream_t)stream;
    setup_smem_limits();
    const int64_t np = net->np;
    net->P = net->alloc<float>(np);
    net->G = net->alloc<float>(np);
    net->M1 = net->alloc<float>(np);
    net->M2 = net->alloc<float>(np);
    net->Pb = net->alloc<bf16>(np);
    const int64_t F = max_frames;
    net->a1 = net->alloc<float>(F * S.c1 * S.h1 * S.w1);
    net->da1 = net->alloc<float>(F * S.c1 * S.h1 * S.w1);
    net->a2 = net->alloc<float>(F * S.D);
    net->dz2 = net->alloc<float>(F * S.D);
    net->z = net->alloc<float>(F * 2 * S.D);
    net->dz = net->alloc<float>(F * 2 * S.D);
    net->a3 = net->alloc<float>(F * S.hidden);
    net->da3 = net->alloc<float>(F * S.hidden);
    net->dstart = net->alloc<int>(F + 1);
    net->dacc = net->alloc<double>(2);
    net->wmap = net->alloc<float>((size_t)S.h * S.w);
    cudaStream_t st = net->stream;
    WLR_CUDA(cudaMemsetAsync(net->P, 0, sizeof(float) * np, st));
    WLR_CUDA(cudaMemsetAsync(net->G, 0, sizeof(float) * np, st));
    WLR_CUDA(cudaMemsetAsync(net->M1, 0, sizeof(float) * np, st));
    WLR_CUDA(cudaMemsetAsync(net->M2, 0, sizeof(float) * np, st));
    // weights N(0, 2 / fan_in), one SplitMix64 stream position per parameter index
    const int64_t fan[4] = {18, 9LL * S.c1, 2LL * S.D, S.hidden};
    for (int l = 0; l < 4; ++l) {
      const int64_t o = net->lay.off[2 * l], n = net->lay.off[2 * l + 1] - o;
      init_normal<<<grid_for(n), 256, 0, st>>>(net->P + o, n, o, seed, (float)std::sqrt(2.0 / fan[l]));
    }
    to_bf16<<<grid_for(np), 256, 0, st>>>(net->P, net->Pb, np);
    check_launch(net, 5);
    WLR_CUDA(cudaStreamSynchronize(st));
    return WLR_OK;
  });
  if (st != WLR_OK) {
    delete net;
    return st;
  }
  *out = net;
  return WLR_OK;
}

wlr_status wlr_ws_destroy(wlr_ws_net net) {
  delete net;
  return WLR_OK;
}

int64_t wlr_ws_param_count(wlr_ws_net net) { return net ? net->np : 0; }

wlr_status wlr_ws_get_params(wlr_ws_net net, float* out, wlr_memory mem) {
  return net_guard(net, [&]() -> wlr_status {
    if (!out) throw Fail{WLR_ERR_INVALID_ARG, "out must be non-NULL"};
    WLR_CUDA(cudaMemcpyAsync(out, net->P, sizeof(float) * net->np,
                             mem == WLR_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, net->stream));
    WLR_CUDA(cudaStreamSynchronize(net->stream));
    return WLR_OK;
  });
}

wlr_status wlr_ws_get_grads(wlr_ws_net net, float* out, wlr_memory mem) {
  return net_guard(net, [&]() -> wlr_status {
    if (!out) throw Fail{WLR_ERR_INVALID_ARG, "out must be non-NULL"};
    WLR_CUDA(cudaMemcpyAsync(out, net->G, sizeof(float) * net->np,
                             mem == WLR_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, net->stream));
    WLR_CUDA(cudaStreamSynchronize(net->stream));
    return WLR_OK;
  });
}

wlr_status wlr_ws_set_params(wlr_ws_net net, const float* in, wlr_memory mem) {
  return net_guard(net, [&]() -> wlr_status {
    if (!in) throw Fail{WLR_ERR_INVALID_ARG, "in must be non-NULL"};
    WLR_CUDA(cudaMemcpyAsync(net->P, in, sizeof(float) * net->np,
                             mem == WLR_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, net->stream));
    to_bf16<<<grid_for(net->np), 256, 0, net->stream>>>(net->P, net->Pb, net->np);
    check_launch(net, 1);
    WLR_CUDA(cudaStreamSynchronize(net->stream));
    return WLR_OK;
  });
}

wlr_status wlr_ws_prepare(wlr_ws_net net, const float* A, int64_t lda, const float* W1, int64_t ldw,
                          int32_t H, int32_t W, int32_t n, int32_t k, float* X) {
  return net_guard(net, [&]() -> wlr_status {
    const Shape& S = net->sh;
    if (!A || !W1 || !X) throw Fail{WLR_ERR_INVALID_ARG, "A, W1 and X must be non-NULL"};
    if (H < 1 || W < 1 || n < 1 || k < 1 || H % S.h || W % S.w || H / S.h != W / S.w ||
        lda < (int64_t)H * W || ldw < (int64_t)H * W)
      throw Fail{WLR_ERR_INVALID_ARG, "need H = f h, W = f w for one integer f, lda, ldw >= H W"};
    const int f = H / S.h;
    cudaStream_t st = net->stream;
    WLR_CUDA(cudaMemsetAsync(net->dacc, 0, 2 * sizeof(double), st));
    const int64_t tot = (int64_t)n * S.h * S.w;
    prep_frames<<<std::min(grid_for(tot), 1024), 256, 0, st>>>(A, lda, W, f, S.h, S.w, n, X, net->dacc);
    prep_wmap<<<std::min(grid_for((int64_t)S.h * S.w), 1024), 256, 0, st>>>(W1, ldw, W, f, S.h, S.w, k, net->wmap, net->dacc);
    prep_finish<<<grid_for(tot), 256, 0, st>>>(X, net->wmap, S.h, S.w, n, net->dacc);
    check_launch(net, 3);
    return WLR_OK;
  });
}

wlr_status wlr_ws_forward(wlr_ws_net net, const float* X, int32_t frames, const int32_t* clip_start,
                          int32_t nclips, float* Omega) {
  return net_guard(net, [&]() -> wlr_status {
    const Shape& S = net->sh;
    if (!X || !Omega || !clip_start) throw Fail{WLR_ERR_INVALID_ARG, "X, Omega and clip_start must be non-NULL"};
    if (frames < 1 || frames > net->max_frames || nclips < 1 || nclips > frames)
      throw Fail{WLR_ERR_INVALID_ARG, "need 1 <= nclips <= frames <= max_frames"};
    if (clip_start[0] != 0 || clip_start[nclips] != frames)
      throw Fail{WLR_ERR_INVALID_ARG, "clip_start must run from 0 to frames"};
    for (int c = 0; c < nclips; ++c)
      if (clip_start[c + 1] <= clip_start[c]) throw Fail{WLR_ERR_INVALID_ARG, "clips must be non-empty"};
    cudaStream_t st = net->stream;
    WLR_CUDA(cudaMemcpyAsync(net->dstart, clip_start, sizeof(int) * (nclips + 1), cudaMemcpyHostToDevice, st));
    const bf16* Pb = net->Pb;
    const int64_t* o = net->lay.off;
    const int F = frames;
    conv_fwd<<<grid_for((int64_t)F * S.c1 * S.h1 * S.w1), 256, 0, st>>>(X, F, 2, S.h, S.w, Pb + o[0], Pb + o[1], S.c1, net->a1);
    conv_fwd<<<grid_for((int64_t)F * S.D), 256, 0, st>>>(net->a1, F, S.c1, S.h1, S.w1, Pb + o[2], Pb + o[3], S.c2, net->a2);
    ctx_forward<<<nclips, 256, 0, st>>>(net->a2, net->dstart, S.D, net->z);
    check_launch(net, 3);
    gemm<MODE_NT, bf16>(st, net->z, 2 * S.D, Pb + o[4], 2 * S.D, F, S.hidden, 2 * S.D, Pb + o[5], true, nullptr, 0, net->a3, S.hidden);
    gemm<MODE_NT, bf16>(st, net->a3, S.hidden, Pb + o[6], S.hidden, F, S.rmax, S.hidden, Pb + o[7], false, nullptr, 0, Omega, S.rmax);
    check_launch(net, 2);
    net->Xin = X;
    net->frames = F;
    net->nclips = nclips;
    // the host clip_start may be freed by the caller once the copy has run
    WLR_CUDA(cudaStreamSynchronize(st));
    return WLR_OK;
  });
}

wlr_status wlr_ws_backward(wlr_ws_net net, const float* dOmega) {
  return net_guard(net, [&]() -> wlr_status {
    const Shape& S = net->sh;
    if (!dOmega) throw Fail{WLR_ERR_INVALID_ARG, "dOmega must be non-NULL"};
    if (net->frames < 1) throw Fail{WLR_ERR_NOT_READY, "call wlr_ws_forward first"};
    cudaStream_t st = net->stream;
    const bf16* Pb = net->Pb;
    const int64_t* o = net->lay.off;
    float* G = net->G;
    const int F = net->frames;
    // fc2: dW4 = dOm^T a3, db4, da3 = (dOm W4) o (a3 > 0)
    gemm<MODE_TN, float>(st, dOmega, S.rmax, net->a3, S.hidden, S.rmax, S.hidden, F, nullptr, false, nullptr, 0, G + o[6], S.hidden);
    col_sum<<<(S.rmax + 31) / 32, 256, 0, st>>>(dOmega, F, S.rmax, G + o[7]);
    gemm<MODE_NN, bf16>(st, dOmega, S.rmax, Pb + o[6], S.hidden, F, S.hidden, S.rmax, nullptr, false, net->a3, S.hidden, net->da3, S.hidden);
    // fc1: dW3 = dz3^T z, db3, dz = dz3 W3
    gemm<MODE_TN, float>(st, net->da3, S.hidden, net->z, 2 * S.D, S.hidden, 2 * S.D, F, nullptr, false, nullptr, 0, G + o[4], 2 * S.D);
    col_sum<<<(S.hidden + 31) / 32, 256, 0, st>>>(net->da3, F, S.hidden, G + o[5]);
    gemm<MODE_NN, bf16>(st, net->da3, S.hidden, Pb + o[4], 2 * S.D, F, 2 * S.D, S.hidden, nullptr, false, nullptr, 0, net->dz, 2 * S.D);
    // context, then the relu of conv2
    ctx_backward<<<net->nclips, 256, 0, st>>>(net->dz, net->a2, net->dstart, S.D, net->dz2);
    // conv2: dWc2, db2 from (dz2, a1); da1 = conv2^T dz2 masked by a1 > 0
    conv_bwd_weight<<<S.c2 * S.c1 * 9 + S.c2, 256, 0, st>>>(net->dz2, net->a1, F, S.c2, S.c1, S.h1, S.w1, G + o[2], G + o[3]);
    conv_bwd_data<<<grid_for((int64_t)F * S.c1 * S.h1 * S.w1), 256, 0, st>>>(net->dz2, F, S.c2, S.c1, S.h1, S.w1, Pb + o[2], net->a1, net->da1);
    // conv1: dWc1, db1 from (da1, X)
    conv_bwd_weight<<<S.c1 * 2 * 9 + S.c1, 256, 0, st>>>(net->da1, net->Xin, F, S.c1, 2, S.h, S.w, G + o[0], G + o[1]);
    check_launch(net, 10);
    return WLR_OK;
  });
}

wlr_status wlr_ws_adam(wlr_ws_net net, float lr, float beta1, float beta2, float eps, float grad_scale) {
  return net_guard(net, [&]() -> wlr_status {
    if (!(lr >= 0.f) || !(beta1 >= 0.f && beta1 < 1.f) || !(beta2 >= 0.f && beta2 < 1.f) || !(eps > 0.f))
      throw Fail{WLR_ERR_INVALID_ARG, "need lr >= 0, 0 <= beta < 1, eps > 0"};
    net->adam_t += 1;
    const float c1 = (float)(1.0 - std::pow((double)beta1, net->adam_t));
    const float c2 = (float)(1.0 - std::pow((double)beta2, net->adam_t));
    adam_kernel<<<grid_for(net->np), 256, 0, net->stream>>>(net->P, net->Pb, net->G, net->M1, net->M2, net->np,
                                                          lr, beta1, beta2, eps, grad_scale, c1, c2);
    check_launch(net, 1);
    return WLR_OK;
  });
}

wlr_status wlr_ws_loss(wlr_ws_net net, const float* A, int64_t lda, int32_t m, int32_t n, int32_t k,
                       const float* Omega_c, int32_t r, const float* V, int64_t ldv, double* loss,
                       float* dOmega_c) {
  return net_guard(net, [&]() -> wlr_status {
    const Shape& S = net->sh;
    if (!A || !Omega_c || !V || !loss || !dOmega_c) throw Fail{WLR_ERR_INVALID_ARG, "NULL pointer"};
    if (m < 1 || n < 1 || r < 1 || r > S.rmax || r > n || k < 0 || k > r || lda < m || ldv < m)
      throw Fail{WLR_ERR_INVALID_ARG, "need 0 <= k <= r <= min(r_max, n), lda, ldv >= m"};
    cudaStream_t st = net->stream;
    const int nblk = (m + GR - 1) / GR;
    size_t off = 0;
    const size_t bY = align256(sizeof(float) * (size_t)m * r);
    const size_t bP = align256(sizeof(double) * (size_t)nblk * 2 * r * r);
    const size_t bG = align256(sizeof(double) * 2 * r * r);
    const size_t bS = align256(sizeof(float) * 2 * r * r);
    unsigned char* base = (unsigned char*)net->scratch_at_least(2 * bY + bP + bG + bS);
    float* Y = (float*)(base + off); off += bY;
    float* dY = (float*)(base + off); off += bY;
    double* part = (double*)(base + off); off += bP;
    double* GT = (double*)(base + off); off += bG;
    float* P12 = (float*)(base + off);
    basis_from_omega<float><<<grid_for((int64_t)m * r), 256, 0, st>>>(A, lda, m, n, k, Omega_c, S.rmax, r, Y, m);
    check_launch(net, 1);
    gram(net, st, Y, false, m, 0, r, Y, false, m, 0, r, nullptr, 0, m, 1, part, GT);           // G = Y^T Y
    gram(net, st, V, false, ldv, 0, r, Y, false, m, 0, r, nullptr, 0, m, 1, part, GT + r * r); // T = V^T Y
    loss_small<<<1, 256, sizeof(double) * (4 * r * r + r), st>>>(GT, r, loss, P12, P12 + r * r);
    form_dy<<<grid_for((int64_t)m * r), 256, 0, st>>>(V, ldv, Y, m, r, P12, P12 + r * r, dY);
    omega_grad<<<n, 256, 0, st>>>(A, lda, m, dY, r, S.rmax, 1.0 / n, dOmega_c);
    check_launch(net, 3);
    return WLR_OK;
  });
}

int64_t wlr_ws_launches(wlr_ws_net net) { return net ? net->launches : 0; }

wlr_status wlr_get_basis(wlr_handle h, float* V, int64_t ldv) {
  return handle_guard(h, [&]() -> wlr_status {
    const Dims d = h->impl->dims();
    if (!V || ldv < d.m) throw Fail{WLR_ERR_INVALID_ARG, "V must be non-NULL with ldv >= m"};
    if (d.r > 64) throw Fail{WLR_ERR_UNSUPPORTED, "r <= 64 only"};
    const SolverBase::View v = h->impl->view(true);
    cudaStream_t st = v.stream;
    const int m = d.m, k = d.k, n2 = d.n2, s = d.s, r = d.r;
    setup_smem_limits();
    const int nblk = (m + GR - 1) / GR;
    double *Z = nullptr, *part = nullptr, *S = nullptr, *Rinv = nullptr, *CV = nullptr;
    std::vector<void*> tmp;
    auto dal = [&](size_t bytes) {
      void* p = nullptr;
      WLR_CUDA(cudaMalloc(&p, std::max<size_t>(bytes, 8)));
      tmp.push_back(p);
      return (double*)p;
    };
    try {
      Z = dal(sizeof(double) * (size_t)m * r);
      part = dal(sizeof(double) * (size_t)nblk * r * r);
      S = dal(sizeof(double) * r * r);
      Rinv = dal(sizeof(double) * r * r);
      CV = dal(sizeof(double) * (size_t)k * std::max(s, 1));
      if (v.fp64) {
        if (s > 0) cv_product<double><<<grid_for((int64_t)k * s), 256, 0, st>>>((const double*)v.C, (const double*)v.Vs, k, n2, s, CV);
        basis_columns<double><<<grid_for((int64_t)m * r), 256, 0, st>>>((const double*)v.A, v.lda, (const double*)v.X1, m, k, n2, s, (const double*)v.Vs, CV, Z);
      } else {
        if (s > 0) cv_product<float><<<grid_for((int64_t)k * s), 256, 0, st>>>((const float*)v.C, (const float*)v.Vs, k, n2, s, CV);
        basis_columns<float><<<grid_for((int64_t)m * r), 256, 0, st>>>((const float*)v.A, v.lda, (const float*)v.X1, m, k, n2, s, (const float*)v.Vs, CV, Z);
      }
      if (cudaGetLastError() != cudaSuccess) throw Fail{WLR_ERR_CUDA, "kernel launch failed"};
      for (int pass = 0; pass < 2; ++pass) {
        const size_t smem = sizeof(double) * GR * (2 * r);
        gram_partial<double, double><<<dim3(nblk, 1), 256, smem, st>>>(Z, m, 0, r, Z, m, 0, r, nullptr, 0, m, part, (int64_t)r * r);
        gram_reduce<<<dim3((r * r + 255) / 256, 1), 256, 0, st>>>(part, nblk, (int64_t)r * r, r * r, S);
        chol_inverse<<<1, 256, sizeof(double) * (2 * r * r + r), st>>>(S, r, Rinv);
        right_mul_upper<<<grid_for(m), 256, 0, st>>>(Z, m, r, Rinv);
      }
      copy_cols<float><<<grid_for((int64_t)m * r), 256, 0, st>>>(Z, m, r, V, ldv);
      if (cudaGetLastError() != cudaSuccess) throw Fail{WLR_ERR_CUDA, "kernel launch failed"};
      WLR_CUDA(cudaStreamSynchronize(st));
    } catch (...) {
      cudaStreamSynchronize(st);
      for (void* p : tmp) cudaFree(p);
      throw;
    }
    for (void* p : tmp) cudaFree(p);
    return WLR_OK;
  });
}

wlr_status wlr_set_init_learned(wlr_handle h, wlr_ws_net net, int32_t H, int32_t W, int32_t fallback,
                                int32_t* used_learned) {
  if (used_learned) *used_learned = 0;
  if (!net) {
    if (h) h->last_error = "NULL network";
    return WLR_ERR_INVALID_ARG;
  }
  return handle_guard(h, [&]() -> wlr_status {
    const Dims d = h->impl->dims();
    const Shape& S = net->sh;
    const int m = d.m, n = d.n, k = d.k, r = d.r;
    if ((int64_t)H * W != m) throw Fail{WLR_ERR_INVALID_ARG, "H W must equal m"};
    if (r > S.rmax) throw Fail{WLR_ERR_INVALID_ARG, "r exceeds the network's r_max"};
    if (n > net->max_frames) throw Fail{WLR_ERR_INVALID_ARG, "n exceeds the network's max_frames"};
    const SolverBase::View v = h->impl->view(false);
    if (v.fp64) throw Fail{WLR_ERR_UNSUPPORTED, "learned initialisation for float handles only"};
    const float* A = (const float*)v.A;
    const float* W1 = (const float*)v.W1;
    // the network works on its own stream: order it after the handle's work
    cudaEvent_t ev;
    WLR_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    cudaEventRecord(ev, v.stream);
    cudaStreamWaitEvent(net->stream, ev, 0);
    cudaEventDestroy(ev);
    const int nblk = (m + GR - 1) / GR;
    size_t off = 0;
    const size_t bX = align256(sizeof(float) * (size_t)n * 2 * S.h * S.w);
    const size_t bO = align256(sizeof(float) * (size_t)n * S.rmax);
    const size_t bU = align256(sizeof(double) * (size_t)m * r);
    const size_t bP = align256(sizeof(double) * (size_t)nblk * k * (r * r + r));
    const size_t bG = align256(sizeof(double) * (size_t)k * (r * r + r));
    const size_t bY = align256(sizeof(double) * (size_t)r * k);
    const size_t bX1 = align256(sizeof(float) * (size_t)m * k);
    unsigned char* base = (unsigned char*)net->scratch_at_least(bX + bO + bU + bP + bG + bY + bX1);
    float* X = (float*)(base + off); off += bX;
    float* Om = (float*)(base + off); off += bO;
    double* U = (double*)(base + off); off += bU;
    double* part = (double*)(base + off); off += bP;
    double* Gb = (double*)(base + off); off += bG;
    double* Yc = (double*)(base + off); off += bY;
    float* X1 = (float*)(base + off);
    wlr_status st = wlr_ws_prepare(net, A, v.lda, W1, v.ldw, H, W, n, k, X);
    if (st != WLR_OK) throw Fail{st, net->last_error};
    const int32_t cs[2] = {0, n};
    st = wlr_ws_forward(net, X, n, cs, 1, Om);
    if (st != WLR_OK) throw Fail{st, net->last_error};
    cudaStream_t s = net->stream;
    basis_from_omega<double><<<grid_for((int64_t)m * r), 256, 0, s>>>(A, v.lda, m, n, k, Om, S.rmax, r, U, m);
    check_launch(net, 1);
    // per weighted frame a: [U^T D_a U | U^T D_a A1(:, a)] (r x r, then r), D_a = W1(:, a)^2
    {
      const int64_t pe = (int64_t)r * r + r;
      const size_t smem = sizeof(double) * GR * (r + r);
      // U^T D_a U: X = U (weights), Y = U; U^T D_a A1: X = U (weights), Y = A1(:, a)
      gram_partial<double, double><<<dim3(nblk, k), 256, smem, s>>>(U, m, 0, r, U, m, 0, r, W1, v.ldw, m, part, pe);
      gram_partial<double, float><<<dim3(nblk, k), 256, sizeof(double) * GR * (r + 1), s>>>(
          U, m, 0, r, A, v.lda, v.lda, 1, W1, v.ldw, m, part + (int64_t)r * r, pe);
      gram_reduce<<<dim3((unsigned)((pe + 255) / 256), k), 256, 0, s>>>(part, nblk, pe, (int)pe, Gb);
      wproj_solve<<<k, 256, sizeof(double) * (r * r + 2 * r), s>>>(Gb, r, Yc);
      wproj_apply<<<grid_for((int64_t)m * k), 256, 0, s>>>(U, m, r, Yc, k, X1);
      check_launch(net, 5);
    }
    WLR_CUDA(cudaStreamSynchronize(s));
    h->impl->set_init(WLR_INIT_USER, X1, m, WLR_F32, WLR_MEM_DEVICE, 0);
    bool learned = true;
    if (fallback) {
      // the objective judges the two starts: F_0 = F(X1_0, C_0, D_0) of one iteration from
      // each (the value wlr_step returns); the plain start wins ties
      double FL = 0.0, FA = 0.0;
      h->impl->step(&FL);
      h->impl->set_init(WLR_INIT_A1, nullptr, 0, WLR_F32, WLR_MEM_DEVICE, 0);
      h->impl->step(&FA);
      if (FL < FA) h->impl->set_init(WLR_INIT_USER, X1, m, WLR_F32, WLR_MEM_DEVICE, 0);
      else {
        h->impl->set_init(WLR_INIT_A1, nullptr, 0, WLR_F32, WLR_MEM_DEVICE, 0);
        learned = false;
      }
    }
    if (used_learned) *used_learned = learned ? 1 : 0;
    return WLR_OK;
  });
}

}  // extern "C"
