// Tensor-core (tcgen05 + TMA) split-m Gram for the tall-skinny product of the sWLR
// iteration: part[c] = X(rows of chunk c)^T Y(rows of chunk c) with X = Q1 (m x P, P <= 32)
// and Y = [Q1 | A2].  FP32-grade accuracy from three TF32 products per operand pair
// (hi*hi + hi*lo + lo*hi with hi, lo the nearest-TF32 split of each FP32 value), summed by
// the tensor cores in FP32 over 32-row slabs and across slabs in float hi + lo pairs.
// The chunk partials are summed in double afterwards.
//
// Layout: every operand is a column-major m x cols FP32 matrix, so for the MMA (D = A B^T,
// A: M x K, B: N x K) both operands are K-major with K = the row index of the matrices.
// TMA brings 32 rows (128 bytes) of 128 (A) or 32 (B) columns per tile into shared memory
// with the 128-byte swizzle; one thread issues the MMAs into a tensor-memory accumulator.
// Every wait on an mbarrier is bounded by a 2-second clock; on expiry the kernel records an
// error bit, stops issuing work and still frees its tensor memory.
#pragma once

#include <cuda.h>

#include "wlr_common.cuh"

namespace wlr {
namespace tc {

constexpr int BM = 128;             // MMA M = rows of X^T handled (P <= 128)
constexpr int BN = 128;             // MMA N = columns of Y per CTA
constexpr int BK = 32;              // rows of the matrices per stage (128 bytes of FP32)
constexpr int STAGES = 2;
constexpr int TILE_BYTES = 128 * BK * 4;            // 16 KB for a 128 x 32 FP32 tile
constexpr int STAGE_BYTES = 4 * TILE_BYTES;         // X hi, X lo, Y hi, Y lo
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024;  // + 1 KB for 1024-byte alignment
constexpr unsigned TMEM_COLS = 128;
constexpr unsigned long long kWaitNs = 2000000000ull;    // 2 s cap on every wait
constexpr int ERRBIT_TIMEOUT = 16;

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ unsigned long long now_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
// Wait for the phase with the given parity to complete; false after limit_ns.
__device__ __forceinline__ bool mbar_try(uint64_t* bar, unsigned parity) {
  unsigned done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(done)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return done != 0;
}
// The clock is read only once a first try has failed (most waits of a running pipeline
// find the phase complete), then the wait gives up after limit_ns.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity,
                                          unsigned long long limit_ns = kWaitNs) {
  if (mbar_try(bar, parity)) return true;
  const unsigned long long t0 = now_ns();
  while (true) {
    if (mbar_try(bar, parity)) return true;
    if (now_ns() - t0 > limit_ns) return false;
  }
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x,
                                            int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_u32(dst)),
      "l"(map), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// K-major operand tile with the 128-byte swizzle: 8-row atoms of 1024 bytes (SBO), the
// tile base 1024-byte aligned; the start address moves 32 bytes per 8-element K step.
__device__ __forceinline__ uint64_t sdesc_sw128(unsigned saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);     // start address
  d |= (uint64_t)1 << 16;                        // leading byte offset (unused here)
  d |= (uint64_t)(1024 >> 4) << 32;              // stride byte offset: 8 rows x 128 B
  d |= (uint64_t)1 << 46;                        // descriptor version
  d |= (uint64_t)2 << 61;                        // 128-byte swizzle
  return d;
}
// Instruction descriptor, kind::tf32: D = F32, A = B = TF32, both K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(unsigned d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         unsigned accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void tmem_ld16(unsigned taddr, float (&v)[16]) {
  unsigned r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
        "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Nearest TF32 value (10 explicit mantissa bits; ties away from zero) as an FP32 number.

// x = hi + lo + r with hi = round_tf32(x), lo = round_tf32(x - hi): both parts are exact
// TF32 numbers, so hi*hi, hi*lo and lo*hi are exact FP32 products inside the MMA and the
// dropped terms (lo*lo and the residual r, |r| <= 2^-22 |x|) carry no systematic sign.
static __global__ void split_tf32(const float* __restrict__ src, int64_t lds, int rows, int cols,
                           float* __restrict__ hi, float* __restrict__ lo, int64_t ldd) {
  const int64_t total = (int64_t)rows * cols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = e / rows, i = e - j * rows;
    const float x = src[i + j * lds];
    const float h = round_tf32(x);
    hi[i + j * ldd] = h;
    lo[i + j * ldd] = round_tf32(x - h);
  }
}

// Q1 = X1 R^{-1} written as the TF32 split (hi, lo), leading dimension ldq.
static __global__ void form_q_split(const float* __restrict__ X1, int64_t ldx, const float* __restrict__ Rinv,
                             int m, int k, float* __restrict__ qh, float* __restrict__ ql, int64_t ldq,
                             int full) {
  extern __shared__ unsigned char smem_q[];
  float* Ri = reinterpret_cast<float*>(smem_q);
  for (int e = threadIdx.x; e < k * k; e += blockDim.x) Ri[e] = Rinv[e];
  __syncthreads();
  const int64_t total = (int64_t)m * k;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int a = (int)(e / m);
    const int64_t i = e - (int64_t)a * m;
    float v = 0.f;
    const int bend = full ? k : a + 1;   // Rinv upper triangular unless full
    for (int b = 0; b < bend; ++b) v = fmaf(X1[i + b * ldx], Ri[b + a * k], v);
    const float h = round_tf32(v);
    qh[i + (int64_t)a * ldq] = h;
    ql[i + (int64_t)a * ldq] = round_tf32(v - h);
  }
}

// ------------------------------------------------------------------------------------
// Transposed form with per-slab read-back (the one the solver uses):
//   part[c*pstride + a + col*P] = sum over the rows of chunk c of Y(i, col) X(i, a), stored
//   as the float pair hi + lo in the 8 bytes of the slot (reduce_pairs_split adds them)
// computed as D = Y^T X with the columns of Y on the 128 MMA rows (all TMEM lanes carry
// data) and the P <= TNV columns of X as N = TNV (32 or 64).  Each 32-row slab is
// accumulated by the tensor cores in FP32 into one of two TMEM buffers; while the MMA
// fills the other one, the epilogue warps read the slab back (tcgen05.ld) and add it into
// a float hi + lo pair per entry (TwoSum), so the chunk sum keeps about FP64 accuracy, as
// the SIMT Gram does.  Epilogue warp w (of 4 TNV / 32) reads TMEM lanes 32 (w % 4) ..
// + 31 and columns 32 (w / 4) .. + 31; the next warp issues the TMA loads, the one after it
// the MMAs.  Column tile 0 uses Y1 (= Q1, q1 columns) as Y, tiles t >= 1 use columns
// (t-1)*128 .. of Y2 (= A2).
constexpr int TN = 32;                                   // MMA N for up to 32 columns of X
constexpr int T_STAGES = 4;
// warps that split FP32 A2 tiles: 4, or 2 for N = 64 (whose 8 epilogue warps keep 96 live
// accumulator registers each; more threads would cap the registers below that)
__host__ __device__ constexpr int t_split_warps(int tnv) { return tnv == TN ? 4 : 2; }
constexpr int T_A_BYTES = 128 * BK * 4;                  // Y tile: 128 columns x 32 rows
__host__ __device__ constexpr int t_b_bytes(int tnv) { return tnv * BK * 4; }   // X tile
__host__ __device__ constexpr int t_stage_bytes(int tnv) { return 2 * T_A_BYTES + 2 * t_b_bytes(tnv); }
__host__ __device__ constexpr int t_smem_bytes(int tnv) { return T_STAGES * t_stage_bytes(tnv) + 1024; }
__host__ __device__ constexpr int t_threads(int tnv) { return 32 * (4 * (tnv / 32) + 2 + t_split_warps(tnv)); }

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void tmem_ld32(unsigned taddr, float (&v)[32]) {
  unsigned r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
        "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
        "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
        "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void two_sum_f(float a, float b, float& s, float& e) {
  s = a + b;
  const float bp = s - a;
  const float ap = s - bp;
  e = (a - ap) + (b - bp);
}

//
// With split != 0 the column tiles of Y2 (= A2) come from the FP32 matrix itself (mY2f):
// TMA brings the FP32 tile into the hi slot of the stage, and the split warps
// (t_split_warps, running ahead of the MMA as far as the stages allow) replace it in place by its TF32
// high part and write the low part to the lo slot at the same (swizzled) offsets, then
// release the stage to the MMA warp.  The values are those of the split copies, so the
// result is the same bit for bit, while one pass over A2 reads half the bytes (and the row
// pass reads the same FP32 A2).  Warps: epilogue 0 .. NEPI-1, TMA NEPI, MMA NEPI+1, split
// the rest.
template <int TNV>
static __global__ void __launch_bounds__(t_threads(TNV))
gram_tf32x3_t(const __grid_constant__ CUtensorMap mY1h, const __grid_constant__ CUtensorMap mY1l,
              const __grid_constant__ CUtensorMap mY2h, const __grid_constant__ CUtensorMap mY2l,
              const __grid_constant__ CUtensorMap mXh, const __grid_constant__ CUtensorMap mXl,
              const __grid_constant__ CUtensorMap mY2f, int split,
              int m, int P, int q1, int q2, int chunk_rows, double* __restrict__ part, int64_t pstride,
              int* __restrict__ err) {
  constexpr int NEPI = 4 * (TNV / 32);                  // epilogue warps
  constexpr int NSPL = t_split_warps(TNV);              // split warps
  constexpr int T_B_BYTES = t_b_bytes(TNV), T_STAGE_BYTES = t_stage_bytes(TNV);
  constexpr unsigned T_TMEM_COLS = 2 * TNV;             // two TNV-column accumulators
  extern __shared__ unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t full[T_STAGES], empty[T_STAGES], splt[T_STAGES], accf[2], acce[2];
  __shared__ unsigned tmem_base;
  __shared__ int fail;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tile = blockIdx.x, c = blockIdx.y;
  const bool do_split = split != 0 && tile != 0;
  const int i_begin = c * chunk_rows;
  const int i_end = min(m, i_begin + chunk_rows);
  const int nkb = (i_end - i_begin + BK - 1) / BK;
  const CUtensorMap* yh = tile == 0 ? &mY1h : &mY2h;
  const CUtensorMap* yl = tile == 0 ? &mY1l : &mY2l;
  const int y0 = tile == 0 ? 0 : (tile - 1) * 128;
  const int ncols = tile == 0 ? q1 : min(128, q2 - y0);
  const int gcol0 = tile == 0 ? 0 : q1 + y0;
  const unsigned base = (smem_u32(smem_raw) + 1023u) & ~1023u;
  unsigned char* base_ptr = smem_raw + (base - smem_u32(smem_raw));
  auto a_addr = [&](int s, int lo) { return base + (unsigned)(s * T_STAGE_BYTES + lo * T_A_BYTES); };
  auto b_addr = [&](int s, int lo) {
    return base + (unsigned)(s * T_STAGE_BYTES + 2 * T_A_BYTES + lo * T_B_BYTES);
  };

  if (threadIdx.x == 0) {
    for (int s = 0; s < T_STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
      mbar_init(&splt[s], NSPL);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&accf[b], 1);
      mbar_init(&acce[b], NEPI);
    }
    fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(T_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const unsigned tacc = tmem_base;

  if (warp == NEPI) {
    if (lane == 0) {
      int issued = 0;
      for (int kb = 0; kb < nkb; ++kb) {
        const int s = kb % T_STAGES;
        if (kb >= T_STAGES && !mbar_wait(&empty[s], (unsigned)((kb / T_STAGES - 1) & 1))) {
          atomicOr(&fail, 1);
          break;
        }
        if (*(volatile int*)&fail) break;
        issued = kb + 1;
        const int x = i_begin + kb * BK;
        if (do_split) {
          mbar_expect_tx(&full[s], T_A_BYTES + 2 * T_B_BYTES);
          tma_load_2d(base_ptr + (a_addr(s, 0) - base), &mY2f, &full[s], x, y0);
        } else {
          mbar_expect_tx(&full[s], T_STAGE_BYTES);
          tma_load_2d(base_ptr + (a_addr(s, 0) - base), yh, &full[s], x, y0);
          tma_load_2d(base_ptr + (a_addr(s, 1) - base), yl, &full[s], x, y0);
        }
        tma_load_2d(base_ptr + (b_addr(s, 0) - base), &mXh, &full[s], x, 0);
        tma_load_2d(base_ptr + (b_addr(s, 1) - base), &mXl, &full[s], x, 0);
      }
      // drain: the last fill issued into each stage has landed before the CTA exits (in
      // the normal path these phases completed long ago)
      for (int kb = issued - 1; kb >= 0 && kb >= issued - T_STAGES; --kb)
        if (!mbar_wait(&full[kb % T_STAGES], (unsigned)((kb / T_STAGES) & 1))) atomicOr(&fail, 1);
    }
  } else if (warp == NEPI + 1) {
    if (lane == 0) {
      constexpr uint32_t idesc = idesc_tf32(128, TNV);
      int committed = 0;
      for (int kb = 0; kb < nkb; ++kb) {
        const int s = kb % T_STAGES, b = kb & 1;
        const unsigned ph = (unsigned)((kb / T_STAGES) & 1);
        if (!mbar_wait(&full[s], ph) || (do_split && !mbar_wait(&splt[s], ph)) ||
            (kb >= 2 && !mbar_wait(&acce[b], (unsigned)((kb / 2 - 1) & 1)))) {
          atomicOr(&fail, 1);
          break;
        }
        fence_after();
        const uint64_t yhd = sdesc_sw128(a_addr(s, 0)), yld = sdesc_sw128(a_addr(s, 1));
        const uint64_t xhd = sdesc_sw128(b_addr(s, 0)), xld = sdesc_sw128(b_addr(s, 1));
        const unsigned d = tacc + (unsigned)(b * TNV);
#pragma unroll
        for (int ks = 0; ks < BK / 8; ++ks) {
          const uint64_t adv = (uint64_t)((ks * 32) >> 4);
          mma_tf32(d, yhd + adv, xhd + adv, idesc, ks > 0 ? 1u : 0u);
          mma_tf32(d, yhd + adv, xld + adv, idesc, 1u);
          mma_tf32(d, yld + adv, xhd + adv, idesc, 1u);
        }
        mma_commit(&empty[s]);
        mma_commit(&accf[b]);
        committed = kb + 1;
      }
      // drain: the last commit tracks every MMA this thread issued; wait for it before the
      // tensor memory is freed
      if (committed > 0) {
        const int kl = committed - 1;
        if (!mbar_wait(&accf[kl & 1], (unsigned)((kl / 2) & 1))) atomicOr(&fail, 1);
      }
    }
  } else if (warp >= NEPI + 2) {
    // split warps: stage kb's FP32 tile (hi slot) -> TF32 hi in place and lo in the lo slot,
    // 16 bytes per step over the split warps' threads
    if (do_split) {
      const int t = threadIdx.x - 32 * (NEPI + 2);
      for (int kb = 0; kb < nkb; ++kb) {
        const int s = kb % T_STAGES;
        if (!mbar_wait(&full[s], (unsigned)((kb / T_STAGES) & 1))) {
          atomicOr(&fail, 1);
          break;
        }
        float4* yh = reinterpret_cast<float4*>(base_ptr + (a_addr(s, 0) - base));
        float4* yl = reinterpret_cast<float4*>(base_ptr + (a_addr(s, 1) - base));
        for (int e = t; e < T_A_BYTES / 16; e += 32 * NSPL) {
          const float4 x = yh[e];
          float4 h, l;
          h.x = round_tf32(x.x); l.x = round_tf32(x.x - h.x);
          h.y = round_tf32(x.y); l.y = round_tf32(x.y - h.y);
          h.z = round_tf32(x.z); l.z = round_tf32(x.z - h.z);
          h.w = round_tf32(x.w); l.w = round_tf32(x.w - h.w);
          yh[e] = h;
          yl[e] = l;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive(&splt[s]);
      }
    }
  } else {
    // epilogue warp w: TMEM lanes 32 (w % 4) .. + 31 = columns col = 32 (w % 4) + lane of
    // this tile, X columns a = 32 (w / 4) .. + 31
    const int qd = warp & 3, hf = warp >> 2;
    float hi[32], lo[32];
#pragma unroll
    for (int a = 0; a < 32; ++a) {
      hi[a] = 0.f;
      lo[a] = 0.f;
    }
    bool ok = true;
    for (int kb = 0; ok && kb < nkb; ++kb) {
      const int b = kb & 1;
      if (!mbar_wait(&accf[b], (unsigned)((kb / 2) & 1))) {
        ok = false;
        break;
      }
      fence_after();
      float v[32];
      tmem_ld32(tacc + ((unsigned)(32 * qd) << 16) + (unsigned)(b * TNV + 32 * hf), v);
      fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acce[b]);
#pragma unroll
      for (int a = 0; a < 32; ++a) {
        float sres, e;
        two_sum_f(hi[a], v[a], sres, e);
        hi[a] = sres;
        lo[a] += e;
      }
    }
    if (!ok || *(volatile int*)&fail) {
      if (lane == 0) atomicOr(err, ERRBIT_TIMEOUT);
    } else {
      // each chunk partial leaves as its float pair (hi, lo) in the 8 bytes of its slot;
      // the reduction over the chunks adds the pairs and converts once (FP64 arithmetic,
      // slow on this GPU, stays out of this kernel's tail)
      const int j = 32 * qd + lane;
      if (j < ncols) {
        float2* out = reinterpret_cast<float2*>(part + (int64_t)c * pstride + (int64_t)(gcol0 + j) * P + 32 * hf);
#pragma unroll
        for (int a = 0; a < 32; ++a)
          if (32 * hf + a < P) out[a] = make_float2(hi[a], lo[a]);
      }
    }
  }
  fence_before();
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tacc), "r"(T_TMEM_COLS) : "memory");
}

// ------------------------------------------------------------------------------------
// K = A2^T A2 (step a0, once per clip) on the tensor cores: part[c][p] = the 128 x 64 block
// (bi, bj) = pairs[p] (columns 128 bi .. + 127 by 64 bj .. + 63 of K, the blocks that hold
// entries on or above the diagonal) of A2(rows of chunk c)^T A2(rows of chunk c), in
// 3xTF32 like gram_tf32x3_t.  M = 128 columns on the TMEM lanes, N = 64; the tensor cores
// accumulate a 128-row slab (4 stages of 32 rows) in FP32 into one of two 64-column TMEM
// buffers while the other is read back by the 8 epilogue warps (warp w: lane quadrant
// w % 4, columns 32 (w / 4) .. + 31) and added into float hi + lo pairs with TwoSum; warp 8
// issues the TMA loads, warp 9 the MMAs.  chunk_rows is a multiple of 32, so only the last
// chunk runs past m (TMA fills zeros).
constexpr int KN = 64;                                      // MMA N
constexpr int K_STAGES = 4;
constexpr int K_B_BYTES = KN * BK * 4;                      // 8 KB
constexpr int K_STAGE_BYTES = 2 * T_A_BYTES + 2 * K_B_BYTES;  // A hi, A lo, B hi, B lo
constexpr int K_SMEM_BYTES = K_STAGES * K_STAGE_BYTES + 1024;
constexpr int K_SLAB = 4;                                   // stages per TMEM slab (128 rows)
constexpr unsigned K_TMEM_COLS = 128;                       // two 64-column accumulators
constexpr int K_THREADS = 320;
constexpr int K_TILE = 128 * KN;                            // partial entries per (chunk, pair)

static __global__ void __launch_bounds__(K_THREADS, 1)
gram_kk_tf32x3(const __grid_constant__ CUtensorMap mh, const __grid_constant__ CUtensorMap ml,
               const __grid_constant__ CUtensorMap mh64, const __grid_constant__ CUtensorMap ml64, int m,
               int chunk_rows, const int2* __restrict__ pairs, int npairs, double* __restrict__ part,
               int* __restrict__ err) {
  extern __shared__ unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t full[K_STAGES], empty[K_STAGES], accf[2], acce[2], drain_bar;
  __shared__ unsigned tmem_base;
  __shared__ int fail;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int p = blockIdx.x, c = blockIdx.y;
  const int2 pb = pairs[p];
  const int i_begin = c * chunk_rows;
  const int i_end = min(m, i_begin + chunk_rows);
  const int nkb = (i_end - i_begin + BK - 1) / BK;
  const int nslab = (nkb + K_SLAB - 1) / K_SLAB;
  const unsigned base = (smem_u32(smem_raw) + 1023u) & ~1023u;
  unsigned char* base_ptr = smem_raw + (base - smem_u32(smem_raw));
  auto a_addr = [&](int s, int lo) { return base + (unsigned)(s * K_STAGE_BYTES + lo * T_A_BYTES); };
  auto b_addr = [&](int s, int lo) {
    return base + (unsigned)(s * K_STAGE_BYTES + 2 * T_A_BYTES + lo * K_B_BYTES);
  };

  if (threadIdx.x == 0) {
    for (int s = 0; s < K_STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&accf[b], 1);
      mbar_init(&acce[b], 8);
    }
    mbar_init(&drain_bar, 1);
    fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(K_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const unsigned tacc = tmem_base;

  if (warp == 8) {
    if (lane == 0) {
      int issued = 0;
      for (int kb = 0; kb < nkb; ++kb) {
        const int s = kb % K_STAGES;
        if (kb >= K_STAGES && !mbar_wait(&empty[s], (unsigned)((kb / K_STAGES - 1) & 1))) {
          atomicOr(&fail, 1);
          break;
        }
        if (*(volatile int*)&fail) break;
        issued = kb + 1;
        mbar_expect_tx(&full[s], K_STAGE_BYTES);
        const int x = i_begin + kb * BK;
        tma_load_2d(base_ptr + (a_addr(s, 0) - base), &mh, &full[s], x, pb.x * 128);
        tma_load_2d(base_ptr + (a_addr(s, 1) - base), &ml, &full[s], x, pb.x * 128);
        tma_load_2d(base_ptr + (b_addr(s, 0) - base), &mh64, &full[s], x, pb.y * KN);
        tma_load_2d(base_ptr + (b_addr(s, 1) - base), &ml64, &full[s], x, pb.y * KN);
      }
      // drain the last fill of each stage (see gram_tf32x3_t)
      for (int kb = issued - 1; kb >= 0 && kb >= issued - K_STAGES; --kb)
        if (!mbar_wait(&full[kb % K_STAGES], (unsigned)((kb / K_STAGES) & 1))) atomicOr(&fail, 1);
    }
  } else if (warp == 9) {
    if (lane == 0) {
      constexpr uint32_t idesc = idesc_tf32(128, KN);
      int last_slab = -1;
      for (int kb = 0; kb < nkb; ++kb) {
        const int s = kb % K_STAGES, slab = kb / K_SLAB, b = slab & 1;
        const bool first = kb % K_SLAB == 0;
        if (!mbar_wait(&full[s], (unsigned)((kb / K_STAGES) & 1)) ||
            (first && slab >= 2 && !mbar_wait(&acce[b], (unsigned)((slab / 2 - 1) & 1)))) {
          atomicOr(&fail, 1);
          break;
        }
        fence_after();
        const uint64_t ah = sdesc_sw128(a_addr(s, 0)), al = sdesc_sw128(a_addr(s, 1));
        const uint64_t bh = sdesc_sw128(b_addr(s, 0)), bl = sdesc_sw128(b_addr(s, 1));
        const unsigned d = tacc + (unsigned)(b * KN);
#pragma unroll
        for (int ks = 0; ks < BK / 8; ++ks) {
          const uint64_t adv = (uint64_t)((ks * 32) >> 4);
          mma_tf32(d, ah + adv, bh + adv, idesc, (first && ks == 0) ? 0u : 1u);
          mma_tf32(d, ah + adv, bl + adv, idesc, 1u);
          mma_tf32(d, al + adv, bh + adv, idesc, 1u);
        }
        mma_commit(&empty[s]);
        if (kb % K_SLAB == K_SLAB - 1 || kb == nkb - 1) {
          mma_commit(&accf[b]);
          last_slab = slab;
        } else {
          last_slab = -1;   // MMAs issued after the last slab commit: committed below
        }
      }
      // drain: a commit after the last MMA tracks all of them; wait for it before the
      // tensor memory is freed
      if (nkb > 0) {
        if (last_slab < 0) {
          // (only after a failure: the loop stopped inside a slab)
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                           smem_u32(&drain_bar))
                       : "memory");
          if (!mbar_wait(&drain_bar, 0u)) atomicOr(&fail, 1);
        } else if (!mbar_wait(&accf[last_slab & 1], (unsigned)((last_slab / 2) & 1))) {
          atomicOr(&fail, 1);
        }
      }
    }
  } else {
    // warps 0-7: TMEM lanes 32 (warp % 4) .. +31 (M = columns of block bi), 32 columns of N
    const int q = warp & 3, h = warp >> 2;
    float hi[32], lo[32];
#pragma unroll
    for (int a = 0; a < 32; ++a) {
      hi[a] = 0.f;
      lo[a] = 0.f;
    }
    bool ok = true;
    for (int slab = 0; slab < nslab; ++slab) {
      const int b = slab & 1;
      if (!mbar_wait(&accf[b], (unsigned)((slab / 2) & 1))) {
        ok = false;
        break;
      }
      fence_after();
      float v[32];
      tmem_ld32(tacc + ((unsigned)(32 * q) << 16) + (unsigned)(b * KN + h * 32), v);
      fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acce[b]);
#pragma unroll
      for (int a = 0; a < 32; ++a) {
        float sres, e;
        two_sum_f(hi[a], v[a], sres, e);
        hi[a] = sres;
        lo[a] += e;
      }
    }
    if (!ok || *(volatile int*)&fail) {
      if (lane == 0) atomicOr(err, ERRBIT_TIMEOUT);
    } else {
      double* out = part + ((int64_t)c * npairs + p) * K_TILE + (int64_t)(32 * q + lane) * KN + h * 32;
#pragma unroll
      for (int a = 0; a < 32; ++a) out[a] = (double)hi[a] + (double)lo[a];
    }
  }
  fence_before();
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tacc), "r"(K_TMEM_COLS) : "memory");
}

// K (n2 x n2, FP64) from the chunk partials of gram_kk_tf32x3: the entries with c1 <= c2 of
// every block, summed over the chunks in order, written to both triangles.
static __global__ void reduce_kk(const double* __restrict__ part, int nch, const int2* __restrict__ pairs,
                                 int npairs, int n2, double* __restrict__ K) {
  const int64_t total = (int64_t)npairs * K_TILE;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int p = (int)(e / K_TILE), rc = (int)(e % K_TILE);
    const int r = rc / KN, col = rc % KN;
    const int c1 = pairs[p].x * 128 + r, c2 = pairs[p].y * KN + col;
    if (c1 >= n2 || c2 >= n2 || c1 > c2) continue;
    double v = 0.0;
    for (int c = 0; c < nch; ++c) v += __ldcg(&part[((int64_t)c * npairs + p) * K_TILE + rc]);
    K[c1 + (int64_t)c2 * n2] = v;
    K[c2 + (int64_t)c1 * n2] = v;
  }
}

}  // namespace tc
}  // namespace wlr
