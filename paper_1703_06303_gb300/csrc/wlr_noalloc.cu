// wlr_x1_update_noalloc: the X1 row update (E and the per-row weighted solves) for a
// caller that cannot allocate device memory.  The paper has no counterpart; it is a
// packaging of the same kernels the handle-based solver runs.
//
// All scratch lives in one file-scope device array (kNoallocScratchBytes).  Host code
// never touches that array by name: the first call on a device, with that device
// current, looks up its device address with cudaGetSymbolAddress (and raises the
// kernels' shared-memory limit); later calls reuse the cached address.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/wlr.h"
#include "wlr_kernels.cuh"

namespace {

constexpr size_t kNoallocScratchBytes = (size_t)1 << 20;  // 1 MiB per device
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};
bool g_ready[kMaxDevices] = {};

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Z2 (row-major n2 x NP) = [C^T | V_s | 0]: row j holds C(:, j), then V_s(j, :), then zeros.
__global__ void pack_z2(const float* __restrict__ C, const float* __restrict__ Vs, int k, int n2,
                        int s, int NP, float* __restrict__ Z2) {
  const int64_t total = (int64_t)n2 * NP;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(e / NP), c = (int)(e % NP);
    float v = 0.f;
    if (c < k) v = C[c + (int64_t)j * k];
    else if (c < k + s) v = Vs[j + (int64_t)(c - k) * n2];
    Z2[e] = v;
  }
}

// The caller's status word gets a wlr_status code, not the kernels' error bits: the row
// pass can only report a row system that broke down (WLR_ERR_NOT_SPD).
__global__ void store_err(const int* __restrict__ err, int* __restrict__ out) {
  const int e = *err;
  *out = (e & wlr::ERRBIT_NOT_SPD) ? (int)WLR_ERR_NOT_SPD : (e != 0 ? (int)WLR_ERR_CUDA : (int)WLR_OK);
}

// First call on the current device: find the scratch array's device address and allow
// the row-pass kernels their dynamic shared memory.  Returns nullptr on failure.
void* setup_device(int dev, const char** why) {
  std::lock_guard<std::mutex> lock(g_mu);
  if (g_ready[dev]) return g_scratch_ptr[dev];
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) {
    *why = "cudaGetSymbolAddress failed for the scratch array";
    return nullptr;
  }
  const int limit = 200 * 1024;  // above the largest row-pass need (k = 64, r - k = 32)
  const void* fns[] = {(const void*)wlr::row_pass_fn<float>(8), (const void*)wlr::row_pass_fn<float>(16),
                       (const void*)wlr::row_pass_fn<float>(20), (const void*)wlr::row_pass_fn<float>(24),
                       (const void*)wlr::row_pass_fn<float>(32), (const void*)wlr::row_pass_fn<float>(64)};
  // raise, never lower: the limit is shared with the solver handles of the process
  bool ok = true;
  for (const void* f : fns) {
    cudaFuncAttributes fa;
    ok = ok && cudaFuncGetAttributes(&fa, f) == cudaSuccess;
    if (ok && fa.maxDynamicSharedSizeBytes < limit)
      ok = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, limit) == cudaSuccess;
  }
  if (!ok) {
    *why = "cudaFuncSetAttribute failed";
    return nullptr;
  }
  g_scratch_ptr[dev] = p;
  g_ready[dev] = true;
  return p;
}

// The reason goes where wlr_last_error(NULL) reads it (this entry point has no handle).
wlr_status fail(wlr_status st, const char* msg) {
  wlr::set_global_error(msg);
  return st;
}


// Bytes of scratch a problem needs (each piece padded to 256 bytes).
size_t scratch_bytes(int64_t m, int64_t n, int64_t k, int64_t r) {
  const int64_t n2 = n - k, s = r - k;
  const int64_t NP = ((k + s + 15) / 16) * 16;
  return align256(sizeof(float) * (size_t)(n2 > 0 ? n2 : 1) * NP) +
         align256(sizeof(float) * (size_t)k * k) +
         align256(sizeof(float) * (size_t)k * (s > 0 ? s : 1)) +
         align256(sizeof(double) * (size_t)((m + wlr::RP_BM - 1) / wlr::RP_BM)) + 256;
}

}  // namespace

extern "C" wlr_status wlr_x1_update_noalloc(const float* A, int64_t lda, const float* W1,
                                            int64_t ldw, const float* X1, int64_t m, int64_t n,
                                            int64_t k, int64_t r, const float* C,
                                            const float* Vs, float* X1_next, double* wterm,
                                            int* status, void* cuda_stream) {
  if (!A || !W1 || !X1 || !X1_next || (n > k && !C) || (r > k && n > k && !Vs))
    return fail(WLR_ERR_INVALID_ARG, "a required pointer is NULL");
  if (m < 1 || k < 1 || k > n || r < k || r > (m < n ? m : n) || lda < m || ldw < m)
    return fail(WLR_ERR_INVALID_ARG, "need 1 <= k <= n, k <= r <= min(m, n), lda >= m, ldw >= m");
  if (k > 64 || r - k > 32) return fail(WLR_ERR_UNSUPPORTED, "k <= 64 and r - k <= 32 only");
  if (m > (int64_t)1 << 30) return fail(WLR_ERR_UNSUPPORTED, "m <= 2^30 only");
  const size_t need = scratch_bytes(m, n, k, r);
  if (need > kNoallocScratchBytes)
    return fail(WLR_ERR_UNSUPPORTED,
                "problem needs more scratch than the fixed 1 MiB array");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return fail(WLR_ERR_CUDA, "cudaGetDevice failed");
  const char* why = "";
  unsigned char* base = (unsigned char*)setup_device(dev, &why);
  if (!base) return fail(WLR_ERR_CUDA, why);

  const int mi = (int)m, ki = (int)k, n2 = (int)(n - k), s = (int)(r - k);
  const int NP = ((ki + s + 15) / 16) * 16;
  size_t off = 0;
  float* Z2 = (float*)(base + off);
  off += align256(sizeof(float) * (size_t)(n2 > 0 ? n2 : 1) * NP);
  float* G = (float*)(base + off);
  off += align256(sizeof(float) * (size_t)ki * ki);
  float* CV = (float*)(base + off);
  off += align256(sizeof(float) * (size_t)ki * (s > 0 ? s : 1));
  double* wpart = (double*)(base + off);
  const int nblk = (mi + wlr::RP_BM - 1) / wlr::RP_BM;
  off += align256(sizeof(double) * (size_t)nblk);
  int* err = (int*)(base + off);

  cudaStream_t st = (cudaStream_t)cuda_stream;
  // The error word must start at zero; every other piece is fully overwritten below.
  if (cudaMemsetAsync(err, 0, sizeof(int), st) != cudaSuccess)
    return fail(WLR_ERR_CUDA, "cudaMemsetAsync failed");
  if (n2 > 0) {
    const int g = (int)(((int64_t)n2 * NP + 255) / 256);
    pack_z2<<<g < 4096 ? g : 4096, 256, 0, st>>>(C, Vs, ki, n2, s, NP, Z2);
  }
  wlr::prep_rowpass<float><<<ki, 128, 0, st>>>(C, Vs, ki, n2, s, G, CV);
  const size_t smem = wlr::RowPassSmem<float>::bytes(NP, ki, s);
  const wlr::FinalizeArgs<float> nofin{nullptr, 0, nullptr, nullptr, nullptr, 0, nullptr, nullptr, nullptr};
  wlr::row_pass_fn<float>(ki)<<<nblk, 256, smem, st>>>(A, lda, W1, ldw, X1, Z2, G, CV, mi, n2, ki, s, NP,
                                                      X1_next, wpart, err, nofin,
                                                      wlr::QSplitOut{nullptr, nullptr, 0, nullptr});
  if (wterm) wlr::reduce_partials<double><<<1, 32, 0, st>>>(wpart, 1, nblk, 1, wterm, nullptr);
  if (status) store_err<<<1, 1, 0, st>>>(err, status);
  if (cudaGetLastError() != cudaSuccess) return fail(WLR_ERR_CUDA, "kernel launch failed");
  wlr::set_global_error("");
  return WLR_OK;
}
