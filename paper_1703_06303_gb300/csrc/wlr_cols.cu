// Weighted frames given as an arbitrary index set (wlr_set_data_cols) and the full
// X = (X1, X2) in the caller's column order (wlr_get_x).  Eq. 5 and Algorithm 1 take the k
// weighted frames as the first columns of A; these entry points permute A's columns so
// that they are, and put the result's columns back.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "../../include/wlr.h"
#include "wlr_solver.cuh"

namespace {

// out(:, q) = in(:, perm[q]) for q < n (element size ES bytes; columns of `rows` elements)
template <int ES>
__global__ void gather_cols(const unsigned char* __restrict__ in, int64_t ld_in, int rows, int n,
                            const int* __restrict__ perm, unsigned char* __restrict__ out,
                            int64_t ld_out) {
  const int64_t total = (int64_t)rows * n;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int q = (int)(t / rows), i = (int)(t - (int64_t)q * rows);
    const unsigned char* src = in + ((int64_t)perm[q] * ld_in + i) * ES;
    unsigned char* dst = out + ((int64_t)q * ld_out + i) * ES;
#pragma unroll
    for (int b = 0; b < ES; ++b) dst[b] = src[b];
  }
}

// out(:, perm[q]) = in(:, q)
template <int ES>
__global__ void scatter_cols(const unsigned char* __restrict__ in, int64_t ld_in, int rows, int n,
                             const int* __restrict__ perm, unsigned char* __restrict__ out,
                             int64_t ld_out) {
  const int64_t total = (int64_t)rows * n;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int q = (int)(t / rows), i = (int)(t - (int64_t)q * rows);
    const unsigned char* src = in + ((int64_t)q * ld_in + i) * ES;
    unsigned char* dst = out + ((int64_t)perm[q] * ld_out + i) * ES;
#pragma unroll
    for (int b = 0; b < ES; ++b) dst[b] = src[b];
  }
}

int grid_of(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 1 << 20)); }

template <typename F>
wlr_status guard(wlr_handle h, F&& f) {
  if (!h || !h->impl) {
    wlr::set_global_error("NULL handle");
    return WLR_ERR_INVALID_ARG;
  }
  try {
    const wlr_status st = f();
    if (st == WLR_OK) h->last_error.clear();
    return st;
  } catch (const wlr::Fail& e) {
    h->last_error = e.msg;
    return e.st;
  } catch (const std::bad_alloc&) {
    h->last_error = "host allocation failed";
    return WLR_ERR_OOM;
  }
}

void ensure_perm_dev(wlr_handle h, int n, cudaStream_t st) {
  if (!h->perm_dev) WLR_CUDA(cudaMalloc(&h->perm_dev, sizeof(int) * 65536));
  WLR_CUDA(cudaMemcpyAsync(h->perm_dev, h->perm.data(), sizeof(int) * n, cudaMemcpyHostToDevice, st));
  WLR_CUDA(cudaStreamSynchronize(st));   // the host vector may change after the call
}

}  // namespace

extern "C" wlr_status wlr_set_data_cols(wlr_handle h, const void* A, int64_t lda, const void* W1,
                                        int64_t ldw, wlr_dtype dt, wlr_memory mem,
                                        const int32_t* cols) {
  return guard(h, [&]() -> wlr_status {
    const wlr::Dims d = h->impl->dims();
    const int m = d.m, n = d.n, k = d.k;
    if (!A || !W1 || !cols) throw wlr::Fail{WLR_ERR_INVALID_ARG, "A, W1 and cols must be non-NULL"};
    if (dt != WLR_F32 && dt != WLR_F64) throw wlr::Fail{WLR_ERR_INVALID_ARG, "unknown dtype"};
    if (lda < m || ldw < m) throw wlr::Fail{WLR_ERR_INVALID_ARG, "lda and ldw must be >= m"};
    std::vector<char> seen(n, 0);
    std::vector<int> perm;
    perm.reserve(n);
    for (int a = 0; a < k; ++a) {
      const int c = cols[a];
      if (c < 0 || c >= n || seen[c]) throw wlr::Fail{WLR_ERR_INVALID_ARG, "cols must be k distinct indices in [0, n)"};
      seen[c] = 1;
      perm.push_back(c);
    }
    for (int q = 0; q < n; ++q)
      if (!seen[q]) perm.push_back(q);
    const size_t es = dt == WLR_F64 ? 8 : 4;
    cudaStream_t st = h->impl->user_stream();
    h->perm = perm;
    if (mem == WLR_MEM_DEVICE) {
      const size_t bytes = es * (size_t)m * n;
      if (h->perm_bytes < bytes) {
        if (h->perm_buf) {
          WLR_CUDA(cudaStreamSynchronize(st));
          cudaFree(h->perm_buf);
          h->perm_buf = nullptr;
          h->perm_bytes = 0;
        }
        WLR_CUDA(cudaMalloc(&h->perm_buf, bytes));
        h->perm_bytes = bytes;
      }
      ensure_perm_dev(h, n, st);
      if (es == 8)
        gather_cols<8><<<grid_of((int64_t)m * n), 256, 0, st>>>((const unsigned char*)A, lda, m, n, h->perm_dev,
                                                               (unsigned char*)h->perm_buf, m);
      else
        gather_cols<4><<<grid_of((int64_t)m * n), 256, 0, st>>>((const unsigned char*)A, lda, m, n, h->perm_dev,
                                                               (unsigned char*)h->perm_buf, m);
      if (cudaGetLastError() != cudaSuccess) throw wlr::Fail{WLR_ERR_CUDA, "gather kernel launch failed"};
      h->impl->set_data(h->perm_buf, m, W1, ldw, dt, WLR_MEM_DEVICE);
    } else {
      std::vector<unsigned char> buf(es * (size_t)m * n);
      for (int q = 0; q < n; ++q)
        std::memcpy(buf.data() + es * (size_t)q * m, (const unsigned char*)A + es * (size_t)perm[q] * lda, es * m);
      h->impl->set_data(buf.data(), m, W1, ldw, dt, WLR_MEM_HOST);   // copied; synchronises
    }
    return WLR_OK;
  });
}

extern "C" wlr_status wlr_get_x(wlr_handle h, void* X, int64_t ldx, wlr_dtype dt, wlr_memory mem) {
  return guard(h, [&]() -> wlr_status {
    const wlr::Dims d = h->impl->dims();
    const int m = d.m, n = d.n, k = d.k;
    if (!X || ldx < m) throw wlr::Fail{WLR_ERR_INVALID_ARG, "X must be non-NULL with ldx >= m"};
    if (dt != WLR_F32 && dt != WLR_F64) throw wlr::Fail{WLR_ERR_INVALID_ARG, "unknown dtype"};
    const size_t es = dt == WLR_F64 ? 8 : 4;
    if (h->perm.empty()) {
      // the caller's order is the solver's: X1 and X2 go straight into X
      unsigned char* x = (unsigned char*)X;
      h->impl->get_result(x, ldx, n > k ? x + es * (size_t)k * ldx : nullptr, ldx, dt, mem);
      return WLR_OK;
    }
    cudaStream_t st = h->impl->user_stream();
    if (mem == WLR_MEM_DEVICE) {
      void* tmp = nullptr;
      WLR_CUDA(cudaMalloc(&tmp, es * (size_t)m * n));
      try {
        unsigned char* t = (unsigned char*)tmp;
        h->impl->get_result(t, m, n > k ? t + es * (size_t)k * m : nullptr, m, dt, WLR_MEM_DEVICE);
        ensure_perm_dev(h, n, st);
        if (es == 8)
          scatter_cols<8><<<grid_of((int64_t)m * n), 256, 0, st>>>(t, m, m, n, h->perm_dev, (unsigned char*)X, ldx);
        else
          scatter_cols<4><<<grid_of((int64_t)m * n), 256, 0, st>>>(t, m, m, n, h->perm_dev, (unsigned char*)X, ldx);
        if (cudaGetLastError() != cudaSuccess) throw wlr::Fail{WLR_ERR_CUDA, "scatter kernel launch failed"};
        WLR_CUDA(cudaStreamSynchronize(st));
      } catch (...) {
        cudaStreamSynchronize(st);
        cudaFree(tmp);
        throw;
      }
      cudaFree(tmp);
    } else {
      std::vector<unsigned char> buf(es * (size_t)m * n);
      h->impl->get_result(buf.data(), m, n > k ? buf.data() + es * (size_t)k * m : nullptr, m, dt, WLR_MEM_HOST);
      for (int q = 0; q < n; ++q)
        std::memcpy((unsigned char*)X + es * (size_t)h->perm[q] * ldx, buf.data() + es * (size_t)q * m, es * m);
    }
    return WLR_OK;
  });
}
