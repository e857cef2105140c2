// extern "C" entry points of libwlr.so (declared in include/wlr.h).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <new>
#include <string>
#include <vector>
#include <climits>

#include "wlr_solver.cuh"


namespace {
thread_local std::string g_create_error;
}  // namespace

namespace wlr {
// Message for wlr_last_error(NULL): failures of calls that have no handle.
void set_global_error(const char* msg) { g_create_error = msg ? msg : ""; }
}  // namespace wlr

namespace {

wlr_status fail(wlr_handle h, wlr_status st, const std::string& msg) {
  if (h) h->last_error = msg;
  else g_create_error = msg;
  return st;
}

template <typename F>
wlr_status guarded(wlr_handle h, F&& f) {
  if (!h || !h->impl) return fail(nullptr, WLR_ERR_INVALID_ARG, "NULL handle");
  try {
    wlr_status st = f();
    if (st == WLR_OK) h->last_error.clear();
    return st;
  } catch (const wlr::Fail& e) {
    return fail(h, e.st, e.msg);
  } catch (const std::bad_alloc&) {
    return fail(h, WLR_ERR_OOM, "host allocation failed");
  } catch (...) {
    return fail(h, WLR_ERR_CUDA, "unexpected failure");
  }
}
}  // namespace

extern "C" {

void wlr_default_options(wlr_options* opt) {
  if (!opt) return;
  opt->precision = WLR_PREC_FP32;
  opt->stop = WLR_STOP_RELATIVE;
  opt->eig_block = 0;
  opt->eig_iters = 0;
  opt->eig_iters_cold = 0;
  opt->use_graph = 1;
  opt->seed = 0x1703063032ull;
  opt->autotune = 0;
}

wlr_status wlr_create(wlr_handle* out, int64_t m, int64_t n, int64_t k, int64_t r,
                      const wlr_options* opt, void* cuda_stream) {
  if (!out) return fail(nullptr, WLR_ERR_INVALID_ARG, "out must be non-NULL");
  *out = nullptr;
  if (m < 1 || n < 1 || k < 1 || k > n || r < k || r > std::min(m, n))
    return fail(nullptr, WLR_ERR_INVALID_ARG,
                "need m >= 1, n >= 1, 1 <= k <= n and k <= r <= min(m, n)");
  if (m > (int64_t)1 << 30 || n > 65536)
    return fail(nullptr, WLR_ERR_UNSUPPORTED, "m up to 2^30 and n up to 65536 are supported");
  if (k > 64) return fail(nullptr, WLR_ERR_UNSUPPORTED, "k <= 64 is supported");
  if (r - k > 32) return fail(nullptr, WLR_ERR_UNSUPPORTED, "r - k <= 32 is supported");
  wlr_options o;
  wlr_default_options(&o);
  if (opt) o = *opt;
  if (o.precision != WLR_PREC_FP32 && o.precision != WLR_PREC_FP64)
    return fail(nullptr, WLR_ERR_INVALID_ARG, "unknown precision");
  if (o.stop < WLR_STOP_PAPER || o.stop > WLR_STOP_OBJECTIVE)
    return fail(nullptr, WLR_ERR_INVALID_ARG, "unknown stop rule");
  if (o.eig_iters <= 0) o.eig_iters = 1;
  if (o.eig_iters_cold <= 0) o.eig_iters_cold = 40;
  wlr::Dims d;
  d.m = (int)m;
  d.n = (int)n;
  d.k = (int)k;
  d.r = (int)r;
  d.s = (int)(r - k);
  d.n2 = (int)(n - k);
  const int bmax = std::min(d.n2, 32);
  int b = o.eig_block > 0 ? o.eig_block : std::max(d.s + 8, 2 * d.s);
  b = std::min(b, bmax);
  if (d.s > 0 && b < d.s)
    return fail(nullptr, WLR_ERR_INVALID_ARG, "eig_block must be >= r - k");
  d.b = d.s > 0 ? b : 0;
  d.NP = ((d.k + d.s + 15) / 16) * 16;
  wlr_handle h = new (std::nothrow) wlr_handle_s;
  if (!h) return fail(nullptr, WLR_ERR_OOM, "host allocation failed");
  try {
    cudaStream_t us = (cudaStream_t)cuda_stream;
    h->impl = o.precision == WLR_PREC_FP64 ? wlr::make_solver_f64(d, o, us)
                                           : wlr::make_solver_f32(d, o, us);
  } catch (const wlr::Fail& e) {
    delete h;
    return fail(nullptr, e.st, e.msg);
  } catch (...) {
    delete h;
    return fail(nullptr, WLR_ERR_CUDA, "solver construction failed");
  }
  *out = h;
  return WLR_OK;
}

wlr_status wlr_set_data(wlr_handle h, const void* A, int64_t lda, const void* W1, int64_t ldw,
                        wlr_dtype dt, wlr_memory mem) {
  return guarded(h, [&] {
    if (dt != WLR_F32 && dt != WLR_F64) throw wlr::Fail{WLR_ERR_INVALID_ARG, "unknown dtype"};
    h->impl->set_data(A, lda, W1, ldw, dt, mem);
    h->perm.clear();
    return WLR_OK;
  });
}

wlr_status wlr_set_init(wlr_handle h, wlr_init kind, const void* X1_0, int64_t ldx,
                        wlr_dtype dt, wlr_memory mem, uint64_t seed) {
  return guarded(h, [&] {
    h->impl->set_init(kind, X1_0, ldx, dt, mem, seed);
    return WLR_OK;
  });
}

wlr_status wlr_step(wlr_handle h, double* objective_out) {
  return guarded(h, [&] {
    h->impl->step(objective_out);
    return WLR_OK;
  });
}

wlr_status wlr_solve(wlr_handle h, double tol, int32_t max_iter, int32_t* iters_out,
                     double* objective_out) {
  return guarded(h, [&] {
    int it = 0;
    double F = 0;
    wlr_status st = h->impl->solve(tol, max_iter, &it, &F);
    if (iters_out) *iters_out = it;
    if (objective_out) *objective_out = F;
    if (st == WLR_ERR_NO_CONVERGENCE) h->last_error = "max_iter reached before the stopping rule held";
    return st;
  });
}

wlr_status wlr_solve_batched(wlr_handle* hs, int32_t count, int32_t iters, int32_t* failed_index) {
  if (failed_index) *failed_index = -1;
  if (count < 0 || iters < 0) return fail(nullptr, WLR_ERR_INVALID_ARG, "count and iters must be >= 0");
  if (count == 0) return WLR_OK;
  if (!hs) return fail(nullptr, WLR_ERR_INVALID_ARG, "handles must be non-NULL");
  for (int i = 0; i < count; ++i) {
    if (!hs[i] || !hs[i]->impl) return fail(nullptr, WLR_ERR_INVALID_ARG, "NULL handle in the batch");
    for (int j = 0; j < i; ++j)
      if (hs[j] == hs[i]) return fail(hs[0], WLR_ERR_INVALID_ARG, "a handle appears twice in the batch");
  }
  auto at = [&](int i, wlr_status st) {
    if (failed_index) *failed_index = i;
    return st;
  };
  // warm-up on each handle alone
  std::vector<int> left(count, iters);
  std::vector<char> joined(count, 0);
  for (int i = 0; i < count; ++i) {
    wlr::SolverBase* s = hs[i]->impl;
    const wlr_status st = guarded(hs[i], [&] {
      while (left[i] > 0 && !s->batch_ready()) {
        s->batch_iterate();
        --left[i];
      }
      joined[i] = s->batch_ready() ? 1 : 0;
      return WLR_OK;
    });
    if (st != WLR_OK) return at(i, st);
  }
  int nb = INT32_MAX;
  for (int i = 0; i < count; ++i)
    if (joined[i]) nb = std::min(nb, left[i] / 3);
  if (nb == INT32_MAX) nb = 0;
  if (nb > 0) {
    cudaStream_t bs = nullptr;
    cudaGraph_t parent = nullptr;
    cudaGraphExec_t exec = nullptr;
    auto cleanup = [&] {
      if (bs) cudaStreamSynchronize(bs);
      cudaGetLastError();
      if (exec) cudaGraphExecDestroy(exec);
      if (parent) cudaGraphDestroy(parent);
      if (bs) cudaStreamDestroy(bs);
    };
    auto cuda_fail = [&](cudaError_t e, const char* what) {
      cleanup();
      return fail(hs[0], WLR_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
    };
    cudaError_t e = cudaStreamCreateWithFlags(&bs, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_fail(e, "batch stream");
    e = cudaGraphCreate(&parent, 0);
    if (e != cudaSuccess) return cuda_fail(e, "batch graph");
    for (int i = 0; i < count; ++i) {
      if (!joined[i]) continue;
      cudaGraph_t g = nullptr;
      const wlr_status st = guarded(hs[i], [&] {
        g = hs[i]->impl->batch_capture(3);
        return WLR_OK;
      });
      if (st != WLR_OK) {
        cleanup();
        return at(i, st);
      }
      cudaGraphNode_t node;
      e = cudaGraphAddChildGraphNode(&node, parent, nullptr, 0, g);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) return cuda_fail(e, "batch graph node");
    }
    e = cudaGraphInstantiate(&exec, parent, 0);
    if (e != cudaSuccess) return cuda_fail(e, "batch graph instantiation");
    for (int i = 0; i < count; ++i) {
      if (!joined[i]) continue;
      const wlr_status st = guarded(hs[i], [&] {
        hs[i]->impl->batch_enter(bs);
        return WLR_OK;
      });
      if (st != WLR_OK) {
        cleanup();
        return at(i, st);
      }
    }
    for (int b = 0; b < nb && e == cudaSuccess; ++b) e = cudaGraphLaunch(exec, bs);
    if (e != cudaSuccess) return cuda_fail(e, "batch graph launch");
    for (int i = 0; i < count; ++i) {
      if (!joined[i]) continue;
      const wlr_status st = guarded(hs[i], [&] {
        for (int b = 0; b < nb; ++b) hs[i]->impl->batch_advance(3);
        hs[i]->impl->batch_leave(bs);
        return WLR_OK;
      });
      left[i] -= 3 * nb;
      if (st != WLR_OK) {
        cleanup();
        return at(i, st);
      }
    }
    e = cudaStreamSynchronize(bs);
    cudaGraphExecDestroy(exec);
    exec = nullptr;
    cudaGraphDestroy(parent);
    parent = nullptr;
    cudaStreamDestroy(bs);
    bs = nullptr;
    if (e != cudaSuccess) return fail(hs[0], WLR_ERR_CUDA, std::string("batch: ") + cudaGetErrorString(e));
  }
  // the rest on each handle alone, then every handle's device-side status
  for (int i = 0; i < count; ++i) {
    wlr::SolverBase* s = hs[i]->impl;
    const wlr_status st = guarded(hs[i], [&] {
      for (; left[i] > 0; --left[i]) s->batch_iterate();
      s->batch_finish();
      return WLR_OK;
    });
    if (st != WLR_OK) return at(i, st);
  }
  return WLR_OK;
}

wlr_status wlr_refine(wlr_handle h, double* X1_out, int64_t ldx, wlr_memory mem, double* F_out,
                      double* F_next_out) {
  return guarded(h, [&] {
    if (mem != WLR_MEM_DEVICE && mem != WLR_MEM_HOST) throw wlr::Fail{WLR_ERR_INVALID_ARG, "bad memory kind"};
    h->impl->refine(X1_out, ldx, mem, F_out, F_next_out);
    return WLR_OK;
  });
}

wlr_status wlr_objective(wlr_handle h, double* F_out) {
  return guarded(h, [&] {
    if (!F_out) throw wlr::Fail{WLR_ERR_INVALID_ARG, "F_out must be non-NULL"};
    *F_out = h->impl->objective_exact();
    return WLR_OK;
  });
}

wlr_status wlr_get_result(wlr_handle h, void* X1, int64_t ldx, void* X2, int64_t ldx2,
                          wlr_dtype dt, wlr_memory mem) {
  return guarded(h, [&] {
    h->impl->get_result(X1, ldx, X2, ldx2, dt, mem);
    return WLR_OK;
  });
}

wlr_status wlr_get_factors(wlr_handle h, double* C, double* Vs, double* sigma2) {
  return guarded(h, [&] {
    h->impl->get_factors(C, Vs, sigma2);
    return WLR_OK;
  });
}

wlr_status wlr_get_history(wlr_handle h, double* F, double* rel_err, int32_t cap,
                           int32_t* count_out) {
  return guarded(h, [&] {
    const int n = h->impl->get_history(F, rel_err, cap);
    if (count_out) *count_out = n;
    return WLR_OK;
  });
}

wlr_status wlr_get_iteration(wlr_handle h, int32_t* p_out) {
  return guarded(h, [&] {
    if (!p_out) throw wlr::Fail{WLR_ERR_INVALID_ARG, "p_out must be non-NULL"};
    *p_out = h->impl->iteration();
    return WLR_OK;
  });
}

wlr_status wlr_get_state(wlr_handle h, void* buf, int64_t cap, int64_t* size_out) {
  return guarded(h, [&] {
    const int64_t need = h->impl->state_bytes();
    if (size_out) *size_out = need;
    if (!buf) return WLR_OK;
    if (cap < need) throw wlr::Fail{WLR_ERR_INVALID_ARG, "cap is smaller than the state size"};
    h->impl->get_state(buf);
    return WLR_OK;
  });
}

wlr_status wlr_set_state(wlr_handle h, const void* buf, int64_t size) {
  return guarded(h, [&] {
    h->impl->set_state(buf, size);
    return WLR_OK;
  });
}

wlr_status wlr_destroy(wlr_handle h) {
  if (!h) return WLR_OK;
  delete h->impl;
  delete h;
  return WLR_OK;
}

const char* wlr_status_string(wlr_status s) {
  switch (s) {
    case WLR_OK: return "WLR_OK";
    case WLR_ERR_INVALID_ARG: return "WLR_ERR_INVALID_ARG";
    case WLR_ERR_NONPOSITIVE_WEIGHT: return "WLR_ERR_NONPOSITIVE_WEIGHT";
    case WLR_ERR_RANK_DEFICIENT: return "WLR_ERR_RANK_DEFICIENT";
    case WLR_ERR_NOT_SPD: return "WLR_ERR_NOT_SPD";
    case WLR_ERR_NO_CONVERGENCE: return "WLR_ERR_NO_CONVERGENCE";
    case WLR_ERR_DEVICE_TIMEOUT: return "WLR_ERR_DEVICE_TIMEOUT";
    case WLR_ERR_CUDA: return "WLR_ERR_CUDA";
    case WLR_ERR_OOM: return "WLR_ERR_OOM";
    case WLR_ERR_NOT_READY: return "WLR_ERR_NOT_READY";
    case WLR_ERR_UNSUPPORTED: return "WLR_ERR_UNSUPPORTED";
  }
  return "WLR_ERR_UNKNOWN";
}

const char* wlr_last_error(wlr_handle h) {
  return h ? h->last_error.c_str() : g_create_error.c_str();
}

int64_t wlr_kernel_launches(wlr_handle h) { return (h && h->impl) ? h->impl->launches() : 0; }

}  // extern "C"

extern "C" wlr_status wlr_profile(wlr_handle h, int32_t reps, char* names, int32_t names_cap,
                                  double* ms_total, int32_t* launches, int32_t max_kernels,
                                  int32_t* n_kernels) {
  return guarded(h, [&] {
    if (reps < 1) throw wlr::Fail{WLR_ERR_INVALID_ARG, "reps must be >= 1"};
    auto v = h->impl->profile(reps);
    std::string all;
    const int n = std::min<int>((int)v.size(), max_kernels);
    for (int q = 0; q < n; ++q) {
      if (ms_total) ms_total[q] = v[q].ms;
      if (launches) launches[q] = v[q].launches;
      all += v[q].name;
      all += '\n';
    }
    if (names && names_cap > 0) {
      const size_t c = std::min<size_t>(all.size(), (size_t)names_cap - 1);
      std::memcpy(names, all.data(), c);
      names[c] = 0;
    }
    if (n_kernels) *n_kernels = n;
    return WLR_OK;
  });
}
