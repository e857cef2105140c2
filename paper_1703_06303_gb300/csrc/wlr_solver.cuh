// Host-side driver of the sWLR iteration: workspace, kernel sequence, CUDA graphs.
#pragma once

#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "../../include/wlr.h"

namespace wlr {

// Status-carrying error for the host driver; converted to wlr_status at the ABI.
struct Fail {
  wlr_status st;
  std::string msg;
};

#define WLR_CUDA(call)                                                                 \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess)                                                             \
      throw ::wlr::Fail{e_ == cudaErrorMemoryAllocation ? WLR_ERR_OOM : WLR_ERR_CUDA,  \
                        std::string(#call) + ": " + cudaGetErrorString(e_)};           \
  } while (0)

struct Dims {
  int m, n, k, r, s, n2, b, NP;
};

struct ProfEntry {
  std::string name;
  double ms;
  int launches;
};

// Interface shared by the float and double solvers.
class SolverBase {
 public:
  virtual ~SolverBase() {}
  virtual void set_data(const void* A, int64_t lda, const void* W1, int64_t ldw, wlr_dtype dt,
                        wlr_memory mem) = 0;
  virtual void set_init(wlr_init kind, const void* X1_0, int64_t ldx, wlr_dtype dt,
                        wlr_memory mem, uint64_t seed) = 0;
  virtual void step(double* F) = 0;
  virtual wlr_status solve(double tol, int max_iter, int* iters, double* F) = 0;
  virtual double objective_exact() = 0;
  virtual void get_result(void* X1, int64_t ldx, void* X2, int64_t ldx2, wlr_dtype dt,
                          wlr_memory mem) = 0;
  virtual void get_factors(double* C, double* Vs, double* sigma2) = 0;
  virtual int get_history(double* F, double* rel_err, int cap) = 0;
  virtual int iteration() = 0;
  virtual int64_t launches() const = 0;
  virtual int64_t state_bytes() = 0;
  virtual void get_state(void* buf) = 0;
  virtual void set_state(const void* buf, int64_t size) = 0;
  virtual std::vector<ProfEntry> profile(int reps) = 0;
  virtual void refine(void* X1_out, int64_t ldx, wlr_memory mem, double* Fp, double* Fnext) = 0;

  // Device view for the warm-start code: the data, the current X1 and (with_factors) the
  // factors C (k x n2) and V_s (n2 x s) of its (C, D) step, column-major, element type
  // float or double (fp64).  Work on `stream` is ordered after the handle's and the handle's
  // later work after it.  Pointers stay valid until the next call on the handle.
  struct View {
    const void* A;
    int64_t lda;
    const void* W1;
    int64_t ldw;
    const void* X1;
    const void* C;
    const void* Vs;
    cudaStream_t stream;
    bool fp64;
  };
  // Start the rank-(r-k) subspace iteration from the given basis (n2 x b columns, float or
  // double, column-major, device) instead of a random one: the first min(b, this b) columns
  // are taken, the rest stay random.  Used by the FP64 scorer of a float handle, which then
  // starts from the float iteration's own, nearly converged, subspace.
  virtual void seed_subspace(const void* V, int b, bool fp64) = 0;
  virtual View view(bool with_factors) = 0;
  virtual Dims dims() const = 0;
  virtual cudaStream_t user_stream() const = 0;

  // Batched solve (wlr_solve_batched).  batch_ready: the next iterations replay as a
  // graph (data and init set, warm-up done).  batch_iterate: one iteration on the handle's
  // own stream.  batch_capture: n iterations captured into a graph that is not run; the
  // caller joins the graphs of all handles and launches them.  batch_advance: the host
  // bookkeeping after one launch of that graph.  batch_enter / batch_leave order the batch
  // stream after this handle's earlier work and the handle's later work after the batch.
  // batch_finish: synchronise and raise the handle's device-side errors.
  virtual bool batch_ready() = 0;
  virtual void batch_iterate() = 0;
  virtual cudaGraph_t batch_capture(int n) = 0;
  virtual void batch_advance(int n) = 0;
  virtual void batch_enter(cudaStream_t bs) = 0;
  virtual void batch_leave(cudaStream_t bs) = 0;
  virtual void batch_finish() = 0;
};

SolverBase* make_solver_f32(const Dims& d, const wlr_options& o, cudaStream_t user_stream);
SolverBase* make_solver_f64(const Dims& d, const wlr_options& o, cudaStream_t user_stream);

// Host: set the message that wlr_last_error(NULL) returns (calls without a handle).
void set_global_error(const char* msg);

}  // namespace wlr

// The object behind a wlr_handle.  perm: the caller's column order of A when the weighted
// frames were given as an index set (wlr_set_data_cols): column q of the problem the solver
// sees is the caller's column perm[q]; empty means the identity.
struct wlr_handle_s {
  wlr::SolverBase* impl = nullptr;
  std::string last_error;
  std::vector<int> perm;
  void* perm_buf = nullptr;     // the permuted copy of A (device data)
  size_t perm_bytes = 0;
  int* perm_dev = nullptr;
  ~wlr_handle_s() {
    if (perm_buf) cudaFree(perm_buf);
    if (perm_dev) cudaFree(perm_dev);
  }
};
