// Solver<T>: the sWLR iteration (Algorithm 1 of Dutta & Li) on one CUDA stream.
// Included by wlr_solver_f32.cu and wlr_solver_f64.cu, one instantiation each.
#pragma once

#include <map>
#include <mutex>
#include <tuple>
#include <vector>
#include <climits>
#include <algorithm>
#include <type_traits>

#include <cudaTypedefs.h>

#include "wlr_dstep.cuh"
#include "wlr_plan.h"
#include "wlr_kernels.cuh"
#include "wlr_solver.cuh"
#include "wlr_tc.cuh"

namespace wlr {

template <typename T>
constexpr wlr_dtype dtype_of() {
  return std::is_same<T, float>::value ? WLR_F32 : WLR_F64;
}


template <typename T>
class Solver final : public SolverBase {
 public:
  Solver(const Dims& d, const wlr_options& o, cudaStream_t us) : d_(d), o_(o), ustream_(us) {
    WLR_CUDA(cudaStreamCreateWithFlags(&stream_, cudaStreamNonBlocking));
    WLR_CUDA(cudaStreamCreateWithFlags(&stream2_, cudaStreamNonBlocking));
    WLR_CUDA(cudaEventCreateWithFlags(&ev_fork_, cudaEventDisableTiming));
    WLR_CUDA(cudaEventCreateWithFlags(&ev_join_, cudaEventDisableTiming));
    WLR_CUDA(cudaEventCreateWithFlags(&ev_in_, cudaEventDisableTiming));
    WLR_CUDA(cudaEventCreateWithFlags(&ev_out_, cudaEventDisableTiming));
    WLR_CUDA(cudaEventCreateWithFlags(&ev_batch_, cudaEventDisableTiming));
    WLR_CUDA(cudaHostAlloc((void**)&hbuf_, 4096, cudaHostAllocDefault));
    const int m = d_.m, k = d_.k, n2 = d_.n2, s = d_.s, b = d_.b, NP = d_.NP;
    for (int q = 0; q < 3; ++q) X1buf_[q] = dalloc<T>((size_t)m * k);
    Q1_ = dalloc<T>((size_t)m * k);
    // chunking of the split-m Gram products
    ch_S1_ = chunking(m, 1, 64);
    ch_T_ = chunking(m, (size_t)cdiv(k + n2, 64), 608);
    ch_K_ = chunking(m, (size_t)std::max(1, cdiv(n2, 64)) * std::max(1, cdiv(n2, 64)), 608);
    const size_t L = (size_t)k * k + (size_t)k * n2;
    size_t part_elems = std::max((size_t)ch_S1_.nch * k * k, (size_t)ch_T_.nch * L);
    part_elems = std::max(part_elems, (size_t)ch_K_.nch * n2 * n2);
    part64_ = dalloc<double>(std::max<size_t>(part_elems, 1));
    part_elems_ = std::max<size_t>(part_elems, 1);
    S2T_ = dalloc<double>(L);
    F2_ = dalloc<T>((size_t)k * k);
    R1inv_ = dalloc<T>((size_t)k * k);
    Nm_ = dalloc<T>((size_t)k * k);
    Rinv_ = dalloc<T>((size_t)k * k);
    C_ = dalloc<T>(std::max<size_t>((size_t)k * n2, 1));
    B64_ = dalloc<double>(std::max<size_t>((size_t)k * n2, 1));
    Bh_ = dalloc<float>(std::max<size_t>((size_t)k * n2, 1));
    Bl_ = dalloc<float>(std::max<size_t>((size_t)k * n2, 1));
    Z2_ = dalloc<T>(std::max<size_t>((size_t)n2 * NP, 1));
    Z2prev_ = dalloc<T>(std::max<size_t>((size_t)n2 * NP, 1));
    nblk_coef_ = cdiv(n2, 8);
    bpart_ = dalloc<double>(std::max(nblk_coef_, 1));
    K64_ = dalloc<double>(std::max<size_t>((size_t)n2 * n2, 1));
    G2_ = dalloc<T>(std::max<size_t>((size_t)n2 * n2, 1));
    nblk_prep_ = cdiv(n2, 64);
    prep_part_ = dalloc<double>((size_t)std::max(nblk_prep_, 1) * k * (k + std::max(s, 0)));
    prep_ticket_ = dalloc<unsigned int>(1);
    normA2_ = dalloc<double>(1);
    nblk_eig_ = cdiv(n2, 8);
    const int bb = std::max(b, 1);
    V_ = dalloc<T>((size_t)std::max(n2, 1) * bb);
    Zeig_ = dalloc<T>((size_t)std::max(n2, 1) * bb);
    eigpart_ = dalloc<T>((size_t)std::max(nblk_eig_, 1) * 2 * bb * bb);
    Y_ = dalloc<T>((size_t)bb * bb);
    Mv_ = dalloc<T>((size_t)bb * bb);
    Mz_ = dalloc<T>((size_t)bb * bb);
    theta_ = dalloc<T>(bb);
    HP_ = dalloc<T>(2 * (size_t)bb * bb);
    eig_ticket_ = dalloc<unsigned int>(1);
    fin_ticket_ = dalloc<unsigned int>(1);
    resid_ = dalloc<T>(bb);
    Vs_ = dalloc<T>((size_t)std::max(n2, 1) * std::max(s, 1));
    G_ = dalloc<T>((size_t)k * k);
    CV_ = dalloc<T>((size_t)k * std::max(s, 1));
    CVprev_ = dalloc<T>((size_t)k * std::max(s, 1));
    nblk_row_ = cdiv(m, RP_BM);
    wpart_ = dalloc<double>(nblk_row_);
    x2part_ = dalloc<double>((size_t)nblk_row_ * 8);
    x2sum_ = dalloc<double>(8);
    hist_cap_ = 1 << 16;
    Fhist_ = dalloc<double>(hist_cap_);
    Fcur_ = dalloc<double>(1);
    iter_ = dalloc<int>(1);
    err_ = dalloc<int>(1);
    if (std::is_same<T, float>::value && n2 > 0) setup_tc();
    setup_dstep();
    WLR_CUDA(cudaMemsetAsync(Z2_, 0, sizeof(T) * std::max<size_t>((size_t)n2 * NP, 1), stream_));
    WLR_CUDA(cudaMemsetAsync(Z2prev_, 0, sizeof(T) * std::max<size_t>((size_t)n2 * NP, 1), stream_));
    WLR_CUDA(cudaMemsetAsync(err_, 0, sizeof(int), stream_));
    WLR_CUDA(cudaMemsetAsync(iter_, 0, sizeof(int), stream_));
    WLR_CUDA(cudaMemsetAsync(CV_, 0, sizeof(T) * k * std::max(s, 1), stream_));
    WLR_CUDA(cudaMemsetAsync(CVprev_, 0, sizeof(T) * k * std::max(s, 1), stream_));
    WLR_CUDA(cudaMemsetAsync(bpart_, 0, sizeof(double) * std::max(nblk_coef_, 1), stream_));
    WLR_CUDA(cudaMemsetAsync(prep_ticket_, 0, sizeof(unsigned int), stream_));
    WLR_CUDA(cudaMemsetAsync(eig_ticket_, 0, sizeof(unsigned int), stream_));
    WLR_CUDA(cudaMemsetAsync(fin_ticket_, 0, sizeof(unsigned int), stream_));
    WLR_CUDA(cudaMemsetAsync(G_, 0, sizeof(T) * k * k, stream_));
    // dynamic shared memory limits
    set_smem((const void*)row_pass_fn<T>(k), RowPassSmem<T>::bytes(NP, k, s));
    set_smem((const void*)x2_pass<T>, x2_smem());
    set_smem((const void*)coef_kernel3<T>, sizeof(T) * (2 * k * k + 16 * 64));
    set_smem((const void*)chol1_kernel<T>, sizeof(double) * (2 * k * k + k));
    set_smem((const void*)chol2_kernel<T>, 3 * sizeof(T) * k * k);
    set_smem((const void*)prep_gram<T>, sizeof(T) * 64 * (NP + 1));
    eig_vsmem_ = (size_t)n2 * std::max(b, 1) * sizeof(T) <= 200 * 1024;
    if (eig_vsmem_) set_smem((const void*)eig_mult<T, true>, (size_t)n2 * std::max(b, 1) * sizeof(T));
    WLR_CUDA(cudaStreamSynchronize(stream_));
  }

  ~Solver() override {
    for (auto& g : graphs_) cudaGraphExecDestroy(g.second);
    for (auto& g : graphs3_) cudaGraphExecDestroy(g.second);
    for (auto e : ev_pool_) cudaEventDestroy(e);
    if (scorer_) delete scorer_;
    for (void* p : allocs_) cudaFree(p);
    if (hbuf_) cudaFreeHost(hbuf_);
    cudaEventDestroy(ev_in_);
    cudaEventDestroy(ev_out_);
    cudaEventDestroy(ev_batch_);
    cudaStreamDestroy(stream_);
    cudaStreamDestroy(stream2_);
    cudaEventDestroy(ev_fork_);
    cudaEventDestroy(ev_join_);
  }

  // ------------------------------------------------------------------ ABI methods
  void set_data(const void* A, int64_t lda, const void* W1, int64_t ldw, wlr_dtype dt,
                wlr_memory mem) override {
    const int m = d_.m, n = d_.n, k = d_.k;
    if (!A || !W1) throw Fail{WLR_ERR_INVALID_ARG, "A and W1 must be non-NULL"};
    if (lda < m || ldw < m) throw Fail{WLR_ERR_INVALID_ARG, "lda and ldw must be >= m"};
    begin();
    A_ = adopt_or_copy(A, lda, m, n, dt, mem, &A_own_, &lda_);
    W1_ = adopt_or_copy(W1, ldw, m, k, dt, mem, &W1_own_, &ldw_);
    WLR_CUDA(cudaMemsetAsync(err_, 0, sizeof(int), stream_));
    check_weights<T><<<grid1d((int64_t)m * k), 256, 0, stream_>>>(W1_, ldw_, m, k, err_);
    count(1);
    setup();
    have_data_ = true;
    cd_valid_ = false;
    graphs_clear();
    end();
    const int e = read_err();
    if (e & ERRBIT_BAD_WEIGHT) {
      have_data_ = false;
      throw Fail{WLR_ERR_NONPOSITIVE_WEIGHT, "W1 has an entry <= 0 or not finite (Theorem 2 needs W1 > 0)"};
    }
  }

  void set_init(wlr_init kind, const void* X1_0, int64_t ldx, wlr_dtype dt, wlr_memory mem,
                uint64_t seed) override {
    need_data();
    const int m = d_.m, k = d_.k;
    begin();
    T* X = X1buf_[0];
    if (kind == WLR_INIT_A1) {
      WLR_CUDA(cudaMemcpy2DAsync(X, sizeof(T) * m, A_, sizeof(T) * lda_, sizeof(T) * m, k,
                                 cudaMemcpyDeviceToDevice, stream_));
    } else if (kind == WLR_INIT_RANDOM) {
      random_normal_fill<T><<<grid1d((int64_t)m * k), 256, 0, stream_>>>(X, m, m, k, seed);
      count(1);
    } else if (kind == WLR_INIT_USER) {
      if (!X1_0) throw Fail{WLR_ERR_INVALID_ARG, "X1_0 must be non-NULL for WLR_INIT_USER"};
      if (ldx < m) throw Fail{WLR_ERR_INVALID_ARG, "ldx must be >= m"};
      load_matrix(X, m, X1_0, ldx, m, k, dt, mem);
    } else {
      throw Fail{WLR_ERR_INVALID_ARG, "unknown init kind"};
    }
    cur_ = 0;
    prev_ = -1;
    WLR_CUDA(cudaMemsetAsync(iter_, 0, sizeof(int), stream_));
    WLR_CUDA(cudaMemsetAsync(err_, 0, sizeof(int), stream_));
    eig_cold_ = true;
    cd_valid_ = false;
    iters_host_ = 0;
    rel_err_hist_.clear();
    have_init_ = true;
    end();
  }

  void step(double* F) override {
    need_init();
    begin();
    if (!cd_valid_) compute_cd(cur_, false);
    iterate_once();
    end();
    if (F) {
      WLR_CUDA(cudaMemcpyAsync(hbuf_, Fcur_, sizeof(double), cudaMemcpyDeviceToHost, stream_));
      WLR_CUDA(cudaStreamSynchronize(stream_));
      *F = *(double*)hbuf_;
      raise_err();
    }
  }

  wlr_status solve(double tol, int max_iter, int* iters, double* F) override {
    need_init();
    if (max_iter < 0) throw Fail{WLR_ERR_INVALID_ARG, "max_iter must be >= 0"};
    begin();
    if (!cd_valid_) compute_cd(cur_, false);
    const int stop = o_.stop;
    bool converged = false;
    double Fprev = NAN;
    int it = 0;
    for (; it < max_iter; ++it) {
      if (stop == WLR_STOP_NONE && max_iter - it >= 3 && three_ready()) {
        iterate_three();
        it += 2;
        continue;
      }
      iterate_once();
      if (stop == WLR_STOP_NONE) continue;
      if (stop == WLR_STOP_OBJECTIVE) {
        WLR_CUDA(cudaMemcpyAsync(hbuf_, Fcur_, sizeof(double), cudaMemcpyDeviceToHost, stream_));
        WLR_CUDA(cudaStreamSynchronize(stream_));
        const double Fp = *(double*)hbuf_;
        if (std::isfinite(Fprev) && std::fabs(Fprev - Fp) <= tol * std::fabs(Fp)) {
          converged = true;
          ++it;
          break;
        }
        Fprev = Fp;
        continue;
      }
      // paper / relative: Error_p = ||X_{p+1} - X_p||_F from the exact X2 pass
      double e6[6];
      x2_eval(cur_, prev_, nullptr, 0, e6);
      const double err = std::sqrt(std::max(0.0, e6[1] + e6[3]));
      const double nrm = std::sqrt(std::max(0.0, e6[2] + e6[4]));
      const double rel = nrm > 0 ? err / nrm : INFINITY;
      rel_err_hist_.push_back(rel);
      if ((stop == WLR_STOP_PAPER && (err < tol || rel < tol)) || rel < tol) {
        converged = true;
        ++it;
        break;
      }
    }
    end();
    WLR_CUDA(cudaMemcpyAsync(hbuf_, Fcur_, sizeof(double), cudaMemcpyDeviceToHost, stream_));
    WLR_CUDA(cudaStreamSynchronize(stream_));
    if (iters) *iters = it;
    if (F) *F = *(double*)hbuf_;
    raise_err();
    if (stop != WLR_STOP_NONE && !converged) return WLR_ERR_NO_CONVERGENCE;
    return WLR_OK;
  }

  double objective_exact() override {
    need_init();
    if (std::is_same<T, double>::value) {
      begin();
      qr_coef(cur_);
      if (d_.s > 0) {
        if (!use_dstep_) form_g2_launch();
        converge_eig();
      }
      if (!use_dstep_ || d_.s == 0) prep();
      cd_valid_ = true;
      double e6[6];
      x2_eval(cur_, -1, nullptr, 0, e6);
      end();
      raise_err();
      return e6[0] + e6[5];
    }
    // FP32 handle: score with an FP64 copy of the problem, its subspace iteration started
    // from this handle's current basis (nearly converged; the random start needed hundreds
    // of rounds to reach the same values)
    SolverBase* sc = scorer();
    // the scorer's stream waits on this stream, so the current X1 is complete
    sc->set_init(WLR_INIT_USER, X1buf_[cur_], d_.m, dtype_of<T>(), WLR_MEM_DEVICE, 0);
    if (!eig_cold_) sc->seed_subspace(V_, d_.b, std::is_same<T, double>::value);
    return sc->objective_exact();
  }
  // An FP64 solver on the same data (widened from T), with the widest subspace block, used
  // to score iterates exactly and for the refinement sweep.
  SolverBase* scorer() {
    if (!scorer_) {
      wlr_options so = o_;
      so.precision = WLR_PREC_FP64;
      so.use_graph = 0;
      so.eig_block = std::min(d_.n2, EIG_BMAX);
      Dims sd = d_;
      sd.b = std::max(d_.s, std::min(d_.n2, EIG_BMAX));
      scorer_ = make_solver_f64(sd, so, stream_);
      scorer_->set_data(A_, lda_, W1_, ldw_, dtype_of<T>(), WLR_MEM_DEVICE);
    }
    return scorer_;
  }
  // FP64 refinement sweep: from the current X1_p, the FP64 solver forms C_p and D_p with
  // the eigensolve run to convergence (F~(X1_p) = F(X1_p, C_p, D_p)), takes one loop body
  // of Algorithm 1 to X1_{p+1} and scores it the same way.  This handle's state is kept.
  void refine(void* X1_out, int64_t ldx, wlr_memory mem, double* Fp, double* Fnext) override {
    need_init();
    if (X1_out && ldx < d_.m) throw Fail{WLR_ERR_INVALID_ARG, "ldx must be >= m"};
    SolverBase* sc = scorer();
    sc->set_init(WLR_INIT_USER, X1buf_[cur_], d_.m, dtype_of<T>(), WLR_MEM_DEVICE, 0);
    if (!eig_cold_) sc->seed_subspace(V_, d_.b, std::is_same<T, double>::value);
    const double F0 = sc->objective_exact();
    sc->step(nullptr);
    const double F1 = sc->objective_exact();
    if (X1_out) sc->get_result(X1_out, ldx, nullptr, 0, WLR_F64, mem);
    if (Fp) *Fp = F0;
    if (Fnext) *Fnext = F1;
  }

  void get_result(void* X1, int64_t ldx, void* X2, int64_t ldx2, wlr_dtype dt,
                  wlr_memory mem) override {
    need_init();
    const int m = d_.m, k = d_.k, n2 = d_.n2;
    if (X1 && ldx < m) throw Fail{WLR_ERR_INVALID_ARG, "ldx must be >= m"};
    if (X2 && ldx2 < m) throw Fail{WLR_ERR_INVALID_ARG, "ldx2 must be >= m"};
    begin();
    if (!cd_valid_) compute_cd(cur_, false);
    if (X1) store_matrix(X1, ldx, X1buf_[cur_], m, m, k, dt, mem);
    if (X2 && n2 > 0) {
      const bool direct = (mem == WLR_MEM_DEVICE && dt == dtype_of<T>());
      T* out = direct ? (T*)X2 : scratch_out((size_t)m * n2);
      const int64_t ldo = direct ? ldx2 : m;
      double e6[6];
      x2_eval(cur_, -1, out, ldo, e6);
      if (!direct) store_matrix(X2, ldx2, out, m, m, n2, dt, mem);
    }
    end();
    if (mem == WLR_MEM_HOST) WLR_CUDA(cudaStreamSynchronize(stream_));
    raise_err_async();
  }

  void seed_subspace(const void* V, int b, bool fp64) override {
    need_init();
    const int n2 = d_.n2, nb = std::min(b, d_.b);
    if (d_.s == 0 || n2 == 0 || !V || nb < 1) return;
    begin();
    if (eig_cold_) eig_start();
    if (fp64)
      convert_copy<T, double><<<grid1d((int64_t)n2 * nb), 256, 0, stream_>>>(V_, n2, (const double*)V, n2, n2, nb);
    else
      convert_copy<T, float><<<grid1d((int64_t)n2 * nb), 256, 0, stream_>>>(V_, n2, (const float*)V, n2, n2, nb);
    count(1);
    eig_cold_ = false;
    end();
  }
  View view(bool with_factors) override {
    need_data();
    if (with_factors) {
      need_init();
      begin();
      if (!cd_valid_) compute_cd(cur_, false);
      end();
    }
    return View{A_, lda_, W1_, ldw_, have_init_ ? X1buf_[cur_] : nullptr, C_, Vs_, ustream_,
                std::is_same<T, double>::value};
  }
  Dims dims() const override { return d_; }
  cudaStream_t user_stream() const override { return ustream_; }

  void get_factors(double* C, double* Vs, double* sigma2) override {
    need_init();
    const int k = d_.k, n2 = d_.n2, s = d_.s;
    begin();
    if (!cd_valid_) compute_cd(cur_, false);
    end();
    WLR_CUDA(cudaStreamSynchronize(stream_));
    if (C && k * n2 > 0) copy_to_host_double(C, C_, (size_t)k * n2);
    if (Vs && n2 * s > 0) copy_to_host_double(Vs, Vs_, (size_t)n2 * s);
    if (sigma2 && s > 0) copy_to_host_double(sigma2, theta_, (size_t)s);
    raise_err();
  }

  int get_history(double* F, double* rel_err, int cap) override {
    WLR_CUDA(cudaStreamSynchronize(stream_));
    int p = 0;
    WLR_CUDA(cudaMemcpy(&p, iter_, sizeof(int), cudaMemcpyDeviceToHost));
    const int n = std::min(p, hist_cap_);
    if (F && cap > 0) WLR_CUDA(cudaMemcpy(F, Fhist_, sizeof(double) * std::min(n, cap), cudaMemcpyDeviceToHost));
    if (rel_err) {
      for (int q = 0; q < std::min(n, cap); ++q)
        rel_err[q] = q < (int)rel_err_hist_.size() ? rel_err_hist_[q] : NAN;
    }
    return n;
  }

  int iteration() override {
    WLR_CUDA(cudaStreamSynchronize(stream_));
    int p = 0;
    WLR_CUDA(cudaMemcpy(&p, iter_, sizeof(int), cudaMemcpyDeviceToHost));
    return p;
  }

  int64_t launches() const override { return launches_; }

  // ---- checkpoint: everything the next iteration reads (Algorithm 1's loop state plus
  // the build's carried state), so that a restored handle continues bit for bit
  struct StateHeader {
    char magic[4];     // "WLRS"
    int32_t version;   // 1
    int32_t tbytes;    // sizeof(T)
    int32_t m, n, k, r, b, NP, nbpart;
    int32_t iters_host, p_device, eig_cold, cd_valid, n_rel;
  };
  struct StateArrays {
    size_t x1, z2, g, cv, theta, resid, c, rinv, v, vs, bpart, fhist, rel;
  };
  StateArrays state_counts(int p_device, int n_rel) const {
    const int m = d_.m, k = d_.k, n2 = d_.n2, s = d_.s, b = std::max(d_.b, 1), NP = d_.NP;
    StateArrays c;
    c.x1 = (size_t)m * k;
    c.z2 = (size_t)std::max(n2, 1) * NP;
    c.g = (size_t)k * k;
    c.cv = (size_t)k * std::max(s, 1);
    c.theta = b;
    c.resid = b;
    c.c = (size_t)k * std::max(n2, 1);
    c.rinv = (size_t)k * k;
    c.v = (size_t)std::max(n2, 1) * b;
    c.vs = (size_t)std::max(n2, 1) * std::max(s, 1);
    c.bpart = nbpart();
    c.fhist = std::min(p_device, hist_cap_);
    c.rel = n_rel;
    return c;
  }
  int nbpart() const { return std::max(fuse_front_ ? ds_nc_ : nblk_coef_, 1); }
  static size_t state_size(const StateArrays& c) {
    return sizeof(StateHeader) +
           sizeof(T) * (c.x1 + c.z2 + c.g + c.cv + c.theta + c.resid + c.c + c.rinv + c.v + c.vs) +
           sizeof(double) * (c.bpart + c.fhist + c.rel);
  }
  int64_t state_bytes() override {
    need_init();
    WLR_CUDA(cudaStreamSynchronize(stream_));
    int p = 0;
    WLR_CUDA(cudaMemcpy(&p, iter_, sizeof(int), cudaMemcpyDeviceToHost));
    return (int64_t)state_size(state_counts(p, (int)rel_err_hist_.size()));
  }
  void get_state(void* buf) override {
    need_init();
    WLR_CUDA(cudaStreamSynchronize(stream_));
    int p = 0;
    WLR_CUDA(cudaMemcpy(&p, iter_, sizeof(int), cudaMemcpyDeviceToHost));
    const StateArrays c = state_counts(p, (int)rel_err_hist_.size());
    StateHeader h;
    std::memcpy(h.magic, "WLRS", 4);
    h.version = 1;
    h.tbytes = (int32_t)sizeof(T);
    h.m = d_.m; h.n = d_.n; h.k = d_.k; h.r = d_.r; h.b = d_.b; h.NP = d_.NP;
    h.nbpart = (int32_t)c.bpart;
    h.iters_host = iters_host_;
    h.p_device = p;
    h.eig_cold = eig_cold_ ? 1 : 0;
    h.cd_valid = cd_valid_ ? 1 : 0;
    h.n_rel = (int32_t)c.rel;
    unsigned char* o = (unsigned char*)buf;
    std::memcpy(o, &h, sizeof(h));
    o += sizeof(h);
    auto dl = [&](const void* src, size_t bytes) {
      if (bytes) WLR_CUDA(cudaMemcpy(o, src, bytes, cudaMemcpyDeviceToHost));
      o += bytes;
    };
    dl(X1buf_[cur_], sizeof(T) * c.x1);
    dl(Z2_, sizeof(T) * c.z2);
    dl(G_, sizeof(T) * c.g);
    dl(CV_, sizeof(T) * c.cv);
    dl(theta_, sizeof(T) * c.theta);
    dl(resid_, sizeof(T) * c.resid);
    dl(C_, sizeof(T) * c.c);
    dl(Rinv_, sizeof(T) * c.rinv);
    dl(V_, sizeof(T) * c.v);
    dl(Vs_, sizeof(T) * c.vs);
    dl(bpart_, sizeof(double) * c.bpart);
    dl(Fhist_, sizeof(double) * c.fhist);
    if (c.rel) std::memcpy(o, rel_err_hist_.data(), sizeof(double) * c.rel);
  }
  void set_state(const void* buf, int64_t size) override {
    need_data();
    StateHeader h;
    if (!buf || size < (int64_t)sizeof(h)) throw Fail{WLR_ERR_INVALID_ARG, "state buffer too small"};
    std::memcpy(&h, buf, sizeof(h));
    if (std::memcmp(h.magic, "WLRS", 4) != 0 || h.version != 1)
      throw Fail{WLR_ERR_INVALID_ARG, "not a state buffer of this library (magic/version)"};
    if (h.tbytes != (int32_t)sizeof(T) || h.m != d_.m || h.n != d_.n || h.k != d_.k || h.r != d_.r ||
        h.b != d_.b || h.NP != d_.NP || h.nbpart != nbpart())
      throw Fail{WLR_ERR_INVALID_ARG, "state was saved by a handle with other sizes or precision"};
    if (h.p_device < 0 || h.n_rel < 0 || h.iters_host < 0)
      throw Fail{WLR_ERR_INVALID_ARG, "corrupt state header"};
    const StateArrays c = state_counts(h.p_device, h.n_rel);
    if (size < (int64_t)state_size(c)) throw Fail{WLR_ERR_INVALID_ARG, "state buffer truncated"};
    begin();
    const unsigned char* o = (const unsigned char*)buf + sizeof(h);
    auto ul = [&](void* dst, size_t bytes) {
      if (bytes) WLR_CUDA(cudaMemcpy(dst, o, bytes, cudaMemcpyHostToDevice));
      o += bytes;
    };
    ul(X1buf_[0], sizeof(T) * c.x1);
    ul(Z2_, sizeof(T) * c.z2);
    ul(G_, sizeof(T) * c.g);
    ul(CV_, sizeof(T) * c.cv);
    ul(theta_, sizeof(T) * c.theta);
    ul(resid_, sizeof(T) * c.resid);
    ul(C_, sizeof(T) * c.c);
    ul(Rinv_, sizeof(T) * c.rinv);
    ul(V_, sizeof(T) * c.v);
    ul(Vs_, sizeof(T) * c.vs);
    ul(bpart_, sizeof(double) * c.bpart);
    ul(Fhist_, sizeof(double) * c.fhist);
    rel_err_hist_.assign((const double*)o, (const double*)o + c.rel);
    WLR_CUDA(cudaMemcpy(iter_, &h.p_device, sizeof(int), cudaMemcpyHostToDevice));
    if (c.fhist > 0) {
      double Fl = 0.0;
      WLR_CUDA(cudaMemcpy(&Fl, Fhist_ + (c.fhist - 1), sizeof(double), cudaMemcpyDeviceToHost));
      WLR_CUDA(cudaMemcpy(Fcur_, &Fl, sizeof(double), cudaMemcpyHostToDevice));
    }
    WLR_CUDA(cudaMemsetAsync(err_, 0, sizeof(int), stream_));
    cur_ = 0;
    prev_ = -1;
    iters_host_ = h.iters_host;
    eig_cold_ = h.eig_cold != 0;
    cd_valid_ = h.cd_valid != 0;
    graphs_clear();
    have_init_ = true;
    end();
  }

  // Run reps iterations without graphs, each kernel bracketed by CUDA events on the
  // solver's stream; per kernel name: total milliseconds and launch count.
  std::vector<ProfEntry> profile(int reps) override {
    need_init();
    begin();
    if (!cd_valid_) compute_cd(cur_, false);
    WLR_CUDA(cudaStreamSynchronize(stream_));
    prof_ = true;
    prof_recs_.clear();
    ev_used_ = 0;
    const int saved_graph = o_.use_graph;
    o_.use_graph = 0;
    try {
      for (int q = 0; q < reps; ++q) iterate_once();
      // the setup Gram K = A2^T A2 once more (deterministic: the same K)
      if (reps > 0 && use_tc_k_) tc_gram_k();
    } catch (...) {
      prof_ = false;
      o_.use_graph = saved_graph;
      throw;
    }
    prof_ = false;
    o_.use_graph = saved_graph;
    end();
    WLR_CUDA(cudaStreamSynchronize(stream_));
    std::vector<ProfEntry> out;
    for (auto& r : prof_recs_) {
      float ms = 0.f;
      WLR_CUDA(cudaEventElapsedTime(&ms, r.a, r.b));
      auto it = std::find_if(out.begin(), out.end(), [&](const ProfEntry& e) { return e.name == r.name; });
      if (it == out.end()) out.push_back(ProfEntry{r.name, (double)ms, 1});
      else { it->ms += ms; it->launches += 1; }
    }
    raise_err();
    return out;
  }

 private:

  // ------------------------------------------------------------------ plumbing
  template <typename U>
  U* dalloc(size_t n) {
    void* p = nullptr;
    WLR_CUDA(cudaMalloc(&p, sizeof(U) * std::max<size_t>(n, 1)));
    allocs_.push_back(p);
    return (U*)p;
  }
  // The dynamic shared-memory limit is an attribute of the kernel, shared by every handle
  // of the process: raise it to `bytes` if it is lower, never lower it (a smaller problem
  // set up after a larger one must not break the larger one's launches).
  static cudaError_t raise_smem_limit(const void* fn, size_t bytes) {
    static std::mutex mu;
    std::lock_guard<std::mutex> lock(mu);
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, fn);
    if (e != cudaSuccess) return e;
    if ((size_t)fa.maxDynamicSharedSizeBytes >= bytes) return cudaSuccess;
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  }
  static void set_smem(const void* fn, size_t bytes) {
    if (bytes > 48 * 1024) WLR_CUDA(raise_smem_limit(fn, bytes));
  }
  static int sm_count() {
    int dev = 0, n = 152;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
      cudaGetLastError();
      n = 152;
    }
    return n;
  }
  static int resident(const void* fn, int threads, size_t smem) {
    int b = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, fn, threads, smem) != cudaSuccess || b < 1) {
      cudaGetLastError();
      b = 1;
    }
    return b;
  }
  static int grid1d(int64_t total) {
    return (int)std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, 152 * 16));
  }
  void count(int n) { launches_ += n; }
  cudaEvent_t next_event() {
    if (ev_used_ == ev_pool_.size()) {
      cudaEvent_t e;
      WLR_CUDA(cudaEventCreate(&e));
      ev_pool_.push_back(e);
    }
    return ev_pool_[ev_used_++];
  }
  // Brackets the launches of its lifetime with events when profiling.
  struct Prof {
    Solver* s;
    const char* name;
    cudaEvent_t a = nullptr;
    Prof(Solver* sv, const char* nm) : s(sv), name(nm) {
      if (s->prof_) {
        a = s->next_event();
        cudaEventRecord(a, s->stream_);
      }
    }
    ~Prof() {
      if (s->prof_) {
        cudaEvent_t b = s->next_event();
        cudaEventRecord(b, s->stream_);
        s->prof_recs_.push_back({name, a, b});
      }
    }
  };
  size_t x2_smem() const {
    const int NP = d_.NP;
    return sizeof(T) * ((size_t)RP_BK * RP_BM + (size_t)RP_BK * std::max(NP, EIG_BMAX) +
                        2 * (size_t)RP_BM * (NP + 1));
  }
  void begin() {
    WLR_CUDA(cudaEventRecord(ev_in_, ustream_));
    WLR_CUDA(cudaStreamWaitEvent(stream_, ev_in_, 0));
  }
  void end() {
    WLR_CUDA(cudaEventRecord(ev_out_, stream_));
    WLR_CUDA(cudaStreamWaitEvent(ustream_, ev_out_, 0));
  }
  void need_data() {
    if (!have_data_) throw Fail{WLR_ERR_NOT_READY, "call wlr_set_data first"};
  }
  void need_init() {
    need_data();
    if (!have_init_) throw Fail{WLR_ERR_NOT_READY, "call wlr_set_init first"};
  }
  int read_err() {
    WLR_CUDA(cudaMemcpyAsync(hbuf_ + 64, err_, sizeof(int), cudaMemcpyDeviceToHost, stream_));
    WLR_CUDA(cudaStreamSynchronize(stream_));
    return *(int*)(hbuf_ + 64);
  }
  void raise_err() {
    const int e = read_err();
    // root causes first: a rank-deficient X1 also spoils the row systems downstream
    if (e & ERRBIT_BAD_WEIGHT) throw Fail{WLR_ERR_NONPOSITIVE_WEIGHT, "W1 has an entry <= 0 or not finite"};
    if (e & ERRBIT_RANK_DEFICIENT) throw Fail{WLR_ERR_RANK_DEFICIENT, "Cholesky of X1^T X1 broke down: X1 is not of rank k (Eq. 8 assumes rank k)"};
    if (e & ERRBIT_NOT_SPD) throw Fail{WLR_ERR_NOT_SPD, "a row system diag(W1(i,:)^2) + C C^T was not positive definite"};
    if (e & ERRBIT_EIG) throw Fail{WLR_ERR_RANK_DEFICIENT, "the subspace basis for the rank-(r-k) SVD step lost rank"};
    if (e & tc::ERRBIT_TIMEOUT) throw Fail{WLR_ERR_DEVICE_TIMEOUT, "a bounded wait of the tensor-core pipeline gave up"};
  }
  void raise_err_async() {}

  // A device pointer of type T with leading dimension ld, borrowed when possible.
  const T* adopt_or_copy(const void* src, int64_t ld, int rows, int cols, wlr_dtype dt,
                         wlr_memory mem, T** own, int64_t* ld_out) {
    if (mem == WLR_MEM_DEVICE && dt == dtype_of<T>()) {
      *ld_out = ld;
      return (const T*)src;
    }
    if (!*own) *own = dalloc<T>((size_t)rows * cols);
    load_matrix(*own, rows, src, ld, rows, cols, dt, mem);
    *ld_out = rows;
    return *own;
  }

  // dst (device, T, ld_dst) <- src (dt, mem, ld_src)
  void load_matrix(T* dst, int64_t ld_dst, const void* src, int64_t ld_src, int rows, int cols,
                   wlr_dtype dt, wlr_memory mem) {
    const size_t es = dt == WLR_F32 ? 4 : 8;
    const void* dsrc = src;
    int64_t ld_dsrc = ld_src;
    if (mem == WLR_MEM_HOST) {
      void* stage = staging((size_t)rows * cols * es);
      WLR_CUDA(cudaMemcpy2DAsync(stage, es * rows, src, es * ld_src, es * rows, cols,
                                 cudaMemcpyHostToDevice, stream_));
      dsrc = stage;
      ld_dsrc = rows;
    }
    if (dt == dtype_of<T>()) {
      WLR_CUDA(cudaMemcpy2DAsync(dst, sizeof(T) * ld_dst, dsrc, sizeof(T) * ld_dsrc,
                                 sizeof(T) * rows, cols, cudaMemcpyDeviceToDevice, stream_));
    } else if (dt == WLR_F32) {
      convert_copy<T, float><<<grid1d((int64_t)rows * cols), 256, 0, stream_>>>(
          dst, ld_dst, (const float*)dsrc, ld_dsrc, rows, cols);
      count(1);
    } else {
      convert_copy<T, double><<<grid1d((int64_t)rows * cols), 256, 0, stream_>>>(
          dst, ld_dst, (const double*)dsrc, ld_dsrc, rows, cols);
      count(1);
    }
  }

  // dst (dt, mem, ld_dst) <- src (device, T, ld_src)
  void store_matrix(void* dst, int64_t ld_dst, const T* src, int64_t ld_src, int rows, int cols,
                    wlr_dtype dt, wlr_memory mem) {
    const size_t es = dt == WLR_F32 ? 4 : 8;
    const void* dsrc = src;
    int64_t ld_dsrc = ld_src;
    if (dt != dtype_of<T>()) {
      void* stage = staging((size_t)rows * cols * es);
      if (dt == WLR_F32)
        convert_copy<float, T><<<grid1d((int64_t)rows * cols), 256, 0, stream_>>>(
            (float*)stage, rows, src, ld_src, rows, cols);
      else
        convert_copy<double, T><<<grid1d((int64_t)rows * cols), 256, 0, stream_>>>(
            (double*)stage, rows, src, ld_src, rows, cols);
      count(1);
      dsrc = stage;
      ld_dsrc = rows;
    }
    WLR_CUDA(cudaMemcpy2DAsync(dst, es * ld_dst, dsrc, es * ld_dsrc, es * rows, cols,
                               mem == WLR_MEM_HOST ? cudaMemcpyDeviceToHost
                                                   : cudaMemcpyDeviceToDevice,
                               stream_));
  }

  // replace a device buffer of this handle by a larger one (the old contents are dropped)
  template <typename U>
  U* dregrow(U* old, size_t n) {
    if (old) {
      WLR_CUDA(cudaStreamSynchronize(stream_));
      allocs_.erase(std::find(allocs_.begin(), allocs_.end(), (void*)old));
      cudaFree(old);
    }
    return dalloc<U>(n);
  }
  void* staging(size_t bytes) {
    if (bytes > stage_bytes_) {
      if (stage_) {
        WLR_CUDA(cudaStreamSynchronize(stream_));
        cudaFree(stage_);
        allocs_.erase(std::find(allocs_.begin(), allocs_.end(), stage_));
      }
      stage_ = dalloc<unsigned char>(bytes);
      stage_bytes_ = bytes;
    }
    return stage_;
  }
  T* scratch_out(size_t n) { return (T*)staging2(n * sizeof(T)); }
  void* staging2(size_t bytes) {
    if (bytes > stage2_bytes_) {
      if (stage2_) {
        WLR_CUDA(cudaStreamSynchronize(stream_));
        cudaFree(stage2_);
        allocs_.erase(std::find(allocs_.begin(), allocs_.end(), stage2_));
      }
      stage2_ = dalloc<unsigned char>(bytes);
      stage2_bytes_ = bytes;
    }
    return stage2_;
  }
  void copy_to_host_double(double* dst, const T* src, size_t n) {
    std::vector<T> tmp(n);
    WLR_CUDA(cudaMemcpy(tmp.data(), src, sizeof(T) * n, cudaMemcpyDeviceToHost));
    for (size_t q = 0; q < n; ++q) dst[q] = (double)tmp[q];
  }

  // ------------------------------------------------------------------ tensor-core Gram
  // Q1^T [Q1 A2] on tcgen05 (FP32 path): TF32-split copies of A2 (made in setup) and of Q1
  // (each iteration), TMA tensor maps built once for these library-owned buffers.
  void setup_tc() {
    const int m = d_.m, k = d_.k, n2 = d_.n2;
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &fn, cudaEnableDefault, &q) != cudaSuccess || !fn) {
      cudaGetLastError();
      return;
    }
    auto enc = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    enc_ = (void*)fn;
    ld4_ = ((m + 3) / 4) * 4;
    A2h_ = dalloc<float>((size_t)ld4_ * n2);
    A2l_ = dalloc<float>((size_t)ld4_ * n2);
    auto mk = [&](CUtensorMap* map, const float* p, int cols, int boxc) {
      cuuint64_t dims[2] = {(cuuint64_t)m, (cuuint64_t)cols};
      cuuint64_t strides[1] = {(cuuint64_t)ld4_ * 4};
      cuuint32_t box[2] = {32, (cuuint32_t)boxc};
      cuuint32_t es[2] = {1, 1};
      return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void*)p, dims, strides, box, es,
                 CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                 CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    };
    // K = A2^T A2 (any k): blocks (bi, bj) of 128 x 64 columns holding entries c1 <= c2,
    // about one CTA per SM over the row chunks
    if (!mk(&mA2h_, A2h_, n2, 128) || !mk(&mA2l_, A2l_, n2, 128) || !mk(&mA2h64_, A2h_, n2, tc::KN) ||
        !mk(&mA2l64_, A2l_, n2, tc::KN))
      return;
    {
      std::vector<int2> pr;
      for (int bi = 0; bi < cdiv(n2, 128); ++bi)
        for (int bj = 2 * bi; bj < cdiv(n2, tc::KN); ++bj) pr.push_back(make_int2(bi, bj));
      kk_npairs_ = (int)pr.size();
      kk_pairs_ = dalloc<int2>(pr.size());
      WLR_CUDA(cudaMemcpy(kk_pairs_, pr.data(), sizeof(int2) * pr.size(), cudaMemcpyHostToDevice));
      WLR_CUDA(cudaFuncSetAttribute((const void*)tc::gram_kk_tf32x3, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    tc::K_SMEM_BYTES));
      ch_kk_ = chunking_waves(m, kk_npairs_,
                              sm_count() * resident((const void*)tc::gram_kk_tf32x3, tc::K_THREADS, tc::K_SMEM_BYTES));
      const size_t needk = (size_t)ch_kk_.nch * kk_npairs_ * tc::K_TILE;
      if (needk > part_elems_) {
        part64_ = dregrow(part64_, needk);
        part_elems_ = needk;
      }
    }
    use_tc_k_ = true;
    // Q1^T [Q1 A2] each iteration: the transposed kernel takes up to 64 columns of X
    if (k > 2 * tc::TN) return;
    tn_ = k <= tc::TN ? tc::TN : 2 * tc::TN;
    Q1h_ = dalloc<float>((size_t)ld4_ * k);
    Q1l_ = dalloc<float>((size_t)ld4_ * k);
    if (!mk(&mQh128_, Q1h_, k, 128) || !mk(&mQl128_, Q1l_, k, 128) || !mk(&mQh32_, Q1h_, k, tn_) ||
        !mk(&mQl32_, Q1l_, k, tn_))
      return;
    const void* gfn = tn_ == tc::TN ? (const void*)tc::gram_tf32x3_t<tc::TN> : (const void*)tc::gram_tf32x3_t<2 * tc::TN>;
    WLR_CUDA(cudaFuncSetAttribute(gfn, cudaFuncAttributeMaxDynamicSharedMemorySize, tc::t_smem_bytes(tn_)));
    ch_tc_ = chunking_waves(m, 1 + cdiv(n2, 128),
                            sm_count() * resident(gfn, tc::t_threads(tn_), tc::t_smem_bytes(tn_)));
    const size_t need = (size_t)ch_tc_.nch * ((size_t)k * k + (size_t)k * n2);
    if (need > part_elems_) {
      part64_ = dregrow(part64_, need);
      part_elems_ = need;
    }
    use_tc_ = true;
  }
  // TMA map of the FP32 A2 itself (32 rows x 128 columns, 128-byte swizzle) for the
  // per-iteration Gram, when its leading dimension and base allow TMA (lda a multiple of 4,
  // 16-byte aligned); otherwise the Gram reads the TF32 split copies.
  void tc_map_a2() {
    a2f_ok_ = false;
    if (!use_tc_ || !enc_ || !std::is_same<T, float>::value) return;
    const int m = d_.m, k = d_.k, n2 = d_.n2;
    const float* A2 = (const float*)(A_ + (int64_t)k * lda_);
    if (lda_ % 4 != 0 || ((uintptr_t)A2 & 15) != 0) return;
    auto enc = (PFN_cuTensorMapEncodeTiled_v12000)enc_;
    cuuint64_t dims[2] = {(cuuint64_t)m, (cuuint64_t)n2};
    cuuint64_t strides[1] = {(cuuint64_t)lda_ * 4};
    cuuint32_t box[2] = {32, 128};
    cuuint32_t es[2] = {1, 1};
    a2f_ok_ = enc(&mA2f_, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void*)A2, dims, strides, box, es,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
  }
  void tc_split_a2() {
    tc_map_a2();
    if (!use_tc_k_) return;
    const int m = d_.m, k = d_.k, n2 = d_.n2;
    tc::split_tf32<<<grid1d((int64_t)m * n2), 256, 0, stream_>>>((const float*)(A_ + (int64_t)k * lda_), lda_, m, n2,
                                                                  A2h_, A2l_, ld4_);
    count(1);
  }
  // part64 <- chunk partials of Q1^T [Q1 A2] with Q1 = X1 Rpre (k x (k + n2) per chunk)
  void tc_gram(const T* X1, const T* Rpre, bool fork = false) {
    const int m = d_.m, k = d_.k, n2 = d_.n2;
    if (q_from_row_pass_ && Rpre == Rinv_) {
      // the row pass that made X1 has already written Q1 = X1 Rinv_ (same sums, same order)
      q_from_row_pass_ = false;
    } else {
      q_from_row_pass_ = false;
      Prof pf(this, "form_q_split");
      tc::form_q_split<<<grid1d((int64_t)m * k), 256, sizeof(float) * k * k, stream_>>>(
          (const float*)X1, m, (const float*)Rpre, m, k, Q1h_, Q1l_, ld4_, fuse_front_ ? 1 : 0);
      count(1);
    }
    if (fork) fork_kv();
    {
      Prof pf(this, "gram_tf32x3_t");
      dim3 g(1 + cdiv(n2, 128), ch_tc_.nch);
      const int64_t pstride = (int64_t)k * k + (int64_t)k * n2;
      const CUtensorMap& mf = a2f_ok_ ? mA2f_ : mA2h_;
      const int split = a2f_ok_ ? 1 : 0;
      launch_gram_tc(ch_tc_);
    }
    count(1);
  }
  void launch_gram_tc(const Chunk& ch) {
    const int m = d_.m, k = d_.k, n2 = d_.n2;
    dim3 g(1 + cdiv(n2, 128), ch.nch);
    const int64_t pstride = (int64_t)k * k + (int64_t)k * n2;
    const CUtensorMap& mf = a2f_ok_ ? mA2f_ : mA2h_;
    const int split = a2f_ok_ ? 1 : 0;
    if (tn_ == tc::TN)
      tc::gram_tf32x3_t<tc::TN><<<g, tc::t_threads(tc::TN), tc::t_smem_bytes(tc::TN), stream_>>>(
          mQh128_, mQl128_, mA2h_, mA2l_, mQh32_, mQl32_, mf, split, m, k, k, n2, ch.rows, part64_, pstride, err_);
    else
      tc::gram_tf32x3_t<2 * tc::TN><<<g, tc::t_threads(2 * tc::TN), tc::t_smem_bytes(2 * tc::TN), stream_>>>(
          mQh128_, mQl128_, mA2h_, mA2l_, mQh32_, mQl32_, mf, split, m, k, k, n2, ch.rows, part64_, pstride, err_);
  }
  // Autotuner of the per-iteration Gram's row chunks (options.autotune): the whole-wave
  // rule's chunk count and its neighbours (half, two thirds, 3/2 and twice as many chunks)
  // are each launched on this problem's own A2 (one warm-up, then three launches timed by
  // CUDA events) and the fastest is kept, for every handle of this (m, n2, k) in the
  // process.  The partials it writes are scratch (the next iteration rewrites them).
  void autotune_gram() {
    const int m = d_.m, k = d_.k, n2 = d_.n2;
    static std::mutex mu;
    static std::map<std::tuple<int, int, int, int>, Chunk> cache;
    const auto key = std::make_tuple(m, n2, k, a2f_ok_ ? 1 : 0);
    {
      std::lock_guard<std::mutex> lock(mu);
      auto it = cache.find(key);
      if (it != cache.end()) {
        ch_tc_ = it->second;
        return;
      }
    }
    auto chunk_of = [&](int n) {
      n = std::max(1, std::min(128, n));
      const int rows = std::max(32, ((cdiv(m, n) + 31) / 32) * 32);
      return Chunk{cdiv(m, rows), rows};
    };
    const Chunk rule = ch_tc_;
    std::vector<Chunk> cand = {rule};
    for (int n : {rule.nch / 2, (2 * rule.nch) / 3, (3 * rule.nch) / 2, 2 * rule.nch}) {
      const Chunk c = chunk_of(n);
      bool dup = false;
      for (const Chunk& e : cand) dup = dup || e.nch == c.nch;
      if (!dup) cand.push_back(c);
    }
    size_t need = 0;
    for (const Chunk& c : cand) need = std::max(need, (size_t)c.nch * ((size_t)k * k + (size_t)k * n2));
    if (need > part_elems_) {
      part64_ = dregrow(part64_, need);
      part_elems_ = need;
    }
    cudaEvent_t e0, e1;
    WLR_CUDA(cudaEventCreate(&e0));
    WLR_CUDA(cudaEventCreate(&e1));
    Chunk best = rule;
    float best_ms = 1e30f;
    for (const Chunk& c : cand) {
      launch_gram_tc(c);
      WLR_CUDA(cudaEventRecord(e0, stream_));
      for (int rep = 0; rep < 3; ++rep) launch_gram_tc(c);
      WLR_CUDA(cudaEventRecord(e1, stream_));
      WLR_CUDA(cudaEventSynchronize(e1));
      float ms = 0.f;
      WLR_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      count(4);
      if (ms < best_ms) {
        best_ms = ms;
        best = c;
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ch_tc_ = best;
    std::lock_guard<std::mutex> lock(mu);
    cache.emplace(key, best);
  }

  // ------------------------------------------------------------------ kernels
  // part64 <- chunked partials of X^T [Y1 Y2] (Y1: q1 columns, Y2: the rest).  With Rq,
  // X and Y1 are Q1 = X Rq (formed inside the kernel; float path only).
  void gram(const T* X, int64_t ldx, const T* Y1, int64_t ldy1, int q1, const T* Y2, int64_t ldy2,
            int P, int Q, int64_t stride, const Chunk& ch, const T* Rq = nullptr) {
    if (P <= 0 || Q <= 0) return;
    const int m = d_.m;
    Prof pf(this, "gram_tn");
    const bool fuse = Rq != nullptr;
#define WLR_GRAM(PT, QT, NTH)                                                                    \
  do {                                                                                          \
    dim3 g(cdiv(P, PT), cdiv(Q, QT), ch.nch);                                                   \
    if (fuse)                                                                                   \
      gram_tn<T, PT, QT, true><<<g, NTH, 0, stream_>>>(X, ldx, Y1, ldy1, q1, Y2, ldy2, Rq, m, P, Q, \
                                                       ch.rows, part64_, stride, 0);            \
    else                                                                                        \
      gram_tn<T, PT, QT, false><<<g, NTH, 0, stream_>>>(X, ldx, Y1, ldy1, q1, Y2, ldy2, nullptr, m, \
                                                        P, Q, ch.rows, part64_, stride, 0);     \
  } while (0)
    if (P <= 32 && Q <= 32) WLR_GRAM(32, 32, 64);
    else if (P <= 32) WLR_GRAM(32, 64, 128);
    else WLR_GRAM(64, 64, 256);
#undef WLR_GRAM
    count(1);
  }
  // pairs: the partials are float pairs (the tensor-core Gram), else doubles
  void reduce64(int64_t stride, int nch, int64_t len, double* out64, int kf = 0, T* Fout = nullptr,
                bool pairs = false) {
    if (len <= 0) return;
    Prof pf(this, "reduce_partials");
    if (pairs)
      reduce_pairs_split<T><<<(unsigned)cdiv(len, 32), 256, 0, stream_>>>(part64_, stride, nch, len, out64, kf, Fout);
    else
      reduce_partials_split<double, T><<<(unsigned)cdiv(len, 32), 256, 0, stream_>>>(part64_, stride, nch, len, out64,
                                                                                      nullptr, kf, Fout);
    count(1);
  }

  // once per problem (step a0): ||A2||^2 and K = A2^T A2
  void setup() {
    const int m = d_.m, k = d_.k, n2 = d_.n2;
    const T* A2 = A_ + (int64_t)k * lda_;
    if (n2 == 0) {
      WLR_CUDA(cudaMemsetAsync(normA2_, 0, sizeof(double), stream_));
      return;
    }
    const int nb = 304;
    sumsq_partial<T><<<nb, 256, 0, stream_>>>(A2, lda_, m, n2, wpart_scratch(nb));
    reduce_partials<double><<<1, 32, 0, stream_>>>(wpart_scratch(nb), 1, nb, 1, normA2_, nullptr);
    count(2);
    tc_split_a2();
    if (o_.autotune && use_tc_) autotune_gram();
    if (use_tc_k_) {
      tc_gram_k();
    } else {
      gram(A2, lda_, A2, lda_, n2, nullptr, 0, n2, n2, (int64_t)n2 * n2, ch_K_);
      reduce64((int64_t)n2 * n2, ch_K_.nch, (int64_t)n2 * n2, K64_);
    }
    if (use_dstep_ && Kh_) {
      split_pair<<<grid1d((int64_t)n2 * n2), 256, 0, stream_>>>(K64_, (int64_t)n2 * n2, Kh_, Kl_);
      count(1);
    }
  }
  // K = A2^T A2 on the tensor cores (3xTF32, from the split copies of A2)
  void tc_gram_k() {
    const int n2 = d_.n2;
    {
      Prof pf(this, "gram_kk_tf32x3");
      tc::gram_kk_tf32x3<<<dim3(kk_npairs_, ch_kk_.nch), tc::K_THREADS, tc::K_SMEM_BYTES, stream_>>>(
          mA2h_, mA2l_, mA2h64_, mA2l64_, d_.m, ch_kk_.rows, kk_pairs_, kk_npairs_, part64_, err_);
      WLR_CUDA(cudaGetLastError());
    }
    {
      Prof pf(this, "reduce_kk");
      tc::reduce_kk<<<grid1d((int64_t)kk_npairs_ * tc::K_TILE), 256, 0, stream_>>>(part64_, ch_kk_.nch, kk_pairs_,
                                                                                kk_npairs_, n2, K64_);
    }
    count(2);
  }
  double* wpart_scratch(int n) {
    if (!sumsq_part_) sumsq_part_ = dalloc<double>(std::max(n, 304));
    return sumsq_part_;
  }

  // steps a1 + a2 for X1 = X1buf_[xi].  precond: the first CholeskyQR factor is the
  // previous iteration's R (X1 moves little per iteration, so X1 R_prev^{-1} is already
  // nearly orthonormal and the second factor recovers the exact R = R2 R_prev); else a
  // full CholeskyQR2 from S1 = X1^T X1.
  // fused: stop after the summed Gram (the D-step cluster kernel takes the second factor
  // and B, C); front_rpre_ tells it which first factor to use
  void qr_coef(int xi, bool precond = false, bool fused = false) {
    const int m = d_.m, k = d_.k, n2 = d_.n2, NP = d_.NP;
    const T* X1 = X1buf_[xi];
    const T* A2 = A_ + (int64_t)k * lda_;
    const T* Rpre = Rinv_;
    if (!precond) {
      gram(X1, m, X1, m, k, nullptr, 0, k, k, (int64_t)k * k, ch_S1_);
      {
        Prof pf(this, "chol1");
        chol1_kernel<T><<<1, 256, sizeof(double) * (2 * k * k + k), stream_>>>(part64_, ch_S1_.nch, k, R1inv_, err_);
      }
      count(1);
      Rpre = R1inv_;
    }
    const int64_t L = (int64_t)k * k + (int64_t)k * n2;
    int nchT = ch_T_.nch;
    if (use_tc_) {
      // tensor cores (tcgen05 + TMA), Q1 = X1 Rpre split into TF32 hi + lo
      tc_gram(X1, Rpre, fused);
      nchT = ch_tc_.nch;
    } else if (std::is_same<T, float>::value) {
      // Q1 = X1 Rpre formed slab by slab inside the Gram kernel
      gram(X1, m, nullptr, 0, k, A2, lda_, k, k + n2, L, ch_T_, Rpre);
    } else {
      {
        Prof pf(this, "form_q");
        form_q<T><<<grid1d((int64_t)m * k), 256, sizeof(T) * k * k, stream_>>>(X1, m, Rpre, m, k, Q1_);
      }
      count(1);
      gram(Q1_, m, Q1_, m, k, A2, lda_, k, k + n2, L, ch_T_);
    }
    // Q1^T [Q1 A2] summed over the chunks by all SMs; chol2 and coef read the sum
    reduce64(L, nchT, L, S2T_, k, k <= 32 ? F2_ : nullptr, use_tc_);
    if (fused) {
      front_rpre_ = Rpre;
      return;
    }
    {
      Prof pf(this, "chol2");
      if (k <= 32)
        chol2_warp<T><<<1, 32, 0, stream_>>>(F2_, k, Rpre, Nm_, Rinv_, err_);
      else
        chol2_kernel<T><<<1, 256, 3 * sizeof(T) * k * k, stream_>>>(S2T_, 1, L, k, Rpre, Nm_, Rinv_, err_);
    }
    count(1);
    if (n2 > 0) {
      Prof pf(this, "coef");
      coef_kernel3<T><<<nblk_coef_, 256, sizeof(T) * (2 * k * k + 16 * 64), stream_>>>(
          S2T_, 1, L, Nm_, Rinv_, k, n2, NP, C_, B64_, Bh_, Bl_, Z2_, bpart_);
      count(1);
    }
  }
  void form_g2_launch() {
    const int n2 = d_.n2;
    dim3 g(cdiv(n2, 32), cdiv(n2, 32));
    Prof pf(this, "form_g2");
    form_g2_df<T><<<g, 256, 0, stream_>>>(K64_, B64_, Bh_, Bl_, d_.k, n2, G2_);
    count(1);
  }
  void eig_iteration(bool cold = false) {
    const int n2 = d_.n2, b = d_.b, s = d_.s;
    {
      Prof pf(this, "eig_mult");
      if (eig_vsmem_)
        eig_mult<T, true><<<nblk_eig_, 256, (size_t)n2 * b * sizeof(T), stream_>>>(G2_, V_, n2, b, Zeig_, eigpart_,
                                                                                   eig_ticket_, HP_);
      else
        eig_mult<T, false><<<nblk_eig_, 256, 0, stream_>>>(G2_, V_, n2, b, Zeig_, eigpart_, eig_ticket_, HP_);
    }
    {
      Prof pf(this, "eig_small");
      eig_small<T><<<1, 32, 0, stream_>>>(HP_, b, cold ? (sizeof(T) == 4 ? 12 : 24) : (sizeof(T) == 4 ? 1 : 6), Y_, Mv_, Mz_,
                                          theta_, resid_, err_);
    }
    Prof pf(this, "eig_update");
    eig_update<T><<<cdiv(n2, 8), 256, 0, stream_>>>(V_, Zeig_, Y_, Mv_, Mz_, n2, b, s, d_.k,
                                                    d_.NP, Vs_, Z2_);
    count(3);
  }
  // The fused cluster kernel of step a3 (and of G, C V_s): used when s > 0, b <= 32, the
  // device runs a cluster of 16 (or else 8) CTAs with the kernel's shared memory.
  void setup_dstep() {
    const int n2 = d_.n2, k = d_.k, b = d_.b, s = d_.s;
    if (s <= 0 || n2 <= 0 || b > DS_BM) return;
    // the front stage (second factor, B, C inside the cluster) for k <= 32
    const bool front = k <= 32;
    ds_ne_ = std::max(b * b, front ? k * k : 0) <= DS_THREADS ? 1 : 2;
    const void* fn = ds_ne_ == 1 ? (const void*)dstep_cluster<T, 1> : (const void*)dstep_cluster<T, 2>;
    // the steady-state step with the front stage has a kernel of its own (dstep_front),
    // exchanging partial sums by remote stores where one slot per worker fits (push),
    // else by remote loads
    auto front_fn = [&](bool push) {
      if (push) return ds_ne_ == 1 ? (const void*)dstep_front<T, 1, true> : (const void*)dstep_front<T, 2, true>;
      return ds_ne_ == 1 ? (const void*)dstep_front<T, 1, false> : (const void*)dstep_front<T, 2, false>;
    };
    // a cluster of nc CTAs of `bytes` shared memory each can run fn
    auto fits = [&](const void* f, int nc, size_t bytes) {
      if (bytes > 225 * 1024) return false;
      if (nc > 8 && cudaFuncSetAttribute(f, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
        cudaGetLastError();
        return false;
      }
      if (raise_smem_limit(f, bytes) != cudaSuccess) {
        cudaGetLastError();
        return false;
      }
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(nc);
      cfg.blockDim = dim3(DS_THREADS);
      cfg.dynamicSmemBytes = bytes;
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeClusterDimension;
      attr[0].val.clusterDim.x = nc;
      attr[0].val.clusterDim.y = 1;
      attr[0].val.clusterDim.z = 1;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      int ncl = 0;
      if (cudaOccupancyMaxActiveClusters(&ncl, f, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return false;
      }
      return ncl >= 1;
    };
    for (int nc : {16, 8}) {
      if (n2 < nc) continue;
      const size_t bytes = sizeof(T) * DsLayout::make<T>(n2, k, b, s, cdiv(n2, nc)).total;
      if (!fits(fn, nc, bytes)) continue;
      size_t bytes_f = 0;
      bool push = false;
      if (front) {
        for (bool p : {true, false}) {
          const size_t bf = sizeof(T) * DfLayout::make<T>(k, b, s, df_rows(n2, nc), nc - 1, p).total;
          if (fits(front_fn(p), nc, bf)) {
            bytes_f = bf;
            push = p;
            break;
          }
        }
        if (bytes_f == 0) continue;
      }
      ds_nc_ = nc;
      ds_smem_ = bytes;
      ds_smem_f_ = bytes_f;
      ds_push_ = push;
      use_dstep_ = true;
      break;
    }
    if (!use_dstep_) return;
    fuse_front_ = front;
    if (fuse_front_) {
      bpart_ = dalloc<double>(std::max(nblk_coef_, ds_nc_));
      WLR_CUDA(cudaMemsetAsync(bpart_, 0, sizeof(double) * std::max(nblk_coef_, ds_nc_), stream_));
    }
    ZKh_ = dalloc<T>((size_t)n2 * b);
    if (std::is_same<T, float>::value) {
      Kh_ = dalloc<float>((size_t)n2 * n2);
      Kl_ = dalloc<float>((size_t)n2 * n2);
      ZKl_ = dalloc<T>((size_t)n2 * b);
    }
  }
  // q subspace steps: K V on all SMs, then the cluster kernel (which also leaves
  // G = C C^T and C V_s for the row pass)
  // K V for the current basis (all SMs)
  void kv_launch(cudaStream_t st) {
    const int n2 = d_.n2, b = d_.b;
    const T *Kh, *Kl;
    if constexpr (std::is_same<T, float>::value) {
      Kh = Kh_;
      Kl = Kl_;
    } else {
      Kh = K64_;
      Kl = nullptr;
    }
    const int64_t warps = (int64_t)n2 * cdiv(b, KV_CG);
    kv_pair<T><<<cdiv(warps, 8), 256, 0, st>>>(Kh, Kl, V_, n2, b, ZKh_, ZKl_);
    count(1);
  }
  // K V of step a3 depends only on the basis V, which nothing changes before the D-step:
  // start it on the side stream next to the Gram kernel of step a1 (one CTA per SM, which
  // leaves room beside it); dstep_run waits for it
  void keep_prev_factors(cudaStream_t st) {
    const int k = d_.k, n2 = d_.n2, s = d_.s, NP = d_.NP;
    if (n2 > 0) WLR_CUDA(cudaMemcpyAsync(Z2prev_, Z2_, sizeof(T) * (size_t)n2 * NP, cudaMemcpyDeviceToDevice, st));
    if (s > 0) WLR_CUDA(cudaMemcpyAsync(CVprev_, CV_, sizeof(T) * (size_t)k * s, cudaMemcpyDeviceToDevice, st));
    copies_deferred_ = false;
  }
  void fork_kv() {
    if (!use_dstep_ || eig_cold_ || prof_ || kv_pending_) return;
    WLR_CUDA(cudaEventRecord(ev_fork_, stream_));
    WLR_CUDA(cudaStreamWaitEvent(stream2_, ev_fork_, 0));
    if (copies_deferred_) keep_prev_factors(stream2_);
    kv_launch(stream2_);
    WLR_CUDA(cudaEventRecord(ev_join_, stream2_));
    kv_pending_ = true;
  }
  void dstep_run(int q, bool cold, bool front = false) {
    const int n2 = d_.n2, b = d_.b;
    if (copies_deferred_) keep_prev_factors(stream_);   // not forked after all: copy here
    DstepArgs<T> a = {};
    if constexpr (std::is_same<T, float>::value) {
      a.Bh = Bh_;
      a.Bl = Bl_;
    } else {
      a.Bh = B64_;
      a.Bl = nullptr;
    }
    a.ZKh = ZKh_;
    a.ZKl = ZKl_;
    a.Z2 = Z2_;
    a.V = V_;
    a.Vs = Vs_;
    a.theta = theta_;
    a.resid = resid_;
    a.G = G_;
    a.CV = CV_;
    a.err = err_;
    a.n2 = n2;
    a.k = d_.k;
    a.b = b;
    a.s = d_.s;
    a.NP = d_.NP;
    a.sweeps = cold ? (sizeof(T) == 4 ? 12 : 24) : (sizeof(T) == 4 ? 1 : 6);
    a.S2T = S2T_;
    a.F2 = F2_;
    a.R1inv = front_rpre_;
    a.Nout = Nm_;
    a.Rinv = Rinv_;
    a.Cout = C_;
    a.bpart = bpart_;
    // the series form of the second factor leaves a full R^{-1}, which the tensor-core
    // path's Q1 formation (form_q_split, the row pass) takes as such
    a.series = use_tc_ ? 1 : 0;
    if constexpr (std::is_same<T, float>::value) {
      a.B64 = nullptr;
      a.Bho = Bh_;
      a.Blo = Bl_;
    } else {
      a.B64 = B64_;
      a.Bho = nullptr;
      a.Blo = nullptr;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(ds_nc_);
    cfg.blockDim = dim3(DS_THREADS);
    cfg.dynamicSmemBytes = ds_smem_;
    cfg.stream = stream_;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = ds_nc_;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    for (int t = 0; t < q; ++t) {
      if (t == 0 && kv_pending_) {
        // K V was started on the side stream when the iteration began (V has not changed)
        WLR_CUDA(cudaStreamWaitEvent(stream_, ev_join_, 0));
        kv_pending_ = false;
      } else {
        Prof pf(this, "kv_pair");
        kv_launch(stream_);
      }
      a.front = front && t == 0 ? 1 : 0;
      if (a.front) {
        Prof pf(this, "dstep");
        cfg.dynamicSmemBytes = ds_smem_f_;
        if (ds_push_) {
          if (ds_ne_ == 1)
            WLR_CUDA(cudaLaunchKernelEx(&cfg, dstep_front<T, 1, true>, a));
          else
            WLR_CUDA(cudaLaunchKernelEx(&cfg, dstep_front<T, 2, true>, a));
        } else {
          if (ds_ne_ == 1)
            WLR_CUDA(cudaLaunchKernelEx(&cfg, dstep_front<T, 1, false>, a));
          else
            WLR_CUDA(cudaLaunchKernelEx(&cfg, dstep_front<T, 2, false>, a));
        }
        cfg.dynamicSmemBytes = ds_smem_;
      } else {
        Prof pf(this, "dstep");
        if (ds_ne_ == 1)
          WLR_CUDA(cudaLaunchKernelEx(&cfg, dstep_cluster<T, 1>, a));
        else
          WLR_CUDA(cudaLaunchKernelEx(&cfg, dstep_cluster<T, 2>, a));
      }
      count(1);
    }
  }
  void eig_start() {
    eig_random_start<T><<<grid1d((int64_t)d_.n2 * d_.b), 256, 0, stream_>>>(V_, d_.n2, d_.b, o_.seed);
    count(1);
  }
  void prep() {
    const int k = d_.k, n2 = d_.n2, s = d_.s, NP = d_.NP;
    if (n2 == 0) return;  // G = 0 (cleared at construction), CV unused
    Prof pf(this, "prep_gram");
    prep_gram<T><<<nblk_prep_, 256, sizeof(T) * 64 * (NP + 1), stream_>>>(Z2_, n2, k, s, NP, prep_part_,
                                                                        prep_ticket_, G_, CV_);
    count(1);
  }
  // steps a1..a3 (+ the small products for a4/a5) for X1 = X1buf_[xi]
  void compute_cd(int xi, bool warm, bool precond = false) {
    qr_coef(xi, precond, fuse_front_);
    if (d_.s > 0) {
      int q = warm ? o_.eig_iters : o_.eig_iters_cold;
      bool cold = false;
      if (eig_cold_) {
        eig_start();
        q = o_.eig_iters_cold;
        eig_cold_ = false;
        cold = true;
      }
      if (use_dstep_) {
        dstep_run(q, cold, fuse_front_);   // also G = C C^T and C V_s
      } else {
        form_g2_launch();
        for (int t = 0; t < q; ++t) eig_iteration(cold);
        prep();
      }
    } else {
      prep();
    }
    cd_valid_ = true;
  }
  // iterate the subspace step until the wanted Ritz values settle (FP64 scoring)
  void converge_eig() {
    if (eig_cold_) {
      eig_start();
      eig_cold_ = false;
    }
    // rounds of ten subspace steps until the Ritz values stop changing: every value to
    // 1e-15 of the largest, or their sum (what F~ depends on: sum_{j <= s} sigma_j^2 and a
    // D that is unique up to ties sigma_s = sigma_{s+1}) to 1e-14 of itself; with nearly
    // equal sigma_s and sigma_{s+1} the single values can take hundreds of rounds while
    // the sum has long settled
    const int s = d_.s;
    std::vector<T> prev(s, (T)0), now(s);
    double sum_prev = 0.0;
    for (int round = 0; round < 400; ++round) {
      if (use_dstep_) dstep_run(10, true);
      else
        for (int t = 0; t < 10; ++t) eig_iteration(true);
      WLR_CUDA(cudaMemcpyAsync(hbuf_ + 128, theta_, sizeof(T) * s, cudaMemcpyDeviceToHost, stream_));
      WLR_CUDA(cudaStreamSynchronize(stream_));
      std::memcpy(now.data(), hbuf_ + 128, sizeof(T) * s);
      double diff = 0, top = std::fabs((double)now[0]), sum = 0.0;
      for (int c = 0; c < s; ++c) {
        diff = std::max(diff, std::fabs((double)now[c] - (double)prev[c]));
        sum += (double)now[c];
      }
      prev = now;
      const bool settled = round > 0 && (diff <= 1e-15 * std::max(top, 1e-300) ||
                                         std::fabs(sum - sum_prev) <= 1e-14 * std::max(std::fabs(sum), 1e-300));
      sum_prev = sum;
      if (settled) break;
    }
  }

  // step a4 + a5 + objective, then a1..a3 for the new X1 (one loop body of Algorithm 1)
  void iteration_body(int xi, int xo, bool steady) {
    const int m = d_.m, k = d_.k, n2 = d_.n2, s = d_.s, NP = d_.NP;
    const size_t smem = RowPassSmem<T>::bytes(NP, k, s);
    const int g = nblk_row_;

    {
      Prof pf(this, "row_pass");
      FinalizeArgs<T> fin{bpart_, n2 > 0 ? (fuse_front_ ? ds_nc_ : nblk_coef_) : 0, normA2_, theta_, Fhist_, hist_cap_, iter_, Fcur_,
                          fin_ticket_};
      // steady state on the tensor-core path: the next CholeskyQR's Q1 = X1_{p+1} R_p^{-1}
      // (R_p^{-1} is final before this pass) is formed by the row pass itself
      q_from_row_pass_ = steady && use_tc_ && std::is_same<T, float>::value && row_kp(k) <= 32;
      QSplitOut qo{nullptr, nullptr, 0, nullptr};
      if (q_from_row_pass_) qo = QSplitOut{Q1h_, Q1l_, ld4_, (const float*)Rinv_};
      row_pass_fn<T>(k)<<<g, 256, smem, stream_>>>(A_, lda_, W1_, ldw_, X1buf_[xi], Z2_, G_, CV_, m, n2, k, s, NP,
                                                  X1buf_[xo], wpart_, err_, fin, qo);
    }
    count(1);
    // keep the factors of X1_p for Error_p.  When the K V kernel will be started on the
    // side stream (tensor-core Gram, fused front stage, warm subspace), the copies go there
    // too, off the critical path: the row pass above was their last reader before them and
    // the cluster kernel, which joins the side stream, is the next writer of Z2 and CV.
    copies_deferred_ = use_tc_ && fuse_front_ && use_dstep_ && !eig_cold_ && !prof_ && !kv_pending_;
    if (!copies_deferred_) keep_prev_factors(stream_);
    compute_cd(xo, true, steady);
  }

  // iterations after set_init that use the full CholeskyQR2 before switching to the
  // previous-R preconditioned form (and to graph replay)
  static constexpr int kFullQrIters = 3;

  void iterate_once() {
    const int xi = cur_, xo = (cur_ + 1) % 3;
    const bool steady = iters_host_ >= kFullQrIters;
    if (o_.use_graph && !eig_cold_ && steady) {
      auto it = graphs_.find(xi);
      if (it == graphs_.end()) {
        cudaGraph_t graph;
        const int64_t before = launches_;
        WLR_CUDA(cudaStreamBeginCapture(stream_, cudaStreamCaptureModeThreadLocal));
        try {
          iteration_body(xi, xo, true);
        } catch (...) {
          cudaStreamEndCapture(stream_, &graph);
          throw;
        }
        WLR_CUDA(cudaStreamEndCapture(stream_, &graph));
        cudaGraphExec_t exec;
        WLR_CUDA(cudaGraphInstantiate(&exec, graph, 0));
        cudaGraphDestroy(graph);
        graph_launch_count_ = launches_ - before;
        launches_ = before;
        it = graphs_.emplace(xi, exec).first;
      }
      WLR_CUDA(cudaGraphLaunch(it->second, stream_));
      launches_ += graph_launch_count_;
    } else {
      iteration_body(xi, xo, steady);
    }
    prev_ = xi;
    cur_ = xo;
    ++iters_host_;
  }
  void graphs_clear() {
    for (auto& g : graphs_) cudaGraphExecDestroy(g.second);
    graphs_.clear();
    for (auto& g : graphs3_) cudaGraphExecDestroy(g.second);
    graphs3_.clear();
  }
  // Three steady-state iterations (one turn of the X1 buffers) as one CUDA graph, cached
  // per starting buffer: fewer graph launches when nothing is read back between iterations.
  bool three_ready() const { return o_.use_graph && cd_valid_ && !eig_cold_ && iters_host_ >= kFullQrIters && !prof_; }
  void iterate_three() {
    auto it = graphs3_.find(cur_);
    if (it == graphs3_.end()) {
      cudaGraph_t graph = batch_capture(3);
      cudaGraphExec_t exec;
      const cudaError_t e = cudaGraphInstantiate(&exec, graph, 0);
      cudaGraphDestroy(graph);
      WLR_CUDA(e);
      graph3_launch_count_ = batch_launch_count_;
      it = graphs3_.emplace(cur_, exec).first;
    }
    WLR_CUDA(cudaGraphLaunch(it->second, stream_));
    prev_ = (cur_ + 2) % 3;
    iters_host_ += 3;
    launches_ += graph3_launch_count_;
  }

  // ------------------------------------------------------------------ batched solve
  bool batch_ready() override {
    need_init();
    return o_.use_graph && cd_valid_ && !eig_cold_ && iters_host_ >= kFullQrIters;
  }
  void batch_iterate() override {
    need_init();
    begin();
    if (!cd_valid_) compute_cd(cur_, false);
    iterate_once();
    end();
  }
  cudaGraph_t batch_capture(int n) override {
    if (!batch_ready()) throw Fail{WLR_ERR_NOT_READY, "handle not warmed up for batched replay"};
    cudaGraph_t graph = nullptr;
    const int64_t before = launches_;
    WLR_CUDA(cudaStreamBeginCapture(stream_, cudaStreamCaptureModeThreadLocal));
    try {
      for (int q = 0; q < n; ++q) {
        const int xi = (cur_ + q) % 3;
        iteration_body(xi, (xi + 1) % 3, true);
      }
    } catch (...) {
      cudaStreamEndCapture(stream_, &graph);
      if (graph) cudaGraphDestroy(graph);
      launches_ = before;
      throw;
    }
    WLR_CUDA(cudaStreamEndCapture(stream_, &graph));
    batch_launch_count_ = launches_ - before;
    launches_ = before;
    return graph;
  }
  void batch_advance(int n) override {
    prev_ = (cur_ + n - 1) % 3;
    cur_ = (cur_ + n) % 3;
    iters_host_ += n;
    launches_ += batch_launch_count_;
  }
  void batch_enter(cudaStream_t bs) override {
    begin();
    WLR_CUDA(cudaEventRecord(ev_batch_, stream_));
    WLR_CUDA(cudaStreamWaitEvent(bs, ev_batch_, 0));
  }
  void batch_leave(cudaStream_t bs) override {
    WLR_CUDA(cudaEventRecord(ev_batch_, bs));
    WLR_CUDA(cudaStreamWaitEvent(stream_, ev_batch_, 0));
    end();
  }
  void batch_finish() override {
    WLR_CUDA(cudaStreamSynchronize(stream_));
    raise_err();
  }

  // exact evaluation of the current (and previous) iterate; result sums in e6
  void x2_eval(int xi, int xp, T* out, int64_t ldo, double* e6) {
    const int m = d_.m, k = d_.k, n2 = d_.n2, s = d_.s, NP = d_.NP;
    const T* X1p = xp >= 0 ? X1buf_[xp] : nullptr;
    x2_pass<T><<<nblk_row_, 256, x2_smem(), stream_>>>(A_, lda_, W1_, ldw_, X1buf_[xi], Z2_, CV_, X1p,
                                                      X1p ? Z2prev_ : nullptr, X1p ? CVprev_ : nullptr,
                                                      m, n2, k, s, NP, out, ldo, x2part_);
    reduce_partials<double><<<1, 32, 0, stream_>>>(x2part_, 8, nblk_row_, 6, x2sum_, nullptr);
    count(2);
    WLR_CUDA(cudaMemcpyAsync(hbuf_ + 256, x2sum_, sizeof(double) * 6, cudaMemcpyDeviceToHost, stream_));
    WLR_CUDA(cudaStreamSynchronize(stream_));
    std::memcpy(e6, hbuf_ + 256, sizeof(double) * 6);
  }

  // ------------------------------------------------------------------ state
  Dims d_;
  wlr_options o_;
  cudaStream_t ustream_ = nullptr, stream_ = nullptr;
  cudaEvent_t ev_in_ = nullptr, ev_out_ = nullptr, ev_batch_ = nullptr;
  unsigned char* hbuf_ = nullptr;
  std::vector<void*> allocs_;
  int64_t launches_ = 0, graph_launch_count_ = 0, batch_launch_count_ = 0;

  const T* A_ = nullptr;
  int64_t lda_ = 0;
  T* A_own_ = nullptr;
  const T* W1_ = nullptr;
  int64_t ldw_ = 0;
  T* W1_own_ = nullptr;
  bool have_data_ = false, have_init_ = false, cd_valid_ = false, eig_cold_ = true;
  int cur_ = 0, prev_ = -1, iters_host_ = 0;
  std::vector<double> rel_err_hist_;

  T* X1buf_[3] = {nullptr, nullptr, nullptr};
  T *Q1_ = nullptr, *R1inv_ = nullptr, *Nm_ = nullptr, *Rinv_ = nullptr;
  double *part64_ = nullptr, *S2T_ = nullptr;
  T* F2_ = nullptr;   // S2 - I for the second Cholesky factor (k <= 32)
  bool use_dstep_ = false;   // fused cluster kernel for step a3
  cudaStream_t stream2_ = nullptr;   // side stream for K V
  cudaEvent_t ev_fork_ = nullptr, ev_join_ = nullptr;
  bool kv_pending_ = false;
  bool copies_deferred_ = false;   // Z2, CV -> previous-iterate copies left to fork_kv
  bool fuse_front_ = false;  // ... with the second factor and B, C in front (k <= 32)
  const T* front_rpre_ = nullptr;
  int ds_nc_ = 0, ds_ne_ = 1;
  size_t ds_smem_ = 0, ds_smem_f_ = 0;
  bool ds_push_ = false;     // dstep_front exchanges by remote stores
  float *Kh_ = nullptr, *Kl_ = nullptr;   // K as a float pair (float path)
  T *ZKh_ = nullptr, *ZKl_ = nullptr;     // K V (high, low)
  T *C_ = nullptr, *Z2_ = nullptr, *Z2prev_ = nullptr;
  double *B64_ = nullptr, *bpart_ = nullptr, *K64_ = nullptr, *prep_part_ = nullptr;
  float *Bh_ = nullptr, *Bl_ = nullptr;
  unsigned int *prep_ticket_ = nullptr, *eig_ticket_ = nullptr, *fin_ticket_ = nullptr;
  T* HP_ = nullptr;
  // tensor-core Gram (FP32 path)
  bool use_tc_ = false;     // Q1^T [Q1 A2] on the tensor cores (k <= 32)
  bool use_tc_k_ = false;   // K = A2^T A2 on the tensor cores
  bool q_from_row_pass_ = false;   // the last row pass wrote Q1 (consumed by tc_gram)
  int tn_ = 32;             // MMA N of the Q1^T [Q1 A2] kernel (32 or 64 columns of Q1)
  int64_t ld4_ = 0;
  size_t part_elems_ = 0;
  float *A2h_ = nullptr, *A2l_ = nullptr, *Q1h_ = nullptr, *Q1l_ = nullptr;
  CUtensorMap mA2h_, mA2l_, mQh128_, mQl128_, mQh32_, mQl32_, mA2h64_, mA2l64_;
  CUtensorMap mA2f_;          // FP32 A2 itself (per-iteration Gram, split in shared memory)
  bool a2f_ok_ = false;
  void* enc_ = nullptr;       // cuTensorMapEncodeTiled
  int2* kk_pairs_ = nullptr;   // column-block pairs of the tensor-core K
  int kk_npairs_ = 0;
  Chunk ch_kk_{1, 32};
  Chunk ch_tc_{1, 32};
  int nblk_prep_ = 0;
  bool eig_vsmem_ = false;
  T* G2_ = nullptr;
  double* normA2_ = nullptr;
  T *V_ = nullptr, *Zeig_ = nullptr, *eigpart_ = nullptr, *Y_ = nullptr, *Mv_ = nullptr, *Mz_ = nullptr;
  T *theta_ = nullptr, *resid_ = nullptr, *Vs_ = nullptr;
  T *G_ = nullptr, *CV_ = nullptr, *CVprev_ = nullptr;
  double *wpart_ = nullptr, *x2part_ = nullptr, *x2sum_ = nullptr, *Fhist_ = nullptr, *Fcur_ = nullptr;
  double* sumsq_part_ = nullptr;
  int *iter_ = nullptr, *err_ = nullptr;
  int hist_cap_ = 0, nblk_coef_ = 0, nblk_eig_ = 0, nblk_row_ = 0;
  Chunk ch_S1_{1, 32}, ch_T_{1, 32}, ch_K_{1, 32};
  void* stage_ = nullptr;
  size_t stage_bytes_ = 0;
  void* stage2_ = nullptr;
  size_t stage2_bytes_ = 0;
  std::map<int, cudaGraphExec_t> graphs_;
  std::map<int, cudaGraphExec_t> graphs3_;   // three iterations from X1 buffer key
  int64_t graph3_launch_count_ = 0;
  SolverBase* scorer_ = nullptr;
  struct ProfRec {
    const char* name;
    cudaEvent_t a, b;
  };
  bool prof_ = false;
  std::vector<ProfRec> prof_recs_;
  std::vector<cudaEvent_t> ev_pool_;
  size_t ev_used_ = 0;
};

}  // namespace wlr
