// double instantiation of the sWLR solver.
#include "wlr_solver_impl.cuh"

namespace wlr {
SolverBase* make_solver_f64(const Dims& d, const wlr_options& o, cudaStream_t us) {
  return new Solver<double>(d, o, us);
}
}  // namespace wlr
