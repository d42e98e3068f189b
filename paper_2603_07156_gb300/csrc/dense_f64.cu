// Dense passes with float64 anchored matrix and float64 arithmetic.
#include "dense_launch.cuh"

namespace ibsn {

template <>
cudaError_t launch_dense<double>(Pass p, DenseArgs<double>& A, int nsm, cudaStream_t st, PassGeom* geom) {
  return launch_dense_t<double>(p, A, nsm, st, geom);
}

int dense_max_blocks_f64(int64_t n, int nsm) { return dense_max_blocks_t<double>(n, nsm); }

}  // namespace ibsn
