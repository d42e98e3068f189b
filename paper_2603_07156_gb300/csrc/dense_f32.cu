// Dense passes with float32 anchored matrix and float32 per-entry arithmetic
// (mixed precision: float64 row/column totals).
#define IBSN_FF_PASSES
#include "dense_launch.cuh"

namespace ibsn {

template <>
cudaError_t launch_dense<float>(Pass p, DenseArgs<float>& A, int nsm, cudaStream_t st, PassGeom* geom) {
  return launch_dense_t<float>(p, A, nsm, st, geom);
}

int dense_max_blocks_f32(int64_t n, int nsm) { return dense_max_blocks_t<float>(n, nsm); }

cudaError_t launch_dense_ff(Pass p, DenseArgs<float>& A, int nsm, cudaStream_t st, PassGeom* geom) {
  return launch_dense_ff_t(p, A, nsm, st, geom);
}

}  // namespace ibsn
