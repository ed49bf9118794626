// Tiled interior stage kernel (placeholder until the tiled kernel lands).
#include "common.cuh"
#include "launch.h"

namespace sbp {

template <typename T>
cudaError_t launch_stage_interior(const StageArgs<T>&, int, const Box&, cudaStream_t) {
  return cudaErrorNotSupported;
}
template cudaError_t launch_stage_interior<float>(const StageArgs<float>&, int, const Box&, cudaStream_t);
template cudaError_t launch_stage_interior<double>(const StageArgs<double>&, int, const Box&, cudaStream_t);

}  // namespace sbp
