// Cluster-resident coarse-grid cycle, FP32 instantiations.
#include "cmg_tail_launch.cuh"

namespace cmg {
template <>
cudaError_t launch_tail_cycle<float>(const TailParams<float>& P, cudaStream_t s) {
  return tail::launch<float>(P, s);
}
}  // namespace cmg
