// Cluster-resident coarse-grid cycle, FP64 instantiations.
#include "cmg_tail_launch.cuh"

namespace cmg {
template <>
cudaError_t launch_tail_cycle<double>(const TailParams<double>& P, cudaStream_t s) {
  return tail::launch<double>(P, s);
}

bool tail_supported(int N, int elem_bytes, int coarse_m) {
  const SampleMap m = choose_map(N, elem_bytes, 0);
  return m.spl <= 4 && (coarse_m == 1 || coarse_m == 9);
}
}  // namespace cmg
