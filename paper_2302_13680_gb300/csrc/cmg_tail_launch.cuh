// Launcher of the cluster-resident coarse-grid cycle for one precision.
#pragma once

#include "cmg_tail.cuh"

namespace cmg {
namespace tail {

// Cluster size chosen once per kernel instantiation: the largest of 16
// (non-portable), 8, 4 for which the occupancy query reports an active
// cluster; -1 if none.
template <typename T, int V, int SPL, int MM>
cudaError_t launch_one(const TailParams<T>& P, cudaStream_t s) {
  auto kern = tail_cycle_kernel<T, V, SPL, MM>;
  static int cs = 0;
  if (cs == 0) {
    (void)cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    const int sizes[3] = {16, 8, 4};
    for (int c : sizes) {
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(c, 1, 1);
      cfg.blockDim = dim3(kTailThreads, 1, 1);
      cfg.dynamicSmemBytes = 0;
      cfg.stream = s;
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeClusterDimension;
      attr[0].val.clusterDim.x = c;
      attr[0].val.clusterDim.y = 1;
      attr[0].val.clusterDim.z = 1;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      int num = 0;
      if (cudaOccupancyMaxActiveClusters(&num, kern, &cfg) == cudaSuccess && num > 0) {
        cs = c;
        break;
      }
      (void)cudaGetLastError();
    }
    if (cs == 0) cs = -1;
  }
  if (cs < 0) return cudaErrorNotSupported;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(cs, 1, 1);
  cfg.blockDim = dim3(kTailThreads, 1, 1);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cs;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;   // the kernel starts with pdl_enter
  attr[1].val.programmaticStreamSerializationAllowed = pdl_enabled() ? 1 : 0;
  cfg.attrs = attr;
  cfg.numAttrs = 2;
  const cudaError_t e = cudaLaunchKernelEx(&cfg, kern, P);
  count_launches(1);
  return e;
}

template <typename T, int V, int SPL>
cudaError_t launch_mm(const TailParams<T>& P, cudaStream_t s) {
  switch (P.cm) {
    case 1: return launch_one<T, V, SPL, 1>(P, s);
    case 9: return launch_one<T, V, SPL, 9>(P, s);
    default: return cudaErrorNotSupported;
  }
}

template <typename T>
cudaError_t launch(const TailParams<T>& P, cudaStream_t s) {
  const SampleMap m = choose_map(P.cN, sizeof(T), 0);
  if (m.spl > 4 || P.nlev > kTailMax || P.cN > kTailThreads * 8) return cudaErrorNotSupported;
  const int vmax = 16 / (int)sizeof(T);
  if (m.V == 1) {
    switch (m.spl) {
      case 1: return launch_mm<T, 1, 1>(P, s);
      case 2: return launch_mm<T, 1, 2>(P, s);
      case 4: return launch_mm<T, 1, 4>(P, s);
    }
  } else if (m.V == vmax) {
    constexpr int VV = 16 / sizeof(T);
    switch (m.spl) {
      case 1: return launch_mm<T, VV, 1>(P, s);
      case 2: return launch_mm<T, VV, 2>(P, s);
      case 4: return launch_mm<T, VV, 4>(P, s);
    }
  }
  return cudaErrorNotSupported;
}

}  // namespace tail
}  // namespace cmg
