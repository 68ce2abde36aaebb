// Ops<__half>: kernels and launchers for the f16 storage format.
#include "lb_ops_impl.cuh"

namespace trt {
template struct Ops<__half>;
}  // namespace trt
