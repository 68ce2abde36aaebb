// Ops<float>: kernels and launchers for the f32 storage format.
#include "lb_ops_impl.cuh"

namespace trt {
template struct Ops<float>;
}  // namespace trt
