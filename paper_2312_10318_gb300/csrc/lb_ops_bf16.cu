// Ops<__nv_bfloat16>: kernels and launchers for the bf16 storage format.
#include "lb_ops_impl.cuh"

namespace trt {
template struct Ops<__nv_bfloat16>;
}  // namespace trt
