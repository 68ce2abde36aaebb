// Ops<f64dw>: FP64 storage with double-word FP32 collision arithmetic.
#include "lb_ops_impl.cuh"

namespace trt {
template struct Ops<f64dw>;
}  // namespace trt
