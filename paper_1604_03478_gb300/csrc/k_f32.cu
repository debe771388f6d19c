// k_f32.cu -- kernels with FP32 storage of the shifted distributions.
#include "launch_impl.cuh"

template struct lbm::Launch<float>;
