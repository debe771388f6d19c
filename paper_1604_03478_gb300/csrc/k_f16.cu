// k_f16.cu -- kernels with FP16 storage of the shifted distributions
// (f - w rho0, g - w Tm); arithmetic stays FP32.
#include "launch_impl.cuh"

template struct lbm::Launch<__half>;
