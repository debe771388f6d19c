// ens_f16_k2.cu -- the batched form's persistent kernel for FP16 storage and
// 2 z-planes per item, in a translation unit of its own (parallel build).
#include "ensemble_kernel.cuh"

const void *lbm::ens_kernel_f16_k2() { return (const void *)lbm::k_ensemble<__half, 2>; }
