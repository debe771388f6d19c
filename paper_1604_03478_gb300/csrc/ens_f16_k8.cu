// ens_f16_k8.cu -- the batched form's persistent kernel for FP16 storage and
// 8 z-planes per item, in a translation unit of its own (parallel build).
#include "ensemble_kernel.cuh"

const void *lbm::ens_kernel_f16_k8() { return (const void *)lbm::k_ensemble<__half, 8>; }
