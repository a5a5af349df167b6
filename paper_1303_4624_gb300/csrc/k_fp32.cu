// k_fp32.cu - kernels and launchers of the fp32 storage form.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#define LBM_STORE float
#define LBM_OPS kOpsFP32
#include "k_storage.inl"
