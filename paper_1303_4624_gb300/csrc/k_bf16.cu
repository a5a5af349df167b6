// k_bf16.cu - kernels and launchers of the bf16 storage form.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#define LBM_STORE __nv_bfloat16
#define LBM_OPS kOpsBF16
#include "k_storage.inl"
