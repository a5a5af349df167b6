// k_fp16.cu - kernels and launchers of the fp16 storage form.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#define LBM_STORE __half
#define LBM_OPS kOpsFP16
#include "k_storage.inl"
