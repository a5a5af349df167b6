// k_fp64.cu - kernels and launchers of the fp64 storage form.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#define LBM_STORE double
#define LBM_OPS kOpsFP64
#include "k_storage.inl"

namespace lbm {
// The audit reduction is storage-independent; it lives in this translation unit.
cudaError_t launch_audit_reduce(const double* partials, int nblocks, double* out,
                                cudaStream_t st) {
  k_audit_reduce<<<1, 256, 0, st>>>(partials, nblocks, out);
  return cudaGetLastError();
}
cudaError_t launch_sum_reduce(const double* partials, long long n, double* out, cudaStream_t st) {
  k_sum_reduce<<<1, 256, 0, st>>>(partials, n, out);
  return cudaGetLastError();
}
}  // namespace lbm
