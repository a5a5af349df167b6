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
// Validation of the initial fields on the device: rho > 0, T > 0 and every value
// finite (NaN fails every comparison).  *first_bad (preset to all ones) receives the
// smallest (index << 2 | field) of a bad value, field 0 rho, 1 U, 2 T.
static __global__ void k_check_fields(const double* __restrict__ rho, const double* __restrict__ U,
                                      const double* __restrict__ T, long long n, long long begin,
                                      long long end, int D,
                                      unsigned long long* __restrict__ first_bad) {
  for (long long i = begin + (long long)blockIdx.x * blockDim.x + threadIdx.x; i < end;
       i += (long long)gridDim.x * blockDim.x) {
    int field = -1;
    const double r = rho[i], t = T[i];
    if (!(r > 0.0 && r <= 1.7976931348623157e308)) field = 0;
    else {
      for (int d = 0; d < D; ++d)
        if (!(fabs(U[(size_t)d * n + i]) <= 1.7976931348623157e308)) field = 1;
      if (field < 0 && !(t > 0.0 && t <= 1.7976931348623157e308)) field = 2;
    }
    if (field >= 0) atomicMin(first_bad, ((unsigned long long)i << 2) | (unsigned long long)field);
  }
}

cudaError_t launch_check_fields(const double* rho, const double* U, const double* T, long long n,
                                long long begin, long long end, int D,
                                unsigned long long* first_bad, cudaStream_t st) {
  const long long nb = (end - begin + 255) / 256;
  if (nb <= 0) return cudaSuccess;
  k_check_fields<<<(unsigned)(nb < 4096 ? nb : 4096), 256, 0, st>>>(rho, U, T, n, begin, end, D,
                                                                    first_bad);
  return cudaGetLastError();
}

cudaError_t launch_sum_reduce(const double* partials, long long n, double* out, cudaStream_t st) {
  k_sum_reduce<<<1, 256, 0, st>>>(partials, n, out);
  return cudaGetLastError();
}
}  // namespace lbm
