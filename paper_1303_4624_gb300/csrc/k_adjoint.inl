// k_adjoint.inl - launchers of the adjoint kernels of one storage form.  Included
// by k_storage.inl inside its anonymous namespace (S = the storage element type),
// kept apart from the forward launchers.

// Adjoint arithmetic type: FP64 for the FP64 form, else FP32.
using L = std::conditional<std::is_same<S, double>::value, double, float>::type;

// The adjoint kernel for this grid: 32-bit element indices (FP32 adjoint) when
// Q ncell fits them.
using AdjointFn = void (*)(const S*, const L*, const double*, L*, double*, Grid, double);
template <int M, bool kFirst>
AdjointFn adjoint_kernel(const Grid& g) {
  if constexpr (std::is_same<L, float>::value) {
    if ((unsigned long long)Model<M>::Q * (unsigned long long)g.ncell <= 0xFFFFFFFFull)
      return k_adjoint<M, S, L, kFirst, true>;
  }
  return k_adjoint<M, S, L, kFirst, false>;
}

template <int M>
cudaError_t adjoint_m(const void* state_n, const void* nu_next, const double* dldrho, void* nu_out,
                      double* omega_acc, const Grid& g, double omega, cudaStream_t st) {
  const int bx = cell_block_x(g.nx);
  const dim3 grid((unsigned)((g.nx + bx - 1) / bx), (unsigned)g.ny, (unsigned)g.nz);
  constexpr int smem = adj_smem_bytes<M, L>();
  const AdjointFn kern = dldrho ? adjoint_kernel<M, true>(g) : adjoint_kernel<M, false>(g);
  if constexpr (smem > 0) {
    // Dynamic shared memory above the 48 KB default needs the opt-in, once per device.
    static std::mutex mu;
    static int done_dev[16] = {-1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(mu);
    if (done_dev[dev & 15] != dev) {
      const AdjointFn all[4] = {k_adjoint<M, S, L, true, false>, k_adjoint<M, S, L, false, false>,
                                k_adjoint<M, S, L, true, true>, k_adjoint<M, S, L, false, true>};
      for (int k = 0; k < 4 && e == cudaSuccess; ++k)
        e = cudaFuncSetAttribute(all[k], cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
      if (e != cudaSuccess) return e;
      done_dev[dev & 15] = dev;
    }
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = dim3(bx);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (dldrho)
    return cudaLaunchKernelEx(&cfg, kern, static_cast<const S*>(state_n),
                              static_cast<const L*>(nullptr), dldrho, static_cast<L*>(nu_out),
                              omega_acc, g, omega);
  return cudaLaunchKernelEx(&cfg, kern, static_cast<const S*>(state_n),
                            static_cast<const L*>(nu_next), static_cast<const double*>(nullptr),
                            static_cast<L*>(nu_out), omega_acc, g, omega);
}

template <int M>
cudaError_t grad_init_m(const void* nu0, const double* fields, double* d_rho, double* d_U,
                        double* d_T, const Grid& g, cudaStream_t st) {
  const int bx = cell_block_x(g.nx);
  const dim3 grid((unsigned)((g.nx + bx - 1) / bx), (unsigned)g.ny, (unsigned)g.nz);
  k_grad_init<M, L><<<grid, bx, 0, st>>>(static_cast<const L*>(nu0), fields, d_rho, d_U, d_T, g);
  return cudaGetLastError();
}

cudaError_t adjoint_step(int m, const void* state_n, const void* nu_next, const double* dldrho,
                         void* nu_out, double* omega_acc, const Grid& g, double omega,
                         cudaStream_t st) {
  return m == 0 ? adjoint_m<0>(state_n, nu_next, dldrho, nu_out, omega_acc, g, omega, st)
                : adjoint_m<1>(state_n, nu_next, dldrho, nu_out, omega_acc, g, omega, st);
}
cudaError_t grad_init(int m, const void* nu0, const double* fields, double* d_rho, double* d_U,
                      double* d_T, const Grid& g, cudaStream_t st) {
  return m == 0 ? grad_init_m<0>(nu0, fields, d_rho, d_U, d_T, g, st)
                : grad_init_m<1>(nu0, fields, d_rho, d_U, d_T, g, st);
}
