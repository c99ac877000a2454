// Instantiation of the Krylov kernel with FP64 vectors (512 threads per CTA,
// 128 registers per thread); also the operator-only kernel and the rounding
// self-check.
#define ETD_RED_MAX_NT 512
#include "krylov_impl.cuh"

namespace etd {

PhipmKernels phipm_kernels_f64() { return phipm_kernels<double, 512>(); }

// The operator alone, and the rounding self-check.
template <int N>
__global__ void apply_kernel(const ApplyArgs a) {
  const int ncomp = *a.ncomp;
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < ncomp; k += (long long)gridDim.x * blockDim.x) {
    const long long p = a.idx[k];
    a.y[p] = stencil<double, N>(a.x, p, a.g, a.diag[k], a.beta_field, a.beta_c, a.cfac);
  }
}

__global__ void round_check_kernel(const double* __restrict__ x, float* __restrict__ lib, float* __restrict__ hw,
                                   long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    lib[i] = to_f32_rn(x[i]);
    hw[i] = __double2float_rn(x[i]);
  }
}

cudaError_t launch_round_check(const double* x, float* lib, float* hw, long long n, cudaStream_t stream) {
  if (n <= 0) return cudaSuccess;
  const long long nb = (n + 255) / 256;
  round_check_kernel<<<(unsigned)(nb < 4096 ? nb : 4096), 256, 0, stream>>>(x, lib, hw, n);
  return cudaGetLastError();
}

cudaError_t launch_apply(const ApplyArgs& a, cudaStream_t stream) {
  switch (a.g.ndim) {
    case 2: apply_kernel<2><<<152 * 4, 256, 0, stream>>>(a); break;
    case 3: apply_kernel<3><<<152 * 4, 256, 0, stream>>>(a); break;
    case 4: apply_kernel<4><<<152 * 4, 256, 0, stream>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace etd
