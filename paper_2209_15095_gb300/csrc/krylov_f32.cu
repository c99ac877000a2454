// Instantiation of the Krylov kernel with FP32 vectors and 512 threads per
// CTA (128 registers per thread): the problems off the 4-node groups,
// whose per-point paths are latency-bound and would spill at fewer registers.
#define ETD_RED_MAX_NT 512
#include "krylov_impl.cuh"

namespace etd {

PhipmKernels phipm_kernels_f32() { return phipm_kernels<float, 512>(); }

}  // namespace etd
