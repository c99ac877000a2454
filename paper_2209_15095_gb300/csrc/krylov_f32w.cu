// Instantiation of the Krylov kernel with FP32 vectors and 768 threads per
// CTA (80 registers per thread) for problems on the 4-node groups: their
// passes are bound by the bytes each SM keeps in flight.  Measured at 512^3
// (one mixed ETD2 step, same GPU): 512 / 768 / 1024 threads 10.2 / 9.8 /
// 11.4 ms; at star3d (15.9k points) 768 threads cost the Krylov launch 15%
// and at twoball3d (114k points per species) 11% (register spills in the
// per-point paths), so those keep 512.
#define ETD_RED_MAX_NT 768
#include "krylov_impl.cuh"

namespace etd {

PhipmKernels phipm_kernels_f32w() { return phipm_kernels<float, 768>(); }

}  // namespace etd
