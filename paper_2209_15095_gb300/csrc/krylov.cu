// Launch of the adaptive Krylov kernel (krylov_impl.cuh): picks the
// instantiation by precision and, for FP32, by `wide` (the caller's choice of
// the 768-thread kernel for problems on the 4-node groups), loads the unit's
// constants on first use, and runs it as a cooperative launch (one CTA per SM).
#include "kernels.cuh"

namespace etd {

PhipmKernels phipm_kernels_f64();
PhipmKernels phipm_kernels_f32();
PhipmKernels phipm_kernels_f32w();

namespace {
struct Variant {
  PhipmKernels k;
  bool loaded = false;
};
Variant& f64() {
  static Variant v{phipm_kernels_f64()};
  return v;
}
Variant& f32() {
  static Variant v{phipm_kernels_f32()};
  return v;
}
Variant& f32w() {
  static Variant v{phipm_kernels_f32w()};
  return v;
}

template <typename T>
Variant& variant(bool wide) {
  if (sizeof(T) == 8) return f64();
  return wide ? f32w() : f32();
}
}  // namespace

template <typename T>
cudaError_t launch_phipm(const PhipmArgs<T>& a, int nblocks, cudaStream_t stream, bool wide) {
  Variant& v = variant<T>(wide);
  if (!v.loaded) {
    cudaError_t e = v.k.load_consts();
    if (e != cudaSuccess) return e;
    v.loaded = true;
  }
  const bool adj = a.mode == MODE_ADJ_LAMBDA || a.mode == MODE_ADJ_Y;
  if (a.g.ndim < 2 || a.g.ndim > 4) return cudaErrorInvalidValue;
  void* fn = v.k.fn[a.g.ndim - 2][adj ? 1 : 0];
  if (nblocks > MAX_BLOCKS) return cudaErrorInvalidValue;
  cudaError_t e = cudaMemsetAsync(&a.st->barrier, 0, sizeof(unsigned), stream);
  if (e != cudaSuccess) return e;
  void* args[] = {(void*)&a};
  const size_t dsm = adj ? v.k.adj_smem : 0;
  return cudaLaunchCooperativeKernel(fn, nblocks, v.k.nt, args, dsm, stream);
}

// CTAs of a launch: one per SM, if every instantiation the context may
// launch (the adjoint ones with their dynamic shared memory, which for the
// 768-thread kernel exceeds the default 48 KB of a block) fits once per SM.
int phipm_max_blocks(int ndim, bool fp32) {
  if (ndim < 2 || ndim > 4) return 0;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  Variant* vs[2] = {fp32 ? &f32() : &f64(), fp32 ? &f32w() : nullptr};
  int per = 1;
  for (Variant* v : vs) {
    if (!v) continue;
    for (int adj = 0; adj < 2; ++adj) {
      void* fn = v->k.fn[ndim - 2][adj];
      const size_t dsm = adj ? v->k.adj_smem : 0;
      if (adj && cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dsm) != cudaSuccess)
        return 0;
      int p = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p, fn, v->k.nt, dsm) != cudaSuccess) return 0;
      per = min(per, p);
    }
  }
  return per * sms;
}

template cudaError_t launch_phipm<double>(const PhipmArgs<double>&, int, cudaStream_t, bool);
template cudaError_t launch_phipm<float>(const PhipmArgs<float>&, int, cudaStream_t, bool);

}  // namespace etd
