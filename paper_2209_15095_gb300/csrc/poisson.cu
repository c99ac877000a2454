// Embedded-boundary Poisson solve (Sec. 2: div(beta grad u) = f with Dirichlet
// data, interior ghost points; Sec. 4.1 applies it to a virus-shaped domain).
//
// At the computational points the discrete problem is C u + b = f, with C the
// matrix-free EB operator (the stencil of the Krylov kernel with dt = 1) and
// b the boundary-data term of the ghost values (per point, the face slots'
// coefficient times the boundary value).  C is symmetric negative definite
// (Sec. 2), so the kernel runs conjugate gradients on A = -C, A u = b - f,
// FP64, as one persistent cooperative kernel: per iteration one stencil pass
// with the dot product <p, A p>, one update pass with |r|^2, and the search
// direction update, each followed by a bounded grid barrier.  Reductions are
// deterministic (fixed order, every CTA sums the per-CTA partials alike), so
// every CTA takes the same stopping decision.
#include "common.cuh"
#include "kernels.cuh"

namespace etd {

constexpr int PS_NT = 512;

__device__ __forceinline__ double* ps_part(double* part, int& red) {
  double* b = part + (red & 1) * (4 * MAX_BLOCKS);
  ++red;
  return b;
}

// (C x)_p: the EB stencil on the grid vector x (zero off the computational
// set) with cfac = 1 / h^2.
template <int N>
__device__ __forceinline__ double cstencil(const double* __restrict__ x, long long p, const GridDev& g, double Dk,
                                           const double* __restrict__ bfield, double bc, double cfac) {
  const double xp = __ldcg(x + p);
  if (bfield == nullptr) {
    double s = -0.0;  // x + (-0) == x: the first add is free
#pragma unroll
    for (int d = 0; d < N; ++d) s += __ldcg(x + p - g.stride[d]) + __ldcg(x + p + g.stride[d]);
    return cfac * (bc * s - Dk * xp);
  }
  const double bp = __ldg(bfield + p);
  double s = -0.0;
#pragma unroll
  for (int d = 0; d < N; ++d) {
    const long long st = g.stride[d];
    s += 0.5 * (bp + __ldg(bfield + p - st)) * __ldcg(x + p - st);
    s += 0.5 * (bp + __ldg(bfield + p + st)) * __ldcg(x + p + st);
  }
  return cfac * (s - Dk * xp);
}

template <int N>
__global__ void __launch_bounds__(PS_NT, 1) poisson_kernel(const PoissonArgs a) {
  const SpeciesDev<double>& S = a.S;
  const GridDev& g = a.g;
  const int ncomp = *S.ncomp;
  const long long gtid = dealt_tid();
  const long long gth = (long long)gridDim.x * blockDim.x;
  const double cfac = 1.0 / (g.h * g.h);
  constexpr int SL = 2 * N * (N == 2 ? 2 : 1);
  unsigned bar = 0;
  int red = 0;
  double* const x = S.Yc;                 // compact: iterate
  double* const r = (double*)S.V1c;       // compact: residual
  double* const q = (double*)S.V2c;       // compact: A p
  double* const P = (double*)S.Yg;        // grid: search direction (zero off the set)
  __shared__ double s_tot[2];
  // x_0 from the caller's u; P holds x_0 to apply C to it
  for (long long k = gtid; k < ncomp; k += gth) {
    const long long p = __ldg(S.idx + k);
    const double v = a.u[p];
    x[k] = v;
    P[p] = v;
  }
  if (!grid_barrier(a.st, bar, 70)) return;
  // r_0 = (b - f) - A x_0 = (b - f) + C x_0;  |r_0|^2, |b - f|^2
  {
    double rr = 0.0, bb = 0.0;
    for (long long k = gtid; k < ncomp; k += gth) {
      const long long p = __ldg(S.idx + k);
      double rhs = -a.f[p];
      if (S.bco && S.bval) {
#pragma unroll
        for (int i = 0; i < SL; ++i) {
          const double cf = S.bco[k * SL + i];
          if (cf != 0.0) rhs = fma(cf, S.bval[k * SL + i], rhs);
        }
      }
      const double cx = cstencil<N>(P, p, g, __ldg(S.diag + k), S.beta_field, S.beta_c, cfac);
      const double rk = rhs + cx;
      r[k] = rk;
      rr = fma(rk, rk, rr);
      bb = fma(rhs, rhs, bb);
    }
    double v[2] = {rr, bb};
    double* pb = ps_part(a.part, red);
    block_partials<2>(v, pb);
    if (!grid_barrier(a.st, bar, 71)) return;
    double tot[2];
    grid_totals<2>(pb, tot);
    if (threadIdx.x == 0) {
      s_tot[0] = tot[0];
      s_tot[1] = tot[1];
    }
    __syncthreads();
  }
  double rr = s_tot[0];
  const double bnorm = sqrt(s_tot[1]);
  const double stop = a.tol * (bnorm > 0.0 ? bnorm : 1.0);
  // P = r_0
  for (long long k = gtid; k < ncomp; k += gth) P[__ldg(S.idx + k)] = r[k];
  if (!grid_barrier(a.st, bar, 72)) return;
  int it = 0;
  bool converged = sqrt(rr) <= stop;
  while (!converged && it < a.max_iter) {
    // q = A P, <P, q>
    double pq = 0.0;
    for (long long k = gtid; k < ncomp; k += gth) {
      const long long p = __ldg(S.idx + k);
      const double qk = -cstencil<N>(P, p, g, __ldg(S.diag + k), S.beta_field, S.beta_c, cfac);
      q[k] = qk;
      pq = fma(__ldcg(P + p), qk, pq);
    }
    {
      double v[2] = {pq, 0.0};
      double* pb = ps_part(a.part, red);
      block_partials<2>(v, pb);
      if (!grid_barrier(a.st, bar, 73)) return;
      double tot[2];
      grid_totals<2>(pb, tot);
      pq = tot[0];
    }
    if (!(pq > 0.0) || !isfinite(pq)) {  // A is positive definite: breakdown only on bad data
      if (threadIdx.x == 0) atomicOr(&a.st->err, ERRF_NONFINITE);
      return;
    }
    const double alpha = rr / pq;
    // x += alpha P, r -= alpha q, |r|^2
    double rn = 0.0;
    for (long long k = gtid; k < ncomp; k += gth) {
      const long long p = __ldg(S.idx + k);
      x[k] = fma(alpha, __ldcg(P + p), x[k]);
      const double rk = fma(-alpha, q[k], r[k]);
      r[k] = rk;
      rn = fma(rk, rk, rn);
    }
    {
      double v[2] = {rn, 0.0};
      double* pb = ps_part(a.part, red);
      block_partials<2>(v, pb);
      if (!grid_barrier(a.st, bar, 74)) return;
      double tot[2];
      grid_totals<2>(pb, tot);
      rn = tot[0];
    }
    ++it;
    converged = sqrt(rn) <= stop;
    if (converged || it >= a.max_iter) {
      rr = rn;
      break;
    }
    const double beta = rn / rr;
    rr = rn;
    // P = r + beta P (own entries only; the stencil reads after the barrier)
    for (long long k = gtid; k < ncomp; k += gth) {
      const long long p = __ldg(S.idx + k);
      P[p] = fma(beta, __ldcg(P + p), r[k]);
    }
    if (!grid_barrier(a.st, bar, 75)) return;
  }
  // the solution at the computational points; other nodes keep their values
  for (long long k = gtid; k < ncomp; k += gth) a.u[__ldg(S.idx + k)] = x[k];
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    a.out[0] = (double)it;
    a.out[1] = bnorm > 0.0 ? sqrt(rr) / bnorm : sqrt(rr);
    if (!converged) atomicOr(&a.st->err, ERRF_KRYLOV);
  }
}

cudaError_t launch_poisson(const PoissonArgs& a, cudaStream_t stream) {
  void* fn;
  switch (a.g.ndim) {
    case 2: fn = (void*)poisson_kernel<2>; break;
    case 3: fn = (void*)poisson_kernel<3>; break;
    case 4: fn = (void*)poisson_kernel<4>; break;
    default: return cudaErrorInvalidValue;
  }
  int dev = 0, sms = 0, per = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, PS_NT, 0);
  if (e != cudaSuccess) return e;
  if (per < 1) return cudaErrorLaunchOutOfResources;
  e = cudaMemsetAsync(&a.st->barrier, 0, sizeof(unsigned), stream);
  if (e != cudaSuccess) return e;
  PoissonArgs c = a;
  void* args[] = {(void*)&c};
  return cudaLaunchCooperativeKernel(fn, min(sms, MAX_BLOCKS), PS_NT, args, 0, stream);
}

}  // namespace etd
