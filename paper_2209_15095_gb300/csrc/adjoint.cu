// Adjoint of the ETD2 step on a frozen domain: pointwise combination of the
// phi-function actions, the ETD2 right-hand vectors at a quadrature time, and
// the face contraction that gives the gradient with respect to a node field
// beta.  The phi-function actions themselves come from the Krylov kernel.
//
// With lambda = dL/du_{n+1}, Phi_k = phi_k(dt C) lambda (C symmetric):
//   dL/du_n      = Phi_0 + dt F'(u_n) (Phi_1 + Phi_2) + (contribution of the later step)
//   dL/du_{n-1} += -dt F'(u_{n-1}) Phi_2
//   dL/dalpha   += dt <Phi_1 + Phi_2, dF/dalpha(u_n)> - dt <Phi_2, dF/dalpha(u_{n-1})>
// and, for beta, d(mu^T C y)/d beta_f = -h^-2 (mu_p - mu_q)(y_p - y_q) on a face
// between computational points, -h^-2 (1 - w_f) mu_p y_p on a face to a ghost
// point, half of it to each end node (beta_f is the mean of the two nodes).
#include "common.cuh"
#include "kernels.cuh"

namespace etd {

constexpr int ADJ_NT = 256;
constexpr int ADJ_BLOCKS = 608;

// F, F' and dF/dalpha of the single-species reactions
__device__ __forceinline__ void reaction_terms(int kind, const double* rp, double u, double& F, double& dF,
                                               double& dFa) {
  switch (kind) {
    case 1:
      F = u * (1.0 - u);
      dF = 1.0 - 2.0 * u;
      dFa = 0.0;
      break;
    case 2:
      F = rp[0] * u * (1.0 - u / rp[1]);
      dF = rp[0] * (1.0 - 2.0 * u / rp[1]);
      dFa = u * (1.0 - u / rp[1]);
      break;
    default:
      F = 0.0;
      dF = 0.0;
      dFa = 0.0;
  }
}

__global__ void __launch_bounds__(ADJ_NT) adjoint_combine_kernel(const AdjointArgs a) {
  double part = 0.0;
  const long long G = a.g.size;
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < G; p += (long long)gridDim.x * blockDim.x) {
    if ((a.kind[p] & 3) != K_COMP) {
      a.lam[p] = 0.0;
      a.acc[p] = 0.0;
      continue;
    }
    double F, dFn, dFan, dFm, dFam;
    reaction_terms(a.reaction, a.rp, a.un[p], F, dFn, dFan);
    reaction_terms(a.reaction, a.rp, a.unm1[p], F, dFm, dFam);
    const double p0 = a.P0[p], p1 = a.P1[p], p2 = a.P2[p];
    double lam = p0 + a.dt * dFn * (p1 + p2) + a.acc[p];
    double acc = -a.dt * dFm * p2;
    if (a.first) {  // u_{-1} is u_0
      lam += acc;
      acc = 0.0;
    }
    part += a.dt * (p1 + p2) * dFan - a.dt * p2 * dFam;
    a.lam[p] = lam;
    a.acc[p] = acc;
  }
  double v[1] = {part};
  block_partials<1>(v, a.part);
}

// Sums the per-block partials in block order and adds them to grad_params[0].
__global__ void adjoint_alpha_finish_kernel(const double* part, int nblocks, double* grad_params) {
  if (threadIdx.x != 0) return;
  double s = 0.0;
  for (int b = 0; b < nblocks; ++b) s += part[b];
  grad_params[0] += s;
}

cudaError_t launch_adjoint_combine(const AdjointArgs& a, cudaStream_t stream) {
  adjoint_combine_kernel<<<ADJ_BLOCKS, ADJ_NT, 0, stream>>>(a);
  adjoint_alpha_finish_kernel<<<1, 32, 0, stream>>>(a.part, ADJ_BLOCKS, a.grad_params);
  return cudaGetLastError();
}

__global__ void __launch_bounds__(ADJ_NT) adjoint_rhs_kernel(const AdjointArgs a, double s1, double s2, double* v1,
                                                            double* v2) {
  const int ncomp = *a.ncomp;
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < ncomp;
       k += (long long)gridDim.x * blockDim.x) {
    const long long p = a.idx[k];
    double F, Fm, d1, d2;
    reaction_terms(a.reaction, a.rp, a.un[p], F, d1, d2);
    reaction_terms(a.reaction, a.rp, a.unm1[p], Fm, d1, d2);
    v1[p] = s1 * (a.dt * F);
    v2[p] = s2 * (a.dt * (F - Fm));
  }
}

cudaError_t launch_adjoint_rhs(const AdjointArgs& a, double s1, double s2, double* v1, double* v2,
                               cudaStream_t stream) {
  adjoint_rhs_kernel<<<ADJ_BLOCKS, ADJ_NT, 0, stream>>>(a, s1, s2, v1, v2);
  return cudaGetLastError();
}

template <int N>
__global__ void __launch_bounds__(ADJ_NT) beta_contract_kernel(const AdjointArgs a, const double* __restrict__ mu,
                                                              const double* __restrict__ y, double coef,
                                                              double* grad_beta) {
  const int ncomp = *a.ncomp;
  const double inv_h2 = 1.0 / (a.g.h * a.g.h);
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < ncomp;
       k += (long long)gridDim.x * blockDim.x) {
    const long long p = a.idx[k];
    const double mp = mu[p], yp = y[p];
    double own = 0.0;
#pragma unroll
    for (int d = 0; d < N; ++d) {
#pragma unroll
      for (int si = 0; si < 2; ++si) {
        const long long q = p + (si == 0 ? -a.g.stride[d] : a.g.stride[d]);
        if ((a.kind[q] & 3) == K_COMP) {
          own += 0.5 * (-(mp - mu[q]) * (yp - y[q]) * inv_h2);
        } else {
          const double gw = a.facew[k * (2 * N) + 2 * d + si];
          const double df = -gw * mp * yp * inv_h2;
          own += 0.5 * df;
          atomicAdd(grad_beta + q, coef * (0.5 * df));
        }
      }
    }
    grad_beta[p] += coef * own;
  }
}

// All quadrature times in one pass: per face the weighted sum over i of
// the face derivative, then one update per node (and one atomic per ghost
// face).
template <int N>
__global__ void __launch_bounds__(ADJ_NT) beta_contract_multi_kernel(const AdjointArgs a, double* grad_beta) {
  const int ncomp = *a.ncomp;
  const double inv_h2 = 1.0 / (a.g.h * a.g.h);
  const int nq = a.nq;
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < ncomp;
       k += (long long)gridDim.x * blockDim.x) {
    const long long p = a.idx[k];
    double own = 0.0;
#pragma unroll
    for (int d = 0; d < N; ++d) {
#pragma unroll
      for (int si = 0; si < 2; ++si) {
        const long long q = p + (si == 0 ? -a.g.stride[d] : a.g.stride[d]);
        double f = 0.0;
        if ((a.kind[q] & 3) == K_COMP) {
          for (int i = 0; i < nq; ++i) {
            const double* mu = a.muq[i];
            const double* y = a.yq[i];
            f = fma(a.wq[i], -(mu[p] - mu[q]) * (y[p] - y[q]), f);
          }
          own += 0.5 * (f * inv_h2);
        } else {
          const double gw = a.facew[k * (2 * N) + 2 * d + si];
          for (int i = 0; i < nq; ++i) f = fma(a.wq[i], -gw * a.muq[i][p] * a.yq[i][p], f);
          const double df = 0.5 * (f * inv_h2);
          own += df;
          atomicAdd(grad_beta + q, df);
        }
      }
    }
    grad_beta[p] += own;
  }
}

cudaError_t launch_beta_contract_multi(const AdjointArgs& a, double* grad_beta, cudaStream_t stream) {
  switch (a.g.ndim) {
    case 2: beta_contract_multi_kernel<2><<<ADJ_BLOCKS, ADJ_NT, 0, stream>>>(a, grad_beta); break;
    case 3: beta_contract_multi_kernel<3><<<ADJ_BLOCKS, ADJ_NT, 0, stream>>>(a, grad_beta); break;
    case 4: beta_contract_multi_kernel<4><<<ADJ_BLOCKS, ADJ_NT, 0, stream>>>(a, grad_beta); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_beta_contract(const AdjointArgs& a, const double* mu, const double* y, double coef,
                                 double* grad_beta, cudaStream_t stream) {
  switch (a.g.ndim) {
    case 2: beta_contract_kernel<2><<<ADJ_BLOCKS, ADJ_NT, 0, stream>>>(a, mu, y, coef, grad_beta); break;
    case 3: beta_contract_kernel<3><<<ADJ_BLOCKS, ADJ_NT, 0, stream>>>(a, mu, y, coef, grad_beta); break;
    case 4: beta_contract_kernel<4><<<ADJ_BLOCKS, ADJ_NT, 0, stream>>>(a, mu, y, coef, grad_beta); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace etd
