// Adaptive Krylov evaluation of y = phi_0(A) v_0 + phi_1(A) v_1 + ... + phi_p(A) v_p,
// p = 2 or 3 (Sec. 3.3, Eq. 3.9), by time-stepping the equivalent ODE of
// Eq. 3.10 (y' = A y + v_1 + t v_2 + t^2/2 v_3, y(0) = v_0, y = y(1)), A = dt C
// with C the matrix-free embedded-boundary operator of Sec. 2, and the ETD
// steps of Sec. 3.1-3.2 built on it.
//
// One persistent cooperative kernel runs the whole call: the ETD2 right-hand
// vectors, every substep (w_1, w_2 matvecs, the IOM2/Lanczos basis with fused
// dot products, the small augmented-matrix exponential, the error estimate
// and the step-size controller) and the final combination, with bounded grid
// barriers between dependent sweeps.  Every CTA sums the per-CTA partials in
// the same order and runs the same controller on the same bits, so all
// decisions are identical across CTAs without a broadcast.
//
// Substep from t_k with step tau (p = 2):
//   w_1 = A y + v_1 + t_k v_2,  w_2 = A w_1 + v_2,  beta = |w_2|
//   IOM2: z = A v_j, h_jj = <z, v_j>, h_{j-1,j} = <z, v_{j-1}>,
//         z -= h_jj v_j + h_{j-1,j} v_{j-1}, h_{j+1,j} = |z|
//   check every 5 vectors and at m_max:
//     err = tau^3 beta h_{m+1,m} |e_m^T phi_3(tau H_m) e_1| <= tol tau s,
//     s = max(|y(t_k)|, |v_1|, |v_2|)
//   on failure at m_max shrink tau <- tau max(0.2, 0.9 (tol tau |y| / err)^(1/(m+1)))
//   y <- y + tau w_1 + tau^2 beta V_m phi_2(tau H_m) e_1
//   tau_next = min(1 - t, tau min(2, 0.9 (tol tau |y| / err)^(1/(m+1))))
// p = 3: w_1 = A y + v_1 + t_k v_2 + t_k^2/2 v_3, w_2 = A w_1 + v_2 + t_k v_3,
// w_3 = A w_2 + v_3, beta = |w_3|, err = tau^4 beta h_{m+1,m} |e_m^T phi_4(tau H_m) e_1|,
//   y <- y + tau w_1 + tau^2/2 w_2 + tau^3 beta V_m phi_3(tau H_m) e_1.
// Basis vectors are stored unnormalised (v_j = V_j / |V_j|) so that the
// normalisation costs no extra sweep; on the 4-node groups of large FP32
// problems the basis is built by the one-pass form of the symmetric Lanczos
// recurrence (quad_pass_1).
//
// This header holds the kernel; krylov_f64.cu, krylov_f32.cu and
// krylov_f32w.cu instantiate it (FP64 with 512 threads per CTA; FP32 with
// 512, and with 768 for problems on the 4-node groups) and krylov.cu
// launches it.  A unit may define ETD_RED_MAX_NT (the block-reduction width)
// before including it.
#pragma once
#include "common.cuh"
#include "kernels.cuh"

namespace etd {

constexpr int CHECK_EVERY = 5;
constexpr double TAU_MIN = 1e-6;
constexpr double BREAKDOWN_REL = 1e-12;
constexpr float TAYLOR_THETA = 8.0f;
constexpr int MAX_SUBSTEPS = 20000;  // bounded work per call
// From SPLIT_MIN computational points on, a Krylov vector costs two passes
// (V_j = w_j at the own points; after a barrier Z_j = A V_j and the sums)
// instead of one pass that rebuilds w_j at all 2N + 1 stencil points: about
// 15 instead of 30 FP64 instructions per point, which is what bounds FP64 at
// those sizes, for one more barrier and 2 more vector accesses per point.
// Each thread then keeps SPLIT_U points in flight.  FP32 problems of that
// size on the 4-node groups take one pass per vector instead (quad_pass_1).
template <typename T>
constexpr int SPLIT_MIN = sizeof(T) == 8 ? (1 << 17) : QUAD_MIN_POINTS;
template <typename T>
constexpr int SPLIT_U = sizeof(T) == 8 ? 2 : 4;
template <typename T>
constexpr int SPLIT_UB = sizeof(T) == 8 ? 2 : 3;  // the stencil pass (register bound)

// 1/k!: each translation unit that instantiates the kernel has its own copy
// (filled by load_inv_fact before its first launch)
static __constant__ double c_inv_fact[64];

static cudaError_t load_inv_fact() {
  double f[64];
  f[0] = 1.0;
  for (int k = 1; k < 64; ++k) f[k] = f[k - 1] / (double)k;
  return cudaMemcpyToSymbol(c_inv_fact, f, sizeof(f));
}

struct Ctl {
  double alpha[MAX_M + 2];
  double up[MAX_M + 2];
  double low[MAX_M + 2];
  double scale[MAX_M + 2];  // 1 / |V_j|
  double coef[MAX_M + 2];   // tau^p beta phi_p(tau H) e_1, times scale
  float chi[MAX_M + 2];     // coef as a sum of two floats (FP32 basis sum)
  float clo[MAX_M + 2];
  double yexp[64];
  // controller scalars
  double t, tau, ynorm, beta, err, hn;
  int m, accepted, breakdown, last, abort, nrej;
  int trace0;  // trace entries of earlier launches of the step (block 0)
  int nquad, qoff;  // quad list: length, and this block's first entry
  int qcached;      // the list of the current domain is already built
  int nq_sp[2];     // per species: list length (0: no quad path)
  int wb_done[2];   // per species: the last combination wrote u (no write-back)
};

// ---------------------------------------------------------------------------
// small exponential: x = exp(K) e_{M-1} for the augmented matrix
//   K = [[tau H_m, e_1, 0], [0, 0, I_p], [0, 0, 0]],  M = m + p + 1 <= 64,
// by Taylor series with a shift and scaling, exp(K) = e^mu exp((K - mu I)/s)^s,
// unnormalised powers accumulated with 1/k!.  Warp-cooperative: lane owns
// rows lane and lane+32.
// On return c.yexp[0..m-1] = phi_{p+1}(tau H_m) e_1.
// s steps of the degree-deg Taylor polynomial of the tridiagonal-plus-
// coupling matrix held as (A, B, C) per row (lane r: rows r and r + 32).
// TWO is a template argument so that the second half's FP64 work is absent,
// not predicated off, when M <= 32: a predicated-off FP64 instruction still
// takes its issue slot.
template <bool TWO>
__device__ __forceinline__ void taylor_steps(int m, int s, int deg, const double (&A)[2], const double (&B)[2],
                                             const double (&C)[2], double (&x)[2]) {
  const int lane = threadIdx.x & 31;
  for (int it = 0; it < s; ++it) {
    double P0 = x[0], P1 = x[1], acc0 = x[0], acc1 = x[1];
    for (int k = 1; k <= deg; ++k) {
      double dn0 = __shfl_up_sync(0xffffffffu, P0, 1);
      double up0 = __shfl_down_sync(0xffffffffu, P0, 1);
      const double pm = __shfl_sync(0xffffffffu, (!TWO || m < 32) ? P0 : P1, m & 31);
      if (lane == 0) dn0 = pm;
      if (TWO) {
        double dn1 = __shfl_up_sync(0xffffffffu, P1, 1);
        double up1 = __shfl_down_sync(0xffffffffu, P1, 1);
        const double b31 = __shfl_sync(0xffffffffu, P0, 31);
        const double b32 = __shfl_sync(0xffffffffu, P1, 0);
        if (lane == 0) dn1 = b31;
        if (lane == 31) {
          up0 = b32;
          up1 = 0.0;
        }
        P1 = fma(C[1], up1, fma(B[1], dn1, A[1] * P1));
        acc1 = fma(c_inv_fact[k], P1, acc1);
      } else {
        if (lane == 31) up0 = 0.0;
      }
      P0 = fma(C[0], up0, fma(B[0], dn0, A[0] * P0));
      acc0 = fma(c_inv_fact[k], P0, acc0);
    }
    x[0] = acc0;
    x[1] = acc1;
  }
}

static __device__ void small_expm_warp(const Ctl& c, int m, int p, double tau, double* yexp) {
  const int lane = threadIdx.x & 31;
  const int M = m + p + 1;
  // Gershgorin interval [L, U] of the augmented matrix (rows m.. have centre
  // 0 and radius at most 1); FP32 suffices, it only picks the shift and the
  // scaling.  exp(K) = e^mu exp(K - mu I) for any mu: mu is the interval's
  // midpoint (floored at -300 so that neither factor overflows), which
  // about halves the norm bound that sets the number of Taylor terms.
  const float ft = (float)tau;
  float L = -1.f, U = 1.f;
  for (int r = lane; r < m; r += 32) {
    const float cr = ft * (float)c.alpha[r];
    const float rr = ft * ((r > 0 ? fabsf((float)c.low[r - 1]) : 0.f) + (r + 1 < m ? fabsf((float)c.up[r + 1]) : 0.f)) +
                     (r == 0 ? 1.f : 0.f);
    L = fminf(L, cr - rr);
    U = fmaxf(U, cr + rr);
  }
  for (int o = 16; o > 0; o >>= 1) {
    L = fminf(L, __shfl_xor_sync(0xffffffffu, L, o));
    U = fmaxf(U, __shfl_xor_sync(0xffffffffu, U, o));
  }
  const float mu = fmaxf(0.5f * (L + U), -300.f);
  const float nb = fmaxf(U - mu, mu - L);
  const int s = max(1, (int)ceilf(nb / TAYLOR_THETA));
  const float th = nb / (float)s;
  int deg = 1;
  {
    float term = th;
    while (deg < 60 && term > 1e-18f) {
      ++deg;
      term *= __fdividef(th, (float)deg);
    }
  }
  const double inv_s = 1.0 / (double)s;
  const double dmu = (double)mu;
  double A[2], B[2], C[2], x[2];
  for (int h = 0; h < 2; ++h) {
    const int r = lane + 32 * h;
    if (r < m) {
      A[h] = (tau * c.alpha[r] - dmu) * inv_s;
      B[h] = r > 0 ? tau * c.low[r - 1] * inv_s : 0.0;
      C[h] = r + 1 < m ? tau * c.up[r + 1] * inv_s : 0.0;
    } else if (r < M) {
      A[h] = -dmu * inv_s;
      B[h] = 0.0;
      C[h] = r < M - 1 ? inv_s : 0.0;
    } else {
      A[h] = B[h] = C[h] = 0.0;
    }
    x[h] = (r == M - 1) ? 1.0 : 0.0;
  }
  // row 0 has no lower neighbour: that slot carries its coupling to x_m
  if (lane == 0) B[0] = inv_s;
  if (M > 32) taylor_steps<true>(m, s, deg, A, B, C, x);
  else taylor_steps<false>(m, s, deg, A, B, C, x);
  const double emu = exp(dmu);
  if (lane < m) yexp[lane] = x[0] * emu;
  if (lane + 32 < m) yexp[lane + 32] = x[1] * emu;
  __syncwarp();
}

// Combination coefficients from yexp = phi_{p+1}(tau H_m) e_1 (one warp):
// out_r = tau^p beta (phi_p(tau H_m) e_1)_r / |V_r|, with phi_p(X) e_1 =
// X phi_{p+1}(X) e_1 + e_1 / p!  (p = 0 .. 3).
static __device__ void coef_row(const Ctl& c, int m, int p, double tau, const double* yexp, double* out) {
  const int lane = threadIdx.x & 31;
  double taup = 1.0, invf = 1.0;
  for (int i = 1; i <= p; ++i) {
    taup *= tau;
    invf /= (double)i;
  }
  for (int r = lane; r < m; r += 32) {
    double hy = c.alpha[r] * yexp[r];
    if (r > 0) hy = fma(c.low[r - 1], yexp[r - 1], hy);
    if (r + 1 < m) hy = fma(c.up[r + 1], yexp[r + 1], hy);
    const double php = fma(tau, hy, r == 0 ? invf : 0.0);
    out[r] = taup * c.beta * php * c.scale[r];
  }
  __syncwarp();
}

// After small_expm_warp: err and the combination coefficients (warp 0):
// err = tau^{p+1} beta h_{m+1,m} |e_m^T phi_{p+1}(tau H_m) e_1|.
static __device__ void finish_check(Ctl& c, int m, int p, double tau) {
  coef_row(c, m, p, tau, c.yexp, c.coef);
  if ((threadIdx.x & 31) == 0) {
    double taup = 1.0;
    for (int i = 1; i <= p; ++i) taup *= tau;
    c.err = taup * tau * c.beta * c.hn * fabs(c.yexp[m - 1]);
  }
  __syncwarp();
}

// ---------------------------------------------------------------------------
// (A x)_p with A = cfac (beta S - D) (SCALED), or (B x)_p = (A x)_p / cfac.
template <typename T, int N, bool SCALED = true>
__device__ __forceinline__ T stencil(const T* __restrict__ x, long long p, const GridDev& g, T Dk,
                                     const double* __restrict__ bfield, T bc, T cfac) {
  const T xp = __ldcg(x + p);
  // the sums start from -0: x + (-0) == x exactly, so the first add is free
  if (bfield == nullptr) {
    T s = T(-0.0);
#pragma unroll
    for (int d = 0; d < N; ++d) s += __ldcg(x + p - g.stride[d]) + __ldcg(x + p + g.stride[d]);
    return SCALED ? cfac * (bc * s - Dk * xp) : bc * s - Dk * xp;
  }
  const double bp = __ldg(bfield + p);
  T s = T(-0.0);
#pragma unroll
  for (int d = 0; d < N; ++d) {
    const long long st = g.stride[d];
    s += T(0.5 * (bp + __ldg(bfield + p - st))) * __ldcg(x + p - st);
    s += T(0.5 * (bp + __ldg(bfield + p + st))) * __ldcg(x + p + st);
  }
  return SCALED ? cfac * (s - Dk * xp) : s - Dk * xp;
}

__device__ __forceinline__ double reaction(int kind, const double* rp, int species, double u, double v) {
  switch (kind) {
    case 1: return u * (1.0 - u);
    case 2: return rp[0] * u * (1.0 - u / rp[1]);
    case 3:
      if (species == 0) return u * (1.0 - u - rp[0] * v);
      return rp[2] * v * (1.0 - v - rp[1] * u);
    default: return 0.0;
  }
}

// The caller's source and boundary-data terms of F at computational point k
// (grid node p): src[p] plus, over the point's contiguous face slots, the
// boundary coefficient times the boundary value (empty slots have
// coefficient 0 and are skipped, their values being NaN).
template <typename T, int N>
__device__ __forceinline__ double extra_F(const SpeciesDev<T>& S, long long k, long long p) {
  double e = 0.0;
  if (S.src) e += S.src[p];
  if (S.bco && S.bval) {
    constexpr int SL = 2 * N * (N == 2 ? 2 : 1);
    const long long b = k * SL;
#pragma unroll
    for (int i = 0; i < SL; ++i) {
      const double cf = S.bco[b + i];
      if (cf != 0.0) e = fma(cf, S.bval[b + i], e);
    }
  }
  return e;
}

template <typename T>
__device__ __forceinline__ T diag_of(const SpeciesDev<T>& S, int k);
template <>
__device__ __forceinline__ double diag_of<double>(const SpeciesDev<double>& S, int k) { return __ldg(S.diag + k); }
template <>
__device__ __forceinline__ float diag_of<float>(const SpeciesDev<float>& S, int k) { return __ldg(S.diagf + k); }

// Exact widening to FP64.  For a float, normal values are widened on the
// integer pipe (rebias the exponent, shift the mantissa): the hardware
// conversion is an FP64-pipe instruction, which costs as much as an FMA.
// Zero, subnormal, infinite and NaN values take the hardware conversion.
__device__ __forceinline__ double to_f64(double x) { return x; }
__device__ __forceinline__ double to_f64(float x) {
  const unsigned f = __float_as_uint(x);
  const unsigned e = (f >> 23) & 0xffu;
  if (e - 1u < 254u) {
    const unsigned hi = (f & 0x80000000u) | ((e + 896u) << 20) | ((f & 0x7fffffu) >> 3);
    const unsigned lo = (f & 7u) << 29;
    return __hiloint2double((int)hi, (int)lo);
  }
  return (double)x;
}

// Rounding of an FP64 value to FP32, to nearest with ties to even (IEEE
// 754), on the integer pipe where the result is a normal float: the FP32
// exponent is the FP64 one rebiased (1023 -> 127), the 23 mantissa bits are
// the top of the 52, and the 29 bits dropped decide the rounding (above
// half: up; exactly half: up when the kept mantissa is odd).  A carry out
// of the mantissa increments the exponent, and one out of the largest
// exponent gives the infinity bit pattern, as the rounding rule does.
// Results that would be subnormal, zero, infinite or NaN take the hardware
// conversion (an FP64-pipe instruction, as costly as an FMA on this GPU).
__device__ __forceinline__ float to_f32_rn(double x) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const unsigned ex = (hi >> 20) & 0x7ffu;
  if (ex - 897u < 254u) {
    const unsigned m = ((hi & 0xfffffu) << 3) | (lo >> 29);
    const unsigned r = lo & 0x1fffffffu;
    const unsigned up = (r > 0x10000000u || (r == 0x10000000u && (m & 1u))) ? 1u : 0u;
    return __uint_as_float((hi & 0x80000000u) | (((ex - 896u) << 23) + m + up));
  }
  return (float)x;
}
template <typename T>
__device__ __forceinline__ T to_T(double x);
template <>
__device__ __forceinline__ double to_T<double>(double x) { return x; }
template <>
__device__ __forceinline__ float to_T<float>(double x) { return to_f32_rn(x); }

// w = ca Z + cb V1 + cc V2 at grid node q (zero off the computational set,
// since all three arrays are).
template <typename T>
__device__ __forceinline__ T wval(const T* __restrict__ Z, const T* __restrict__ V1, const T* __restrict__ V2,
                                  long long q, T ca, T cb, T cc) {
  return ca * __ldcg(Z + q) + cb * __ldcg(V1 + q) + cc * __ldcg(V2 + q);
}

// Node loop over the computational points with U points per thread and
// iteration: the indices of the U points are loaded first, then body(kk, pp)
// issues all of its loads before its stores, so that a thread waits on memory
// about twice per U points instead of twice per point.  U = 1 is the plain
// loop.  pp[u] < 0 marks a slot past the end.
template <int U, typename Body>
__device__ __forceinline__ void node_loop(long long gtid, long long gth, int ncomp, const int* __restrict__ idx,
                                          Body&& body) {
  // the indices of the next iteration are loaded before this one's body, so
  // that their latency overlaps its data loads
  int nx[U];
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const long long k = gtid + u * gth;
    nx[u] = k < ncomp ? __ldg(idx + k) : -1;
  }
  for (long long k0 = gtid; k0 < ncomp; k0 += U * gth) {
    long long kk[U], pp[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      kk[u] = k0 + u * gth;
      pp[u] = nx[u];
      const long long kn = kk[u] + U * gth;
      nx[u] = kn < ncomp ? __ldg(idx + kn) : -1;
    }
    body(kk, pp);
  }
}

// FP32 vectors: two points in flight per thread for problems of at least
// SPLIT_MIN points, one below (where the loop is latency-bound on barriers
// anyway).  FP64: one point (FP64 issue bounds these loops at those sizes,
// and two points would spill registers).
template <typename T, typename Body>
__device__ __forceinline__ void node_loop_sized(long long gtid, long long gth, int ncomp, const int* __restrict__ idx,
                                                Body&& body) {
  if (sizeof(T) == 4 && ncomp >= SPLIT_MIN<T>) node_loop<2>(gtid, gth, ncomp, idx, body);
  else node_loop<1>(gtid, gth, ncomp, idx, body);
}

#define NL_U(kk) ((int)(sizeof(kk) / sizeof((kk)[0])))

// Runs phipm for one species; returns false if the kernel must stop.
// Two partial-sum buffers used alternately: between two reductions that use
// the same buffer every CTA has passed a barrier after reading it.
__device__ __forceinline__ double* part_buf(double* part, int& red) {
  double* b = part + (red & 1) * (4 * MAX_BLOCKS);
  ++red;
  return b;
}

// sum_i coef_i V_i[p] for an FP32 basis with error-free FP32 transformations
// (Ogita, Rump & Oishi 2005, Dot2): coef_i = chi_i + clo_i as two floats,
// chi_i V_i exactly as a product and its FMA-computed error, the running sum
// by TwoSum, all error terms (and clo_i V_i) in a second float.  About 2^-46
// relative to sum |coef_i V_i|, at FP32 rate instead of one FP64 FMA per
// basis vector.
__device__ __forceinline__ void dot2_step(float& s, float& e, float chi, float clo, float a) {
  const float pr = __fmul_rn(chi, a);
  const float pe = __fmaf_rn(chi, a, -pr);
  const float t = __fadd_rn(s, pr);
  const float z = __fsub_rn(t, s);
  const float te = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(pr, z));
  s = t;
  e = __fadd_rn(e, __fadd_rn(te, __fmaf_rn(clo, a, pe)));
}

__device__ __forceinline__ double basis_sum_f32(const Ctl& c, const float* __restrict__ V, long long vs, long long p,
                                                int m) {
  float s = 0.f, e = 0.f;
#pragma unroll 4
  for (int i = 0; i < m; ++i) dot2_step(s, e, c.chi[i], c.clo[i], __ldcg(V + (long long)i * vs + p));
  return to_f64(s) + to_f64(e);
}

// ---------------------------------------------------------------------------
// Quad path of the large FP32 problems (constant beta, last axis a
// multiple of 4 nodes).  The passes run over the aligned groups of 4 nodes
// that hold computational points, with 16-byte loads and stores of the grid
// vectors and no per-point index: every grid vector is zero off the
// computational set (the set-up zeroes them, the passes keep them so), so
// the other lanes of a group compute zeros.  More bytes in flight per
// thread than the per-point loop, whose dependent index-then-data loads
// keep the passes latency-bound.
__device__ __forceinline__ float4 ld4(const float* p) { return __ldcg(reinterpret_cast<const float4*>(p)); }
__device__ __forceinline__ void st4(float* p, float4 v) { __stcg(reinterpret_cast<float4*>(p), v); }

struct QuadSums {
  double d1, d2, d3;
};

// A thread's sum over the groups it visits of a group's four FP32 products:
// the products of a group are summed in FP32 (an FMA chain, about 2^-23 of
// that group sum, in no fixed direction), and the group sums are
// accumulated without error into s + c by TwoSum (Knuth), so the rounding
// does not grow with the number of groups.  A quarter of the FP32
// instructions of a Dot2 sum of every product.
struct AccG {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add4(const float (&a)[4], const float (&b)[4]) {
    const float p = __fmaf_rn(a[3], b[3], __fmaf_rn(a[2], b[2], __fmaf_rn(a[1], b[1], __fmul_rn(a[0], b[0]))));
    const float t = __fadd_rn(s, p), z = __fsub_rn(t, s);
    c = __fadd_rn(c, __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(p, z)));
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

// groups per thread and iteration in quad_pass_1 (two measured slower at
// 512^3: 322 against 262 us per pass; the registers, not the index loads,
// bound the loads in flight)
constexpr int QP_U = 1;

__device__ __forceinline__ void prefetch_l2(const void* p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }

// Top bit of a group's list entry qk: its 4 nodes are computational and
// have the diagonal of a row whose 2N faces all reach computational
// points, D = 2N beta (the domain set-up stores exactly that value there,
// and a ghost face of weight 0 gives it too), so the passes take D and the
// class word without loading them.
constexpr int QK_FULL = (int)0x80000000u;
constexpr int QK_INDEX = 0x7fffffff;
// the class word of a full group (4 computational nodes), not loaded
constexpr unsigned QK_FULL_KIND = 0x02020202u;
static_assert(K_COMP == 2, "QK_FULL_KIND holds K_COMP in every byte");
template <typename T, int N>
__device__ __forceinline__ float quad_d_int(const SpeciesDev<T>& S) {
  return (float)((double)(2 * N) * S.beta_c);
}
// Loop over this thread's entries q = gtid, gtid + gth, ... of the group
// list.  The entries (the group's index and its first list index) are
// loaded two iterations ahead, so that an iteration's data loads never wait
// on its index loads: body(p4, k0, full, pn4) gets the group's first node,
// its first list index, whether it is a full interior group (QK_FULL), and
// the first node of the thread's next group (-1 if none), whose lines the
// body prefetches into L2.  With one 512-thread CTA
// per SM the passes are bound by the bytes in flight: the prefetches add to
// them without registers.
template <typename Body>
__device__ __forceinline__ void quad_loop(const int* __restrict__ qidx, const int* __restrict__ qk, int nq,
                                          long long gtid, long long gth, Body&& body) {
  long long q = gtid;
  int pa = q < nq ? __ldg(qidx + q) : -1, ka = q < nq ? __ldg(qk + q) : 0;
  int pb = q + gth < nq ? __ldg(qidx + q + gth) : -1, kb = q + gth < nq ? __ldg(qk + q + gth) : 0;
  for (; q < nq; q += gth) {
    const long long q2 = q + 2 * gth;
    const int pc = q2 < nq ? __ldg(qidx + q2) : -1, kc = q2 < nq ? __ldg(qk + q2) : 0;
    body((long long)pa << 2, ka & QK_INDEX, ka < 0, pb >= 0 ? (long long)pb << 2 : -1ll);
    pa = pb;
    ka = kb;
    pb = pc;
    kb = kc;
  }
}

// One pass per Krylov vector on groups of 4 nodes, in the form of the
// symmetric Lanczos recurrence that Paige recommends (u_j = A v_j -
// beta_j v_{j-1}, alpha_j = <u_j, v_j>, beta_{j+1} = |u_j - alpha_j v_j|):
//   V_j = c1 Wp + c2 Vp   at the group and its 2N stencil neighbours
//         (Wp = u_{j-1} and Vp = v_{j-1}, up to their scale factors),
//   Z_j = A V_j at the computational points (0 at the group's other nodes),
//   W_j = Z_j + c3 Vp     (u_j),
// stores V_j and W_j, and sums |V_j|^2, <W_j, V_j>, |W_j|^2 (this thread's
// AccG sums), from which alpha_j and beta_{j+1} follow without another
// pass.  Two vectors are read (each with its stencil) and two written.  A
// V_j value is formed by the same two roundings wherever it is formed, so
// Z_j is A applied to the stored V_j.  Inlined into the kernel: out of line
// its 20-odd register arguments and the saves around the call cost the
// 768-thread kernel 8% per pass at 512^3 (4.93 against 5.34 ms for 19 passes).
template <int N>
__device__ __forceinline__ QuadSums quad_pass_1(const float* __restrict__ Wp, const float* __restrict__ Vp,
                                                float* __restrict__ Vj, float* __restrict__ Wn, float c1, float c2,
                                                float c3, const uint8_t* __restrict__ kind,
                                                const float* __restrict__ diagf, const int* __restrict__ qidx,
                                                const int* __restrict__ qk, int nq, const GridDev& g, float cfac,
                                                float bc, float dint, long long gtid, long long gth) {
  constexpr int U = QP_U;
  long long st[N > 1 ? N - 1 : 1];
#pragma unroll
  for (int d = 0; d < N - 1; ++d) st[d] = g.stride[d];
  AccG d1, d2, d3;
  const auto vnew = [c1, c2](float w, float v) { return __fmaf_rn(c2, v, __fmul_rn(c1, w)); };
  // this iteration's groups q + u gth, the next iteration's, and (loaded
  // here) the one after: an iteration's data loads never wait on its index
  // loads, and the next iteration's lines are prefetched into L2
  int pc[U], kc[U], pn[U], kn[U];
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const long long q0 = gtid + u * gth, q1 = gtid + (U + u) * gth;
    pc[u] = q0 < nq ? __ldg(qidx + q0) : -1;
    kc[u] = q0 < nq ? __ldg(qk + q0) : 0;
    pn[u] = q1 < nq ? __ldg(qidx + q1) : -1;
    kn[u] = q1 < nq ? __ldg(qk + q1) : 0;
  }
  for (long long q = gtid; q < nq; q += U * gth) {
    int pf[U], kf[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const long long q2 = q + (2 * U + u) * gth;
      pf[u] = q2 < nq ? __ldg(qidx + q2) : -1;
      kf[u] = q2 < nq ? __ldg(qk + q2) : 0;
      if (pn[u] >= 0 && (pn[u] & 7) == 0) {
        // the next groups' own lines and those of their upper neighbours
        // along the first axis (the only ones no earlier group brought in),
        // by the lane whose group starts a 128-byte line of the FP32 vectors
        const long long pn4 = (long long)pn[u] << 2;
        prefetch_l2(Wp + pn4);
        prefetch_l2(Vp + pn4);
        prefetch_l2(Wp + pn4 + st[0]);
        prefetch_l2(Vp + pn4 + st[0]);
      }
    }
    float4 wc[U], vc[U], sacc[U], dg[U];
    float wl[U], wr[U], vl[U], vr[U];
    unsigned kw[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (pc[u] < 0) continue;
      const long long p4 = (long long)pc[u] << 2;
      const int k0 = kc[u] & QK_INDEX;
      wc[u] = ld4(Wp + p4);
      vc[u] = ld4(Vp + p4);
      wl[u] = __ldcg(Wp + p4 - 1);
      wr[u] = __ldcg(Wp + p4 + 4);
      vl[u] = __ldcg(Vp + p4 - 1);
      vr[u] = __ldcg(Vp + p4 + 4);
      float4 sa = make_float4(-0.f, -0.f, -0.f, -0.f);  // as stencil()
#pragma unroll
      for (int d = 0; d < N - 1; ++d) {
        const float4 wm = ld4(Wp + p4 - st[d]), wq = ld4(Wp + p4 + st[d]);
        const float4 vm = ld4(Vp + p4 - st[d]), vq = ld4(Vp + p4 + st[d]);
        sa.x += vnew(wm.x, vm.x) + vnew(wq.x, vq.x);
        sa.y += vnew(wm.y, vm.y) + vnew(wq.y, vq.y);
        sa.z += vnew(wm.z, vm.z) + vnew(wq.z, vq.z);
        sa.w += vnew(wm.w, vm.w) + vnew(wq.w, vq.w);
      }
      sacc[u] = sa;
      kw[u] = kc[u] < 0 ? QK_FULL_KIND : __ldg(reinterpret_cast<const unsigned*>(kind + p4));
      dg[u] = kc[u] < 0 ? make_float4(dint, dint, dint, dint)
                        : make_float4(__ldg(diagf + k0), __ldg(diagf + k0 + 1), __ldg(diagf + k0 + 2),
                                      __ldg(diagf + k0 + 3));
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (pc[u] < 0) continue;
      const long long p4 = (long long)pc[u] << 2;
      // V_j along the last axis: the group's left neighbour, its 4 nodes, its right neighbour
      const float x[6] = {vnew(wl[u], vl[u]), vnew(wc[u].x, vc[u].x), vnew(wc[u].y, vc[u].y),
                          vnew(wc[u].z, vc[u].z), vnew(wc[u].w, vc[u].w), vnew(wr[u], vr[u])};
      const float so[4] = {sacc[u].x, sacc[u].y, sacc[u].z, sacc[u].w};
      const float vp[4] = {vc[u].x, vc[u].y, vc[u].z, vc[u].w};
      float z[4];
      int rank = 0;
#pragma unroll
      for (int l = 0; l < 4; ++l) {
        const bool comp = ((kw[u] >> (8 * l)) & 3u) == K_COMP;
        const float D = rank == 0 ? dg[u].x : rank == 1 ? dg[u].y : rank == 2 ? dg[u].z : dg[u].w;
        // as stencil(): the last axis is added last
        const float az = cfac * (bc * (so[l] + (x[l] + x[l + 2])) - D * x[l + 1]);
        z[l] = comp ? az + c3 * vp[l] : 0.f;
        rank += comp ? 1 : 0;
      }
      st4(Vj + p4, make_float4(x[1], x[2], x[3], x[4]));
      st4(Wn + p4, make_float4(z[0], z[1], z[2], z[3]));
      const float xv[4] = {x[1], x[2], x[3], x[4]};
      d1.add4(xv, xv);
      d2.add4(z, xv);
      d3.add4(z, z);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      pc[u] = pn[u];
      kc[u] = kn[u];
      pn[u] = pf[u];
      kn[u] = kf[u];
    }
  }
  return QuadSums{d1.value(), d2.value(), d3.value()};
}

// out = A X + a1 + c2 a2 + c3 a3 on groups of 4 nodes (the first NT terms;
// a1, a2, a3 compact, at the group's list indices), 0 at the group's other
// nodes: the w_j passes and P_0.  With SUMS: |X|^2, <out, X> and |out|^2
// (this thread's AccG sums).  Out of line: inlined, the three w passes took
// twice as long at 512^3 (register pressure in the kernel).
template <int N, int NT, bool SUMS>
__device__ __noinline__ QuadSums quad_stencil(const float* __restrict__ X, float* __restrict__ out,
                                              const float* __restrict__ a1, const float* __restrict__ a2,
                                              const float* __restrict__ a3, float c2, float c3,
                                              const uint8_t* __restrict__ kind, const float* __restrict__ diagf,
                                              const int* __restrict__ qidx, const int* __restrict__ qk, int nq,
                                              const GridDev& g, float cfac, float bc, float dint, long long gtid,
                                              long long gth) {
  long long st[N > 1 ? N - 1 : 1];
#pragma unroll
  for (int d = 0; d < N - 1; ++d) st[d] = g.stride[d];
  AccG d1, d2, d3;
  quad_loop(qidx, qk, nq, gtid, gth, [&](long long p4, int k0, bool full, long long pn4) {
    if (pn4 >= 0 && (pn4 & 31) == 0) {  // a lane per 128-byte line
      prefetch_l2(X + pn4);
      prefetch_l2(X + pn4 + st[0]);
    }
    const float4 vc = ld4(X + p4);
    const float vl = __ldcg(X + p4 - 1), vr = __ldcg(X + p4 + 4);
    float4 sacc = make_float4(-0.f, -0.f, -0.f, -0.f);  // as stencil()
#pragma unroll
    for (int d = 0; d < N - 1; ++d) {
      const float4 m = ld4(X + p4 - st[d]), pq = ld4(X + p4 + st[d]);
      sacc.x += m.x + pq.x;
      sacc.y += m.y + pq.y;
      sacc.z += m.z + pq.z;
      sacc.w += m.w + pq.w;
    }
    const unsigned kw = full ? QK_FULL_KIND : __ldg(reinterpret_cast<const unsigned*>(kind + p4));
    float dg[4], t1[4], t2[4], t3[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      dg[r] = full ? dint : __ldg(diagf + k0 + r);
      t1[r] = NT >= 1 ? __ldcg(a1 + k0 + r) : 0.f;
      t2[r] = NT >= 2 ? __ldcg(a2 + k0 + r) : 0.f;
      t3[r] = NT >= 3 ? __ldcg(a3 + k0 + r) : 0.f;
    }
    const float v[4] = {vc.x, vc.y, vc.z, vc.w};
    const float so[4] = {sacc.x, sacc.y, sacc.z, sacc.w};
    const float sx[4] = {vl + vc.y, vc.x + vc.z, vc.y + vc.w, vc.z + vr};
    float z[4];
    int rank = 0;
#pragma unroll
    for (int l = 0; l < 4; ++l) {
      z[l] = 0.f;
      if (((kw >> (8 * l)) & 3u) != K_COMP) continue;
      const int r = rank++;
      const float D = r == 0 ? dg[0] : r == 1 ? dg[1] : r == 2 ? dg[2] : dg[3];
      float w = cfac * (bc * (so[l] + sx[l]) - D * v[l]);
      if (NT >= 1) w = w + (r == 0 ? t1[0] : r == 1 ? t1[1] : r == 2 ? t1[2] : t1[3]);
      if (NT >= 2) w = w + c2 * (r == 0 ? t2[0] : r == 1 ? t2[1] : r == 2 ? t2[2] : t2[3]);
      if (NT >= 3) w = w + c3 * (r == 0 ? t3[0] : r == 1 ? t3[1] : r == 2 ? t3[2] : t3[3]);
      z[l] = w;
    }
    st4(out + p4, make_float4(z[0], z[1], z[2], z[3]));
    if (SUMS) {
      d1.add4(v, v);
      d2.add4(z, v);
      d3.add4(z, z);
    }
  });
  return QuadSums{d1.value(), d2.value(), d3.value()};
}

// The combination y <- y + tau w_1 (+ tau^2/2 w_2) + sum_i coef_i V_i on
// groups of 4 nodes: per computational point the arithmetic of the per-point
// loop (the same Dot2 basis sum in the same order, so the same bits), with
// 16-byte loads of the basis vectors, ten in flight: the basis size is a
// multiple of 5 but for m_max or a breakdown (the error check runs every 5
// vectors).  Measured per launch with the earlier two-pass kernel at 256^3 /
// 512^3 (10 / 20 vectors): 5 in flight 1.378 / 14.11 ms, 8 1.376 / 14.01,
// 10 1.342 / 13.51, 16 1.390 / 13.72.  Writes y (compact, FP64) and its FP32
// grid copy (0 at the group's other nodes), and, for the last substep, y
// into ufin at the computational points (the kernel then skips its
// write-back); returns this thread's sum of the squares of the FP32 copy
// (the controller's scale).  Inlined into the kernel: 1.59 against 1.80 ms
// at 512^3 out of line.
static __device__ __forceinline__ double quad_combination(const float* __restrict__ chi,
                                                          const float* __restrict__ clo, int m, double tau,
                                                          const float* __restrict__ V, long long vs,
                                                          const float* __restrict__ W1g, const float* __restrict__ W2g,
                                                          double* __restrict__ Yc, float* __restrict__ Yg,
                                                          double* __restrict__ ufin, const uint8_t* __restrict__ kind,
                                                          const int* __restrict__ qidx, const int* __restrict__ qk,
                                                          int nq, long long gtid, long long gth) {
  Acc<float> yn;  // |y|^2 of the FP32 copy: the controller's scale only
  const double h2 = 0.5 * tau * tau;
  quad_loop(qidx, qk, nq, gtid, gth, [&](long long p4, int k0, bool full, long long pn4) {
    if (pn4 >= 0 && (pn4 & 31) == 0)  // a lane per 128-byte line
      for (int i = 0; i < m; ++i) prefetch_l2(V + (long long)i * vs + pn4);
    const unsigned kw = full ? QK_FULL_KIND : __ldg(reinterpret_cast<const unsigned*>(kind + p4));
    float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f, e0 = 0.f, e1 = 0.f, e2 = 0.f, e3 = 0.f;
#pragma unroll 10
    for (int i = 0; i < m; ++i) {
      const float4 a4 = ld4(V + (long long)i * vs + p4);
      const float ch = chi[i], cl = clo[i];
      dot2_step(s0, e0, ch, cl, a4.x);
      dot2_step(s1, e1, ch, cl, a4.y);
      dot2_step(s2, e2, ch, cl, a4.z);
      dot2_step(s3, e3, ch, cl, a4.w);
    }
    const float4 w1 = ld4(W1g + p4);
    const float4 w2 = W2g ? ld4(W2g + p4) : make_float4(0.f, 0.f, 0.f, 0.f);
    const float sl[4] = {s0, s1, s2, s3}, el[4] = {e0, e1, e2, e3};
    const float w1l[4] = {w1.x, w1.y, w1.z, w1.w}, w2l[4] = {w2.x, w2.y, w2.z, w2.w};
    float yo[4];
    int rank = 0;
#pragma unroll
    for (int l = 0; l < 4; ++l) {
      yo[l] = 0.f;
      if (((kw >> (8 * l)) & 3u) != K_COMP) continue;
      const long long k = k0 + rank;
      ++rank;
      double y = fma(tau, to_f64(w1l[l]), __ldcg(Yc + k)) + (to_f64(sl[l]) + to_f64(el[l]));
      if (W2g) y = fma(h2, to_f64(w2l[l]), y);
      Yc[k] = y;
      if (ufin != nullptr) ufin[p4 + l] = y;
      yo[l] = to_f32_rn(y);
      yn.add(yo[l], yo[l]);
    }
    st4(Yg + p4, make_float4(yo[0], yo[1], yo[2], yo[3]));
  });
  return yn.value();
}

template <typename T, int N>
__device__ __forceinline__ bool quad_full(const SpeciesDev<T>& S, int ncomp, int q, long long k) {
  if (k + 3 >= ncomp || __ldg(S.idx + k + 3) != 4 * q + 3) return false;
  const float di = quad_d_int<T, N>(S);
  return __ldg(S.diagf + k) == di && __ldg(S.diagf + k + 1) == di && __ldg(S.diagf + k + 2) == di &&
         __ldg(S.diagf + k + 3) == di;
}

// Builds the quad list from the sorted list of computational points: each
// warp takes a contiguous range of list indices (ranges in block, then warp
// order); a list index starts a group when its group differs from the
// previous index's.  Counts per warp, one grid barrier for the per-block
// totals, then ordered writes at the warp's offset (warp ballots, no block
// barrier in the loop), then a grid barrier: the passes read entries other
// CTAs wrote.  Eight 32-index loads in flight per warp.  Returns false if
// the kernel must stop.
template <typename T, int N>
__device__ bool build_quads(const PhipmArgs<T>& a, const SpeciesDev<T>& S, int ncomp, Ctl& c, unsigned& bar,
                            int& red) {
  constexpr int QU = 8;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const long long nwt = (long long)gridDim.x * nw;
  const long long per = ((long long)ncomp + nwt - 1) / nwt;
  const long long gw = (long long)blockIdx.x * nw + wid;
  const long long kw0 = min((long long)ncomp, gw * per);
  const long long kw1 = min((long long)ncomp, kw0 + per);
  const int* __restrict__ idx = S.idx;
  __shared__ int s_wc[32];
  int cnt = 0;
  for (long long kb = kw0; kb < kw1; kb += 32 * QU) {
    int q[QU], qp[QU];
#pragma unroll
    for (int u = 0; u < QU; ++u) {
      const long long k = kb + u * 32 + lane;
      q[u] = k < kw1 ? (__ldg(idx + k) >> 2) : -1;
      qp[u] = (k < kw1 && k > 0) ? (__ldg(idx + k - 1) >> 2) : -2;
    }
#pragma unroll
    for (int u = 0; u < QU; ++u) cnt += (q[u] >= 0 && qp[u] != q[u]) ? 1 : 0;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  if (lane == 0) s_wc[wid] = cnt;
  __syncthreads();
  double* pb = part_buf(a.part, red);
  if (threadIdx.x == 0) {
    int tot = 0;
    for (int w = 0; w < nw; ++w) tot += s_wc[w];
    pb[blockIdx.x] = (double)tot;
  }
  if (!grid_barrier(a.st, bar, 20)) return false;
  if (threadIdx.x == 0) {
    long long off = 0, tot = 0;
    for (int b = 0; b < (int)gridDim.x; ++b) {
      const long long x = (long long)__ldcg(pb + b);
      if (b < (int)blockIdx.x) off += x;
      tot += x;
    }
    c.qoff = (int)off;
    c.nquad = (int)tot;
  }
  __syncthreads();
  int base = c.qoff;
  for (int w = 0; w < wid; ++w) base += s_wc[w];
  const unsigned below = (1u << lane) - 1u;
  for (long long kb = kw0; kb < kw1; kb += 32 * QU) {
    int q[QU], qp[QU];
#pragma unroll
    for (int u = 0; u < QU; ++u) {
      const long long k = kb + u * 32 + lane;
      q[u] = k < kw1 ? (__ldg(idx + k) >> 2) : -1;
      qp[u] = (k < kw1 && k > 0) ? (__ldg(idx + k - 1) >> 2) : -2;
    }
#pragma unroll
    for (int u = 0; u < QU; ++u) {
      const bool head = q[u] >= 0 && qp[u] != q[u];
      const unsigned bal = __ballot_sync(0xffffffffu, head);
      if (head) {
        const int pos = base + __popc(bal & below);
        const long long k = kb + u * 32 + lane;
        S.qidx[pos] = q[u];
        S.qk[pos] = (int)k | (quad_full<T, N>(S, ncomp, q[u], k) ? QK_FULL : 0);
      }
      base += __popc(bal);
    }
  }
  return grid_barrier(a.st, bar, 26);
}

// Output fields of the adjoint modes: out[r][p] = (y(t_k) + shift_r w_1)[p]
// (shift == nullptr: 0) + sum_i rows[r][i] V_i[p] at the computational
// points, rows r0 .. r0 + NC - 1 in one sweep (FP64 accumulation).
template <typename T, int NC>
__device__ __forceinline__ void multi_out_sweep(const SpeciesDev<T>& S, int ncomp, int m, const double* rows,
                                                double* const* outs, const double* shift, long long vs,
                                                long long gtid, long long gth) {
  for (long long k = gtid; k < ncomp; k += gth) {
    const long long p = __ldg(S.idx + k);
    double acc[NC];
#pragma unroll
    for (int r = 0; r < NC; ++r) acc[r] = 0.0;
    for (int i = 0; i < m; ++i) {
      const double v = to_f64(__ldcg(S.V + (long long)i * vs + p));
#pragma unroll
      for (int r = 0; r < NC; ++r) acc[r] = fma(rows[r * 64 + i], v, acc[r]);
    }
    if (shift) {
      const double y0 = __ldcg(S.Yc + k), w1 = to_f64(__ldcg(S.W1g + p));
#pragma unroll
      for (int r = 0; r < NC; ++r) acc[r] = fma(shift[r], w1, y0) + acc[r];
    }
#pragma unroll
    for (int r = 0; r < NC; ++r) outs[r][p] = acc[r];
  }
}

template <typename T>
__device__ __noinline__ void multi_out(const SpeciesDev<T>& S, int ncomp, int m, const double* rows, int nr,
                                       double* const* outs, const double* shift, long long vs, long long gtid,
                                       long long gth) {
  for (int rb = 0; rb < nr; rb += 6) {
    const double* rw = rows + rb * 64;
    const double* sh = shift ? shift + rb : nullptr;
    switch (min(6, nr - rb)) {
      case 1: multi_out_sweep<T, 1>(S, ncomp, m, rw, outs + rb, sh, vs, gtid, gth); break;
      case 2: multi_out_sweep<T, 2>(S, ncomp, m, rw, outs + rb, sh, vs, gtid, gth); break;
      case 3: multi_out_sweep<T, 3>(S, ncomp, m, rw, outs + rb, sh, vs, gtid, gth); break;
      case 4: multi_out_sweep<T, 4>(S, ncomp, m, rw, outs + rb, sh, vs, gtid, gth); break;
      case 5: multi_out_sweep<T, 5>(S, ncomp, m, rw, outs + rb, sh, vs, gtid, gth); break;
      default: multi_out_sweep<T, 6>(S, ncomp, m, rw, outs + rb, sh, vs, gtid, gth); break;
    }
  }
}

// Dynamic shared memory of the adjoint modes: coefficient rows, then one
// small-exponential scratch row per warp.
constexpr int ADJ_ROWS = ADJ_NQ_MAX + 3;
constexpr size_t adj_smem(int nt) { return (size_t)(ADJ_ROWS + nt / 32) * 64 * sizeof(double); }

// MODE_ADJ_LAMBDA after the basis on lambda is accepted at tau = 1: rows 0 .. 2
// = beta phi_k(H_m) e_1 (k = 0, 1, 2; rows 0 and 1 from the accepting check,
// row 2 from phi_2 = the p = 1 exponential's phi_{p+1}), rows 3 + i = beta
// exp(tq[i] H_m) e_1, each exponential on its own warp; then the outputs.
template <typename T>
__device__ __noinline__ void adj_lambda_outputs(const PhipmArgs<T>& a, const SpeciesDev<T>& S, int sidx, Ctl& c, int ncomp,
                                   long long vs, long long gtid, long long gth) {
  extern __shared__ double adj_sm[];
  double* rows = adj_sm;
  const int m = c.m, nr = 3 + a.nq;
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  double* ye = adj_sm + ADJ_ROWS * 64 + wid * 64;
  if (m > 0) {
    for (int r = wid; r < nr; r += nw) {
      double* out = rows + r * 64;
      if (r == 0) {
        for (int i = lane; i < m; i += 32) out[i] = c.coef[i];
        __syncwarp();
      } else if (r == 1) {
        for (int i = lane; i < m; i += 32) out[i] = c.beta * c.yexp[i] * c.scale[i];
        __syncwarp();
      } else if (r == 2) {
        small_expm_warp(c, m, 1, 1.0, ye);
        for (int i = lane; i < m; i += 32) out[i] = c.beta * ye[i] * c.scale[i];
        __syncwarp();
      } else {
        const double sq = a.tq[r - 3];
        small_expm_warp(c, m, 0, sq, ye);
        coef_row(c, m, 0, sq, ye, out);
      }
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0 && a.stats) {
    a.stats->substeps[sidx] += 1;
    a.stats->iters[sidx] += m;
    const int ti = a.stats->trace_len[sidx];
    if (ti < TRACE_MAX) {
      a.stats->trace_m[sidx][ti] = m;
      a.stats->trace_tau[sidx][ti] = 1.0;
      a.stats->trace_len[sidx] = ti + 1;
    }
  }
  __syncthreads();
  multi_out<T>(S, ncomp, m, rows, nr, const_cast<double* const*>(a.out), nullptr, vs, gtid, gth);
}

// MODE_ADJ_Y within an accepted substep [t, t1] (basis on w_2, P = 2): for
// every output time tq[i] in (t, t1], y(tq[i]) = y(t) + s w_1 + s^2 beta V_m
// phi_2(s H_m) e_1 with s = tq[i] - t (the same basis serves every s <= tau;
// its error estimate shrinks with s).  Returns false if the kernel must stop.
template <typename T>
__device__ __noinline__ bool adj_y_outputs(const PhipmArgs<T>& a, const SpeciesDev<T>& S, Ctl& c, int ncomp, long long vs,
                              long long gtid, long long gth, unsigned& bar, double t) {
  extern __shared__ double adj_sm[];
  __shared__ double s_shift[ADJ_NQ_MAX];
  __shared__ int s_which[ADJ_NQ_MAX];
  const double t1 = c.last ? 1.0 : t + c.tau;
  int nr = 0;
  for (int i = 0; i < a.nq; ++i) {
    if (t < a.tq[i] && a.tq[i] <= t1) {
      if (threadIdx.x == 0) {
        s_which[nr] = i;
        s_shift[nr] = a.tq[i] - t;
      }
      ++nr;
    }
  }
  if (nr == 0) return true;
  __syncthreads();
  double* rows = adj_sm;
  const int m = c.m;
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  double* ye = adj_sm + ADJ_ROWS * 64 + wid * 64;
  __shared__ double* s_out[ADJ_NQ_MAX];
  for (int r = threadIdx.x; r < nr; r += blockDim.x) s_out[r] = a.out[s_which[r]];
  for (int r = wid; r < nr; r += nw) {
    double* out = rows + r * 64;
    if (m > 0) {
      small_expm_warp(c, m, 2, s_shift[r], ye);
      coef_row(c, m, 2, s_shift[r], ye, out);
    } else {
      for (int i = lane; i < 64; i += 32) out[i] = 0.0;
      __syncwarp();
    }
  }
  __syncthreads();
  multi_out<T>(S, ncomp, m, rows, nr, s_out, s_shift, vs, gtid, gth);
  // the substep's combination rewrites y(t) next
  return grid_barrier(a.st, bar, 25);
}

// Whether a species takes the quad path: FP32 vectors, at least SPLIT_MIN
// points, a group list in the workspace, constant beta, the last axis a
// multiple of 4 nodes.
template <typename T, int N>
__device__ __forceinline__ bool use_quads(const SpeciesDev<T>& S, const GridDev& g, int ncomp) {
  return sizeof(T) == 4 && ncomp >= SPLIT_MIN<T> && S.qidx != nullptr && S.beta_field == nullptr &&
         (g.n[N - 1] & 3) == 0;
}

// Makes the species' group list ready and records its length in
// c.nq_sp[sidx].  The list is built once per domain: the flag is read
// before this launch's build can set it (block 0 sets it after the build's
// last grid barrier, which every CTA reaches only after reading it).
template <typename T, int N>
__device__ bool ensure_quads(const PhipmArgs<T>& a, const SpeciesDev<T>& S, int sidx, int ncomp, Ctl& c,
                             unsigned& bar, int& red) {
  if (threadIdx.x == 0) {
    c.qcached = S.qmeta != nullptr && __ldcg(S.qmeta) == 1;
    if (c.qcached) c.nquad = __ldcg(S.qmeta + 1);
  }
  __syncthreads();
  if (!c.qcached) {
    if (!build_quads<T, N>(a, S, ncomp, c, bar, red)) return false;
    if (S.qmeta != nullptr && blockIdx.x == 0 && threadIdx.x == 0) {
      S.qmeta[1] = c.nquad;
      S.qmeta[0] = 1;
    }
  }
  if (threadIdx.x == 0) c.nq_sp[sidx] = c.nquad;
  __syncthreads();
  return true;
}

// The ETD2 set-up (one species, F from the reaction alone, no F_{n-2}) on
// the groups of 4 nodes: per group 16-byte loads and stores of u, F_{n-1},
// the validity bytes and the FP32 copy of y, and the compact y, v_1, v_2 at
// the group's list indices; per computational point the arithmetic of the
// per-point set-up.  Inlined into the kernel (0.66 against 0.70 ms at 512^3
// out of line).  Nodes of the group off the computational set keep
// their F_{n-1} and validity bytes (rewritten unchanged) and get y = 0 in
// the FP32 copy.  sums: this thread's |y|^2, |v_1|^2, |v_2|^2 of the stored
// FP32 values.
static __device__ __forceinline__ void quad_setup_etd2(const PhipmArgs<float>& a, const SpeciesDev<float>& S, int nq,
                                                    long long gtid, long long gth, double* sums) {
  const bool u16 = (reinterpret_cast<uintptr_t>(S.u) & 15u) == 0;
  AccG sy, s1, s2;
  quad_loop(S.qidx, S.qk, nq, gtid, gth, [&](long long p4, int k0, bool full, long long pn4) {
    if (pn4 >= 0 && (pn4 & 15) == 0) {  // a lane per 128-byte line of the FP64 fields
      prefetch_l2(S.u + pn4);
      prefetch_l2(S.Fprev + pn4);
    }
    const unsigned kw = full ? QK_FULL_KIND : __ldg(reinterpret_cast<const unsigned*>(S.kind + p4));
    const unsigned fw = __ldcg(reinterpret_cast<const unsigned*>(S.fvalid + p4));
    double u[4], fp[4];
    if (u16) {
      const double2 u0 = __ldcg(reinterpret_cast<const double2*>(S.u + p4));
      const double2 u1 = __ldcg(reinterpret_cast<const double2*>(S.u + p4 + 2));
      u[0] = u0.x;
      u[1] = u0.y;
      u[2] = u1.x;
      u[3] = u1.y;
    } else {
#pragma unroll
      for (int l = 0; l < 4; ++l) u[l] = __ldcg(S.u + p4 + l);
    }
    {
      const double2 f0 = __ldcg(reinterpret_cast<const double2*>(S.Fprev + p4));
      const double2 f1 = __ldcg(reinterpret_cast<const double2*>(S.Fprev + p4 + 2));
      fp[0] = f0.x;
      fp[1] = f0.y;
      fp[2] = f1.x;
      fp[3] = f1.y;
    }
    float yg[4], v1f[4], v2f[4];
    unsigned fwn = fw;
    int r = 0;
#pragma unroll
    for (int l = 0; l < 4; ++l) {
      yg[l] = v1f[l] = v2f[l] = 0.f;
      if (((kw >> (8 * l)) & 3u) != K_COMP) continue;
      const double F = reaction(a.reaction, a.rp, 0, u[l], 0.0);
      const double Fp = ((fw >> (8 * l)) & 1u) ? fp[l] : F;
      const double v1 = a.dt * F;
      const double v2 = a.etd1 ? 0.0 : a.dt * (F - Fp);
      const long long k = k0 + r;
      ++r;
      yg[l] = to_f32_rn(u[l]);
      v1f[l] = to_f32_rn(v1);
      v2f[l] = to_f32_rn(v2);
      S.Yc[k] = u[l];
      S.V1c[k] = v1f[l];
      S.V2c[k] = v2f[l];
      fp[l] = F;
      fwn = (fwn & ~(0xffu << (8 * l))) | (1u << (8 * l));
    }
    st4(S.Yg + p4, make_float4(yg[0], yg[1], yg[2], yg[3]));
    __stcg(reinterpret_cast<double2*>(S.Fprev + p4), make_double2(fp[0], fp[1]));
    __stcg(reinterpret_cast<double2*>(S.Fprev + p4 + 2), make_double2(fp[2], fp[3]));
    __stcg(reinterpret_cast<unsigned*>(S.fvalid + p4), fwn);
    sy.add4(yg, yg);
    s1.add4(v1f, v1f);
    s2.add4(v2f, v2f);
  });
  sums[0] = sy.value();
  sums[1] = s1.value();
  sums[2] = s2.value();
}

template <typename T, int N, bool ADJ>
__device__ bool phipm_species(const PhipmArgs<T>& a, const SpeciesDev<T>& S, int sidx, Ctl& c, unsigned& bar,
                              int& red, double ynorm2, double vscale) {
  const GridDev& g = a.g;
  const int ncomp = *S.ncomp;
  const long long gtid = dealt_tid();
  const long long gthreads = (long long)gridDim.x * blockDim.x;
  const T cfac = (T)a.cfac;
  const T bc = (T)S.beta_c;
  const float dint = quad_d_int<T, N>(S);  // the diagonal of the full groups (QK_FULL)
  const double anorm = a.dt * (*S.gersh);
  const int m_max = a.m_max;
  // highest phi index: 2 or 3 (any other value of a.p: 2); 0 for the basis
  // on lambda of the adjoint (V_0 = lambda, written by the set-up)
  const int P = ADJ && a.mode == MODE_ADJ_LAMBDA ? 0 : a.p == 3 ? 3 : 2;
  const long long vs = g.size;
  // large problems: split Lanczos pass (see SPLIT_MIN), on aligned groups of
  // 4 nodes where the layout allows
  const bool split = ncomp >= SPLIT_MIN<T>;
  // FP64 split passes: Z_j = B V_j with B = A / cfac (one FP64 multiply less
  // per point); the Lanczos scalars take the factor: zfac = cfac
  const bool zb = sizeof(T) == 8 && split;
  const double zfac = zb ? a.cfac : 1.0;
  // the group list was made ready at kernel start (ensure_quads)
  const bool quad = use_quads<T, N>(S, g, ncomp);
  if (quad) {
    if (threadIdx.x == 0) c.nquad = c.nq_sp[sidx];
    __syncthreads();
  }
  // the statistics accumulate over the launches of one step (zeroed by the host)
  if (blockIdx.x == 0 && threadIdx.x == 0) c.trace0 = a.stats ? a.stats->trace_len[sidx] : 0;
  double* pb = nullptr;
  if (threadIdx.x == 0) {
    c.t = 0.0;
    c.tau = 1.0;
    c.ynorm = fmax(fmax(sqrt(ynorm2), vscale), 1e-300);
    c.abort = 0;
  }
  __syncthreads();
  int nsub = 0;
  while (c.t < 1.0) {
    if (nsub >= MAX_SUBSTEPS) {
      if (threadIdx.x == 0) atomicOr(&a.st->err, ERRF_KRYLOV);
      return false;
    }
    if (threadIdx.x == 0) {
      c.last = c.tau >= 1.0 - c.t;
      if (c.last) c.tau = 1.0 - c.t;
      c.nrej = 0;
    }
    __syncthreads();
    const double t = c.t;
    bool qw = P == 0;  // P = 0: no w_j passes
    if constexpr (sizeof(T) == 4) {
      if (quad && !qw) {
        // the w_j passes on groups of 4 nodes
        const int nq = c.nquad;
        const float tt = (float)t;
        if (P == 3) {
          quad_stencil<N, 3, false>(S.Yg, S.W1g, S.V1c, S.V2c, S.V3c, tt, (float)(0.5 * t * t), S.kind, S.diagf,
                          S.qidx, S.qk, nq, g, cfac, bc, dint, gtid, gthreads);
          if (!grid_barrier(a.st, bar, 10)) return false;
          quad_stencil<N, 2, false>(S.W1g, S.W2g, S.V2c, S.V3c, nullptr, tt, 0.f, S.kind, S.diagf, S.qidx, S.qk, nq, g,
                          cfac, bc, dint, gtid, gthreads);
          if (!grid_barrier(a.st, bar, 16)) return false;
          quad_stencil<N, 1, false>(S.W2g, S.V, S.V3c, nullptr, nullptr, 0.f, 0.f, S.kind, S.diagf, S.qidx, S.qk, nq, g,
                          cfac, bc, dint, gtid, gthreads);
        } else {
          quad_stencil<N, 2, false>(S.Yg, S.W1g, S.V1c, S.V2c, nullptr, tt, 0.f, S.kind, S.diagf, S.qidx, S.qk, nq, g,
                          cfac, bc, dint, gtid, gthreads);
          if (!grid_barrier(a.st, bar, 10)) return false;
          quad_stencil<N, 1, false>(S.W1g, S.V, S.V2c, nullptr, nullptr, 0.f, 0.f, S.kind, S.diagf, S.qidx, S.qk, nq, g,
                          cfac, bc, dint, gtid, gthreads);
        }
        qw = true;
      }
    }
    if (qw) {
    } else
    if (P == 3) {
      // w_1 = A y + v_1 + t v_2 + t^2/2 v_3, w_2 = A w_1 + v_2 + t v_3,
      // w_3 = A w_2 + v_3 -> V_0 (one point per thread: register bound)
      const T tt = (T)t, th2 = (T)(0.5 * t * t);
      node_loop<1>(gtid, gthreads, ncomp, S.idx, [&](const auto& kk, const auto& pp) {
        if (pp[0] < 0) return;
        const T ay = stencil<T, N>(S.Yg, pp[0], g, diag_of<T>(S, (int)kk[0]), S.beta_field, bc, cfac);
        const T a1 = __ldcg(S.V1c + kk[0]), a2 = __ldcg(S.V2c + kk[0]), a3 = __ldcg(S.V3c + kk[0]);
        S.W1g[pp[0]] = ay + a1 + tt * a2 + th2 * a3;
      });
      if (!grid_barrier(a.st, bar, 10)) return false;
      node_loop<1>(gtid, gthreads, ncomp, S.idx, [&](const auto& kk, const auto& pp) {
        if (pp[0] < 0) return;
        const T aw = stencil<T, N>(S.W1g, pp[0], g, diag_of<T>(S, (int)kk[0]), S.beta_field, bc, cfac);
        const T a2 = __ldcg(S.V2c + kk[0]), a3 = __ldcg(S.V3c + kk[0]);
        S.W2g[pp[0]] = aw + a2 + tt * a3;
      });
      if (!grid_barrier(a.st, bar, 16)) return false;
      node_loop<1>(gtid, gthreads, ncomp, S.idx, [&](const auto& kk, const auto& pp) {
        if (pp[0] < 0) return;
        const T aw = stencil<T, N>(S.W2g, pp[0], g, diag_of<T>(S, (int)kk[0]), S.beta_field, bc, cfac);
        S.V[pp[0]] = aw + __ldcg(S.V3c + kk[0]);
      });
    } else {
      // w_1 = A y + v_1 + t v_2
      node_loop_sized<T>(gtid, gthreads, ncomp, S.idx, [&](const auto& kk, const auto& pp) {
        constexpr int U = NL_U(kk);
        T ay[U], a1[U], a2[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          if (pp[u] < 0) continue;
          ay[u] = stencil<T, N>(S.Yg, pp[u], g, diag_of<T>(S, (int)kk[u]), S.beta_field, bc, cfac);
          a1[u] = __ldcg(S.V1c + kk[u]);
          a2[u] = __ldcg(S.V2c + kk[u]);
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
          if (pp[u] >= 0) S.W1g[pp[u]] = ay[u] + a1[u] + (T)t * a2[u];
      });
      if (!grid_barrier(a.st, bar, 10)) return false;
      // w_2 = A w_1 + v_2 -> V_0 (unnormalised)
      node_loop_sized<T>(gtid, gthreads, ncomp, S.idx, [&](const auto& kk, const auto& pp) {
        constexpr int U = NL_U(kk);
        T aw[U], a2[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          if (pp[u] < 0) continue;
          aw[u] = stencil<T, N>(S.W1g, pp[u], g, diag_of<T>(S, (int)kk[u]), S.beta_field, bc, cfac);
          a2[u] = __ldcg(S.V2c + kk[u]);
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
          if (pp[u] >= 0) S.V[pp[u]] = aw[u] + a2[u];
      });
    }
    if (!grid_barrier(a.st, bar, 11)) return false;
    // P_0: Z_0 = A V_0, |V_0|^2, <Z_0, V_0> (and |Z_0|^2 on the 4-node groups)
    bool qp0 = false;
    if constexpr (sizeof(T) == 4) {
      if (quad) {
        const QuadSums qs = quad_stencil<N, 0, true>(S.V, S.Z[0], nullptr, nullptr, nullptr, 0.f, 0.f, S.kind, S.diagf,
                                            S.qidx, S.qk, c.nquad, g, cfac, bc, dint, gtid, gthreads);
        double v[3] = {qs.d1, qs.d2, qs.d3};
        pb = part_buf(a.part, red);
        block_partials<3>(v, pb);
        qp0 = true;
      }
    }
    if (!qp0) {
      Acc<T> d1, d2;
      node_loop_sized<T>(gtid, gthreads, ncomp, S.idx, [&](const auto& kk, const auto& pp) {
        constexpr int U = NL_U(kk);
        T vv[U], zz[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          if (pp[u] < 0) continue;
          vv[u] = __ldcg(S.V + pp[u]);
          zz[u] = zb ? stencil<T, N, false>(S.V, pp[u], g, diag_of<T>(S, (int)kk[u]), S.beta_field, bc, cfac)
                     : stencil<T, N>(S.V, pp[u], g, diag_of<T>(S, (int)kk[u]), S.beta_field, bc, cfac);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
          if (pp[u] < 0) continue;
          S.Z[0][pp[u]] = zz[u];
          d1.add(vv[u], vv[u]);
          d2.add(zz[u], vv[u]);
        }
      });
      double v[2] = {d1.value(), d2.value()};
      pb = part_buf(a.part, red);
      block_partials<2>(v, pb);
    }
    if (!grid_barrier(a.st, bar, 12)) return false;
    {
      double tot[3] = {0.0, 0.0, 0.0};
      if (quad) {
        grid_totals<3>(pb, tot);
      } else {
        double t2[2];
        grid_totals<2>(pb, t2);
        tot[0] = t2[0];
        tot[1] = t2[1];
      }
      if (threadIdx.x == 0) {
        c.beta = sqrt(tot[0]);
        if (!isfinite(c.beta) || !isfinite(tot[1]) || !isfinite(tot[2])) {
          atomicOr(&a.st->err, ERRF_NONFINITE);
          c.abort = 1;
        }
        const double s0 = c.beta > 0.0 ? 1.0 / c.beta : 0.0;
        c.scale[0] = s0;
        c.alpha[0] = zfac * tot[1] * s0 * s0;
        c.up[0] = 0.0;
        c.m = 0;
        c.accepted = 0;
        c.breakdown = 0;
        if (quad && c.beta > 0.0) {
          // one-pass recurrence: beta_1 = |A v_0 - alpha_0 v_0| from the three
          // sums (v_0 = s0 V_0): the state of a basis of one vector
          const double b1 = sqrt(fmax((tot[2] - tot[1] * tot[1] / tot[0]) * s0 * s0, 0.0));
          c.low[0] = b1;
          c.up[1] = b1;
          c.hn = b1;
          c.m = 1;
          c.breakdown = b1 < BREAKDOWN_REL * anorm;
        }
      }
      __syncthreads();
      if (c.abort) return false;
    }
    // error check of the basis of c.m vectors (warp 0), then every thread reads c.accepted
    const auto check = [&]() {
      if (threadIdx.x < 32) {
        small_expm_warp(c, c.m, P, c.tau, c.yexp);
        finish_check(c, c.m, P, c.tau);
        if (threadIdx.x == 0) {
          if (c.breakdown) c.err = 0.0;
          c.accepted = c.err <= a.tol * c.tau * c.ynorm;
        }
      }
      __syncthreads();
    };
    if (c.beta > 0.0 && quad) {
      if constexpr (sizeof(T) == 4) {
        // Groups of 4 nodes: one pass per Krylov vector (quad_pass_1).
        // Before pass j: alpha_{j-1}, beta_j and the scale s of V_{j-1}
        // (1/|V_0| for V_0, 1 after); V_j = (u_{j-1} - alpha_{j-1} v_{j-1}) / beta_j
        // with u_0 = A v_0 = s Z_0; u_j = A v_j - beta_j v_{j-1} -> Z[j & 1].
        // After it: alpha_j = <u_j, V_j> / |V_j|^2, beta_{j+1}^2 =
        // |u_j|^2 - <u_j, V_j>^2 / |V_j|^2; H is symmetric tridiagonal.
        if (c.m == m_max || c.breakdown) check();
        for (int j = 1; j < m_max && !c.accepted; ++j) {
          const double sp = c.scale[j - 1], bj = c.low[j - 1];
          const float c1 = (float)(sp / bj), c2 = (float)(-c.alpha[j - 1] * sp / bj), c3 = (float)(-bj * sp);
          const QuadSums qs = quad_pass_1<N>(S.Z[(j - 1) & 1], S.V + (long long)(j - 1) * vs, S.V + (long long)j * vs,
                                             S.Z[j & 1], c1, c2, c3, S.kind, S.diagf, S.qidx, S.qk, c.nquad, g, cfac,
                                             bc, dint, gtid, gthreads);
          double v[3] = {qs.d1, qs.d2, qs.d3};
          pb = part_buf(a.part, red);
          block_partials<3>(v, pb);
          if (!grid_barrier(a.st, bar, 13)) return false;
          double tot[3];
          grid_totals<3>(pb, tot);
          if (threadIdx.x == 0) {
            const double aj = tot[1] / tot[0];
            const double bn = sqrt(fmax(tot[2] - tot[1] * aj, 0.0));
            if (!isfinite(aj) || !isfinite(bn)) {
              atomicOr(&a.st->err, ERRF_NONFINITE);
              c.abort = 1;
            }
            c.alpha[j] = aj;
            c.scale[j] = 1.0;
            c.low[j] = bn;
            c.up[j + 1] = bn;
            c.hn = bn;
            c.m = j + 1;
            c.breakdown = bn < BREAKDOWN_REL * anorm;
          }
          __syncthreads();
          if (c.abort) return false;
          if (c.m % CHECK_EVERY == 0 || c.m == m_max || c.breakdown) check();
        }
      }
    }
    if (c.beta > 0.0) {
      if (!quad) {
      // Pass P_j (one grid barrier each) rebuilds
      //   w_j = z_{j-1} - h_{j-1,j-1} v_{j-1} - h_{j-2,j-1} v_{j-2}
      // at every stencil point from Z_{j-1} = A V_{j-1}, V_{j-1}, V_{j-2}
      // (all unnormalised), stores V_j = w_j and Z_j = A w_j, and sums
      // |w_j|^2, <A w_j, w_j>, <A w_j, V_{j-1}>.  After the barrier:
      //   h_{j,j-1} = |w_j|, h_jj = <A w_j, w_j>/|w_j|^2,
      //   h_{j-1,j} = <A w_j, V_{j-1}> / (|w_j| |V_{j-1}|),
      // the same classical Gram-Schmidt coefficients as z = A v_j,
      // <z, v_j>, <z, v_{j-1}>, with the normalisation deferred.
      for (int j = 1; j <= m_max; ++j) {
        const T ca = (T)(c.scale[j - 1] * zfac);              // coefficient of Z_{j-1}
        const T cb = (T)(-c.alpha[j - 1] * c.scale[j - 1]);    // of V_{j-1}
        const T cc = j >= 2 ? (T)(-c.up[j - 1] * c.scale[j - 2]) : T(0);  // of V_{j-2}
        const T* Zp = S.Z[(j - 1) & 1];
        T* Zn = S.Z[j & 1];
        const T* V1 = S.V + (long long)(j - 1) * vs;
        const T* V2 = S.V + (long long)(j >= 2 ? j - 2 : 0) * vs;
        T* Vj = S.V + (long long)j * vs;
        if (split) {
          // pass A_j: V_j = w_j at the own points only
          constexpr int U = SPLIT_U<T>;
          node_loop<U>(gtid, gthreads, ncomp, S.idx, [&](const auto& kk, const auto& pp) {
            T zv[U], v1v[U], v2v[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
              if (pp[u] < 0) continue;
              zv[u] = __ldcg(Zp + pp[u]);
              v1v[u] = __ldcg(V1 + pp[u]);
              v2v[u] = __ldcg(V2 + pp[u]);
            }
#pragma unroll
            for (int u = 0; u < U; ++u)
              if (pp[u] >= 0) Vj[pp[u]] = ca * zv[u] + cb * v1v[u] + cc * v2v[u];
          });
          if (!grid_barrier(a.st, bar, 15)) return false;
          // pass B_j: Z_j = A V_j from the stored V_j, and the three sums
          Acc<T> d1, d2, d3;
          node_loop<SPLIT_UB<T>>(gtid, gthreads, ncomp, S.idx, [&](const auto& kk, const auto& pp) {
            constexpr int UB = NL_U(kk);
            T zv[UB], wv[UB], v1v[UB];
#pragma unroll
            for (int u = 0; u < UB; ++u) {
              if (pp[u] < 0) continue;
              zv[u] = zb ? stencil<T, N, false>(Vj, pp[u], g, diag_of<T>(S, (int)kk[u]), S.beta_field, bc, cfac)
                         : stencil<T, N>(Vj, pp[u], g, diag_of<T>(S, (int)kk[u]), S.beta_field, bc, cfac);
              wv[u] = __ldcg(Vj + pp[u]);
              v1v[u] = __ldcg(V1 + pp[u]);
            }
#pragma unroll
            for (int u = 0; u < UB; ++u) {
              if (pp[u] < 0) continue;
              Zn[pp[u]] = zv[u];
              d1.add(wv[u], wv[u]);
              d2.add(zv[u], wv[u]);
              d3.add(zv[u], v1v[u]);
            }
          });
          double v[3] = {d1.value(), d2.value(), d3.value()};
          pb = part_buf(a.part, red);
          block_partials<3>(v, pb);
        } else {
          Acc<T> d1, d2, d3;
          for (long long k = gtid; k < ncomp; k += gthreads) {
            const long long p = __ldg(S.idx + k);
            const T w = wval<T>(Zp, V1, V2, p, ca, cb, cc);
            const T v1 = __ldcg(V1 + p);
            T s = T(-0.0);  // as stencil()
            const double* bf = S.beta_field;
            if (bf == nullptr) {
#pragma unroll
              for (int d = 0; d < N; ++d)
                s += wval<T>(Zp, V1, V2, p - g.stride[d], ca, cb, cc) + wval<T>(Zp, V1, V2, p + g.stride[d], ca, cb, cc);
              s = bc * s;
            } else {
              const double bp = __ldg(bf + p);
#pragma unroll
              for (int d = 0; d < N; ++d) {
                const long long st = g.stride[d];
                s += T(0.5 * (bp + __ldg(bf + p - st))) * wval<T>(Zp, V1, V2, p - st, ca, cb, cc);
                s += T(0.5 * (bp + __ldg(bf + p + st))) * wval<T>(Zp, V1, V2, p + st, ca, cb, cc);
              }
            }
            const T z = cfac * (s - diag_of<T>(S, (int)k) * w);
            Vj[p] = w;
            Zn[p] = z;
            d1.add(w, w);
            d2.add(z, w);
            d3.add(z, v1);
          }
          double v[3] = {d1.value(), d2.value(), d3.value()};
          pb = part_buf(a.part, red);
          block_partials<3>(v, pb);
        }
        if (!grid_barrier(a.st, bar, 13)) return false;
        {
          double tot[3];
          grid_totals<3>(pb, tot);
          if (threadIdx.x == 0) {
            const double hn = sqrt(tot[0]);
            if (!isfinite(hn) || !isfinite(tot[1]) || !isfinite(tot[2])) {
              atomicOr(&a.st->err, ERRF_NONFINITE);
              c.abort = 1;
            }
            c.low[j - 1] = hn;
            c.hn = hn;
            c.m = j;
            c.breakdown = hn < BREAKDOWN_REL * anorm;
            const double sj = c.breakdown ? 0.0 : 1.0 / hn;
            c.scale[j] = sj;
            c.alpha[j] = zfac * tot[1] * sj * sj;
            c.up[j] = zfac * tot[2] * sj * c.scale[j - 1];
          }
          __syncthreads();
          if (c.abort) return false;
        }
        if (c.m % CHECK_EVERY == 0 || c.m == m_max || c.breakdown) {
          check();
          if (c.accepted) break;
        }
      }
      }
      // rejections at m_max: shrink tau, reuse the basis (the adjoint's basis
      // on lambda is not time-stepped: the host falls back instead)
      if (!c.accepted && !(ADJ && a.mode == MODE_ADJ_LAMBDA)) {
        const int m = c.m;
        for (;;) {
          if (threadIdx.x == 0) {
            const double tolabs = a.tol * c.tau * c.ynorm;
            const double fac = fmax(0.2, 0.9 * pow(tolabs / c.err, 1.0 / (m + 1)));
            c.tau *= fac;
            c.last = 0;
            c.nrej += 1;
            if (c.tau < TAU_MIN) {
              atomicOr(&a.st->err, ERRF_KRYLOV);
              c.abort = 1;
            }
          }
          __syncthreads();
          if (c.abort) return false;
          if (threadIdx.x < 32) {
            small_expm_warp(c, m, P, c.tau, c.yexp);
            finish_check(c, m, P, c.tau);
            if (threadIdx.x == 0) c.accepted = c.err <= a.tol * c.tau * c.ynorm;
          }
          __syncthreads();
          if (c.accepted) break;
        }
      }
    } else {
      if (threadIdx.x == 0) {
        c.err = 0.0;
        c.m = 0;
      }
      __syncthreads();
    }
    if constexpr (ADJ) {
      if (a.mode == MODE_ADJ_LAMBDA) {
        if (c.m > 0 && !c.accepted) {
          if (blockIdx.x == 0 && threadIdx.x == 0 && a.stats) a.stats->single_basis_missed = 1;
          return true;
        }
        adj_lambda_outputs<T>(a, S, sidx, c, ncomp, vs, gtid, gthreads);
        return true;
      }
      if (a.mode == MODE_ADJ_Y && !adj_y_outputs<T>(a, S, c, ncomp, vs, gtid, gthreads, bar, t)) return false;
    }
    // y <- y + tau w_1 + sum_i coef_i V_i ; |y|^2
    {
      const int m = c.m;
      const double tau = c.tau;
      Acc<double> yn;
      if constexpr (sizeof(T) == 4) {
        // coefficients split into two floats for the FP32 basis sum
        for (int i = threadIdx.x; i < m; i += blockDim.x) {
          const float hi = (float)c.coef[i];
          c.chi[i] = hi;
          c.clo[i] = (float)(c.coef[i] - (double)hi);
        }
        __syncthreads();
      }
      bool qdone = false;
      if constexpr (sizeof(T) == 4) {
        if (quad) {
          // the last substep of an ETD2 step or a combination writes u itself
          double* ufin = c.last && (a.mode == MODE_ETD2 || a.mode == MODE_GIVEN) ? S.u : nullptr;
          yn.s = quad_combination(c.chi, c.clo, m, tau, S.V, vs, S.W1g, P == 3 ? S.W2g : nullptr, S.Yc, S.Yg, ufin,
                                  S.kind, S.qidx, S.qk, c.nquad, gtid, gthreads);
          if (ufin != nullptr && threadIdx.x == 0) c.wb_done[sidx] = 1;
          qdone = true;
        }
      }
      for (long long k = qdone ? (long long)ncomp : gtid; k < ncomp; k += gthreads) {
        const long long p = __ldg(S.idx + k);
        double sum;
        if constexpr (sizeof(T) == 4) {
          sum = basis_sum_f32(c, S.V, vs, p, m);
        } else {
          sum = 0.0;
          for (int i = 0; i < m; ++i) sum = fma(c.coef[i], to_f64(__ldcg(S.V + (long long)i * vs + p)), sum);
        }
        double y = fma(tau, (double)__ldcg(S.W1g + p), __ldcg(S.Yc + k)) + sum;
        if (P == 3) y = fma(0.5 * tau * tau, (double)__ldcg(S.W2g + p), y);
        S.Yc[k] = y;
        S.Yg[p] = (T)y;
        yn.add(y, y);
      }
      double v[1] = {yn.value()};
      pb = part_buf(a.part, red);
      block_partials<1>(v, pb);
    }
    if (!grid_barrier(a.st, bar, 14)) return false;
    {
      double tot[1];
      grid_totals<1>(pb, tot);
      if (threadIdx.x == 0) {
        const int m = c.m;
        if (blockIdx.x == 0 && a.stats) {
          StatsDev* st = a.stats;
          const int ti = c.trace0 + nsub;  // after the entries of earlier launches of the step
          if (ti < TRACE_MAX) {          // the trace keeps the first TRACE_MAX substeps
            st->trace_m[sidx][ti] = m;
            st->trace_tau[sidx][ti] = c.tau;
          }
          st->rejections[sidx] += c.nrej;
          st->iters[sidx] += m;
        }
        double grow;
        if (c.err == 0.0) grow = 2.0;
        else grow = fmin(2.0, 0.9 * pow(a.tol * c.tau * c.ynorm / c.err, 1.0 / (m + 1)));
        c.t = c.last ? 1.0 : c.t + c.tau;
        if (c.t < 1.0) c.tau = fmin(1.0 - c.t, c.tau * grow);
        c.ynorm = fmax(fmax(sqrt(tot[0]), vscale), 1e-300);
        if (!isfinite(c.ynorm)) {
          atomicOr(&a.st->err, ERRF_NONFINITE);
          c.abort = 1;
        }
      }
      __syncthreads();
      if (c.abort) return false;
    }
    ++nsub;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0 && a.stats) {
    a.stats->substeps[sidx] += nsub;
    a.stats->trace_len[sidx] = min(c.trace0 + nsub, TRACE_MAX);
  }
  return true;
}

// ADJ: the instantiation that also runs the adjoint modes (MODE_ADJ_*),
// kept apart so that their code adds nothing to the other launches.  NT:
// threads per CTA (one CTA per SM), which fixes the registers per thread.
template <typename T, int N, bool ADJ, int NT>
__global__ void __launch_bounds__(NT, 1) phipm_kernel(const PhipmArgs<T> a) {
  __shared__ Ctl c;
  unsigned bar = 0;
  int red = 0;
  double* pb = nullptr;
  const GridDev& g = a.g;
  const long long gtid = dealt_tid();
  const long long gthreads = (long long)gridDim.x * blockDim.x;
  // ---- set-up: y = v_0, v_1 .. v_p for every species (reads every species'
  // fields before any is overwritten)
  double sums[2][4] = {{0.0, 0.0, 0.0, 0.0}, {0.0, 0.0, 0.0, 0.0}};
  // MODE_STAGE: which fields' F values the stage needs
  bool need[4] = {false, false, false, false};
  if (a.mode == MODE_STAGE)
    for (int i = 0; i < 4; ++i)
      for (int j = 0; j < 3; ++j) need[i] = need[i] || a.stage.coef[j][i] != 0.0;
  // the group lists of the species on the quad path (built once per domain)
  for (int s = 0; s < a.nspecies; ++s) {
    if (threadIdx.x == 0) {
      c.nq_sp[s] = 0;
      c.wb_done[s] = 0;
    }
    __syncthreads();
    if (use_quads<T, N>(a.sp[s], g, *a.sp[s].ncomp) && !ensure_quads<T, N>(a, a.sp[s], s, *a.sp[s].ncomp, c, bar, red))
      return;
  }
  for (int s = 0; s < a.nspecies; ++s) {
    const SpeciesDev<T>& S = a.sp[s];
    const int ncomp = *S.ncomp;
    Acc<double> acc, acc1, acc2, acc3;
    if constexpr (sizeof(T) == 4) {
      if (c.nq_sp[s] > 0 && a.mode == MODE_ETD2 && a.nspecies == 1 && !a.ms3 && !S.src && !S.bco) {
        double q3[3];
        quad_setup_etd2(a, S, c.nq_sp[s], gtid, gthreads, q3);
        sums[s][0] = q3[0];
        sums[s][1] = q3[1];
        sums[s][2] = q3[2];
        sums[s][3] = 0.0;
        continue;
      }
    }
    // the other modes: norms of the stored values (FP32 contexts: error-free
    // FP32 pairs, no FP64 work)
    Acc<T> at, at1, at2, at3;
    if (a.mode == MODE_STAGE) {
      // a stage of ETD3RK / ETD4RK: F of each needed field (with the other
      // species' same field, masked to its computational set); one point per
      // thread (register bound)
      node_loop<1>(gtid, gthreads, ncomp, S.idx, [&](const auto& kk, const auto& pp) {
        if (pp[0] < 0) return;
        const long long k = kk[0], p = pp[0];
        double Fi[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          if (!need[i]) continue;
          const double ui = i == 0 ? S.u[p] : S.stg[i - 1][p];
          double other = 0.0;
          if (a.nspecies == 2) {
            const SpeciesDev<T>& O = a.sp[1 - s];
            if ((O.kind[p] & 3) == K_COMP) other = i == 0 ? O.u[p] : O.stg[i - 1][p];
          }
          Fi[i] = s == 0 ? reaction(a.reaction, a.rp, 0, ui, other) : reaction(a.reaction, a.rp, 1, other, ui);
        }
        const int f0 = a.stage.v0_field;
        const double y = f0 == 0 ? S.u[p] : S.stg[f0 - 1][p];
        double vv[3];
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          double t = 0.0;
#pragma unroll
          for (int i = 0; i < 4; ++i) t = fma(a.stage.coef[j][i], Fi[i], t);
          vv[j] = a.dt * t;
        }
        S.Yc[k] = y;
        S.Yg[p] = (T)y;
        S.V1c[k] = (T)vv[0];
        S.V2c[k] = (T)vv[1];
        if (a.p == 3) S.V3c[k] = (T)vv[2];
        acc.add(y, y);
        acc1.add(vv[0], vv[0]);
        acc2.add(vv[1], vv[1]);
        acc3.add(vv[2], vv[2]);
      });
    } else {
      node_loop_sized<T>(gtid, gthreads, ncomp, S.idx, [&](const auto& kk, const auto& pp) {
        constexpr int U = NL_U(kk);
        double y[U], v1[U], v2[U], v3[U];
#pragma unroll
        for (int q = 0; q < U; ++q) {
          if (pp[q] < 0) continue;
          const long long p = pp[q];
          v3[q] = 0.0;
          if (a.mode == MODE_GIVEN) {
            y[q] = a.given[0][p];
            v1[q] = a.given[1][p];
            v2[q] = a.given[2][p];
            if (a.p == 3) v3[q] = a.given[3][p];
          } else if (a.mode == MODE_ADJ_LAMBDA) {
            y[q] = a.given[0][p];
            v1[q] = 0.0;
            v2[q] = 0.0;
          } else if (a.mode == MODE_EXPLICIT || a.mode == MODE_ADJ_Y) {
            const double u = a.given[0][p], um = a.given[1][p];
            const double F = reaction(a.reaction, a.rp, 0, u, 0.0);
            const double Fm = reaction(a.reaction, a.rp, 0, um, 0.0);
            y[q] = u;
            v1[q] = a.dt * F;
            v2[q] = a.dt * (F - Fm);
          } else {
            // MODE_ETD2 (v2 = 0 for ETD1), or the second ETD2RK stage MODE_RK2
            // (u holds a_n, F_prev holds F_n: v0 = v1 = 0, v2 = dt (F(a_n) - F_n))
            const double u = S.u[p];
            double other = 0.0;
            if (a.nspecies == 2) {
              const SpeciesDev<T>& O = a.sp[1 - s];
              other = (O.kind[p] & 3) == K_COMP ? O.u[p] : 0.0;
            }
            double F = s == 0 ? reaction(a.reaction, a.rp, 0, u, other) : reaction(a.reaction, a.rp, 1, other, u);
            if (S.src || S.bco) F += extra_F<T, N>(S, kk[q], p);
            const unsigned fv = S.fvalid[p];
            const double Fp = (fv & 1u) ? S.Fprev[p] : F;
            // multistep ETD3 with both earlier values: F_{n-2}
            const bool three = a.ms3 && (fv & 2u);
            const double Fpp = three ? S.Fprev2[p] : Fp;
            if (a.mode == MODE_ETD2) {
              // F_{n-2} <- F_{n-1} <- F_n in place: only this thread reads
              // this species' history at p (the other species reads u)
              if (a.ms3 && (fv & 1u)) S.Fprev2[p] = Fp;
              S.Fprev[p] = F;
              S.fvalid[p] = a.ms3 ? (uint8_t)(1u | ((fv & 1u) << 1)) : (uint8_t)1;
            }
            const bool rk2 = a.mode == MODE_RK2;
            y[q] = rk2 ? 0.0 : u;
            v1[q] = rk2 ? 0.0 : a.dt * F;
            // ETD3 from two earlier values, else ETD2 from one (ETD1: none)
            v2[q] = a.etd1 ? 0.0 : three ? a.dt * (1.5 * F - 2.0 * Fp + 0.5 * Fpp) : a.dt * (F - Fp);
            if (three) v3[q] = a.dt * (F - 2.0 * Fp + Fpp);
          }
        }
#pragma unroll
        for (int q = 0; q < U; ++q) {
          if (pp[q] < 0) continue;
          const long long k = kk[q], p = pp[q];
          const T yt = to_T<T>(y[q]), v1t = to_T<T>(v1[q]), v2t = to_T<T>(v2[q]);
          S.Yc[k] = y[q];
          S.Yg[p] = yt;
          S.V1c[k] = v1t;
          S.V2c[k] = v2t;
          if (a.mode == MODE_ADJ_LAMBDA) S.V[p] = yt;  // V_0 = lambda
          at.add(yt, yt);
          at1.add(v1t, v1t);
          at2.add(v2t, v2t);
          if (a.p == 3) {
            const T v3t = to_T<T>(v3[q]);
            S.V3c[k] = v3t;
            at3.add(v3t, v3t);
          }
        }
      });
    }
    sums[s][0] = acc.value() + at.value();
    sums[s][1] = acc1.value() + at1.value();
    sums[s][2] = acc2.value() + at2.value();
    sums[s][3] = acc3.value() + at3.value();
  }
  // |y(0)|^2, |v_1|^2, |v_2|^2, |v_3|^2 per species (one grid barrier each;
  // two block sums of two quantities into the halves of one partial buffer)
  double tot[2][4];
  for (int s = 0; s < a.nspecies; ++s) {
    double v01[2] = {sums[s][0], sums[s][1]}, v23[2] = {sums[s][2], sums[s][3]};
    pb = part_buf(a.part, red);
    block_partials<2>(v01, pb);
    block_partials<2>(v23, pb + 2 * MAX_BLOCKS);
    if (!grid_barrier(a.st, bar, 1)) return;
    double t01[2], t23[2];
    grid_totals<2>(pb, t01);
    grid_totals<2>(pb + 2 * MAX_BLOCKS, t23);
    tot[s][0] = t01[0];
    tot[s][1] = t01[1];
    tot[s][2] = t23[0];
    tot[s][3] = t23[1];
  }
  for (int s = 0; s < a.nspecies; ++s) {
    const double vscale = fmax(fmax(sqrt(tot[s][1]), sqrt(tot[s][2])), sqrt(tot[s][3]));
    if (!phipm_species<T, N, ADJ>(a, a.sp[s], s, c, bar, red, tot[s][0], vscale)) return;
  }
  if (!grid_barrier(a.st, bar, 2)) return;
  // the adjoint modes' outputs are written by the species loop
  if (ADJ && (a.mode == MODE_ADJ_LAMBDA || a.mode == MODE_ADJ_Y)) return;
  // ---- write back: new values at computational points, 0 elsewhere
  for (int s = 0; s < a.nspecies; ++s) {
    const SpeciesDev<T>& S = a.sp[s];
    const int ncomp = *S.ncomp;
    const bool add = a.mode == MODE_RK2;  // u <- a_n + the second stage's result
    // a stage of ETD3RK / ETD4RK may write a stage field instead of u
    const int outf = a.mode == MODE_STAGE ? a.stage.out_field : 0;
    double* const dst = outf == 0 ? S.u : S.stg[outf - 1];
    if (!c.wb_done[s]) node_loop_sized<T>(gtid, gthreads, ncomp, S.idx, [&](const auto& kk, const auto& pp) {
      constexpr int U = NL_U(kk);
      double y[U], b[U];
#pragma unroll
      for (int q = 0; q < U; ++q) {
        if (pp[q] < 0) continue;
        y[q] = __ldcg(S.Yc + kk[q]);
        b[q] = add ? S.u[pp[q]] : 0.0;
      }
#pragma unroll
      for (int q = 0; q < U; ++q)
        if (pp[q] >= 0) dst[pp[q]] = add ? b[q] + y[q] : y[q];
    });
    if (outf != 0) continue;  // stage fields are read at computational points only
    // Off the computational set: u = 0 and the validity bits cleared (the
    // set-up wrote those of the computational points).  A lane per block of
    // 16 consecutive nodes, consecutive blocks on consecutive lanes: one
    // 16-byte load of their classes, 16-byte zero stores of u by pairs
    // where u is 16-byte aligned, one 16-byte read-modify-write of their
    // validity bytes; a block of computational nodes only is skipped.  Per
    // class word, t has byte i = 1 when node i is not computational (class
    // bits x = 2 ^ (kind & 3) nonzero).  The last size % 16 nodes, or every
    // node if the class or validity array is not 16-byte aligned, one per lane.
    const bool u16 = (reinterpret_cast<uintptr_t>(S.u) & 15u) == 0;
    const bool b16 = ((reinterpret_cast<uintptr_t>(S.kind) | reinterpret_cast<uintptr_t>(S.fvalid)) & 15u) == 0;
    const long long nblk = b16 ? g.size >> 4 : 0;
    const long long ptid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    for (long long b = ptid; b < nblk; b += gthreads) {
      const uint4 kv = __ldg(reinterpret_cast<const uint4*>(S.kind) + b);
      const unsigned kw[4] = {kv.x, kv.y, kv.z, kv.w};
      unsigned t[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const unsigned x = (kw[j] & 0x03030303u) ^ 0x02020202u;
        t[j] = (x | (x >> 1)) & 0x01010101u;
      }
      if ((t[0] | t[1] | t[2] | t[3]) == 0u) continue;
      double* ub = S.u + (b << 4);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        if (t[j] == 0u) continue;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const bool n0 = (t[j] >> (16 * h)) & 1u, n1 = (t[j] >> (16 * h + 8)) & 1u;
          double* up = ub + 4 * j + 2 * h;
          if (n0 && n1 && u16) {
            *reinterpret_cast<double2*>(up) = make_double2(0.0, 0.0);
          } else {
            if (n0) up[0] = 0.0;
            if (n1) up[1] = 0.0;
          }
        }
      }
      if (a.mode == MODE_ETD2) {
        uint4* vp = reinterpret_cast<uint4*>(S.fvalid) + b;
        uint4 ov = __ldcg(vp);
        ov.x &= ~(t[0] * 0xffu);
        ov.y &= ~(t[1] * 0xffu);
        ov.z &= ~(t[2] * 0xffu);
        ov.w &= ~(t[3] * 0xffu);
        __stcg(vp, ov);
      }
    }
    for (long long p = (nblk << 4) + ptid; p < g.size; p += gthreads) {
      if ((__ldg(S.kind + p) & 3) != K_COMP) {
        S.u[p] = 0.0;
        if (a.mode == MODE_ETD2) S.fvalid[p] = 0;
      }
    }
  }
}

// The kernels of one precision and CTA size, for the entries below.
template <typename T, int NT>
PhipmKernels phipm_kernels() {
  PhipmKernels k;
  k.fn[0][0] = (void*)phipm_kernel<T, 2, false, NT>;
  k.fn[0][1] = (void*)phipm_kernel<T, 2, true, NT>;
  k.fn[1][0] = (void*)phipm_kernel<T, 3, false, NT>;
  k.fn[1][1] = (void*)phipm_kernel<T, 3, true, NT>;
  k.fn[2][0] = (void*)phipm_kernel<T, 4, false, NT>;
  k.fn[2][1] = (void*)phipm_kernel<T, 4, true, NT>;
  k.nt = NT;
  k.adj_smem = adj_smem(NT);
  k.load_consts = load_inv_fact;
  return k;
}

}  // namespace etd
