// Shared device utilities: grid descriptor, node kinds, status flags, the
// bounded grid barrier, deterministic block/grid reductions, FP32
// error-free accumulation.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace etd {

constexpr int MAXD = 4;
constexpr int MAX_M = 61;           // largest Krylov basis (m + p + 1 <= 64)
constexpr int MAX_BLOCKS = 1024;    // partial-sum slots per reduction quantity

// Unsigned division of n < 2^31 by a divisor d >= 1 fixed at set-up, on the
// integer pipe: with s = ceil(log2 d) and m = floor(2^32 (2^s - d) / d) + 1,
// n / d = (umulhi(m, n) + n) >> s (the round-up method of Granlund &
// Montgomery 1994; the sum cannot overflow for n < 2^31).  A division by a
// runtime divisor otherwise goes through float conversions, which GB300
// issues at its FP64 rate.
struct FastDiv {
  unsigned m;
  int s;
  __host__ __device__ FastDiv() : m(1u), s(0) {}
  __host__ explicit FastDiv(unsigned d) : s(0) {
    while ((1ull << s) < (unsigned long long)d) ++s;
    m = (unsigned)(((1ull << 32) * ((1ull << s) - d)) / d + 1ull);
  }
  __device__ __forceinline__ unsigned div(unsigned n) const { return (__umulhi(m, n) + n) >> s; }
};

struct GridDev {
  int ndim;
  int n[MAXD];
  long long stride[MAXD];
  long long size;
  double lo[MAXD];
  double h;
  FastDiv sdiv[MAXD];  // by stride[d]
  // bit-plane geometry of the level-set work sets (rows along the last axis
  // padded to 32-bit words): by the words per row and by the row strides
  // stride[d] / n[ndim - 1] of the other axes
  FastDiv wdiv, rdiv[MAXD];
};

// Fills the FastDiv members of g from ndim, n and stride (host side).
inline void grid_divisors(GridDev& g) {
  const long long nx = g.n[g.ndim - 1];
  for (int d = 0; d < g.ndim; ++d) {
    g.sdiv[d] = FastDiv((unsigned)g.stride[d]);
    g.rdiv[d] = FastDiv((unsigned)(g.stride[d] / nx > 0 ? g.stride[d] / nx : 1));
  }
  g.wdiv = FastDiv((unsigned)((nx + 31) / 32));
}

// node class in the low two bits of a kind byte
enum : uint8_t { K_OUT = 0, K_GHOST = 1, K_COMP = 2 };

// device status word bits (DevStatus::err)
enum : int {
  ERRF_DOMAIN = 1,     // an inside node within 3 nodes of the box edge
  ERRF_TIMEOUT = 2,    // a bounded device wait gave up
  ERRF_KRYLOV = 4,     // tolerance not met at tau_min
  ERRF_NONFINITE = 8,  // NaN / Inf in a reduction
  ERRF_CAPACITY = 16,  // a list or trace outgrew its buffer
  ERRF_UNSUPPORTED = 32,  // boundary data at a case-3 face with N >= 3
};

struct DevStatus {
  int err;
  int nclamp;           // ghost weights clamped to [0, 1]
  int timeout_site;
  int pad;
  double gersh[2];      // Gershgorin bound of C per species (max row sum of |C|)
  unsigned int barrier; // grid-barrier arrival counter (reset before each cooperative launch)
  unsigned int pad2;
  unsigned long long wait_ns;  // limit of every device wait in ns (0: BARRIER_LIMIT_NS)
};

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void red_release_add_u32(unsigned* p, unsigned v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid-wide barrier for a cooperative launch: a monotonically increasing
// arrival counter (reset to 0 before the launch).  Barrier number `k`
// (1-based, identical in every CTA) completes when the counter reaches
// k * gridDim.x.  Ordering: __syncthreads orders the CTA's accesses before
// thread 0's gpu-scope release add; the waiting thread's gpu-scope acquire
// load and the following __syncthreads order them before every later access
// of its CTA.  Every wait is bounded: from the first unsuccessful poll, the
// clock and the status word are checked every 16 polls (every poll when the
// limit is below 1 ms); after st->wait_ns (default BARRIER_LIMIT_NS, ~1 s)
// the status word gets ERRF_TIMEOUT and the call returns false, after which
// the kernel must return.  A CTA that sees another CTA's ERRF_TIMEOUT stops
// waiting too, so every CTA returns.
constexpr unsigned long long BARRIER_LIMIT_NS = 1000000000ull;
constexpr unsigned long long BARRIER_SHORT_NS = 1000000ull;

__device__ __forceinline__ bool grid_barrier(DevStatus* st, unsigned& k, int site) {
  __shared__ int s_ok;
  ++k;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    red_release_add_u32(&st->barrier, 1u);
    // the limit's load is issued before the first poll and has returned by
    // the time that poll's result is known: it adds no latency
    unsigned long long w = *((volatile unsigned long long*)&st->wait_ns);
    const unsigned target = k * gridDim.x;
    unsigned long long t0 = 0;
    unsigned polls = 0;
    while (ld_acquire_u32(&st->barrier) < target) {
      // an opaque update of w: its tests stay after the poll instead of
      // being hoisted above the first one (which would wait for the load)
      asm volatile("" : "+l"(w));
      if (polls == 0) t0 = global_ns();
      ++polls;
      const bool short_limit = w != 0ull && w < BARRIER_SHORT_NS;
      if (short_limit || (polls & 15u) == 0u) {
        if (global_ns() - t0 >= (w != 0ull ? w : BARRIER_LIMIT_NS)) {
          atomicOr(&st->err, ERRF_TIMEOUT);
          atomicExch(&st->timeout_site, site);
          ok = 0;
          break;
        }
        // another CTA gave up: stop waiting for it
        if (*((volatile int*)&st->err) & ERRF_TIMEOUT) { ok = 0; break; }
      }
    }
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// Index of this thread in the node loops: 32-index chunks dealt round-robin
// over the CTAs (chunk j to warp j / gridDim of CTA j % gridDim), a
// bijection onto [0, gridDim * blockDim).  A problem smaller than the grid
// then spreads over every SM instead of filling the first CTAs, whose FP64
// pipes are shared by all of their warps.
__device__ __forceinline__ long long dealt_tid() {
  return (long long)(threadIdx.x & 31) + 32ll * ((long long)blockIdx.x + (long long)gridDim.x * (threadIdx.x >> 5));
}

// ---------------------------------------------------------------- reductions
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Staging area of the block reductions: up to 3 quantities of up to
// RED_MAX_NT threads, one instance per kernel (a translation unit may raise
// the thread count by defining ETD_RED_MAX_NT first).
#ifndef ETD_RED_MAX_NT
#define ETD_RED_MAX_NT 512
#endif
constexpr int RED_MAX_NQ = 3, RED_MAX_NT = ETD_RED_MAX_NT;
__device__ __forceinline__ double* red_stage() {
  __shared__ double s_stage[RED_MAX_NQ * RED_MAX_NT];
  return s_stage;
}

// Sum of NQ per-thread values over the block (blockDim.x <= RED_MAX_NT); thread 0
// of warp q writes the block's total of quantity q to
// part[q * MAX_BLOCKS + blockIdx.x].  The values go through shared memory
// and warp q sums quantity q (lane-strided, then a warp tree): FP64 adds run
// on NQ warps instead of every warp's shuffle tree, and the order is fixed.
template <int NQ>
__device__ __forceinline__ void block_partials(const double (&v)[NQ], double* part) {
  static_assert(NQ <= RED_MAX_NQ, "too many quantities");
  double* st = red_stage();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nt = blockDim.x;
#pragma unroll
  for (int q = 0; q < NQ; ++q) st[q * RED_MAX_NT + threadIdx.x] = v[q];
  __syncthreads();
  if (wid < NQ) {
    const double* row = st + wid * RED_MAX_NT;
    double x0 = 0.0, x1 = 0.0;
    for (int t = lane; t < nt; t += 64) {
      x0 += row[t];
      if (t + 32 < nt) x1 += row[t + 32];
    }
    const double x = warp_sum(x0 + x1);
    if (lane == 0) part[wid * MAX_BLOCKS + blockIdx.x] = x;
  }
  __syncthreads();
}

// After a grid barrier: every CTA sums the per-block partials in the same
// fixed order (warp q sums quantity q: lane-strided, then a warp tree), so
// every CTA obtains the same bits.  Result broadcast to the whole block.
template <int NQ>
__device__ __forceinline__ void grid_totals(const double* part, double (&out)[NQ]) {
  __shared__ double s_tot[NQ];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (wid < NQ) {
    double x = 0.0;
    for (int b = lane; b < (int)gridDim.x; b += 32) x += __ldcg(part + wid * MAX_BLOCKS + b);
    x = warp_sum(x);
    if (lane == 0) s_tot[wid] = x;
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < NQ; ++q) out[q] = s_tot[q];
  __syncthreads();
}

// FP32 error-free accumulation of products (TwoProduct via fma + TwoSum,
// Ogita, Rump & Oishi 2005): s + c carries the sum to about twice single
// precision.  Intrinsics keep the compiler from contracting or reassociating.
struct Dot2f {
  float s, c;
  __device__ __forceinline__ Dot2f() : s(0.f), c(0.f) {}
  __device__ __forceinline__ void add(float a, float b) {
    float p = __fmul_rn(a, b);
    float pe = __fmaf_rn(a, b, -p);
    float t = __fadd_rn(s, p);
    float z = __fsub_rn(t, s);
    float e = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(p, z));
    s = t;
    c = __fadd_rn(c, __fadd_rn(e, pe));
  }
  __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

template <typename T>
struct Acc;
template <>
struct Acc<double> {
  double s = 0.0;
  __device__ __forceinline__ void add(double a, double b) { s = fma(a, b, s); }
  __device__ __forceinline__ double value() const { return s; }
};
template <>
struct Acc<float> {
  Dot2f d;
  __device__ __forceinline__ void add(float a, float b) { d.add(a, b); }
  __device__ __forceinline__ double value() const { return d.value(); }
};

}  // namespace etd
