// Level-set step of the free-boundary algorithm (Sec. 4.3, Algorithm Steps
// 1-2; Stefan condition of Eq. free), as one persistent cooperative kernel.
//
// Local level set (after Peng, Merriman, Osher, Zhao & Kang 1999): phi is
// clamped to [-G, G], G = 6h; the update set T is {|phi| < G} grown by one
// node along every axis; the work list holds T grown by three more nodes (the
// reach of the WENO5 stencil).  Out-of-box neighbours repeat the edge value.
//
// Phases of levelset_advance:
//   1. extension of u (Aslam 2004 quadratic normal extrapolation):
//      n = grad phi/|grad phi| (central; |grad phi| floored at 1e-12);
//      u_n = n.grad u on computational points whose neighbours are
//      computational (valid1), u_nn = n.grad u_n on valid2; three
//      pseudo-time sweeps q_tau + n.grad q = s (first-order upwind along n,
//      step h/(2 sqrt N), ceil(12 sqrt N) steps) for u_nn (s = 0) on T minus
//      valid2, u_n (s = u_nn) on T minus valid1, u (s = u_n) on T minus the
//      computational points;
//   2. Stefan speed at every node of T: x_G = x - phi n,
//      V = mu max(0, (4 u(x_G - h n) - u(x_G - 2h n)) / (2h)), N-linear
//      interpolation of the extended u (points clamped to the box);
//   3. phi_t + V |grad phi| = 0: Godunov Hamiltonian on HJ-WENO5 one-sided
//      derivatives (Jiang & Peng 2000, eps = 1e-6), Shu-Osher TVD-RK3,
//      max(1, ceil(dt max V N / (0.5 h))) substeps, then clamp;
//   4. optionally reinitialisation phi_t + S(phi_0)(|grad phi| - 1) = 0,
//      S = phi_0 / sqrt(phi_0^2 + h^2) (Sussman, Smereka & Osher 1994), same
//      spatial scheme upwinded by the sign of S, TVD-RK3 with pseudo-step
//      0.5 h / sqrt N, ceil(12 sqrt N) steps, on a work set rebuilt from the
//      advected phi, then clamp.
#include <cmath>

#include "common.cuh"
#include "levelset.cuh"

namespace etd {

constexpr int LS_NT = 512;
constexpr double BAND = 6.0;
constexpr double WENO_EPS = 1e-6;
constexpr double GRAD_FLOOR = 1e-12;

enum : uint8_t {
  F_T = 1, F_T1 = 2, F_T2 = 4, F_T3 = 8, F_V0 = 16, F_V1 = 32, F_V2 = 64, F_S = 128
};
enum : int { LS_ADVANCE = 0, LS_PREPARE = 1 };

// Bit planes of the work-set build: one bit per node, rows along the last
// (contiguous) axis padded to whole 32-bit words.
enum : int { P_S = 0, P_T, P_T1, P_T2, P_T3, P_V0, P_V1, P_V2, NPLANES };

struct BitGeo {
  int nx;        // nodes per row (last axis)
  int W;         // words per row
  long long R;   // rows
  long long nw;  // words per plane
};

__host__ __device__ __forceinline__ BitGeo bit_geo(const GridDev& g) {
  BitGeo b;
  b.nx = g.n[g.ndim - 1];
  b.W = (b.nx + 31) / 32;
  b.R = g.size / b.nx;
  b.nw = b.R * b.W;
  return b;
}

struct LsArgs {
  GridDev g;
  LevelsetBufs b;
  DevStatus* st;
  const uint8_t* kind;
  double* phi;
  double* u;
  double dt;
  double mu;
  int mode;
  int reinit;
  int mixed;  // FP32 WENO/Godunov arithmetic away from the interface
};

LevelsetBufs levelset_carve(const GridDev& g, const std::function<char*(size_t)>& take) {
  const size_t G = (size_t)g.size;
  LevelsetBufs b;
  b.lflag = (uint8_t*)take(G);
  b.bits = (uint32_t*)take((size_t)NPLANES * (size_t)bit_geo(g).nw * sizeof(uint32_t));
  b.list = (int*)take(G * sizeof(int));
  b.slist = (int*)take(G * sizeof(int));
  b.lcoord = (ushort4*)take(G * sizeof(ushort4));
  b.count = (int*)take(4 * sizeof(int));
  b.cta_count = (int*)take(MAX_BLOCKS * sizeof(int));
  b.sw = (int*)take(8 * sizeof(int));
  b.vmax = (double*)take(sizeof(double));
  b.nsub = (int*)take(sizeof(int));
  b.info = (int*)take(8 * sizeof(int));
  b.nrm = (double*)take((size_t)g.ndim * G * sizeof(double));
  b.V = (double*)take(G * sizeof(double));
  b.S0 = (double*)take(G * sizeof(double));
  for (int i = 0; i < 6; ++i) b.q[i] = (double*)take(G * sizeof(double));
  b.p1 = (double*)take(G * sizeof(double));
  b.p2 = (double*)take(G * sizeof(double));
  b.gidx = (int*)take(G * sizeof(int));
  return b;
}

// axis indices of node p (grids hold fewer than 2^31 nodes: 32-bit division)
template <int N>
__device__ __forceinline__ void coords(const GridDev& g, long long p, int* ix) {
  unsigned rem = (unsigned)p;
#pragma unroll
  for (int d = 0; d < N; ++d) {
    const unsigned st = (unsigned)g.stride[d];
    const unsigned q = g.sdiv[d].div(rem);
    ix[d] = (int)q;
    rem -= q * st;
  }
}

template <int N>
__device__ __forceinline__ void unpack(ushort4 c, int* ix) {
  ix[0] = c.x;
  ix[1] = c.y;
  if (N > 2) ix[2] = c.z;
  if (N > 3) ix[3] = c.w;
}

__device__ __forceinline__ long long nbr(const GridDev& g, long long p, const int* ix, int d, int k) {
  int i = ix[d] + k;
  i = i < 0 ? 0 : (i > g.n[d] - 1 ? g.n[d] - 1 : i);
  return p + (long long)(i - ix[d]) * g.stride[d];
}

// ------------------------------------------------------------------ WENO5
// Both one-sided HJ-WENO5 derivatives at a node from six consecutive
// differences q_0..q_5 (q_k = f_{i+k-2} - f_{i+k-3}, optionally divided by
// h), in the equivalent form of Jiang & Peng (2000): with e_k = q_{k+1} - q_k,
//   d- = c - Phi(e0, e1, e2, e3),   d+ = c + Phi(e4, e3, e2, e1),
//   c  = (7 (q2 + q3) - (q1 + q4)) / 12,
//   Phi(a,b,c,d) = w0 (a - 2b + c) / 3 + (w2 - 1/2)(b - 2c + d) / 6,
// w_k = alpha_k / sum alpha, alpha = (1, 6, 3) / (eps' + I_k)^2 with
// I_0 = (13/3)(a-b)^2 + (a-3b)^2, I_1 = (13/3)(b-c)^2 + (b+c)^2,
// I_2 = (13/3)(c-d)^2 + (3c-d)^2.  I_k is 4 times the smoothness indicator
// of the usual weighted form with eps = 1e-6 (on divided differences), so
// eps' = 4 eps (times h^2 on undivided ones) gives the same weights; the
// usual weighted sum of the three candidate stencils is the same number up
// to rounding.
//
// The terms are kept scaled by 12, which leaves no constant factor to
// multiply by: with d_k = (eps' + I_k)^2, A = d1 d2, B = d0 d2, C = d0 d1,
// W = A + 6B + 3C (the sum of the alphas times d0 d1 d2) and
// V = 3C - A - 6B (= 2 W (w2 - 1/2) with w2 the normalised weight),
//   12 Phi = 4 (A X + V Y / 4) / W,   X = (a-b) - (b-c),  Y = b - 2c + d,
//   12 c   = 7 (q2 + q3) - (q1 + q4).
// The two sides share the differences, 12 c, the squares (a-b)^2 of common
// pairs and Y (the same on both).
template <typename C>
struct Weno5Terms {
  C cen;     // 12 c
  C num[2];  // A X + V Y / 4 of the minus and plus sides
  C W[2];
};

template <typename C>
__device__ __forceinline__ Weno5Terms<C> weno5_terms(const C* q, C epsw) {
  constexpr C k13 = C(13.0 / 3.0);
  const C e0 = q[1] - q[0], e1 = q[2] - q[1], e2 = q[3] - q[2], e3 = q[4] - q[3], e4 = q[5] - q[4];
  Weno5Terms<C> t;
  t.cen = fma(C(7), q[2] + q[3], -(q[1] + q[4]));
  // minus side (a,b,c,d) = (e0,e1,e2,e3): third differences (ta, tb, tc);
  // plus side (e4,e3,e2,e1): (td, -tc, -tb)
  const C ta = e0 - e1, tb = e1 - e2, tc = e2 - e3, td = e4 - e3;
  const C sa = ta * ta, sb = tb * tb, sc = tc * tc, sd = td * td;
  const C um0 = fma(C(-3), e1, e0), um1 = e1 + e2, um2 = fma(C(3), e2, -e3);
  const C up0 = fma(C(-3), e3, e4), up1 = e3 + e2, up2 = fma(C(3), e2, -e1);
  const C Y4 = C(0.25) * (tb - tc);
#pragma unroll
  for (int side = 0; side < 2; ++side) {
    // eps' + I_k
    const C s0 = side == 0 ? fma(k13, sa, fma(um0, um0, epsw)) : fma(k13, sd, fma(up0, up0, epsw));
    const C s1 = side == 0 ? fma(k13, sb, fma(um1, um1, epsw)) : fma(k13, sc, fma(up1, up1, epsw));
    const C s2 = side == 0 ? fma(k13, sc, fma(um2, um2, epsw)) : fma(k13, sb, fma(up2, up2, epsw));
    const C X = side == 0 ? ta - tb : td + tc;
    const C d0 = s0 * s0, d1 = s1 * s1, d2 = s2 * s2;
    const C A = d1 * d2, B = d0 * d2, Cc = d0 * d1;
    const C AB = fma(C(6), B, A);
    t.W[side] = fma(C(3), Cc, AB);
    t.num[side] = fma(A, X, fma(C(3), Cc, -AB) * Y4);
  }
  return t;
}

// max(a, b, 0) of doubles on the integer pipe: as signed 64-bit integers,
// the bit patterns of non-negative doubles order like their values and those
// of negative ones lie below that of +0.
__device__ __forceinline__ double max0(double a, double b) {
  const long long m = max(__double_as_longlong(a), __double_as_longlong(b));
  return __longlong_as_double(max(m, 0LL));
}
__device__ __forceinline__ float max0(float a, float b) { return fmaxf(fmaxf(a, b), 0.f); }

// 12 max(d-, -d+, 0) (outward) or its mirror image, with r_s = 4 / W_s.
// outward: max(max(d-, 0)^2, min(d+, 0)^2) = max(d-, -d+, 0)^2 (a square is
// monotone on the non-negatives); inward: the mirror image.  Exact sign
// flips and no branch, so that no work of the other case is issued
// predicated off.
template <typename C>
__device__ __forceinline__ C weno5_upwind(const Weno5Terms<C>& t, C r0, C r1, bool positive) {
  const C dm = fma(-t.num[0], r0, t.cen), dp = fma(t.num[1], r1, t.cen);
  return max0(positive ? dm : -dm, positive ? -dp : dp);
}

// Constants of the Godunov evaluations of one grid, computed once.
struct WenoK {
  double epsw;     // eps' on undivided FP64 differences: 4 eps h^2
  double inv_h;    // 1 / h
  double inv_h12;  // 1 / (12 h): the scale of the FP64 result
};

__device__ __forceinline__ WenoK weno_k(double h) {
  WenoK k;
  k.epsw = 4.0 * WENO_EPS * h * h;
  k.inv_h = 1.0 / h;
  k.inv_h12 = 1.0 / (12.0 * h);
  return k;
}

// The seven values along axis d as six differences: FP64 undivided, or
// FP32-mixed (values rounded to FP32, differences divided by h in FP32; an
// eps' scaled by h^2 would leave the FP32 normal range).
template <typename C, int N>
__device__ __forceinline__ void axis_diffs(const GridDev& g, const double* __restrict__ src, long long p, const int* ix,
                                           int d, double inv_h, C* q) {
  double f[7];
#pragma unroll
  for (int k = -3; k <= 3; ++k) f[k + 3] = __ldcg(src + nbr(g, p, ix, d, k));
  if constexpr (sizeof(C) == 8) {
#pragma unroll
    for (int k = -2; k <= 3; ++k) q[k + 2] = f[k + 3] - f[k + 2];
  } else {
    const C ih = C(inv_h);
    C fc[7];
#pragma unroll
    for (int k = 0; k < 7; ++k) fc[k] = C(f[k]);
#pragma unroll
    for (int k = -2; k <= 3; ++k) q[k + 2] = (fc[k + 3] - fc[k + 2]) * ih;
  }
}

// One axis of the Godunov |grad phi| (godunov, below), scaled by 12: the
// upwind value from the WENO5 pair on the seven values along axis d.
template <typename C, int N>
__device__ __forceinline__ C godunov_mx(const GridDev& g, const double* __restrict__ src, long long p, const int* ix,
                                        int d, bool positive, const WenoK& k) {
  C q[6];
  axis_diffs<C, N>(g, src, p, ix, d, k.inv_h, q);
  const C epsw = sizeof(C) == 8 ? C(k.epsw) : C(4.0 * WENO_EPS);
  const Weno5Terms<C> t = weno5_terms<C>(q, epsw);
  if constexpr (sizeof(C) == 8) {
    // W_s >= 10 eps'^4 (> 1e-70 for h > 1e-6) and for |q| < 1e18 the
    // product stays finite: it neither underflows nor overflows in FP64
    const C r = C(4) / (t.W[0] * t.W[1]);
    return weno5_upwind<C>(t, t.W[1] * r, t.W[0] * r, positive);
  } else {
    return weno5_upwind<C>(t, C(4) / t.W[0], C(4) / t.W[1], positive);
  }
}

// 4 / (W0 W1) of every axis.  When each product lies within 2^(+-1000/N)
// one division serves all axes (prefix and suffix products of the others);
// otherwise one division per axis.
template <int N>
__device__ __forceinline__ void weno5_recips(const Weno5Terms<double>* t, double* r) {
  constexpr unsigned LIM = 1000 / N;
  double D[N];
  bool shared = true;
#pragma unroll
  for (int d = 0; d < N; ++d) {
    D[d] = t[d].W[0] * t[d].W[1];
    const unsigned e = (unsigned)__double2hiint(D[d]) >> 20;  // biased exponent (D > 0)
    shared = shared && e - (1023u - LIM) <= 2u * LIM;
  }
  if (shared) {
    double pre[N];
    pre[0] = 1.0;
#pragma unroll
    for (int d = 1; d < N; ++d) pre[d] = pre[d - 1] * D[d - 1];
    const double rP = 4.0 / (pre[N - 1] * D[N - 1]);
    double suf = 1.0;
#pragma unroll
    for (int d = N - 1; d >= 0; --d) {
      r[d] = (rP * pre[d]) * suf;
      suf *= D[d];
    }
  } else {
#pragma unroll
    for (int d = 0; d < N; ++d) r[d] = 4.0 / D[d];
  }
}

// Godunov |grad phi| at node p from array src; positive: outward motion.
// FP64 (C = double): undivided differences, eps' scaled by h^2, every axis's
// terms first so that one division serves the node, one factor 1/(12 h) at
// the end.  FP32-mixed (C = float): WENO5 and Godunov in FP32, no FP64
// arithmetic (this GPU issues one FP64 warp instruction per ~80 cycles per
// SM sub-partition).
template <typename C, int N>
__device__ double godunov(const GridDev& g, const double* __restrict__ src, long long p, const int* ix,
                          bool positive, const WenoK& k) {
  if constexpr (sizeof(C) == 8) {
    Weno5Terms<double> t[N];
#pragma unroll
    for (int d = 0; d < N; ++d) {
      double q[6];
      axis_diffs<double, N>(g, src, p, ix, d, k.inv_h, q);
      t[d] = weno5_terms<double>(q, k.epsw);
    }
    double r[N];
    weno5_recips<N>(t, r);
    double acc = 0.0;
#pragma unroll
    for (int d = 0; d < N; ++d) {
      const double mx = weno5_upwind<double>(t[d], t[d].W[1] * r[d], t[d].W[0] * r[d], positive);
      acc = fma(mx, mx, acc);
    }
    return sqrt(acc) * k.inv_h12;
  } else {
    float acc = 0.f;
#pragma unroll
    for (int d = 0; d < N; ++d) {
      const float mx = godunov_mx<float, N>(g, src, p, ix, d, positive, k);
      acc = fma(mx, mx, acc);
    }
    return (double)(sqrtf(acc) * (1.f / 12.f));
  }
}

// ------------------------------------------------------------ work lists
struct LsCtx {
  unsigned bar;
  int red;
  long long wlo, whi;  // this CTA's words of the bit planes
};

// valid-node mask of word wi of a row
__device__ __forceinline__ unsigned tail_mask(const BitGeo& bg, int wi) {
  const int left = bg.nx - 32 * wi;
  return left >= 32 ? 0xffffffffu : ((1u << left) - 1u);
}

// |x| < G decided on the bit patterns (G > 0 finite): non-negative doubles
// order like their bits, and NaN compares false
__device__ __forceinline__ bool abs_below(double x, unsigned long long Gbits) {
  return ((unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull) < Gbits;
}

// Planes S (|phi| < G), T, T1, T2, T3 (each the previous dilated by one
// node along every axis) and, with `kind`, V0 (computational), V1, V2 (each
// the previous eroded the same way); out-of-box neighbours repeat the edge
// node.  Then the ordered list of T3 nodes with their axis indices and
// flags.  Returns false if the kernel must stop.
template <int N>
__device__ bool build_work_set(const LsArgs& a, LsCtx& c, bool with_valid, int slot) {
  const GridDev& g = a.g;
  const BitGeo bg = bit_geo(g);
  uint32_t* const pl = a.b.bits;
  const unsigned long long Gbits = (unsigned long long)__double_as_longlong(BAND * g.h);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  // row strides in words and row extents of the first N - 1 axes
  long long rsw[N > 1 ? N - 1 : 1];
  unsigned rstr[N > 1 ? N - 1 : 1];
#pragma unroll
  for (int d = 0; d < N - 1; ++d) {
    rstr[d] = (unsigned)(g.stride[d] / bg.nx);
    rsw[d] = (long long)rstr[d] * bg.W;
  }
  // pass A: a lane per node, UA consecutive words per warp and iteration
  // (their loads issued before any is used; where rows are whole words, a
  // word's nodes are 32 w .. 32 w + 31 and every load is a predicated select)
  constexpr int UA = 8;
  const bool whole = bg.nx == 32 * bg.W;
  for (long long w0 = c.wlo + (long long)wid * UA; w0 < c.whi; w0 += (long long)nwarp * UA) {
    double ph[UA];
    uint8_t kd[UA];
    bool in[UA];
#pragma unroll
    for (int u = 0; u < UA; ++u) {
      const long long w = w0 + u;
      long long p = 32 * w + lane;
      in[u] = w < c.whi;
      if (!whole && in[u]) {
        const unsigned r = g.wdiv.div((unsigned)w);
        const int x = (int)((unsigned)w - r * (unsigned)bg.W) * 32 + lane;
        in[u] = x < bg.nx;
        p = (long long)r * bg.nx + x;
      }
      ph[u] = in[u] ? a.phi[p] : 0.0;
      kd[u] = in[u] && with_valid ? a.kind[p] : (uint8_t)0;
    }
#pragma unroll
    for (int u = 0; u < UA; ++u) {
      const unsigned ws = __ballot_sync(0xffffffffu, in[u] && abs_below(ph[u], Gbits));
      const unsigned wv = __ballot_sync(0xffffffffu, in[u] && (kd[u] & 3) == K_COMP);
      if (lane == 0 && w0 + u < c.whi) {
        pl[P_S * bg.nw + w0 + u] = ws;
        if (with_valid) pl[P_V0 * bg.nw + w0 + u] = wv;
      }
    }
  }
  if (!grid_barrier(a.st, c.bar, 20)) return false;
  // passes B..E: dilation S -> T -> T1 -> T2 -> T3; erosion V0 -> V1 -> V2
  int cnt = 0;
  for (int pass = 0; pass < 4; ++pass) {
    const uint32_t* src = pl + (P_S + pass) * bg.nw;
    uint32_t* dst = pl + (P_T + pass) * bg.nw;
    const bool vpass = with_valid && pass < 2;
    const uint32_t* vsrc = pl + (P_V0 + pass) * bg.nw;
    uint32_t* vdst = pl + (P_V1 + pass) * bg.nw;
    for (long long w = c.wlo + threadIdx.x; w < c.whi; w += blockDim.x) {
      unsigned r = g.wdiv.div((unsigned)w);
      const int wi = (int)((unsigned)w - r * (unsigned)bg.W);
      int ir[N > 1 ? N - 1 : 1];
#pragma unroll
      for (int d = 0; d < N - 1; ++d) {
        ir[d] = (int)g.rdiv[d].div(r);
        r -= (unsigned)ir[d] * rstr[d];
      }
      const unsigned tm = tail_mask(bg, wi);
      const unsigned sv = __ldcg(src + w);
      unsigned any = sv | (sv << 1) | (sv >> 1);
      if (wi > 0) any |= __ldcg(src + w - 1) >> 31;
      if (wi + 1 < bg.W) any |= __ldcg(src + w + 1) << 31;
#pragma unroll
      for (int d = 0; d < N - 1; ++d) {
        if (ir[d] > 0) any |= __ldcg(src + w - rsw[d]);
        if (ir[d] < g.n[d] - 1) any |= __ldcg(src + w + rsw[d]);
      }
      any &= tm;
      dst[w] = any;
      if (pass == 3) cnt += __popc(any);
      if (vpass) {
        const unsigned v = __ldcg(vsrc + w);
        const unsigned lft = (v << 1) | (wi > 0 ? __ldcg(vsrc + w - 1) >> 31 : (v & 1u));
        const unsigned rgt =
            (v >> 1) | (wi + 1 < bg.W ? __ldcg(vsrc + w + 1) << 31 : (v & (1u << ((bg.nx - 1) & 31))));
        unsigned all = v & lft & rgt;
#pragma unroll
        for (int d = 0; d < N - 1; ++d) {
          all &= ir[d] > 0 ? __ldcg(vsrc + w - rsw[d]) : v;
          all &= ir[d] < g.n[d] - 1 ? __ldcg(vsrc + w + rsw[d]) : v;
        }
        vdst[w] = all & tm;
      }
    }
    if (pass == 3) {
      for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
      __shared__ int s_c[LS_NT / 32];
      if (lane == 0) s_c[wid] = cnt;
      __syncthreads();
      if (threadIdx.x == 0) {
        int t = 0;
        for (int k = 0; k < nwarp; ++k) t += s_c[k];
        a.b.cta_count[blockIdx.x] = t;
      }
      __syncthreads();
    }
    if (!grid_barrier(a.st, c.bar, 21 + pass)) return false;
  }
  // ordered compaction of T3: this CTA's offset, then a block scan of the
  // per-word counts, then each thread expands its word
  __shared__ int s_off, s_tot;
  __shared__ int s_w[LS_NT / 32];
  if (wid == 0) {
    int off = 0, tot = 0;
    for (int b = lane; b < (int)gridDim.x; b += 32) {
      const int v = __ldcg(a.b.cta_count + b);
      if (b < (int)blockIdx.x) off += v;
      tot += v;
    }
    for (int o = 16; o > 0; o >>= 1) {
      off += __shfl_xor_sync(0xffffffffu, off, o);
      tot += __shfl_xor_sync(0xffffffffu, tot, o);
    }
    if (lane == 0) {
      s_off = off;
      if (blockIdx.x == 0) {
        a.b.count[0] = tot;
        a.b.info[slot] = tot;
      }
    }
  }
  __syncthreads();
  int run = s_off;
  int tcnt = 0;
  const uint32_t* T3 = pl + P_T3 * bg.nw;
  for (long long base = c.wlo; base < c.whi; base += blockDim.x) {
    const long long w = base + threadIdx.x;
    const unsigned v = w < c.whi ? __ldcg(T3 + w) : 0u;
    const int cw = __popc(v);
    int incl = cw;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    if (lane == 31) s_w[wid] = incl;
    __syncthreads();
    int woff = 0;
    if (threadIdx.x == 0) {
      int t = 0;
      for (int k = 0; k < nwarp; ++k) t += s_w[k];
      s_tot = t;
    }
    for (int k = 0; k < wid; ++k) woff += s_w[k];
    if (v) {
      unsigned r = g.wdiv.div((unsigned)w);
      const int wi = (int)((unsigned)w - r * (unsigned)bg.W);
      int ix[N];
#pragma unroll
      for (int d = 0; d < N - 1; ++d) {
        ix[d] = (int)g.rdiv[d].div(r);
        r -= (unsigned)ix[d] * rstr[d];
      }
      const long long row0 = (long long)(g.wdiv.div((unsigned)w)) * bg.nx;
      const unsigned wT = __ldcg(pl + P_T * bg.nw + w), wT1 = __ldcg(pl + P_T1 * bg.nw + w),
                     wT2 = __ldcg(pl + P_T2 * bg.nw + w);
      unsigned wV0 = 0, wV1 = 0, wV2 = 0;
      if (with_valid) {
        wV0 = __ldcg(pl + P_V0 * bg.nw + w);
        wV1 = __ldcg(pl + P_V1 * bg.nw + w);
        wV2 = __ldcg(pl + P_V2 * bg.nw + w);
      }
      tcnt += __popc(wT);
      int pos = run + woff + incl - cw;
      unsigned rest = v;
      while (rest) {
        const int b = __ffs(rest) - 1;
        rest &= rest - 1u;
        ix[N - 1] = 32 * wi + b;
        const unsigned m = 1u << b;
        uint8_t f = F_T3;
        if (wT & m) f |= F_T;
        if (wT1 & m) f |= F_T1;
        if (wT2 & m) f |= F_T2;
        if (wV0 & m) f |= F_V0;
        if (wV1 & m) f |= F_V1;
        if (wV2 & m) f |= F_V2;
        a.b.list[pos] = (int)(row0 + ix[N - 1]);
        a.b.lcoord[pos] = make_ushort4((unsigned short)ix[0], (unsigned short)ix[1],
                                       (unsigned short)(N > 2 ? ix[2] : 0), (unsigned short)(N > 3 ? ix[3] : 0));
        a.b.lflag[pos] = f;
        ++pos;
      }
    }
    __syncthreads();
    run += s_tot;
    __syncthreads();
  }
  for (int o = 16; o > 0; o >>= 1) tcnt += __shfl_xor_sync(0xffffffffu, tcnt, o);
  if (lane == 0 && tcnt) atomicAdd(&a.b.info[slot + 1], tcnt);
  return grid_barrier(a.st, c.bar, 25);
}

// Number of extension solves whose region holds a work-list entry with
// flags f: the regions T minus V2 (u_nn), T minus V1 (u_n) and T minus V0 (u)
// are nested because V2 lies in V1 and V1 in V0.
__device__ __forceinline__ int sweep_level(uint8_t f) {
  if (!(f & F_T)) return 0;
  if (!(f & F_V0)) return 3;
  if (!(f & F_V1)) return 2;
  return (f & F_V2) ? 0 : 1;
}

// Extension sweeps of the mixed variant: the same first-order upwind
// iteration as the FP64 sweeps (three sweeps of K Jacobi passes over the
// regions of levels >= 1, >= 2, 3; each sweep's result is the next one's
// source), in FP32 arithmetic on FP32 copies of the fields, two passes per
// grid barrier.  One pass at a region entry p is
//   q'(p) = c0 q(p) + sum_d a_d q(u_d) + ds,   a_d = dtau |n_d| / h, c0 = 1 - sum_d a_d,
// with u_d the upwind neighbour along d and ds = dtau s(p); nodes off the
// region keep their values.  Two passes in one update from the values before
// both:
//   q''(p) = c0 q'(p) + sum_d a_d q'(u_d) + ds
//          = D + c0^2 q(p) + sum_d a_d (c0 + c0(u_d)) q(u_d) + sum_de a_d a_e(u_d) q(u_de),
//   D = (1 + c0) ds + sum_d a_d ds(u_d),
// where a neighbour u_d off the region contributes a_d (c0 + 1) q(u_d) and
// nothing else.  A node met twice (u_de = u_ed; u_dd = p where the upwind
// direction turns) keeps one term with the summed weight.  Each region entry
// has a thread of its own when the region is at most one entry per thread;
// larger regions take one pass per barrier.  The fields arrive in FP64 and the
// extended u leaves in FP64.
template <typename T>
__device__ __forceinline__ T tfma(T x, T y, T z) {
  if constexpr (sizeof(T) == 4) return fmaf(x, y, z);
  else return fma(x, y, z);
}
template <typename T>
__device__ __forceinline__ T tabs(T x) {
  if constexpr (sizeof(T) == 4) return fabsf(x);
  else return fabs(x);
}

template <int N, typename T>
__device__ bool ext_sweeps_pair(const LsArgs& a, LsCtx& c, int n, long long cap, int K, double dtau, double dth,
                               const double* const* Q0) {
  constexpr int NTM = 1 + N + N * N;  // terms of a two-pass update
  const GridDev& g = a.g;
  const long long gtid = (long long)blockIdx.x * blockDim.x + threadIdx.x, gth = (long long)gridDim.x * blockDim.x;
  const long long jt = dealt_tid();
  const int* const swl = a.b.slist;
  const int sc1 = __ldcg(a.b.sw + 1), sc2 = __ldcg(a.b.sw + 2), sc3 = __ldcg(a.b.sw + 3);
  const long long len0 = (long long)sc1 + sc2 + sc3;
  constexpr bool F32 = sizeof(T) == 4;
  const T dtf = (T)dtau, dthf = (T)dth;
  // ping-pong fields of the three sweeps: in FP64 the fields' own buffers;
  // in FP32 copies in the FP64 ping-pong partners, which that path leaves
  // unused (each holds two FP32 fields)
  T* F[6];
  if constexpr (F32) {
#pragma unroll
    for (int sw = 0; sw < 3; ++sw) {
      F[2 * sw] = reinterpret_cast<T*>(a.b.q[2 * sw + 1]);
      F[2 * sw + 1] = F[2 * sw] + cap;
    }
  } else {
#pragma unroll
    for (int i = 0; i < 6; ++i) F[i] = reinterpret_cast<T*>(a.b.q[i]);
  }
  for (long long i = gtid; i < n; i += gth) {
    const long long p = __ldcg(a.b.list + i);
#pragma unroll
    for (int sw = 0; sw < 3; ++sw) {
      const T v = (T)__ldcg(Q0[sw] + p);
      if (F32) F[2 * sw][p] = v;
      F[2 * sw + 1][p] = v;
    }
  }
  // The thread's region entry is the same node in every sweep (the regions
  // are prefixes of one sweep list): its upwind nodes and coefficients, and
  // those of its upwind neighbours with their sweep levels, once.
  int p = 0, up[N], lev[N], tu[N][N];
  T c0 = T(0), ad[N], c0u[N], au[N][N];
  if (jt < len0) {
    const long long i = __ldcg(swl + jt);
    p = __ldcg(a.b.list + i);
    int ix[N];
    unpack<N>(__ldcg(a.b.lcoord + i), ix);
    T asum = T(0);
#pragma unroll
    for (int d = 0; d < N; ++d) {
      const double nd = __ldcg(a.b.nrm + d * cap + i);
      up[d] = (int)nbr(g, p, ix, d, nd > 0.0 ? -1 : 1);
      ad[d] = dthf * tabs((T)nd);
      asum += ad[d];
    }
    c0 = T(1) - asum;
    int gi[N];
#pragma unroll
    for (int d = 0; d < N; ++d) gi[d] = __ldcg(a.b.gidx + up[d]);
#pragma unroll
    for (int d = 0; d < N; ++d) {
      const bool ok = gi[d] >= 0 && gi[d] < n;
      const int lp = ok ? __ldcg(a.b.list + gi[d]) : -1;
      const uint8_t f = ok ? __ldcg(a.b.lflag + gi[d]) : (uint8_t)0;
      int ixu[N];
      unpack<N>(ok ? __ldcg(a.b.lcoord + gi[d]) : make_ushort4(0, 0, 0, 0), ixu);
      lev[d] = ok && lp == up[d] ? sweep_level(f) : 0;
      T as = T(0);
#pragma unroll
      for (int e = 0; e < N; ++e) {
        const T ne = ok ? (T)__ldcg(a.b.nrm + e * cap + gi[d]) : T(0);
        au[d][e] = dthf * tabs(ne);
        tu[d][e] = (int)nbr(g, up[d], ixu, e, ne > T(0) ? -1 : 1);
        as += au[d][e];
      }
      c0u[d] = T(1) - as;
    }
  }
  if (!grid_barrier(a.st, c.bar, 53)) return false;
  int si = -1;  // field holding the source (the previous sweep's result)
  for (int sw = 0; sw < 3; ++sw) {
    const long long len = sw == 0 ? len0 : (sw == 1 ? sc2 + sc3 : sc3);
    const bool two = K >= 2 && len <= gth;
    T* const X[2] = {F[2 * sw], F[2 * sw + 1]};
    const T* const src = si < 0 ? nullptr : F[si];
    const bool has = two && jt < len;
    // this sweep's update: membership of the neighbours, source terms (no
    // barrier: nothing written here is read by another thread)
    int ti[NTM];
    T ds = T(0), cq = T(0), D = T(0), tw[NTM];
    unsigned live = 0u;
    if (has) {
      T sd[N];
#pragma unroll
      for (int d = 0; d < N; ++d) sd[d] = src ? __ldcg(src + up[d]) : T(0);
      ds = src ? dtf * __ldcg(src + p) : T(0);
      cq = __ldcg(X[0] + p);
      ti[0] = p;
      tw[0] = c0 * c0;
      live = 1u;
      D = tfma(c0, ds, ds);
#pragma unroll
      for (int d = 0; d < N; ++d) {
        const bool in = lev[d] > sw;
#pragma unroll
        for (int e = 0; e < N; ++e) {
          ti[1 + N + d * N + e] = tu[d][e];
          tw[1 + N + d * N + e] = ad[d] * au[d][e];
        }
        if (in) {
          D = tfma(ad[d], dtf * sd[d], D);
          live |= ((1u << N) - 1u) << (1 + N + d * N);
        }
        ti[1 + d] = up[d];
        tw[1 + d] = ad[d] * (c0 + (in ? c0u[d] : T(1)));
        live |= 1u << (1 + d);
      }
#pragma unroll
      for (int k = 1; k < NTM; ++k) {
        bool done = !((live >> k) & 1u);
#pragma unroll
        for (int k2 = 0; k2 < k; ++k2) {
          if (!done && ((live >> k2) & 1u) && ti[k2] == ti[k]) {
            tw[k2] += tw[k];
            live &= ~(1u << k);
            done = true;
          }
        }
      }
    }
    int cur = 0, it = 0;
    if (two) {
      for (; it + 2 <= K; it += 2) {
        if (has) {
          const T* const qc = X[cur];
          T qv[NTM];
#pragma unroll
          for (int k = 0; k < NTM; ++k) qv[k] = ((live >> k) & 1u) ? __ldcg(qc + ti[k]) : T(0);
          T t = D;
#pragma unroll
          for (int k = 0; k < NTM; ++k) t = tfma(tw[k], qv[k], t);
          cq = t;
          X[cur ^ 1][p] = t;
        }
        if (!grid_barrier(a.st, c.bar, 56)) return false;
        cur ^= 1;
      }
    }
    for (; it < K; ++it) {
      const T* const qc = X[cur];
      T* const qn = X[cur ^ 1];
      if (has) {
        T t = tfma(c0, cq, ds);
#pragma unroll
        for (int d = 0; d < N; ++d) t = tfma(ad[d], __ldcg(qc + up[d]), t);
        cq = t;
        qn[p] = t;
      } else if (!two) {
        for (long long j = jt; j < len; j += gth) {
          const long long i = __ldcg(swl + j);
          const long long q = __ldcg(a.b.list + i);
          int ix[N];
          unpack<N>(__ldcg(a.b.lcoord + i), ix);
          T asum = T(0), qu[N], aw[N];
#pragma unroll
          for (int d = 0; d < N; ++d) {
            const double nd = __ldcg(a.b.nrm + d * cap + i);
            qu[d] = __ldcg(qc + nbr(g, q, ix, d, nd > 0.0 ? -1 : 1));
            aw[d] = dthf * tabs((T)nd);
            asum += aw[d];
          }
          T t = tfma(T(1) - asum, __ldcg(qc + q), src ? dtf * __ldcg(src + q) : T(0));
#pragma unroll
          for (int d = 0; d < N; ++d) t = tfma(aw[d], qu[d], t);
          qn[q] = t;
        }
      }
      if (!grid_barrier(a.st, c.bar, 57)) return false;
      cur ^= 1;
    }
    si = 2 * sw + cur;
  }
  // the swept region of u (level 3) from FP32; the rest of the work list as
  // the FP64 sweeps leave it (its initial values)
  for (long long i = gtid; i < n; i += gth) {
    const long long p = __ldcg(a.b.list + i);
    a.u[p] = sweep_level(__ldcg(a.b.lflag + i)) == 3 ? (double)__ldcg(F[si] + p) : __ldcg(Q0[2] + p);
  }
  return true;
}

// Extension sweeps in FP64 (the plain and the reference arithmetic): three
// sweeps of K Jacobi passes, one pass per grid barrier (see the caller for
// the update).  The extended u goes to the caller's array on the work list.
template <int N>
__device__ bool ext_sweeps_f64(const LsArgs& a, LsCtx& c, int n, long long cap, int K, double dtau, double dth,
                               double* const* UNN, double* const* UN, double* const* U) {
  const GridDev& g = a.g;
  const long long gtid = (long long)blockIdx.x * blockDim.x + threadIdx.x, gth = (long long)gridDim.x * blockDim.x;
  double* const* bufs[3] = {UNN, UN, U};
  const double* src = nullptr;
  constexpr int SW_CACHE = 2;
  const int* const swl = a.b.slist;
  const int sc1 = __ldcg(a.b.sw + 1), sc2 = __ldcg(a.b.sw + 2), sc3 = __ldcg(a.b.sw + 3);
  const long long jt = dealt_tid();
  for (int sw = 0; sw < 3; ++sw) {
    double* const* B = bufs[sw];
    const long long len = sw == 0 ? sc1 + sc2 + sc3 : (sw == 1 ? sc2 + sc3 : sc3);
    for (long long i = gtid; i < n; i += gth) {
      const long long p = __ldcg(a.b.list + i);
      B[1][p] = __ldcg(B[0] + p);
    }
    int cp[SW_CACHE], cup[SW_CACHE][N];
    bool creg[SW_CACHE];
    double cq[SW_CACHE], cds[SW_CACHE], cc0[SW_CACHE], ca[SW_CACHE][N];
#pragma unroll
    for (int r = 0; r < SW_CACHE; ++r) {
      const long long j = jt + r * gth;
      creg[r] = j < len;
      cp[r] = 0;
      cq[r] = cds[r] = cc0[r] = 0.0;
#pragma unroll
      for (int d = 0; d < N; ++d) {
        cup[r][d] = 0;
        ca[r][d] = 0.0;
      }
      if (creg[r]) {
        const long long i = __ldcg(swl + j);
        const long long p = __ldcg(a.b.list + i);
        cp[r] = (int)p;
        cq[r] = __ldcg(B[0] + p);
        cds[r] = src ? dtau * __ldcg(src + p) : 0.0;
        int ix[N];
        unpack<N>(a.b.lcoord[i], ix);
        double asum = 0.0;
#pragma unroll
        for (int d = 0; d < N; ++d) {
          const double nd = __ldcg(a.b.nrm + d * cap + i);
          cup[r][d] = (int)nbr(g, p, ix, d, nd > 0.0 ? -1 : 1);
          ca[r][d] = dth * fabs(nd);
          asum += ca[r][d];
        }
        cc0[r] = 1.0 - asum;
      }
    }
    if (!grid_barrier(a.st, c.bar, 53)) return false;
    int cur = 0;
    for (int it = 0; it < K; ++it) {
      const double* qc = B[cur];
      double* qn = B[cur ^ 1];
#pragma unroll
      for (int r = 0; r < SW_CACHE; ++r) {
        if (!creg[r]) continue;
        double qu[N];
#pragma unroll
        for (int d = 0; d < N; ++d) qu[d] = __ldcg(qc + cup[r][d]);
        double t = fma(cc0[r], cq[r], cds[r]);
#pragma unroll
        for (int d = 0; d < N; ++d) t = fma(ca[r][d], qu[d], t);
        cq[r] = t;
        qn[cp[r]] = t;
      }
      for (long long j = jt + SW_CACHE * gth; j < len; j += gth) {
        const long long i = __ldcg(swl + j);
        const long long p = __ldcg(a.b.list + i);
        int ix[N];
        unpack<N>(a.b.lcoord[i], ix);
        double asum = 0.0, qu[N], ad[N];
#pragma unroll
        for (int d = 0; d < N; ++d) {
          const double nd = __ldcg(a.b.nrm + d * cap + i);
          qu[d] = __ldcg(qc + nbr(g, p, ix, d, nd > 0.0 ? -1 : 1));
          ad[d] = dth * fabs(nd);
          asum += ad[d];
        }
        const double ds = src ? dtau * __ldcg(src + p) : 0.0;
        double t = fma(1.0 - asum, __ldcg(qc + p), ds);
#pragma unroll
        for (int d = 0; d < N; ++d) t = fma(ad[d], qu[d], t);
        qn[p] = t;
      }
      if (!grid_barrier(a.st, c.bar, 53)) return false;
      cur ^= 1;
    }
    src = B[cur];
  }
  // extended u back to the caller's array on the work list
  for (long long i = gtid; i < n; i += gth) {
    const long long p = __ldcg(a.b.list + i);
    a.u[p] = __ldcg(src + p);
  }
  return true;
}

// Stefan speed of the mixed variant at tube node x (axis indices ix, unit
// normal n, level set value phi): V = mu max(0, (4 u(y_1) - u(y_2)) / (2h)),
// y_k = x - (phi + k h) n, u at y_k by N-linear interpolation; the same
// formula as the FP64 path, in FP32.  The sample points are taken relative
// to the node, in grid units (t_d = -(phi + k h) n_d / h, |t_d| <= about 8),
// so that FP32 keeps the interpolation weights to ~1e-6; the cell index is
// clamped in integers as the FP64 path clamps the coordinate to the box.
template <int N>
__device__ double stefan_speed_f32(const GridDev& g, const double* __restrict__ u, const int* ix, const double* nv,
                                   double ph, double mu) {
  const float inv_h = (float)(1.0 / g.h);
  const float phf = (float)ph;
  const float hf = (float)g.h;
  float nf[N];
#pragma unroll
  for (int d = 0; d < N; ++d) nf[d] = (float)nv[d];
  float us[2];
#pragma unroll
  for (int sidx = 0; sidx < 2; ++sidx) {
    const float off = -(phf + (sidx == 0 ? hf : 2.f * hf)) * inv_h;
    float fr[N];
    long long q0 = 0;
#pragma unroll
    for (int d = 0; d < N; ++d) {
      const float t = off * nf[d];
      const float fl = floorf(t);
      int ii = ix[d] + (int)fl;
      float f = t - fl;
      if (ii < 0) {
        ii = 0;
        f = 0.f;
      } else if (ii > g.n[d] - 2) {
        ii = g.n[d] - 2;
        f = 1.f;
      }
      fr[d] = f;
      q0 += (long long)ii * g.stride[d];
    }
    float cv[1 << N];
#pragma unroll
    for (int corner = 0; corner < (1 << N); ++corner) {
      long long q = q0;
#pragma unroll
      for (int d = 0; d < N; ++d)
        if ((corner >> d) & 1) q += g.stride[d];
      cv[corner] = (float)u[q];
    }
#pragma unroll
    for (int d = 0; d < N; ++d) {
#pragma unroll
      for (int corner = 0; corner < (1 << N); corner += 2 << d)
        cv[corner] = fmaf(fr[d], cv[corner + (1 << d)] - cv[corner], cv[corner]);
    }
    us[sidx] = cv[0];
  }
  return (double)((float)mu * fmaxf(0.f, (4.f * us[0] - us[1]) * (0.5f * inv_h)));
}

// TVD-RK3 on the nodes of T (list order); L(src, p) supplied by the caller.
// Stage values p1/p2 hold phi off T (copied when the work set is built).
// The stage list holds the work-list positions of the update set T: entries
// pushed to the front first, then those pushed to the back (read in that
// order), so that warps see one kind of entry (FP64 or FP32 arithmetic).
__device__ __forceinline__ void stage_push(const LsArgs& a, int i, bool front) {
  if (front) a.b.slist[atomicAdd(&a.b.count[1], 1)] = i;
  else a.b.slist[a.g.size - 1 - atomicAdd(&a.b.count[2], 1)] = i;
}

// How the front entries of the stage list (the FP64 ones) are dealt to warps:
// a lane per entry, or an axis per lane.
enum : int { SPLIT_NONE = 0, SPLIT_ALL = 1 };

// One TVD-RK3 step over the stage list.  Front entries go a lane per entry
// (SPLIT_NONE) or have their N axes evaluated on N lanes each (SPLIT_ALL,
// 32 / N entries per warp): the per-axis terms come back by shuffles and are
// summed in axis order as in godunov (which differs only in sharing one
// division among the axes, i.e. in rounding), and a warp issues a third (3D)
// of the FP64 instructions of a warp of whole entries.  This GPU issues about
// one FP64 warp instruction per 80 cycles per SM sub-partition whatever the
// warp's active lanes, so where few FP64 entries leave at most a warp or two
// per sub-partition, split warps finish sooner.  Back entries (FP32 ones) go
// a lane per entry.  L(src, p, ix, i, front) gives the update value of a
// whole entry, LAx(src, p, ix, i, d) the axis term of a split one and
// LFin(i, acc) its update value.
template <int N, typename LFn, typename LAx, typename LFin>
__device__ bool rk3(const LsArgs& a, LsCtx& c, double dt, bool clamp_last, int split, LFn L, LAx LAxis,
                    LFin LFinal) {
  const GridDev& g = a.g;
  const int nf = __ldcg(a.b.count + 1), nb = __ldcg(a.b.count + 2);
  const double G = BAND * g.h;
  // 32-entry chunks dealt round-robin over the CTAs: every SM gets its share
  // of each kind while a warp reads 32 consecutive entries.  Chunk order:
  // whole front, split front, back.
  const int lane = threadIdx.x & 31;
  const long long warp0 = (long long)blockIdx.x + (long long)gridDim.x * (threadIdx.x >> 5);
  const long long wstride = (long long)gridDim.x * (blockDim.x >> 5);
  constexpr int NPW = 32 / N;  // split entries per warp
  const long long nwf = split == SPLIT_NONE ? nf : 0;
  const long long cw = (nwf + 31) / 32;
  const long long cf = ((long long)nf - nwf + NPW - 1) / NPW;
  const long long nchunk = cw + cf + ((long long)nb + 31) / 32;
  for (int stage = 0; stage < 3; ++stage) {
    const double* src = stage == 0 ? a.phi : (stage == 1 ? a.b.p1 : a.b.p2);
    auto update = [&](long long p, double Lv) {
      const double ph = a.phi[p];
      if (stage == 0) {
        a.b.p1[p] = ph + dt * Lv;
      } else if (stage == 1) {
        a.b.p2[p] = 0.75 * ph + 0.25 * (__ldcg(a.b.p1 + p) + dt * Lv);
      } else {
        double v = fma(1.0 / 3.0, ph, 2.0 / 3.0 * (__ldcg(a.b.p2 + p) + dt * Lv));
        if (clamp_last) v = fmin(fmax(v, -G), G);
        a.phi[p] = v;
      }
    };
    for (long long chunk = warp0; chunk < nchunk; chunk += wstride) {
      if (chunk >= cw && chunk < cw + cf) {
        const int sub = lane / N, d = lane - sub * N;
        const long long j = nwf + (chunk - cw) * NPW + sub;
        const bool valid = sub < NPW && j < nf;
        long long i = 0, p = 0;
        double mx = 0.0;
        if (valid) {
          i = __ldcg(a.b.slist + j);
          p = __ldcg(a.b.list + i);
          int ix[N];
          unpack<N>(a.b.lcoord[i], ix);
          mx = LAxis(src, p, ix, i, d);
        }
        double acc = 0.0;
#pragma unroll
        for (int e = 0; e < N; ++e) {
          const double v = __shfl_sync(0xffffffffu, mx, sub * N + e);
          acc = fma(v, v, acc);
        }
        if (valid && d == 0) update(p, LFinal(i, acc));
        continue;
      }
      const bool front = chunk < cw;
      const long long j = front ? 32 * chunk + lane : 32 * (chunk - cw - cf) + lane;
      if (j >= (front ? nwf : (long long)nb)) continue;
      const long long i = __ldcg(a.b.slist + (front ? j : g.size - 1 - j));
      const long long p = __ldcg(a.b.list + i);
      int ix[N];
      unpack<N>(a.b.lcoord[i], ix);
      update(p, L(src, p, ix, i, front));
    }
    if (!grid_barrier(a.st, c.bar, 30 + stage)) return false;
  }
  return true;
}

// copy phi into the RK stage buffers on the work list
template <int N>
__device__ void stage_init(const LsArgs& a) {
  const int n = __ldcg(a.b.count);
  const long long gtid = (long long)blockIdx.x * blockDim.x + threadIdx.x, gth = (long long)gridDim.x * blockDim.x;
  for (long long i = gtid; i < n; i += gth) {
    const long long p = __ldcg(a.b.list + i);
    const double v = a.phi[p];
    a.b.p1[p] = v;
    a.b.p2[p] = v;
  }
}

template <int N>
__device__ bool reinitialise(const LsArgs& a, LsCtx& c) {
  const GridDev& g = a.g;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    a.b.count[1] = 0;
    a.b.count[2] = 0;
  }
  if (!build_work_set<N>(a, c, false, 3)) return false;
  const int n = __ldcg(a.b.count);
  const long long gtid = (long long)blockIdx.x * blockDim.x + threadIdx.x, gth = (long long)gridDim.x * blockDim.x;
  const double h = g.h;
  // mixed path: FP64 within h of the interface (|phi_0| < h, i.e.
  // |S| < 1/sqrt(2)), FP32 WENO/Godunov arithmetic further out; the two
  // kinds go to the two ends of the stage list, the FP64 ones an axis per
  // lane (see rk3)
  const double near_s = 1.0 / sqrt(2.0);
  for (long long i = gtid; i < n; i += gth) {
    const long long p = __ldcg(a.b.list + i);
    const double ph = a.phi[p];
    const double S = ph / sqrt(ph * ph + h * h);
    a.b.S0[i] = S;
    if (a.b.lflag[i] & F_T) stage_push(a, (int)i, !a.mixed || fabs(S) < near_s);
  }
  stage_init<N>(a);
  if (!grid_barrier(a.st, c.bar, 40)) return false;
  const int K = (int)ceil(12.0 * sqrt((double)N));
  const double dtau = 0.5 * h / sqrt((double)N);
  const WenoK wk = weno_k(h);
  auto L = [&](const double* src, long long p, const int* ix, long long i, bool fp64) {
    const double S = __ldcg(a.b.S0 + i);
    const double gr =
        fp64 ? godunov<double, N>(g, src, p, ix, S > 0.0, wk) : godunov<float, N>(g, src, p, ix, S > 0.0, wk);
    return fma(-S, gr, S);  // -S (|grad phi| - 1)
  };
  // FP64 entries an axis per lane (see rk3)
  auto LAx = [&](const double* src, long long p, const int* ix, long long i, int d) {
    return godunov_mx<double, N>(g, src, p, ix, d, __ldcg(a.b.S0 + i) > 0.0, wk);
  };
  auto LFin = [&](long long i, double acc) {
    const double S = __ldcg(a.b.S0 + i);
    return fma(-S, sqrt(acc) * wk.inv_h12, S);
  };
  const int split = a.mixed ? SPLIT_ALL : SPLIT_NONE;
  for (int it = 0; it < K; ++it) {
    if (!rk3<N>(a, c, dtau, it == K - 1, split, L, LAx, LFin)) return false;
  }
  return true;
}

template <int N>
__global__ void __launch_bounds__(LS_NT, 1) levelset_kernel(const LsArgs a) {
  const GridDev& g = a.g;
  LsCtx c;
  c.bar = 0;
  c.red = 0;
  {
    const long long nw = bit_geo(g).nw;
    const long long chunk = (nw + gridDim.x - 1) / gridDim.x;
    c.wlo = min((long long)blockIdx.x * chunk, nw);
    c.whi = min(c.wlo + chunk, nw);
  }
  const long long gtid = (long long)blockIdx.x * blockDim.x + threadIdx.x, gth = (long long)gridDim.x * blockDim.x;
  const double h = g.h;
  const double inv_h = 1.0 / h;
  const double inv_2h = 0.5 * inv_h;
  const double G = BAND * h;

  if (blockIdx.x == 0 && threadIdx.x == 0) {
    for (int i = 0; i < 8; ++i) a.b.info[i] = 0;
    a.b.info[5] = a.reinit;
  }
  if (a.mode == LS_PREPARE) {
    for (long long p = gtid; p < g.size; p += gth) a.phi[p] = fmin(fmax(a.phi[p], -G), G);
    if (!grid_barrier(a.st, c.bar, 50)) return;
    if (a.reinit) reinitialise<N>(a, c);
    return;
  }

  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *a.b.vmax = 0.0;
    a.b.count[1] = 0;
    a.b.count[2] = 0;
    for (int k = 0; k < 8; ++k) a.b.sw[k] = 0;
  }
  if (!build_work_set<N>(a, c, true, 0)) return;
  const int n = __ldcg(a.b.count);
  const long long cap = g.size;
  double* const UNN[2] = {a.b.q[0], a.b.q[1]};
  double* const UN[2] = {a.b.q[2], a.b.q[3]};
  double* const U[2] = {a.b.q[4], a.b.q[5]};
  // normals, u_0, u_n, stage buffers; counts of the sweep levels
  int lc1 = 0, lc2 = 0, lc3 = 0;
  for (long long i = gtid; i < n; i += gth) {
    const long long p = __ldcg(a.b.list + i);
    int ix[N];
    unpack<N>(a.b.lcoord[i], ix);
    // central differences times 1/(2h), one reciprocal of |grad phi|: FP64
    // divisions cost about ten FP64 instructions each.  Mixed variant: the
    // values rounded to FP32 and the arithmetic in FP32 (normals and u_n feed
    // the FP32 extension sweeps and Stefan interpolation)
    const uint8_t f = a.b.lflag[i];
    const bool want_un = (f & F_V1) && (f & F_T2);
    double nv[N];
    double un = 0.0;
    if (a.mixed) {
      const float ih2 = (float)inv_2h;
      float gf[N], s2f = 0.f;
#pragma unroll
      for (int d = 0; d < N; ++d) {
        gf[d] = ((float)a.phi[nbr(g, p, ix, d, 1)] - (float)a.phi[nbr(g, p, ix, d, -1)]) * ih2;
        s2f = fmaf(gf[d], gf[d], s2f);
      }
      const float rnf = 1.f / fmaxf(sqrtf(s2f), (float)GRAD_FLOOR);
      float nf[N];
#pragma unroll
      for (int d = 0; d < N; ++d) {
        nf[d] = gf[d] * rnf;
        nv[d] = (double)nf[d];
        a.b.nrm[d * cap + i] = nv[d];
      }
      if (want_un) {
        float uf = 0.f;
#pragma unroll
        for (int d = 0; d < N; ++d)
          uf = fmaf(nf[d], (float)a.u[nbr(g, p, ix, d, 1)] - (float)a.u[nbr(g, p, ix, d, -1)], uf);
        un = (double)(uf * ih2);
      }
    } else {
      double gr[N];
      double s2 = 0.0;
#pragma unroll
      for (int d = 0; d < N; ++d) {
        gr[d] = (a.phi[nbr(g, p, ix, d, 1)] - a.phi[nbr(g, p, ix, d, -1)]) * inv_2h;
        s2 += gr[d] * gr[d];
      }
      const double rn = 1.0 / fmax(sqrt(s2), GRAD_FLOOR);
#pragma unroll
      for (int d = 0; d < N; ++d) {
        nv[d] = gr[d] * rn;
        a.b.nrm[d * cap + i] = nv[d];
      }
      if (want_un) {
#pragma unroll
        for (int d = 0; d < N; ++d) un += nv[d] * (a.u[nbr(g, p, ix, d, 1)] - a.u[nbr(g, p, ix, d, -1)]);
        un *= inv_2h;
      }
    }
    const int lev = sweep_level(f);
    lc1 += lev == 1;
    lc2 += lev == 2;
    lc3 += lev == 3;
    a.b.gidx[p] = (int)i;
    U[0][p] = (f & F_V0) ? a.u[p] : 0.0;
    UN[0][p] = un;
    a.b.p1[p] = a.phi[p];
    a.b.p2[p] = a.phi[p];
  }
  {
    const int lane = threadIdx.x & 31;
    for (int o = 16; o > 0; o >>= 1) {
      lc1 += __shfl_xor_sync(0xffffffffu, lc1, o);
      lc2 += __shfl_xor_sync(0xffffffffu, lc2, o);
      lc3 += __shfl_xor_sync(0xffffffffu, lc3, o);
    }
    if (lane == 0) {
      if (lc1) atomicAdd(&a.b.sw[1], lc1);
      if (lc2) atomicAdd(&a.b.sw[2], lc2);
      if (lc3) atomicAdd(&a.b.sw[3], lc3);
    }
  }
  if (!grid_barrier(a.st, c.bar, 51)) return;
  // u_nn; the sweep list: entries of level 3, then 2, then 1 (warp-aggregated
  // placement; the order within a level does not matter to a Jacobi sweep)
  {
    const int lane = threadIdx.x & 31;
    const int c3 = __ldcg(a.b.sw + 3), c2 = __ldcg(a.b.sw + 2);
    for (long long base = gtid - lane; base < n; base += gth) {
      const long long i = base + lane;
      int lev = 0;
      if (i < n) {
        const long long p = __ldcg(a.b.list + i);
        const uint8_t f = a.b.lflag[i];
        lev = sweep_level(f);
        double unn = 0.0;
        if ((f & F_V2) && (f & F_T1)) {
          int ix[N];
          unpack<N>(a.b.lcoord[i], ix);
          if (a.mixed) {
            float uf = 0.f;
#pragma unroll
            for (int d = 0; d < N; ++d)
              uf = fmaf((float)__ldcg(a.b.nrm + d * cap + i),
                        (float)__ldcg(UN[0] + nbr(g, p, ix, d, 1)) - (float)__ldcg(UN[0] + nbr(g, p, ix, d, -1)), uf);
            unn = (double)(uf * (float)inv_2h);
          } else {
#pragma unroll
            for (int d = 0; d < N; ++d)
              unn += __ldcg(a.b.nrm + d * cap + i) *
                     (__ldcg(UN[0] + nbr(g, p, ix, d, 1)) - __ldcg(UN[0] + nbr(g, p, ix, d, -1)));
            unn *= inv_2h;
          }
        }
        UNN[0][p] = unn;
      }
#pragma unroll
      for (int L = 1; L <= 3; ++L) {
        const unsigned m = __ballot_sync(0xffffffffu, lev == L);
        if (m) {
          const int leader = __ffs(m) - 1;
          int b0 = 0;
          if (lane == leader) b0 = atomicAdd(&a.b.sw[4 + L], __popc(m));
          b0 = __shfl_sync(0xffffffffu, b0, leader);
          const int seg = L == 3 ? 0 : (L == 2 ? c3 : c3 + c2);
          if (lev == L) a.b.slist[seg + b0 + __popc(m & ((1u << lane) - 1u))] = (int)i;
        }
      }
    }
  }
  if (!grid_barrier(a.st, c.bar, 52)) return;
  // three extrapolation sweeps.  Values off the sweep region never change,
  // so both ping-pong buffers get them once; each pass then touches only the
  // region: the first len_s entries of the sweep list, read in 32-entry
  // chunks dealt round-robin over the CTAs (full warps on every SM).  The
  // first-order upwind step
  //   q' = q - dtau (sum_d n_d D_d q - s),  D_d backward where n_d > 0,
  // is used in the rearranged form q' = c0 q + sum_d a_d q(up_d) + dtau s,
  // a_d = dtau |n_d| / h, c0 = 1 - sum_d a_d (equal up to rounding).  Each
  // thread keeps its first SW_CACHE region entries (node, upwind nodes,
  // coefficients, own value, dtau s) in registers, so a pass issues its N
  // neighbour loads at once and does N + 1 FMAs.
  const int K = (int)ceil(12.0 * sqrt((double)N));
  const double dtau = h / (2.0 * sqrt((double)N));
  const double dth = dtau * inv_h;
  {
    const double* const Q0[3] = {UNN[0], UN[0], U[0]};
    const long long len0 = (long long)__ldcg(a.b.sw + 1) + __ldcg(a.b.sw + 2) + __ldcg(a.b.sw + 3);
    if (a.mixed) {
      if (!ext_sweeps_pair<N, float>(a, c, n, cap, K, dtau, dth, Q0)) return;
    } else if (N <= 3 && len0 <= gth) {
      if (!ext_sweeps_pair<N, double>(a, c, n, cap, K, dtau, dth, Q0)) return;
    } else if (!ext_sweeps_f64<N>(a, c, n, cap, K, dtau, dth, UNN, UN, U)) {
      return;
    }
  }
  if (!grid_barrier(a.st, c.bar, 54)) return;
  // Stefan speed on T
  {
    double vm = 0.0;
    for (long long i = gtid; i < n; i += gth) {
      const long long p = __ldcg(a.b.list + i);
      if (!(a.b.lflag[i] & F_T)) continue;
      int ix[N];
      unpack<N>(a.b.lcoord[i], ix);
      double nv[N];
      const double ph = a.phi[p];
#pragma unroll
      for (int d = 0; d < N; ++d) nv[d] = __ldcg(a.b.nrm + d * cap + i);
      double V;
      if (a.mixed) {
        V = stefan_speed_f32<N>(g, a.u, ix, nv, ph, a.mu);
      } else {
        double xg[N];
#pragma unroll
        for (int d = 0; d < N; ++d) xg[d] = (g.lo[d] + h * ix[d]) - ph * nv[d];
        double us[2];
#pragma unroll
        for (int sidx = 0; sidx < 2; ++sidx) {
          const double dist = sidx == 0 ? h : 2.0 * h;
          int i0[N];
          double fr[N];
          long long q0 = 0;
#pragma unroll
          for (int d = 0; d < N; ++d) {
            double s = ((xg[d] - dist * nv[d]) - g.lo[d]) * inv_h;
            s = fmin(fmax(s, 0.0), (double)(g.n[d] - 1));
            int ii = (int)floor(s);
            ii = min(ii, g.n[d] - 2);
            i0[d] = ii;
            fr[d] = s - ii;
            q0 += (long long)ii * g.stride[d];
          }
          // N-linear interpolation one axis at a time (2^N - 1 lerps; the
          // same value as the sum of corner weights times corner values)
          double cv[1 << N];
#pragma unroll
          for (int corner = 0; corner < (1 << N); ++corner) {
            long long q = q0;
#pragma unroll
            for (int d = 0; d < N; ++d)
              if ((corner >> d) & 1) q += g.stride[d];
            cv[corner] = a.u[q];
          }
#pragma unroll
          for (int d = 0; d < N; ++d) {
#pragma unroll
            for (int corner = 0; corner < (1 << N); corner += 2 << d) cv[corner] = fma(fr[d], cv[corner + (1 << d)] - cv[corner], cv[corner]);
          }
          us[sidx] = cv[0];
        }
        V = a.mu * fmax(0.0, (4.0 * us[0] - us[1]) * inv_2h);
      }
      a.b.V[i] = V;
      stage_push(a, (int)i, true);
      vm = fmax(vm, V);
    }
    for (int o = 16; o > 0; o >>= 1) vm = fmax(vm, __shfl_xor_sync(0xffffffffu, vm, o));
    if ((threadIdx.x & 31) == 0 && vm > 0.0)
      atomicMax((unsigned long long*)a.b.vmax, (unsigned long long)__double_as_longlong(vm));
  }
  if (!grid_barrier(a.st, c.bar, 55)) return;
  // advection
  {
    const double vmax = __ldcg(a.b.vmax);
    double ns = ceil(a.dt * vmax * N / (0.5 * h));
    int nsub = ns < 1.0 ? 1 : (int)fmin(ns, 1e6);
    if (nsub > 100000) {
      if (threadIdx.x == 0) atomicOr(&a.st->err, ERRF_NONFINITE);
      return;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      *a.b.nsub = nsub;
      a.b.info[2] = nsub;
    }
    const double dts = a.dt / nsub;
    const WenoK wk = weno_k(h);
    auto L = [&](const double* s, long long p, const int* ix, long long i, bool) {
      const double gr = a.mixed ? godunov<float, N>(g, s, p, ix, true, wk) : godunov<double, N>(g, s, p, ix, true, wk);
      return -__ldcg(a.b.V + i) * gr;
    };
    for (int sub = 0; sub < nsub; ++sub) {
      auto LAx = [&](const double*, long long, const int*, long long, int) { return 0.0; };
      auto LFin = [&](long long, double) { return 0.0; };
      if (!rk3<N>(a, c, dts, sub == nsub - 1, SPLIT_NONE, L, LAx, LFin)) return;
    }
  }
  if (a.reinit) reinitialise<N>(a, c);
}

static int ls_blocks(int ndim) {
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  void* fn = ndim == 2 ? (void*)levelset_kernel<2> : ndim == 3 ? (void*)levelset_kernel<3> : (void*)levelset_kernel<4>;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, LS_NT, 0) != cudaSuccess || per < 1) return 0;
  return min(sms, MAX_BLOCKS);
}

static cudaError_t launch(const LsArgs& a, cudaStream_t stream) {
  void* fn;
  switch (a.g.ndim) {
    case 2: fn = (void*)levelset_kernel<2>; break;
    case 3: fn = (void*)levelset_kernel<3>; break;
    case 4: fn = (void*)levelset_kernel<4>; break;
    default: return cudaErrorInvalidValue;
  }
  const int nb = ls_blocks(a.g.ndim);
  if (nb <= 0) return cudaErrorLaunchOutOfResources;
  cudaError_t e = cudaMemsetAsync(&a.st->barrier, 0, sizeof(unsigned), stream);
  if (e != cudaSuccess) return e;
  void* args[] = {(void*)&a};
  return cudaLaunchCooperativeKernel(fn, nb, LS_NT, args, 0, stream);
}

cudaError_t launch_levelset_advance(const GridDev& g, const LevelsetBufs& b, DevStatus* st, const uint8_t* kind,
                                    double* phi, double* u, double dt, double mu, bool reinit, bool mixed,
                                    cudaStream_t stream) {
  LsArgs a;
  a.mixed = mixed ? 1 : 0;
  a.g = g;
  a.b = b;
  a.st = st;
  a.kind = kind;
  a.phi = phi;
  a.u = u;
  a.dt = dt;
  a.mu = mu;
  a.mode = LS_ADVANCE;
  a.reinit = reinit ? 1 : 0;
  return launch(a, stream);
}

cudaError_t launch_levelset_prepare(const GridDev& g, const LevelsetBufs& b, DevStatus* st, double* phi, bool reinit,
                                    bool mixed, cudaStream_t stream) {
  LsArgs a;
  a.mixed = mixed ? 1 : 0;
  a.g = g;
  a.b = b;
  a.st = st;
  a.kind = nullptr;
  a.phi = phi;
  a.u = nullptr;
  a.dt = 0.0;
  a.mu = 0.0;
  a.mode = LS_PREPARE;
  a.reinit = reinit ? 1 : 0;
  return launch(a, stream);
}

}  // namespace etd
