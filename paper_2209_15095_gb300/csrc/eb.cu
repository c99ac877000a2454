// Embedded-boundary domain set-up (Sec. 2): point classification, the list of
// computational points in grid order, and per-row diagonal metadata.
//
//  inside         phi < 0 (phi == 0 is outside)
//  ghost          inside with at least one of the 2N axis neighbours outside
//  computational  inside with all 2N axis neighbours inside
//
// Row p of the operator (Sec. 2, cases 1-3):
//   (C u)_p = (1/h^2) [ sum_{faces to computational q} beta_f u_q - D_p u_p ],
//   D_p = sum_{all faces} beta_f - sum_{ghost faces} beta_f w_f,
// where w_f is the weight of u_p in the ghost value: case 2 (line-by-line
// Lagrange, Eq. DirichletLineByLine) w = theta/(1+theta), theta =
// phi_q/(phi_q - phi_r); case 3 (RBF + linear tail, Eq. rbf_ubp) the affine
// interpolant's weight through x_p and the closest boundary points of the
// ghost (Gamma1) and of p (Gamma2); for N >= 3 the affine function vanishing
// on the hyperplane through Gamma1, Gamma2.  w is clamped to [0, 1].
// Ghost-node entries of every stencil input vector are kept at zero, so the
// matrix-free apply needs only D_p per row.
#include "common.cuh"
#include "kernels.cuh"

namespace etd {

constexpr int INIT_NT = 512;  // threads per CTA of the set-up kernel

// x < 0 decided on the bit pattern (integer pipe; FP64 compares are costly
// over the whole grid): sign bit set, and x is neither -0 nor NaN.
__device__ __forceinline__ bool negative(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  return (long long)b < 0 && (b << 1) - 1ull < 0xFFE0000000000000ull;
}

// Case-3 ghost weight (reading for Eq. rbf_ubp, see the header comment).
// p has axis indices ip; q = p + s * e_dq, s = +-1.  FP64 divisions and
// square roots cost about ten FP64 instructions each, so the gradients use
// 1/(2h), unit vectors use rsqrt, and the length test on Gamma2 - Gamma1 is
// made on its square; the decisions are those of the plain formulas up to
// rounding at the thresholds.
// Boundary part of a case-3 ghost value in 2D, u_q = w u_p + c1 u(G1) + c2 u(G2)
// (barycentric coordinates of x_q in the triangle x_p, G1, G2).
struct Case3Bnd {
  double c1, c2, G1[2], G2[2];
  bool ok;  // false: no boundary part defined (N >= 3, or no gradient)
};

template <int N>
__device__ double case3_weight(const GridDev& g, const double* __restrict__ phi, long long p, const int* ip,
                               long long q, int dq, int s, Case3Bnd* bo = nullptr) {
  const double h = g.h;
  const double inv_2h = 0.5 / h;
  double xp[N], xq[N], gp[N], gq[N];
#pragma unroll
  for (int d = 0; d < N; ++d) {
    xp[d] = g.lo[d] + h * ip[d];
    xq[d] = g.lo[d] + h * (ip[d] + (d == dq ? s : 0));
    gp[d] = (phi[p + g.stride[d]] - phi[p - g.stride[d]]) * inv_2h;
    gq[d] = (phi[q + g.stride[d]] - phi[q - g.stride[d]]) * inv_2h;
  }
  const double php = phi[p], phq = phi[q];
  double np2 = 0.0, nq2 = 0.0;
#pragma unroll
  for (int d = 0; d < N; ++d) {
    np2 += gp[d] * gp[d];
    nq2 += gq[d] * gq[d];
  }
  const double fallback = phq / php;
  if (bo) bo->ok = false;
  if (!(np2 > 0.0) || !(nq2 > 0.0)) return fallback;
  const double cq = phq / nq2, cp = php / np2;
  double G1[N], G2[N];
#pragma unroll
  for (int d = 0; d < N; ++d) {
    G1[d] = xq[d] - cq * gq[d];
    G2[d] = xp[d] - cp * gp[d];
  }
  if (N == 2) {
    double e1x = G1[0] - xp[0], e1y = G1[1] - xp[1], e2x = G2[0] - xp[0], e2y = G2[1] - xp[1];
    double det = e1x * e2y - e1y * e2x;
    if (bo) {
      bo->ok = true;
      bo->G1[0] = G1[0];
      bo->G1[1] = G1[N - 1];
      bo->G2[0] = G2[0];
      bo->G2[1] = G2[N - 1];
    }
    if (fabs(det) < 1e-12 * h * h) {
      // degenerate triangle: w = phi_q / phi_p, the rest carried by G1
      if (bo) {
        bo->c1 = 1.0 - fallback;
        bo->c2 = 0.0;
      }
      return fallback;
    }
    double f1x = G1[0] - xq[0], f1y = G1[1] - xq[1], f2x = G2[0] - xq[0], f2y = G2[1] - xq[1];
    if (bo) {
      const double dx = xq[0] - xp[0], dy = xq[1] - xp[1];
      bo->c1 = (dx * e2y - dy * e2x) / det;
      bo->c2 = (e1x * dy - e1y * dx) / det;
    }
    return (f1x * f2y - f1y * f2x) / det;
  } else {
    double nb[N], t[N], n[N];
    double nb2 = 0.0, t2 = 0.0;
#pragma unroll
    for (int d = 0; d < N; ++d) {
      nb[d] = gq[d] + gp[d];
      nb2 += nb[d] * nb[d];
      t[d] = G2[d] - G1[d];
      t2 += t[d] * t[d];
    }
    if (!(nb2 > 0.0)) return fallback;
    const double rnb = rsqrt(nb2);
#pragma unroll
    for (int d = 0; d < N; ++d) nb[d] *= rnb;
    if (t2 >= 1e-24 * h * h) {
      const double rt = rsqrt(t2);
      double dot = 0.0;
#pragma unroll
      for (int d = 0; d < N; ++d) {
        t[d] *= rt;
        dot += nb[d] * t[d];
      }
      double nl2 = 0.0;
#pragma unroll
      for (int d = 0; d < N; ++d) {
        n[d] = nb[d] - dot * t[d];
        nl2 += n[d] * n[d];
      }
      if (!(nl2 > 0.0)) return fallback;
      const double rnl = rsqrt(nl2);
#pragma unroll
      for (int d = 0; d < N; ++d) n[d] *= rnl;
    } else {
#pragma unroll
      for (int d = 0; d < N; ++d) n[d] = nb[d];
    }
    double num = 0.0, den = 0.0;
#pragma unroll
    for (int d = 0; d < N; ++d) {
      num += (xq[d] - G1[d]) * n[d];
      den += (xp[d] - G1[d]) * n[d];
    }
    if (fabs(den) < 1e-12 * h) return fallback;
    return num / den;
  }
}

__device__ __forceinline__ void atomic_max_pos(double* a, double v) {
  // non-negative doubles order like their bit patterns
  atomicMax((unsigned long long*)a, (unsigned long long)__double_as_longlong(v));
}

// Class of a node from phi: inside (phi < 0) with all 2N axis neighbours
// inside and not on the box boundary is computational, inside otherwise a
// ghost; near flags inside-or-not nodes within 3 of the boundary.  Loading
// (node_load) is split from deciding (node_class) so that a warp issues the
// loads of several words before it waits on any of them; neighbour indices
// are clamped into the box (an edge node is a ghost or outside whatever they
// hold).  Grids hold fewer than 2^31 nodes: 32-bit index arithmetic.
template <int N>
struct NodeLoad {
  double v, w[2 * N];
  bool edge, near;
};

template <int N>
__device__ __forceinline__ void node_load(const GridDev& g, const double* __restrict__ phi, long long p,
                                          NodeLoad<N>& L) {
  unsigned rem = (unsigned)p;
  L.edge = false;
  L.near = false;
  long long nb[2 * N];
#pragma unroll
  for (int d = 0; d < N; ++d) {
    const unsigned st = (unsigned)g.stride[d];
    const int i = (int)g.sdiv[d].div(rem);
    rem -= (unsigned)i * st;
    if (i == 0 || i == g.n[d] - 1) L.edge = true;
    if (i < 3 || i > g.n[d] - 4) L.near = true;
    nb[2 * d] = i > 0 ? p - g.stride[d] : p;
    nb[2 * d + 1] = i < g.n[d] - 1 ? p + g.stride[d] : p;
  }
  L.v = phi[p];
#pragma unroll
  for (int j = 0; j < 2 * N; ++j) L.w[j] = phi[nb[j]];
}

template <int N>
__device__ __forceinline__ uint8_t node_class(const NodeLoad<N>& L) {
  if (!negative(L.v)) return K_OUT;
  bool all = !L.edge;
#pragma unroll
  for (int j = 0; j < 2 * N; ++j) all = all && negative(L.w[j]);
  return all ? K_COMP : K_GHOST;
}

// Phase 3: per computational row, D_p and the Gershgorin row sum.  One
// thread per face: a warp holds 32 / (2N) rows with their 2N faces on
// consecutive lanes (warps dealt round-robin over the CTAs); the row's first
// lane sums the face terms in face order.
template <int N>
__device__ void metadata_phase(const MetaArgs& a, int ncomp) {
  constexpr int FPR = 2 * N, RPW = 32 / FPR;
  const GridDev& g = a.g;
  const double h2 = g.h * g.h;
  const int lane = threadIdx.x & 31;
  const int slot = lane / FPR, f = lane % FPR, d = f / 2, si = f % 2;
  const int lead = slot * FPR;
  const long long nwarps = (long long)gridDim.x * (blockDim.x >> 5);
  double gmax = 0.0;
  int nclamp = 0;
  // interior rows (every face to a computational point) with a constant
  // beta: D = 2N beta and the Gershgorin row sum 4N beta / h^2, without the
  // FP64 face sums (FP64 warp instructions are what this phase spends)
  const bool cbeta = a.beta_field == nullptr;
  const double D_int = (double)FPR * a.beta_c;
  const unsigned row_mask = ((1u << FPR) - 1u) << lead;
  bool seen_interior = false;
  for (long long w = (long long)blockIdx.x + (long long)gridDim.x * (threadIdx.x >> 5); w * RPW < ncomp;
       w += nwarps) {
    const long long k = w * RPW + slot;
    const bool act = slot < RPW && k < ncomp;
    double cD = 0.0, cOff = 0.0;
    bool face_comp = false;
    if (act) {
      const long long p = __ldcg(a.idx + k);
      int ip[N];
      {
        unsigned rem = (unsigned)p;
#pragma unroll
        for (int e = 0; e < N; ++e) {
          const unsigned st = (unsigned)g.stride[e];
          ip[e] = (int)g.sdiv[e].div(rem);
          rem -= (unsigned)ip[e] * st;
        }
      }
      const long long s = si == 0 ? -g.stride[d] : g.stride[d];
      const long long q = p + s;
      const int iq = ip[d] + (si == 0 ? -1 : 1);
      const double bf = a.beta_field ? 0.5 * (a.beta_field[p] + a.beta_field[q]) : a.beta_c;
      double gw = 0.0;  // 1 - w on a ghost face, 0 on a face to a computational point
      // boundary-data slots of this face: coefficient of u_Gamma in the row
      // (beta_f c / h^2, the ghost value's weight on the boundary point) and
      // the point; coefficient 0 and a NaN point where there is none
      double bc[2] = {0.0, 0.0}, bx[2][N];
#pragma unroll
      for (int j = 0; j < 2; ++j)
#pragma unroll
        for (int e = 0; e < N; ++e) bx[j][e] = __longlong_as_double(0x7ff8000000000000ll);
      if ((__ldcg(a.kind + q) & 3) == K_COMP) {
        cD = bf;
        cOff = bf;
        face_comp = true;
      } else if (iq <= 0 || iq >= g.n[d] - 1) {
        // ghost on the box boundary: the domain-margin error is already
        // flagged by the classification; keep every access in bounds
        cD = bf;
      } else {
        const long long r = q + s;
        double wv;
        if (!negative(a.phi[r])) {
          const double theta = a.phi[q] / (a.phi[q] - a.phi[r]);
          wv = theta / (1.0 + theta);
          if (a.bco) {
            // case 2: the crossing at x_q + s theta h e_d, weight 1 / (1 + theta)
            bc[0] = bf * (1.0 / (1.0 + theta)) / h2;
#pragma unroll
            for (int e = 0; e < N; ++e)
              bx[0][e] = g.lo[e] + g.h * ip[e] + (e == d ? (si == 0 ? -1.0 : 1.0) * g.h * (1.0 + theta) : 0.0);
          }
        } else {
          Case3Bnd cb;
          wv = case3_weight<N>(g, a.phi, p, ip, q, d, si == 0 ? -1 : 1, a.bco ? &cb : nullptr);
          if (a.bco) {
            if (N == 2 && cb.ok) {
              bc[0] = bf * cb.c1 / h2;
              bc[1] = bf * cb.c2 / h2;
              bx[0][0] = cb.G1[0];
              bx[0][N - 1] = cb.G1[1];
              bx[1][0] = cb.G2[0];
              bx[1][N - 1] = cb.G2[1];
            } else {
              // nonzero boundary data at a case-3 face is defined for N = 2 only
              atomicOr(&a.st->err, ERRF_UNSUPPORTED);
            }
          }
        }
        const double wc = fmin(fmax(wv, 0.0), 1.0);
        if (!(wc == wv)) ++nclamp;
        cD = fma(-bf, wc, bf);
        gw = 1.0 - wc;
      }
      if (a.facew) a.facew[k * FPR + f] = gw;
      if (a.bco) {
        const int J = N == 2 ? 2 : 1;
#pragma unroll
        for (int j = 0; j < J; ++j) {
          const long long slot = (k * FPR + f) * J + j;
          a.bco[slot] = bc[j];
#pragma unroll
          for (int e = 0; e < N; ++e) a.bpts[slot * N + e] = bx[j][e];
        }
      }
    }
    const unsigned fc = __ballot_sync(0xffffffffu, act && face_comp);
    const bool interior = cbeta && (fc & row_mask) == row_mask;
    // the face sums only where some row of this warp iteration has a ghost face
    const unsigned need = __ballot_sync(0xffffffffu, act && f == 0 && !interior);
    double D = D_int, off = D_int;
    if (need) {
      double Ds = 0.0, os = 0.0;
#pragma unroll
      for (int j = 0; j < FPR; ++j) {
        Ds += __shfl_sync(0xffffffffu, cD, lead + j);
        os += __shfl_sync(0xffffffffu, cOff, lead + j);
      }
      if (!interior) {
        D = Ds;
        off = os;
      }
    }
    if (act && f == 0) {
      a.diag[k] = D;
      if (a.diagf) a.diagf[k] = (float)D;
      if (!interior) gmax = fmax(gmax, (D + off) / h2);
      seen_interior = seen_interior || interior;
    }
  }
  // the interior rows' Gershgorin sum, once for all of those this thread wrote
  if (seen_interior) gmax = fmax(gmax, (D_int + D_int) / h2);
  for (int o = 16; o > 0; o >>= 1) {
    gmax = fmax(gmax, __shfl_xor_sync(0xffffffffu, gmax, o));
    nclamp += __shfl_xor_sync(0xffffffffu, nclamp, o);
  }
  if (lane == 0) {
    if (gmax > 0.0) atomic_max_pos(a.gersh, gmax);
    if (nclamp) atomicAdd(&a.st->nclamp, nclamp);
  }
}

// The whole set-up as one persistent cooperative kernel (one CTA per SM):
//   phase 1  classify this CTA's chunk of nodes (whole 32-node words), zero
//            stale vector entries where a computational node stopped being
//            one, count computational nodes (when rows are whole words: a
//            sign plane first, then, after a grid barrier, 32 nodes at a
//            time from it);
//   phase 2  (after a grid barrier) this CTA's offset from the counts of the
//            CTAs before it, then the grid indices of its computational nodes
//            in grid order;
//   phase 3  (after a second barrier) the row metadata.
template <int N>
__global__ void __launch_bounds__(INIT_NT, 1) init_domain_kernel(const ClassifyArgs ca, const MetaArgs ma) {
  const GridDev& g = ca.g;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  unsigned bar = 0;
  // this CTA's 32-node words; the computational-node bit plane follows the
  // per-CTA counts in the scratch
  const long long nw = (g.size + 31) / 32;
  const long long cw = (nw + gridDim.x - 1) / gridDim.x;
  const long long wlo = min((long long)blockIdx.x * cw, nw), whi = min(wlo + cw, nw);
  uint32_t* cbits = (uint32_t*)(ca.tile_count + MAX_BLOCKS);
  if (blockIdx.x == 0 && threadIdx.x == 0) *ma.gersh = 0.0;
  __shared__ int s_w[INIT_NT / 32];
  __shared__ int s_off, s_tot;
  int cnt = 0;
  constexpr int UW = 4;  // words per warp and iteration: their loads overlap
  const int nx = g.n[N - 1];
  if ((nx & 31) == 0) {
    // Rows are whole 32-node words: classify a word at a time from a sign
    // plane (bit set where phi < 0).  A node is computational when it and its
    // 2N neighbours are inside and it is not on the box edge; the x
    // neighbours are the word shifted by one bit (with the end bits of the
    // adjacent words), the others the words one stride away.
    uint32_t* const sbits = cbits + nw;
    constexpr int US = 16;  // words per warp and iteration of the sign plane
    for (long long w0 = wlo + (long long)wid * US; w0 < whi; w0 += (long long)nwarp * US) {
      double v[US];
#pragma unroll
      for (int u = 0; u < US; ++u) v[u] = w0 + u < whi ? ca.phi[32 * (w0 + u) + lane] : 1.0;
#pragma unroll
      for (int u = 0; u < US; ++u) {
        const unsigned b = __ballot_sync(0xffffffffu, negative(v[u]));
        if (lane == 0 && w0 + u < whi) sbits[w0 + u] = b;
      }
    }
    if (!grid_barrier(ca.st, bar, 62)) return;
    // a thread per word: its 32 kinds are written as two 16-byte stores
    for (long long w = wlo + threadIdx.x; w < whi; w += blockDim.x) {
      // axis indices of the word's first node
      int ix[N];
      unsigned rem = (unsigned)(32 * w);
#pragma unroll
      for (int d = 0; d < N; ++d) {
        ix[d] = (int)g.sdiv[d].div(rem);
        rem -= (unsigned)ix[d] * (unsigned)g.stride[d];
      }
      const int x0 = ix[N - 1];
      const unsigned s0 = __ldcg(sbits + w);
      const unsigned sl = x0 > 0 ? __ldcg(sbits + w - 1) : 0u;
      const unsigned sr = x0 + 32 < nx ? __ldcg(sbits + w + 1) : 0u;
      unsigned all = s0 & ((s0 << 1) | (sl >> 31)) & ((s0 >> 1) | (sr << 31));
      unsigned nearm = 0u;  // nodes within 3 nodes of the box edge
#pragma unroll
      for (int d = 0; d < N - 1; ++d) {
        const long long ws = g.stride[d] >> 5;
        all &= ix[d] > 0 ? __ldcg(sbits + w - ws) : 0u;
        all &= ix[d] < g.n[d] - 1 ? __ldcg(sbits + w + ws) : 0u;
        if (ix[d] < 3 || ix[d] > g.n[d] - 4) nearm = 0xffffffffu;
      }
      if (x0 == 0) {
        all &= ~1u;
        nearm |= 0x7u;
      }
      if (x0 + 32 == nx) {
        all &= 0x7fffffffu;
        nearm |= 0xe0000000u;
      }
      if (s0 & nearm) atomicOr(&ca.st->err, ERRF_DOMAIN);
      // kind byte = inside bit + computational bit (K_OUT 0, K_GHOST 1,
      // K_COMP 2); a nibble spreads to one bit per byte by a multiply
      uint4* const kp = reinterpret_cast<uint4*>(ca.kind + 32 * w);
      const uint4 o0 = kp[0], o1 = kp[1];
      const unsigned ow[8] = {o0.x, o0.y, o0.z, o0.w, o1.x, o1.y, o1.z, o1.w};
      unsigned kw[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        kw[q] = ((((s0 >> (4 * q)) & 15u) * 0x204081u) & 0x01010101u) +
                ((((all >> (4 * q)) & 15u) * 0x204081u) & 0x01010101u);
        // nodes that stop being computational: zero their vector entries
        unsigned z = (ow[q] >> 1) & ~(kw[q] >> 1) & 0x01010101u;
        while (z) {
          const long long p = 32 * w + 4 * q + ((__ffs(z) - 1) >> 3);
          z &= z - 1u;
          for (int s = 0; s < ca.nzero; ++s) {
            if (ca.zero_f64[s]) ca.zero_f64[s][p] = 0.0;
            if (ca.zero_f32[s]) ca.zero_f32[s][p] = 0.0f;
          }
          for (int j = 0; j < ca.nbasis; ++j) {
            if (ca.basis_f64) ca.basis_f64[(long long)j * g.size + p] = 0.0;
            if (ca.basis_f32) ca.basis_f32[(long long)j * g.size + p] = 0.0f;
          }
        }
      }
      kp[0] = make_uint4(kw[0], kw[1], kw[2], kw[3]);
      kp[1] = make_uint4(kw[4], kw[5], kw[6], kw[7]);
      cbits[w] = all;
      cnt += __popc(all);
    }
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  } else {
    for (long long w0 = wlo + (long long)wid * UW; w0 < whi; w0 += (long long)nwarp * UW) {
      NodeLoad<N> L[UW];
      uint8_t old[UW];
      bool val[UW];
  #pragma unroll
      for (int u = 0; u < UW; ++u) {
        const long long p = 32 * (w0 + u) + lane;
        val[u] = w0 + u < whi && p < g.size;
        old[u] = K_OUT;
        if (val[u]) {
          node_load<N>(g, ca.phi, p, L[u]);
          old[u] = ca.kind[p] & 3;
        }
      }
  #pragma unroll
      for (int u = 0; u < UW; ++u) {
        const long long p = 32 * (w0 + u) + lane;
        const uint8_t k = val[u] ? node_class<N>(L[u]) : K_OUT;
        if (val[u]) {
          if (k != K_OUT && L[u].near) atomicOr(&ca.st->err, ERRF_DOMAIN);
          if (old[u] == K_COMP && k != K_COMP) {
            for (int s = 0; s < ca.nzero; ++s) {
              if (ca.zero_f64[s]) ca.zero_f64[s][p] = 0.0;
              if (ca.zero_f32[s]) ca.zero_f32[s][p] = 0.0f;
            }
            for (int j = 0; j < ca.nbasis; ++j) {
              if (ca.basis_f64) ca.basis_f64[(long long)j * g.size + p] = 0.0;
              if (ca.basis_f32) ca.basis_f32[(long long)j * g.size + p] = 0.0f;
            }
          }
          ca.kind[p] = k;
        }
        const unsigned bal = __ballot_sync(0xffffffffu, val[u] && k == K_COMP);
        if (lane == 0 && w0 + u < whi) {
          cbits[w0 + u] = bal;
          cnt += __popc(bal);
        }
      }
    }
  }
  if (lane == 0) s_w[wid] = cnt;
  __syncthreads();
  if (threadIdx.x == 0) {
    int t = 0;
    for (int j = 0; j < nwarp; ++j) t += s_w[j];
    ca.tile_count[blockIdx.x] = t;
  }
  if (!grid_barrier(ca.st, bar, 60)) return;
  if (wid == 0) {
    int off = 0, tot = 0;
    for (int b = lane; b < (int)gridDim.x; b += 32) {
      const int v = __ldcg(ca.tile_count + b);
      if (b < (int)blockIdx.x) off += v;
      tot += v;
    }
    for (int o = 16; o > 0; o >>= 1) {
      off += __shfl_xor_sync(0xffffffffu, off, o);
      tot += __shfl_xor_sync(0xffffffffu, tot, o);
    }
    if (lane == 0) {
      s_off = off;
      s_tot = tot;
      if (blockIdx.x == 0) *ma.ncomp = tot;
    }
  }
  __syncthreads();
  // ordered compaction: a thread per word, block scan of the popcounts,
  // then each thread writes its word's nodes
  int run = s_off;
  for (long long base = wlo; base < whi; base += blockDim.x) {
    const long long w = base + threadIdx.x;
    const unsigned v = w < whi ? cbits[w] : 0u;
    const int c = __popc(v);
    int incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    __syncthreads();
    if (lane == 31) s_w[wid] = incl;
    __syncthreads();
    int woff = 0, tot = 0;
    for (int j = 0; j < nwarp; ++j) {
      const int cc = s_w[j];
      if (j < wid) woff += cc;
      tot += cc;
    }
    int pos = run + woff + incl - c;
    unsigned rest = v;
    while (rest) {
      const int b = __ffs(rest) - 1;
      rest &= rest - 1u;
      ma.idx[pos++] = (int)(32 * w + b);
    }
    run += tot;
  }
  const int ncomp = s_tot;
  if (!grid_barrier(ca.st, bar, 61)) return;
  metadata_phase<N>(ma, ncomp);
}

// ints of scratch the set-up kernel needs: one count per CTA, then two bit
// planes (computational nodes, signs of phi) of one bit per node
template <int N>
static void* init_fn() {
  return (void*)init_domain_kernel<N>;
}

cudaError_t launch_init_domain(const ClassifyArgs& ca, const MetaArgs& ma, int* tile_count, int* ncomp_dev,
                               cudaStream_t stream) {
  (void)tile_count;
  (void)ncomp_dev;
  void* fn;
  switch (ma.g.ndim) {
    case 2: fn = init_fn<2>(); break;
    case 3: fn = init_fn<3>(); break;
    case 4: fn = init_fn<4>(); break;
    default: return cudaErrorInvalidValue;
  }
  int dev = 0, sms = 0, per = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, INIT_NT, 0);
  if (e != cudaSuccess) return e;
  if (per < 1) return cudaErrorLaunchOutOfResources;
  const int nb = min(sms, MAX_BLOCKS);
  e = cudaMemsetAsync(&ca.st->barrier, 0, sizeof(unsigned), stream);
  if (e != cudaSuccess) return e;
  ClassifyArgs c1 = ca;
  MetaArgs m1 = ma;
  void* args[] = {(void*)&c1, (void*)&m1};
  return cudaLaunchCooperativeKernel(fn, nb, INIT_NT, args, 0, stream);
}

}  // namespace etd
