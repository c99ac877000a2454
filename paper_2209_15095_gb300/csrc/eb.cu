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

constexpr int SCAN_TILE = 2048;   // nodes per block in the compaction
constexpr int SCAN_NT = 256;

// x < 0 decided on the bit pattern (integer pipe; FP64 compares are costly
// over the whole grid): sign bit set, and x is neither -0 nor NaN.
__device__ __forceinline__ bool negative(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  return (long long)b < 0 && (b << 1) - 1ull < 0xFFE0000000000000ull;
}

// Class of node p from phi; nodes on the box boundary cannot be computational.
// Grids hold fewer than 2^31 nodes: 32-bit index arithmetic.
__device__ __forceinline__ uint8_t classify_node(const GridDev& g, const double* __restrict__ phi, long long p,
                                                 bool& near_edge) {
  unsigned rem = (unsigned)p;
  bool edge = false;
  near_edge = false;
  for (int d = 0; d < g.ndim; ++d) {
    const unsigned st = (unsigned)g.stride[d];
    const int i = (int)(rem / st);
    rem -= (unsigned)i * st;
    if (i == 0 || i == g.n[d] - 1) edge = true;
    if (i < 3 || i > g.n[d] - 4) near_edge = true;
  }
  if (!negative(phi[p])) return K_OUT;
  if (edge) return K_GHOST;
  for (int d = 0; d < g.ndim; ++d) {
    if (!negative(phi[p - g.stride[d]]) || !negative(phi[p + g.stride[d]])) return K_GHOST;
  }
  return K_COMP;
}

// Pass 1: classify, zero stale vector entries where a computational node
// stopped being one, count computational nodes per tile.
__global__ void __launch_bounds__(SCAN_NT) classify_count_kernel(ClassifyArgs a) {
  const GridDev g = a.g;
  const long long base = (long long)blockIdx.x * SCAN_TILE;
  int cnt = 0;
  for (int i = 0; i < SCAN_TILE / SCAN_NT; ++i) {
    long long p = base + threadIdx.x + (long long)i * SCAN_NT;
    if (p >= g.size) break;
    bool near_edge;
    uint8_t k = classify_node(g, a.phi, p, near_edge);
    if (k != K_OUT && near_edge) atomicOr(&a.st->err, ERRF_DOMAIN);
    uint8_t old = a.kind[p] & 3;
    if (old == K_COMP && k != K_COMP) {
      for (int s = 0; s < a.nzero; ++s) {
        if (a.zero_f64[s]) a.zero_f64[s][p] = 0.0;
        if (a.zero_f32[s]) a.zero_f32[s][p] = 0.0f;
      }
      for (int j = 0; j < a.nbasis; ++j) {
        if (a.basis_f64) a.basis_f64[(long long)j * g.size + p] = 0.0;
        if (a.basis_f32) a.basis_f32[(long long)j * g.size + p] = 0.0f;
      }
    }
    a.kind[p] = k;
    cnt += (k == K_COMP);
  }
  __shared__ int s_cnt[SCAN_NT / 32];
  for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  if ((threadIdx.x & 31) == 0) s_cnt[threadIdx.x >> 5] = cnt;
  __syncthreads();
  if (threadIdx.x == 0) {
    int t = 0;
    for (int w = 0; w < SCAN_NT / 32; ++w) t += s_cnt[w];
    a.tile_count[blockIdx.x] = t;
  }
}

// Pass 2: exclusive scan of tile counts by one block.
__global__ void __launch_bounds__(1024) scan_tiles_kernel(int* tile_count, int ntiles, int* total) {
  __shared__ int s_part[1024];
  const int per = (ntiles + 1023) / 1024;
  const int b0 = threadIdx.x * per;
  int sum = 0;
  for (int i = 0; i < per; ++i) {
    int b = b0 + i;
    if (b < ntiles) sum += tile_count[b];
  }
  s_part[threadIdx.x] = sum;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {
    int v = threadIdx.x >= o ? s_part[threadIdx.x - o] : 0;
    __syncthreads();
    s_part[threadIdx.x] += v;
    __syncthreads();
  }
  int run = s_part[threadIdx.x] - sum;  // exclusive prefix of this thread's chunk
  for (int i = 0; i < per; ++i) {
    int b = b0 + i;
    if (b < ntiles) {
      int c = tile_count[b];
      tile_count[b] = run;
      run += c;
    }
  }
  if (threadIdx.x == 1023) *total = s_part[1023];
}

// Pass 3: write the grid indices of computational nodes in grid order.
__global__ void __launch_bounds__(SCAN_NT) scatter_kernel(const GridDev g, const uint8_t* __restrict__ kind,
                                                          const int* __restrict__ tile_offset, int* __restrict__ idx) {
  __shared__ int s_w[SCAN_NT / 32];
  const long long base = (long long)blockIdx.x * SCAN_TILE;
  int run = tile_offset[blockIdx.x];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int i = 0; i < SCAN_TILE / SCAN_NT; ++i) {
    long long p = base + threadIdx.x + (long long)i * SCAN_NT;
    bool f = p < g.size && (kind[p] & 3) == K_COMP;
    unsigned bal = __ballot_sync(0xffffffffu, f);
    int before = __popc(bal & ((1u << lane) - 1u));
    if (lane == 0) s_w[wid] = __popc(bal);
    __syncthreads();
    int woff = 0, tot = 0;
    for (int w = 0; w < SCAN_NT / 32; ++w) {
      int c = s_w[w];
      if (w < wid) woff += c;
      tot += c;
    }
    if (f) idx[run + woff + before] = (int)p;
    run += tot;
    __syncthreads();
  }
}

// Case-3 ghost weight (reading for Eq. rbf_ubp, see the header comment).
// p has axis indices ip; q = p + s * e_dq, s = +-1.
template <int N>
__device__ double case3_weight(const GridDev& g, const double* __restrict__ phi, long long p, const int* ip,
                               long long q, int dq, int s) {
  const double h = g.h;
  double xp[N], xq[N], gp[N], gq[N];
#pragma unroll
  for (int d = 0; d < N; ++d) {
    xp[d] = g.lo[d] + h * ip[d];
    xq[d] = g.lo[d] + h * (ip[d] + (d == dq ? s : 0));
    gp[d] = (phi[p + g.stride[d]] - phi[p - g.stride[d]]) / (2.0 * h);
    gq[d] = (phi[q + g.stride[d]] - phi[q - g.stride[d]]) / (2.0 * h);
  }
  const double php = phi[p], phq = phi[q];
  double np2 = 0.0, nq2 = 0.0;
  for (int d = 0; d < N; ++d) {
    np2 += gp[d] * gp[d];
    nq2 += gq[d] * gq[d];
  }
  const double fallback = phq / php;
  if (!(np2 > 0.0) || !(nq2 > 0.0)) return fallback;
  double G1[N], G2[N];
  for (int d = 0; d < N; ++d) {
    G1[d] = xq[d] - (phq / nq2) * gq[d];
    G2[d] = xp[d] - (php / np2) * gp[d];
  }
  if (N == 2) {
    double e1x = G1[0] - xp[0], e1y = G1[1] - xp[1], e2x = G2[0] - xp[0], e2y = G2[1] - xp[1];
    double det = e1x * e2y - e1y * e2x;
    if (fabs(det) < 1e-12 * h * h) return fallback;
    double f1x = G1[0] - xq[0], f1y = G1[1] - xq[1], f2x = G2[0] - xq[0], f2y = G2[1] - xq[1];
    return (f1x * f2y - f1y * f2x) / det;
  } else {
    double nb[N], t[N], n[N];
    double nbl = 0.0, tl = 0.0;
    for (int d = 0; d < N; ++d) {
      nb[d] = gq[d] + gp[d];
      nbl += nb[d] * nb[d];
      t[d] = G2[d] - G1[d];
      tl += t[d] * t[d];
    }
    nbl = sqrt(nbl);
    tl = sqrt(tl);
    if (!(nbl > 0.0)) return fallback;
    for (int d = 0; d < N; ++d) nb[d] /= nbl;
    if (tl >= 1e-12 * h) {
      double dot = 0.0;
      for (int d = 0; d < N; ++d) {
        t[d] /= tl;
        dot += nb[d] * t[d];
      }
      double nl = 0.0;
      for (int d = 0; d < N; ++d) {
        n[d] = nb[d] - dot * t[d];
        nl += n[d] * n[d];
      }
      nl = sqrt(nl);
      if (!(nl > 0.0)) return fallback;
      for (int d = 0; d < N; ++d) n[d] /= nl;
    } else {
      for (int d = 0; d < N; ++d) n[d] = nb[d];
    }
    double num = 0.0, den = 0.0;
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

// Pass 4: per computational row, D_p and the Gershgorin row sum.  One thread
// per face: a warp holds 32 / (2N) rows with their 2N faces on consecutive
// lanes; the row's first lane sums the face terms in face order.
template <int N>
__global__ void __launch_bounds__(256) metadata_kernel(MetaArgs a) {
  constexpr int FPR = 2 * N, RPW = 32 / FPR;
  const GridDev g = a.g;
  const int ncomp = *a.ncomp;
  const double h2 = g.h * g.h;
  const int lane = threadIdx.x & 31;
  const int slot = lane / FPR, f = lane % FPR, d = f / 2, si = f % 2;
  const int lead = slot * FPR;
  const long long nwarps = (long long)gridDim.x * (blockDim.x >> 5);
  double gmax = 0.0;
  int nclamp = 0;
  for (long long w = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); w * RPW < ncomp; w += nwarps) {
    const long long k = w * RPW + slot;
    const bool act = slot < RPW && k < ncomp;
    double cD = 0.0, cOff = 0.0;
    if (act) {
      const long long p = a.idx[k];
      int ip[N];
      {
        unsigned rem = (unsigned)p;
#pragma unroll
        for (int e = 0; e < N; ++e) {
          const unsigned st = (unsigned)g.stride[e];
          ip[e] = (int)(rem / st);
          rem -= (unsigned)ip[e] * st;
        }
      }
      const long long s = si == 0 ? -g.stride[d] : g.stride[d];
      const long long q = p + s;
      const int iq = ip[d] + (si == 0 ? -1 : 1);
      const double bf = a.beta_field ? 0.5 * (a.beta_field[p] + a.beta_field[q]) : a.beta_c;
      double gw = 0.0;  // 1 - w on a ghost face, 0 on a face to a computational point
      if ((a.kind[q] & 3) == K_COMP) {
        cD = bf;
        cOff = bf;
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
        } else {
          wv = case3_weight<N>(g, a.phi, p, ip, q, d, si == 0 ? -1 : 1);
        }
        const double wc = fmin(fmax(wv, 0.0), 1.0);
        if (!(wc == wv)) ++nclamp;
        cD = fma(-bf, wc, bf);
        gw = 1.0 - wc;
      }
      if (a.facew) a.facew[k * FPR + f] = gw;
    }
    double D = 0.0, off = 0.0;
#pragma unroll
    for (int j = 0; j < FPR; ++j) {
      const double vD = __shfl_sync(0xffffffffu, cD, lead + j);
      const double vO = __shfl_sync(0xffffffffu, cOff, lead + j);
      D += vD;
      off += vO;
    }
    if (act && f == 0) {
      a.diag[k] = D;
      if (a.diagf) a.diagf[k] = (float)D;
      gmax = fmax(gmax, (D + off) / h2);
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    gmax = fmax(gmax, __shfl_xor_sync(0xffffffffu, gmax, o));
    nclamp += __shfl_xor_sync(0xffffffffu, nclamp, o);
  }
  if (lane == 0) {
    atomic_max_pos(a.gersh, gmax);
    if (nclamp) atomicAdd(&a.st->nclamp, nclamp);
  }
}

int scan_tiles(long long size) { return (int)((size + SCAN_TILE - 1) / SCAN_TILE); }

cudaError_t launch_init_domain(const ClassifyArgs& ca, const MetaArgs& ma, int* tile_count, int* ncomp_dev,
                               cudaStream_t stream) {
  const int ntiles = scan_tiles(ca.g.size);
  classify_count_kernel<<<ntiles, SCAN_NT, 0, stream>>>(ca);
  scan_tiles_kernel<<<1, 1024, 0, stream>>>(tile_count, ntiles, ncomp_dev);
  scatter_kernel<<<ntiles, SCAN_NT, 0, stream>>>(ca.g, ca.kind, tile_count, ma.idx);
  cudaMemsetAsync(ma.gersh, 0, sizeof(double), stream);
  const int nb = 152 * 8;
  switch (ma.g.ndim) {
    case 2: metadata_kernel<2><<<nb, 256, 0, stream>>>(ma); break;
    case 3: metadata_kernel<3><<<nb, 256, 0, stream>>>(ma); break;
    case 4: metadata_kernel<4><<<nb, 256, 0, stream>>>(ma); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace etd
