// Tiled Lanczos pass for large 3D FP32 problems with a constant beta: one
// pass per Krylov vector instead of two.
//
// The split passes build V_j = ca Z_{j-1} + cb V_{j-1} + cc V_{j-2} from a
// stored Z_{j-1} = A V_{j-1} and then Z_j = A V_j: 8 vector accesses per
// point and Krylov vector.  Here Z_{j-1} is recomputed from V_{j-1} in shared
// memory: per 64 x 8 x 8 tile of the grid, TMA copies V_{j-1} on the tile
// grown by two nodes, V_{j-2} and the node classes on the tile grown by one;
// A V_{j-1} and w_j = ca A V_{j-1} + cb V_{j-1} + cc V_{j-2} are formed on the
// tile grown by one (w_j = 0 off the computational set), then A w_j and the
// three sums on the tile, and V_j = w_j is stored.  HBM traffic per point is
// about 3 vectors (V_{j-1}, V_{j-2} read, V_j written) and a class byte; the
// halos come from L2.  Two stages: the next tile's copies are in flight while
// this one is computed.
//
// Node classes (per launch, from the domain set-up): tk = 0 off the
// computational set, 1 at a computational node whose diagonal is the
// interior value 2 N beta, 2 at one with any other diagonal, which is then
// read from the full-grid array Dg.
#pragma once
#include <cuda.h>

#include "common.cuh"

namespace etd {

constexpr int TL_X = 64, TL_Y = 8, TL_Z = 8;   // tile (x the last, fastest axis)
constexpr int TL_AX = TL_X + 8;                 // x extent of the staged rows (16-byte aligned start x0 - 4)
constexpr int TL_KX = TL_X + 32;                // x extent of the staged class rows (start x0 - 16)
constexpr int TL_A_BYTES = TL_AX * (TL_Y + 4) * (TL_Z + 4) * 4;  // V_{j-1}, two-node halo
constexpr int TL_B_BYTES = TL_AX * (TL_Y + 2) * (TL_Z + 2) * 4;  // V_{j-2}, one-node halo
constexpr int TL_K_BYTES = TL_KX * (TL_Y + 2) * (TL_Z + 2);      // classes, one-node halo
constexpr int TL_STAGE = TL_A_BYTES + TL_B_BYTES + TL_K_BYTES;
constexpr int TL_SMEM = 2 * TL_STAGE + 128;  // two stages and the two mbarriers
static_assert(TL_A_BYTES % 128 == 0 && TL_B_BYTES % 128 == 0 && TL_K_BYTES % 128 == 0, "stage alignment");

// Everything the tiled pass needs: the tensor maps (V as a 4D array x, y,
// z, basis slot with the two box sizes; the classes as a 3D uint8 array),
// the class and diagonal arrays and the tile grid with its activity flags.
struct TileArgs {
  CUtensorMap tmA;  // V, box TL_AX x (TL_Y + 4) x (TL_Z + 4) x 1
  CUtensorMap tmB;  // V, box TL_AX x (TL_Y + 2) x (TL_Z + 2) x 1
  CUtensorMap tmK;  // tk, box TL_KX x (TL_Y + 2) x (TL_Z + 2)
  int enabled;
  int ntx, nty, ntz, ntiles;
  uint8_t* tk;     // full grid
  float* Dg;       // full grid (read where tk == 2)
  uint8_t* flags;  // per tile: any computational node
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred P1;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 P1, [%1], %2;\n\t"
      "selp.b32 %0, 1, 0, P1;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap* tm, int c0, int c1, int c2, int c3,
                                            uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
      "[%6];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(tm)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* tm, int c0, int c1, int c2,
                                            uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(tm)), "r"(c0), "r"(c1), "r"(c2), "r"(bar)
      : "memory");
}

// Waits for a stage's copies; bounded like the grid barrier (the status
// word's limit, default 1 s).  On timeout ERRF_TIMEOUT is raised and the
// wait goes on, again bounded, so that no copy is still landing in shared
// memory when the CTA returns false.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, DevStatus* st) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long w = *((volatile unsigned long long*)&st->wait_ns);
  const unsigned long long limit = w != 0ull ? w : BARRIER_LIMIT_NS;
  const unsigned long long t0 = global_ns();
  while (!mbar_try_wait(bar, parity)) {
    if (global_ns() - t0 >= limit) {
      atomicOr(&st->err, ERRF_TIMEOUT);
      const unsigned long long t1 = global_ns();
      while (!mbar_try_wait(bar, parity) && global_ns() - t1 < BARRIER_LIMIT_NS) {
      }
      return false;
    }
  }
  return true;
}

// The next active tile of this CTA at or after t (stride gridDim.x), or -1.
__device__ __forceinline__ int tile_next(const TileArgs& ta, int t) {
  for (; t < ta.ntiles; t += gridDim.x)
    if (__ldcg(ta.flags + t)) return t;
  return -1;
}

// Issues the copies of tile t for Krylov vector j into stage s (one thread).
// The copies of V_{j-2} are skipped for j == 1 (its coefficient is 0).
__device__ __forceinline__ void tile_issue(const TileArgs& ta, unsigned char* base, int s, int t, int j) {
  unsigned char* stg = base + s * TL_STAGE;
  const uint32_t bar = smem_u32(base + 2 * TL_STAGE + 8 * s);
  const int tx = t % ta.ntx, r = t / ta.ntx;
  const int ty = r % ta.nty, tz = r / ta.nty;
  const int x0 = tx * TL_X, y0 = ty * TL_Y, z0 = tz * TL_Z;
  // the TMA reads data written by generic stores before the last grid
  // barrier, and overwrites a stage that generic stores wrote
  asm volatile("fence.proxy.async;" ::: "memory");
  mbar_expect_tx(bar, TL_A_BYTES + (j >= 2 ? TL_B_BYTES : 0) + TL_K_BYTES);
  tma_load_4d(smem_u32(stg), &ta.tmA, x0 - 4, y0 - 2, z0 - 2, j - 1, bar);
  if (j >= 2) tma_load_4d(smem_u32(stg + TL_A_BYTES), &ta.tmB, x0 - 4, y0 - 1, z0 - 1, j - 2, bar);
  tma_load_3d(smem_u32(stg + TL_A_BYTES + TL_B_BYTES), &ta.tmK, x0 - 16, y0 - 1, z0 - 1, bar);
}

struct TileSums {
  double d1, d2, d3;
};

// One Krylov vector by the tiled pass (see the file comment): V_j at the
// tile nodes and this thread's FP32 Dot2 sums |w_j|^2, <A w_j, w_j>,
// <A w_j, V_{j-1}>.  The stencil sums follow stencil(): axis 0, then axis 1,
// then the last axis.  `phase` holds the two stages' mbarrier parities
// (identical in every thread).  Returns false if a copy timed out.
static __device__ __noinline__ bool tile_lanczos_pass(const TileArgs& ta, const GridDev& g, float* __restrict__ Vj, int j,
                                               float ca, float cb, float cc, float cfac, float bc, float Dint,
                                               DevStatus* st, unsigned& phase, TileSums& out) {
  extern __shared__ __align__(128) unsigned char tl_smem[];
  Acc<float> d1, d2, d3;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int nx = g.n[2], ny = g.n[1], nz = g.n[0];
  const long long sy = g.stride[1], sz = g.stride[0];
  int t = tile_next(ta, blockIdx.x);
  int s = 0;
  if (t >= 0 && tid == 0) tile_issue(ta, tl_smem, 0, t, j);
  while (t >= 0) {
    const int tn = tile_next(ta, t + gridDim.x);
    if (tn >= 0 && tid == 0) tile_issue(ta, tl_smem, s ^ 1, tn, j);
    if (!mbar_wait(smem_u32(tl_smem + 2 * TL_STAGE + 8 * s), (phase >> s) & 1u, st)) return false;
    phase ^= 1u << s;
    float* sA = reinterpret_cast<float*>(tl_smem + s * TL_STAGE);
    float* sB = reinterpret_cast<float*>(tl_smem + s * TL_STAGE + TL_A_BYTES);
    const uint8_t* sK = tl_smem + s * TL_STAGE + TL_A_BYTES + TL_B_BYTES;
    const int tx = t % ta.ntx, r = t / ta.ntx;
    const int x0 = tx * TL_X, y0 = (r % ta.nty) * TL_Y, z0 = (r / ta.nty) * TL_Z;
    // w_j on the tile grown by one node, in place of V_{j-2} in sB
    constexpr int RX = TL_X + 2, RY = TL_Y + 2, RZ = TL_Z + 2;
    constexpr int AY = TL_AX, AZ = TL_AX * (TL_Y + 4);  // strides in sA
    constexpr int BY = TL_AX, BZ = TL_AX * RY;          // strides in sB
    for (int q = tid; q < RX * RY * RZ; q += nt) {
      const int row = q / RX, xi = q - row * RX;  // xi = x + 1
      const int yi = row % RY, zi = row / RY;     // yi = y + 1, zi = z + 1
      const int iB = zi * BZ + yi * BY + xi + 3;
      const uint8_t k = sK[zi * (TL_KX * RY) + yi * TL_KX + xi + 15];
      float w = 0.f;
      if (k != 0) {
        const int iA = (zi + 1) * AZ + (yi + 1) * AY + xi + 3;
        const float v = sA[iA];
        float sacc = -0.f;  // as stencil()
        sacc += sA[iA - AZ] + sA[iA + AZ];
        sacc += sA[iA - AY] + sA[iA + AY];
        sacc += sA[iA - 1] + sA[iA + 1];
        float D = Dint;
        if (k == 2) {
          const long long p = (long long)(z0 + zi - 1) * sz + (long long)(y0 + yi - 1) * sy + (x0 + xi - 1);
          D = __ldcg(ta.Dg + p);
        }
        const float y = cfac * (bc * sacc - D * v);
        w = j >= 2 ? ca * y + cb * v + cc * sB[iB] : ca * y + cb * v;
      }
      sB[iB] = w;
    }
    __syncthreads();
    // A w_j on the tile, the sums and V_j = w_j
    for (int q = tid; q < TL_X * TL_Y * TL_Z; q += nt) {
      const int x = q % TL_X, row = q / TL_X;
      const int y = row % TL_Y, z = row / TL_Y;
      const int iB = (z + 1) * BZ + (y + 1) * BY + x + 4;
      const float w = sB[iB];
      const uint8_t k = sK[(z + 1) * (TL_KX * RY) + (y + 1) * TL_KX + x + 16];
      if (k != 0) {
        float sacc = -0.f;
        sacc += sB[iB - BZ] + sB[iB + BZ];
        sacc += sB[iB - BY] + sB[iB + BY];
        sacc += sB[iB - 1] + sB[iB + 1];
        float D = Dint;
        const long long p = (long long)(z0 + z) * sz + (long long)(y0 + y) * sy + (x0 + x);
        if (k == 2) D = __ldcg(ta.Dg + p);
        const float zz = cfac * (bc * sacc - D * w);
        const float v1 = sA[(z + 2) * AZ + (y + 2) * AY + x + 4];
        d1.add(w, w);
        d2.add(zz, w);
        d3.add(zz, v1);
      }
      if (x0 + x < nx && y0 + y < ny && z0 + z < nz)
        __stcg(Vj + (long long)(z0 + z) * sz + (long long)(y0 + y) * sy + (x0 + x), w);
    }
    __syncthreads();
    t = tn;
    s ^= 1;
  }
  out.d1 = d1.value();
  out.d2 = d2.value();
  out.d3 = d3.value();
  return true;
}

}  // namespace etd
