// Tiled Lanczos pass for large 3D FP32 problems with a constant beta: one
// pass per Krylov vector instead of two.
//
// The split passes build V_j = ca Z_{j-1} + cb V_{j-1} + cc V_{j-2} from a
// stored Z_{j-1} = A V_{j-1} and then Z_j = A V_j: 8 vector accesses per
// point and Krylov vector.  Here Z_{j-1} is recomputed from V_{j-1} in shared
// memory: per 64 x 8 x 8 tile of the grid, TMA copies V_{j-1} on the tile
// grown by two nodes, V_{j-2} and the row diagonals on the tile grown by one;
// A V_{j-1} and w_j = ca A V_{j-1} + cb V_{j-1} + cc V_{j-2} are formed on the
// tile grown by one (w_j = 0 off the computational set), then A w_j and the
// three sums on the tile, and V_j = w_j is stored.  HBM traffic per point is
// 3 vectors (V_{j-1}, V_{j-2} read, V_j written) and the diagonal; the halos
// come from L2.  Two stages: the next tile's copies are in flight while this
// one is computed.
//
// The diagonals (per launch, from the domain set-up): Dg = D_p (FP32) at the
// computational points and 0 elsewhere, so that Dg != 0 marks the
// computational set (D_p >= the row's interior faces' beta > 0).
#pragma once
#include <cuda.h>

#include "common.cuh"

namespace etd {

constexpr int TL_X = 64, TL_Y = 8, TL_Z = 8;   // tile (x the last, fastest axis)
constexpr int TL_AX = TL_X + 8;                 // x extent of the staged rows (16-byte aligned start x0 - 4)
constexpr int TL_A_BYTES = TL_AX * (TL_Y + 4) * (TL_Z + 4) * 4;  // V_{j-1}, two-node halo
constexpr int TL_B_BYTES = TL_AX * (TL_Y + 2) * (TL_Z + 2) * 4;  // V_{j-2}, one-node halo
constexpr int TL_D_BYTES = TL_B_BYTES;                           // diagonals, one-node halo
constexpr int TL_STAGE = TL_A_BYTES + TL_B_BYTES + TL_D_BYTES;
constexpr int TL_SMEM = 2 * TL_STAGE + 128;  // two stages and the two mbarriers
static_assert(TL_A_BYTES % 128 == 0 && TL_B_BYTES % 128 == 0, "stage alignment");

// Everything the tiled pass needs: the tensor maps (V as a 4D array x, y,
// z, basis slot with the two box sizes; the diagonals as a 3D array), the
// diagonal array and the tile grid with its activity flags.
struct TileArgs {
  CUtensorMap tmA;  // V, box TL_AX x (TL_Y + 4) x (TL_Z + 4) x 1
  CUtensorMap tmB;  // V, box TL_AX x (TL_Y + 2) x (TL_Z + 2) x 1
  CUtensorMap tmD;  // Dg, box TL_AX x (TL_Y + 2) x (TL_Z + 2)
  int enabled;
  int ntx, nty, ntz, ntiles;
  float* Dg;       // full grid: D_p at the computational points, 0 elsewhere
  uint8_t* flags;  // per tile: any computational node
  int* list;       // the active tiles in order (ntiles entries)
  int* cnt;        // per CTA: active tiles in its range (MAX_BLOCKS entries)
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

// Largest number of tiles a CTA takes per pass (its list lives in shared
// memory).
constexpr int TL_CAP = 512;

// This CTA's tiles: entries blockIdx.x + i gridDim.x of the ordered list of
// active tiles (consecutive CTAs take consecutive tiles, so the tiles in
// flight at a time are neighbours and share their halos in L2).  Returns
// their number.
__device__ __forceinline__ int tile_list(const TileArgs& ta, int ntotal, int* s_list) {
  const int n = ntotal > (int)blockIdx.x ? (ntotal - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x : 0;
  for (int i = threadIdx.x; i < n && i < TL_CAP; i += blockDim.x)
    s_list[i] = __ldcg(ta.list + blockIdx.x + (long long)i * gridDim.x);
  __syncthreads();
  return n < TL_CAP ? n : TL_CAP;
}

// Issues the copies of tile t for Krylov vector j into stage s (one thread).
// The copies of V_{j-2} are skipped for j == 1 (its coefficient is 0).  The
// stage was written by generic stores (w_j in place of V_{j-2}): a proxy
// fence on shared memory orders them before the copies.
__device__ __forceinline__ void tile_issue(const TileArgs& ta, unsigned char* base, int s, int t, int j) {
  unsigned char* stg = base + s * TL_STAGE;
  const uint32_t bar = smem_u32(base + 2 * TL_STAGE + 8 * s);
  const int tx = t % ta.ntx, r = t / ta.ntx;
  const int ty = r % ta.nty, tz = r / ta.nty;
  const int x0 = tx * TL_X, y0 = ty * TL_Y, z0 = tz * TL_Z;
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  mbar_expect_tx(bar, TL_A_BYTES + (j >= 2 ? TL_B_BYTES : 0) + TL_D_BYTES);
  tma_load_4d(smem_u32(stg), &ta.tmA, x0 - 4, y0 - 2, z0 - 2, j - 1, bar);
  if (j >= 2) tma_load_4d(smem_u32(stg + TL_A_BYTES), &ta.tmB, x0 - 4, y0 - 1, z0 - 1, j - 2, bar);
  tma_load_3d(smem_u32(stg + TL_A_BYTES + TL_B_BYTES), &ta.tmD, x0 - 4, y0 - 1, z0 - 1, bar);
}

struct TileSums {
  double d1, d2, d3;
};

__device__ __forceinline__ float f4at(const float4& v, int l) {
  return l == 0 ? v.x : l == 1 ? v.y : l == 2 ? v.z : v.w;
}

// One Krylov vector by the tiled pass (see the file comment): V_j at the
// tile nodes and this thread's FP32 Dot2 sums |w_j|^2, <A w_j, w_j>,
// <A w_j, V_{j-1}>.  The stencil sums follow stencil(): axis 0, then axis 1,
// then the last axis.  Threads take groups of 4 nodes along the last axis
// (16-byte shared-memory accesses), in step 1 two groups' loads issued
// before either is computed; the grown region's two boundary columns are
// taken node by node.  s_list / ntl: this CTA's tiles
// (tile_list).  `phase` holds the two stages' mbarrier parities (identical
// in every thread).  Returns false if a copy timed out.
static __device__ __noinline__ bool tile_lanczos_pass(const TileArgs& ta, const GridDev& g, float* __restrict__ Vj,
                                                      int j, float ca, float cb, float cc, float cfac, float bc,
                                                      DevStatus* st, unsigned& phase, const int* s_list, int ntl,
                                                      TileSums& out) {
  extern __shared__ __align__(128) unsigned char tl_smem[];
  static_assert(TL_X == 64 && TL_Y == 8 && TL_Z == 8, "the offsets below assume 64 x 8 x 8 tiles");
  Acc<float> d1, d2, d3;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int nx = g.n[2], ny = g.n[1], nz = g.n[0];
  const long long sy = g.stride[1], sz = g.stride[0];
  constexpr int RY = TL_Y + 2, RZ = TL_Z + 2;
  constexpr int AY = TL_AX, AZ = TL_AX * (TL_Y + 4);  // strides in sA (floats)
  constexpr int BY = TL_AX, BZ = TL_AX * RY;          // strides in sB and sD
  constexpr int QX = TL_X / 4;                        // 4-node groups per row
  constexpr int N1 = QX * RY * RZ;                    // groups of the grown tile (1600)
  constexpr int N2 = QX * TL_Y * TL_Z;                // groups of the tile (1024)
  // node (x, y, z) of the tile (x in [-4, 68)) at sA[(z + 2) AZ + (y + 2) AY
  // + x + 4] (y, z in [-2, 10)) and sB, sD[(z + 1) BZ + (y + 1) BY + x + 4]
  // (y, z in [-1, 9)).  This thread's work: step 1 groups q = tid + 512 u
  // (u < 4), the boundary-column node q = tid (< 200), step 2 groups (u < 2).
  // step 1 group u of this thread: offsets in sA and sB (-1: none)
  auto grp1 = [&](int u, int& iA, int& iB) {
    const int q = tid + u * nt, row = q / QX, x = (q - row * QX) * 4;
    const int y = row % RY - 1, z = row / RY - 1;
    iA = q < N1 ? (z + 2) * AZ + (y + 2) * AY + x + 4 : -1;
    iB = (z + 1) * BZ + (y + 1) * BY + x + 4;
  };
  int ah, bh;
  {
    const int row = tid >> 1, x = (tid & 1) ? TL_X : -1;
    const int y = row % RY - 1, z = row / RY - 1;
    ah = tid < 2 * RY * RZ ? (z + 2) * AZ + (y + 2) * AY + x + 4 : -1;
    bh = (z + 1) * BZ + (y + 1) * BY + x + 4;
  }
  // (the tile-relative grid offset fits 32 bits: z <= 7 and nz >= 8)
  int b2[2], a2[2], o2[2];
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    const int q = tid + u * nt, row = q / QX, x = (q - row * QX) * 4;
    const int y = row % TL_Y, z = row / TL_Y;
    b2[u] = q < N2 ? (z + 1) * BZ + (y + 1) * BY + x + 4 : -1;
    a2[u] = (z + 2) * AZ + (y + 2) * AY + x + 4;
    o2[u] = (int)((long long)z * sz + (long long)y * sy + x);
  }
  // the copies read vectors written by generic stores before the last grid
  // barrier: one global proxy fence per pass (by the issuing thread)
  if (tid == 0) asm volatile("fence.proxy.async.global;" ::: "memory");
  if (ntl > 0 && tid == 0) tile_issue(ta, tl_smem, 0, s_list[0], j);
  for (int it = 0; it < ntl; ++it) {
    const int s = it & 1;
    const int t = s_list[it];
    if (!mbar_wait(smem_u32(tl_smem + 2 * TL_STAGE + 8 * s), (phase >> s) & 1u, st)) return false;
    phase ^= 1u << s;
    const float* sA = reinterpret_cast<const float*>(tl_smem + s * TL_STAGE);
    float* sB = reinterpret_cast<float*>(tl_smem + s * TL_STAGE + TL_A_BYTES);
    const float* sD = reinterpret_cast<const float*>(tl_smem + s * TL_STAGE + TL_A_BYTES + TL_B_BYTES);
    const int tx = t % ta.ntx, r = t / ta.ntx;
    const int x0 = tx * TL_X, y0 = (r % ta.nty) * TL_Y, z0 = (r / ta.nty) * TL_Z;
    auto wval = [&](float v, float sacc, float v2, float D) {
      const float y = cfac * (bc * sacc - D * v);
      return j >= 2 ? ca * y + cb * v + cc * v2 : ca * y + cb * v;
    };
    // 1. w_j on the tile grown by one node, in place of V_{j-2} in sB:
    //    4-node groups for x in [0, 64), two at a time ...
#pragma unroll 1
    for (int u0 = 0; u0 < 4; u0 += 2) {
      float4 D4[2], c[2], zm[2], zp[2], ym[2], yp[2], v2[2];
      float xl[2], xr[2];
      int gA[2], gB[2];
      grp1(u0, gA[0], gB[0]);
      grp1(u0 + 1, gA[1], gB[1]);
#pragma unroll
      for (int v = 0; v < 2; ++v) {
        const int iA = gA[v], iB = gB[v];
        if (iA < 0) continue;
        D4[v] = *reinterpret_cast<const float4*>(sD + iB);
        c[v] = *reinterpret_cast<const float4*>(sA + iA);
        zm[v] = *reinterpret_cast<const float4*>(sA + iA - AZ);
        zp[v] = *reinterpret_cast<const float4*>(sA + iA + AZ);
        ym[v] = *reinterpret_cast<const float4*>(sA + iA - AY);
        yp[v] = *reinterpret_cast<const float4*>(sA + iA + AY);
        xl[v] = sA[iA - 1];
        xr[v] = sA[iA + 4];
        v2[v] = *reinterpret_cast<const float4*>(sB + iB);
      }
#pragma unroll
      for (int v = 0; v < 2; ++v) {
        if (gA[v] < 0) continue;
        float wl[4];
#pragma unroll
        for (int l = 0; l < 4; ++l) {
          const float D = f4at(D4[v], l);
          float sacc = -0.f;  // as stencil()
          sacc += f4at(zm[v], l) + f4at(zp[v], l);
          sacc += f4at(ym[v], l) + f4at(yp[v], l);
          sacc += (l == 0 ? xl[v] : f4at(c[v], l - 1)) + (l == 3 ? xr[v] : f4at(c[v], l + 1));
          wl[l] = D != 0.f ? wval(f4at(c[v], l), sacc, f4at(v2[v], l), D) : 0.f;
        }
        *reinterpret_cast<float4*>(sB + gB[v]) = make_float4(wl[0], wl[1], wl[2], wl[3]);
      }
    }
    // ... and node by node for the columns x = -1 and x = 64
    if (ah >= 0) {
      const float D = sD[bh];
      float w = 0.f;
      if (D != 0.f) {
        float sacc = -0.f;
        sacc += sA[ah - AZ] + sA[ah + AZ];
        sacc += sA[ah - AY] + sA[ah + AY];
        sacc += sA[ah - 1] + sA[ah + 1];
        w = wval(sA[ah], sacc, sB[bh], D);
      }
      sB[bh] = w;
    }
    __syncthreads();
    // the next tile's copies, into the other stage (free since the previous
    // tile's end): they land while step 2 runs.  Issued here rather than
    // before step 1 because the shared-memory proxy fence waits for the
    // issuing thread's global stores, none of which are in flight now.
    if (it + 1 < ntl && tid == 0) tile_issue(ta, tl_smem, s ^ 1, s_list[it + 1], j);
    // 2. A w_j on the tile, the sums and V_j = w_j (one group at a time: the
    //    4 x 3 Dot2 chains of a group already run side by side)
    const long long tbase = (long long)z0 * sz + (long long)y0 * sy + x0;
#pragma unroll
    for (int v = 0; v < 2; ++v) {
      const int iB = b2[v];
      if (iB < 0) continue;
      const float4 c = *reinterpret_cast<const float4*>(sB + iB);
      const float4 D4 = *reinterpret_cast<const float4*>(sD + iB);
      const float4 zm = *reinterpret_cast<const float4*>(sB + iB - BZ);
      const float4 zp = *reinterpret_cast<const float4*>(sB + iB + BZ);
      const float4 ym = *reinterpret_cast<const float4*>(sB + iB - BY);
      const float4 yp = *reinterpret_cast<const float4*>(sB + iB + BY);
      const float xl = sB[iB - 1], xr = sB[iB + 4];
      const float4 v1 = *reinterpret_cast<const float4*>(sA + a2[v]);
#pragma unroll
      for (int l = 0; l < 4; ++l) {
        const float D = f4at(D4, l);
        if (D != 0.f) {
          float sacc = -0.f;
          sacc += f4at(zm, l) + f4at(zp, l);
          sacc += f4at(ym, l) + f4at(yp, l);
          sacc += (l == 0 ? xl : f4at(c, l - 1)) + (l == 3 ? xr : f4at(c, l + 1));
          const float w = f4at(c, l);
          const float zz = cfac * (bc * sacc - D * w);
          d1.add(w, w);
          d2.add(zz, w);
          d3.add(zz, f4at(v1, l));
        }
      }
      const int zr = iB / BZ - 1, yr = (iB - (zr + 1) * BZ) / BY - 1, xg = iB - (zr + 1) * BZ - (yr + 1) * BY - 4;
      if (x0 + xg < nx && y0 + yr < ny && z0 + zr < nz) __stcg(reinterpret_cast<float4*>(Vj + tbase + o2[v]), c);
    }
    __syncthreads();
  }
  out.d1 = d1.value();
  out.d2 = d2.value();
  out.d3 = d3.value();
  return true;
}

}  // namespace etd
