// etd_phi_combination_noalloc: the phi-combination for callers that cannot
// allocate device memory.  All scratch lives in one fixed, file-scope device
// array; the caller passes only the level set, the three input vectors and
// the output.
#include <cstring>

#include "etd_gb300.h"
#include "kernels.cuh"

using namespace etd;

namespace {

// Largest problem the fixed scratch holds: every layout below is carved from
// this array; etd_phi_combination_noalloc rejects larger grids or bases.
constexpr long long NA_MAX_NODES = ETD_NOALLOC_MAX_NODES;
constexpr int NA_MAX_M = ETD_NOALLOC_MAX_M;
constexpr size_t NA_BYTES = ETD_NOALLOC_SCRATCH_BYTES;

constexpr int NA_MAX_DEVICES = 64;
void* g_scratch_addr[NA_MAX_DEVICES];
bool g_scratch_ready[NA_MAX_DEVICES];

}  // namespace

// Every GPU that loads the library holds this array until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[ETD_NOALLOC_SCRATCH_BYTES];

namespace {

// Byte offsets of the buffers in the fixed array for a grid of G nodes and
// a basis of at most m vectors (each buffer 256-byte aligned).  constexpr, so
// that the limits below are checked against the array size at compile time.
struct NaLayout {
  size_t st, stats, part, tiles, kind, idx, ncomp, diag, V, Yg, W1g, Yc, V1c, V2c, Z0, Z1, total;
};
constexpr size_t na_up(size_t o) { return (o + 255) & ~size_t(255); }
constexpr NaLayout na_layout(size_t G, int m) {
  NaLayout L{};
  size_t o = 0;
  L.st = o;
  o = na_up(o + sizeof(DevStatus));
  L.stats = o;
  o = na_up(o + sizeof(StatsDev));
  L.part = o;
  o = na_up(o + sizeof(double) * 8 * MAX_BLOCKS);
  L.tiles = o;
  o = na_up(o + sizeof(int) * ((size_t)init_scratch_ints((long long)G) + 1));
  L.kind = o;
  o = na_up(o + G);
  L.idx = o;
  o = na_up(o + sizeof(int) * G);
  L.ncomp = o;
  o = na_up(o + sizeof(int));
  L.diag = o;
  o = na_up(o + sizeof(double) * G);
  L.V = o;
  o = na_up(o + sizeof(double) * G * (size_t)(m + 1));
  size_t* vec[7] = {&L.Yg, &L.W1g, &L.Yc, &L.V1c, &L.V2c, &L.Z0, &L.Z1};
  for (int i = 0; i < 7; ++i) {
    *vec[i] = o;
    o = na_up(o + sizeof(double) * G);
  }
  L.total = o;
  return L;
}
static_assert(na_layout(ETD_NOALLOC_MAX_NODES, ETD_NOALLOC_MAX_M).total <= ETD_NOALLOC_SCRATCH_BYTES,
              "the documented largest problem must fit the fixed scratch array");

bool grid_of(const etd_grid* grid, GridDev& g) {
  if (!grid || grid->ndim < 2 || grid->ndim > 4) return false;
  memset(&g, 0, sizeof(g));
  g.ndim = grid->ndim;
  long long size = 1;
  for (int d = 0; d < grid->ndim; ++d) {
    if (grid->n[d] < 8 || grid->n[d] > 65535) return false;
    // no wrap-around: stop as soon as the size would pass 2^31 - 1
    if (size > 2147483647LL / grid->n[d]) return false;
    g.n[d] = grid->n[d];
    size *= grid->n[d];
  }
  g.size = size;
  long long s = 1;
  for (int d = grid->ndim - 1; d >= 0; --d) {
    g.stride[d] = s;
    s *= grid->n[d];
  }
  grid_divisors(g);
  const double h0 = (grid->hi[0] - grid->lo[0]) / (grid->n[0] - 1);
  if (!(h0 > 0.0)) return false;
  for (int d = 0; d < grid->ndim; ++d) {
    const double hd = (grid->hi[d] - grid->lo[d]) / (grid->n[d] - 1);
    if (fabs(hd - h0) > 1e-12 * h0) return false;
    g.lo[d] = grid->lo[d];
  }
  g.h = h0;
  return true;
}

}  // namespace

extern "C" etd_status etd_phi_combination_noalloc(const etd_grid* grid, const double* phi, double beta, double dt,
                                                  const double* v0, const double* v1, const double* v2, double* y,
                                                  double krylov_tol, int m_max, void* stream) {
  GridDev g;
  if (!grid_of(grid, g) || !phi || !v0 || !v1 || !v2 || !y || !(dt > 0.0) || !(beta > 0.0) ||
      !(krylov_tol > 0.0) || m_max < 5)
    return ETD_ERR_ARG;
  if (g.size > NA_MAX_NODES || m_max > NA_MAX_M) return ETD_ERR_WORKSPACE;
  cudaStream_t st = (cudaStream_t)stream;

  // One-time set-up per device, with that device current: the host-side name
  // of the array is not a device address, so look the address up.  The
  // cached address belongs to the device's primary context (see the header
  // on resets).
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NA_MAX_DEVICES) return ETD_ERR_CUDA;
  if (st != nullptr) {
    // the kernels run on the stream's device, the array is the current one's
    int sdev = -1;
    if (cudaStreamGetDevice(st, &sdev) != cudaSuccess) return ETD_ERR_CUDA;
    if (sdev != dev) return ETD_ERR_ARG;
  }
  if (!g_scratch_ready[dev]) {
    void* addr = nullptr;
    if (cudaGetSymbolAddress(&addr, g_noalloc_scratch) != cudaSuccess || !addr) return ETD_ERR_CUDA;
    g_scratch_addr[dev] = addr;
    g_scratch_ready[dev] = true;
  }

  // Carve the fixed array.
  const NaLayout L = na_layout((size_t)g.size, m_max);
  if (L.total > NA_BYTES) return ETD_ERR_WORKSPACE;
  char* base = (char*)g_scratch_addr[dev];
  DevStatus* dst = reinterpret_cast<DevStatus*>(base + L.st);
  StatsDev* stats = reinterpret_cast<StatsDev*>(base + L.stats);
  double* part = reinterpret_cast<double*>(base + L.part);
  int* tiles = reinterpret_cast<int*>(base + L.tiles);
  uint8_t* kind = reinterpret_cast<uint8_t*>(base + L.kind);
  int* idx = reinterpret_cast<int*>(base + L.idx);
  int* ncomp = reinterpret_cast<int*>(base + L.ncomp);
  double* diag = reinterpret_cast<double*>(base + L.diag);
  double* V = reinterpret_cast<double*>(base + L.V);
  double* Yg = reinterpret_cast<double*>(base + L.Yg);
  double* W1g = reinterpret_cast<double*>(base + L.W1g);
  double* Yc = reinterpret_cast<double*>(base + L.Yc);
  double* V1c = reinterpret_cast<double*>(base + L.V1c);
  double* V2c = reinterpret_cast<double*>(base + L.V2c);
  double* Z0 = reinterpret_cast<double*>(base + L.Z0);
  double* Z1 = reinterpret_cast<double*>(base + L.Z1);
  const size_t used = L.total;

  // The array keeps the previous call's contents: start from zero (status,
  // node kinds, and the zero entries every stencil input needs off the
  // computational set).
  if (cudaMemsetAsync(g_scratch_addr[dev], 0, used, st) != cudaSuccess) return ETD_ERR_CUDA;

  ClassifyArgs ca;
  memset(&ca, 0, sizeof(ca));
  ca.g = g;
  ca.phi = phi;
  ca.kind = kind;
  ca.tile_count = tiles;
  ca.st = dst;
  ca.nzero = 0;
  ca.nbasis = 0;
  MetaArgs ma;
  memset(&ma, 0, sizeof(ma));
  ma.g = g;
  ma.phi = phi;
  ma.kind = kind;
  ma.idx = idx;
  ma.ncomp = ncomp;
  ma.beta_field = nullptr;
  ma.beta_c = beta;
  ma.diag = diag;
  ma.diagf = nullptr;
  ma.gersh = &dst->gersh[0];
  ma.st = dst;
  if (launch_init_domain(ca, ma, tiles, ncomp, st) != cudaSuccess) return ETD_ERR_CUDA;

  PhipmArgs<double> a;
  memset(&a, 0, sizeof(a));
  a.g = g;
  a.nspecies = 1;
  a.mode = MODE_GIVEN;
  a.m_max = m_max;
  a.dt = dt;
  a.cfac = dt / (g.h * g.h);
  a.tol = krylov_tol;
  SpeciesDev<double>& S = a.sp[0];
  S.idx = idx;
  S.ncomp = ncomp;
  S.diag = diag;
  S.kind = kind;
  S.beta_field = nullptr;
  S.beta_c = beta;
  S.gersh = &dst->gersh[0];
  S.u = y;
  S.V = V;
  S.Yg = Yg;
  S.W1g = W1g;
  S.Yc = Yc;
  S.V1c = V1c;
  S.V2c = V2c;
  S.Z[0] = Z0;
  S.Z[1] = Z1;
  a.given[0] = v0;
  a.given[1] = v1;
  a.given[2] = v2;
  a.part = part;
  a.st = dst;
  a.stats = stats;
  const int nblocks = phipm_max_blocks(g.ndim, false);
  if (nblocks <= 0 || nblocks > MAX_BLOCKS) return ETD_ERR_CUDA;
  if (launch_phipm<double>(a, nblocks, st) != cudaSuccess) return ETD_ERR_CUDA;

  // Synchronise and report device-side errors.
  if (cudaStreamSynchronize(st) != cudaSuccess) return ETD_ERR_CUDA;
  int err = 0;
  if (cudaMemcpy(&err, &dst->err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return ETD_ERR_CUDA;
  if (err & ERRF_TIMEOUT) return ETD_ERR_TIMEOUT;
  if (err & ERRF_NONFINITE) return ETD_ERR_NONFINITE;
  if (err & ERRF_DOMAIN) return ETD_ERR_DOMAIN;
  if (err & ERRF_KRYLOV) return ETD_ERR_KRYLOV;
  if (err) return ETD_ERR_ARG;
  return ETD_OK;
}
