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

struct NaCarver {
  char* base;
  size_t off = 0;
  template <typename T>
  T* take(size_t count) {
    off = (off + 255) & ~size_t(255);
    T* p = reinterpret_cast<T*>(base + off);
    off += count * sizeof(T);
    return p;
  }
};

bool grid_of(const etd_grid* grid, GridDev& g) {
  if (!grid || grid->ndim < 2 || grid->ndim > 4) return false;
  memset(&g, 0, sizeof(g));
  g.ndim = grid->ndim;
  long long size = 1;
  for (int d = 0; d < grid->ndim; ++d) {
    if (grid->n[d] < 8 || grid->n[d] > 65535) return false;
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
  // of the array is not a device address, so look the address up.
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NA_MAX_DEVICES) return ETD_ERR_CUDA;
  if (!g_scratch_ready[dev]) {
    void* addr = nullptr;
    if (cudaGetSymbolAddress(&addr, g_noalloc_scratch) != cudaSuccess || !addr) return ETD_ERR_CUDA;
    g_scratch_addr[dev] = addr;
    g_scratch_ready[dev] = true;
  }

  // Carve the fixed array.
  NaCarver cv{(char*)g_scratch_addr[dev]};
  const size_t G = (size_t)g.size;
  DevStatus* dst = cv.take<DevStatus>(1);
  StatsDev* stats = cv.take<StatsDev>(1);
  double* part = cv.take<double>(8 * MAX_BLOCKS);
  int* tiles = cv.take<int>(init_scratch_ints(g.size) + 1);
  uint8_t* kind = cv.take<uint8_t>(G);
  int* idx = cv.take<int>(G);
  int* ncomp = cv.take<int>(1);
  double* diag = cv.take<double>(G);
  double* V = cv.take<double>(G * (size_t)(m_max + 1));
  double* Yg = cv.take<double>(G);
  double* W1g = cv.take<double>(G);
  double* Yc = cv.take<double>(G);
  double* V1c = cv.take<double>(G);
  double* V2c = cv.take<double>(G);
  double* Z0 = cv.take<double>(G);
  double* Z1 = cv.take<double>(G);
  const size_t used = (cv.off + 255) & ~size_t(255);
  if (used > NA_BYTES) return ETD_ERR_WORKSPACE;

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
