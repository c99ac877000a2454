// C ABI: context, workspace carving, argument checks and launches.
#include <nvtx3/nvToolsExt.h>

#include <cstdio>
#include <cstring>
#include <string>

#include "etd_gb300.h"
#include "kernels.cuh"
#include "levelset.cuh"

using namespace etd;

struct SpeciesBufs {
  uint8_t* kind = nullptr;
  int* idx = nullptr;
  int* ncomp = nullptr;
  double* diag = nullptr;
  float* diagf = nullptr;
  double* Fprev = nullptr;
  double* Fprev2 = nullptr;  // multistep ETD3
  uint8_t* fvalid = nullptr;
  void* V = nullptr;
  void* Yg = nullptr;
  void* W1g = nullptr;
  double* Yc = nullptr;
  void* V1c = nullptr;
  void* V2c = nullptr;
  void* V3c = nullptr;  // phi_3 combinations
  void* W2g = nullptr;
  void* Z[2] = {nullptr, nullptr};
  double* stg[3] = {nullptr, nullptr, nullptr};  // ETD3RK / ETD4RK stage fields
  int* qidx = nullptr;  // FP32 contexts: aligned 4-node groups of the large split passes
  int* qk = nullptr;
  int* qmeta = nullptr;  // the list's validity flag and length (zeroed by every domain set-up)
  const double* beta_field = nullptr;
  // boundary data (params.boundary_data): per point, face and slot
  double* bco = nullptr;
  double* bpts = nullptr;
  // caller's source fields and boundary values at t_n and t_{n+1} (device,
  // caller-owned; the t_{n+1} ones are read by the second ETD2RK stage)
  const double* src[2] = {nullptr, nullptr};
  const double* bval[2] = {nullptr, nullptr};
  bool ready = false;
};

struct etd_ctx {
  etd_grid grid;
  etd_params par;
  GridDev g;
  cudaStream_t stream = nullptr;
  char* ws = nullptr;
  size_t ws_bytes = 0;
  DevStatus* st = nullptr;
  StatsDev* stats = nullptr;
  double* part = nullptr;
  int* tile_count = nullptr;
  double* pout = nullptr;  // 2 doubles: Poisson solve iterations and residual
  SpeciesBufs sp[2];
  LevelsetBufs ls;
  // adjoint (species 0): phi actions, right-hand sides, face weights, and
  // mu(t_i), y(t_i) at the quadrature times
  double* adj[8] = {nullptr};
  double* adj_mu[ADJ_NQ_MAX] = {nullptr};
  double* adj_y[ADJ_NQ_MAX] = {nullptr};
  double* facew = nullptr;
  int nblocks = 0;
  bool fp32 = false;
  int last_nspecies = 0;
  int last_species0 = 0;
  unsigned long long wait_ns = 0;  // host copy of the device-wait limit (0: default)
  // FP32 contexts: each species' computational-point count, copied back
  // after every domain set-up without a wait (pinned, an event per copy);
  // the Krylov launch takes the 768-thread kernel when a species with the
  // latest count that has arrived runs on the 4-node groups
  int* ncomp_host = nullptr;
  cudaEvent_t ncomp_ev[2] = {nullptr, nullptr};
  bool ncomp_pending[2] = {false, false};
  int ncomp_known[2] = {-1, -1};
  std::string err;
  ~etd_ctx() {
    for (cudaEvent_t ev : ncomp_ev)
      if (ev) cudaEventDestroy(ev);
    if (ncomp_host) cudaFreeHost(ncomp_host);
  }
};

namespace {

// NVTX range over an entry point (a named range on the host timeline of a
// profiler; header-only NVTX, inert without one)
struct Range {
  explicit Range(const char* name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
};

struct Carver {
  char* base;
  size_t off = 0;
  template <typename T>
  T* take(size_t count) {
    off = (off + 255) & ~size_t(255);
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += count * sizeof(T);
    return p;
  }
};

bool check_grid(const etd_grid* grid, GridDev& g, std::string& why) {
  if (!grid || grid->ndim < 2 || grid->ndim > 4) {
    why = "ndim must be 2, 3 or 4";
    return false;
  }
  memset(&g, 0, sizeof(g));
  g.ndim = grid->ndim;
  long long size = 1;
  for (int d = 0; d < grid->ndim; ++d) {
    if (grid->n[d] < 8 || grid->n[d] > 65535) {
      why = "each axis needs 8 to 65535 nodes";
      return false;
    }
    // checked before the product, which could otherwise wrap around
    if (size > 2147483647LL / grid->n[d]) {
      why = "grid larger than 2^31 - 1 nodes";
      return false;
    }
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
  double h0 = (grid->hi[0] - grid->lo[0]) / (grid->n[0] - 1);
  if (!(h0 > 0.0)) {
    why = "hi must exceed lo";
    return false;
  }
  for (int d = 0; d < grid->ndim; ++d) {
    double hd = (grid->hi[d] - grid->lo[d]) / (grid->n[d] - 1);
    if (fabs(hd - h0) > 1e-12 * h0) {
      why = "grid spacing must be the same on every axis";
      return false;
    }
    g.lo[d] = grid->lo[d];
  }
  g.h = h0;
  return true;
}

bool check_params(const etd_params* p, std::string& why) {
  if (!p) {
    why = "params is NULL";
    return false;
  }
  if (p->nspecies < 1 || p->nspecies > 2) {
    why = "nspecies must be 1 or 2";
    return false;
  }
  if (p->precision != ETD_PRECISION_FP64 && p->precision != ETD_PRECISION_MIXED) {
    why = "unknown precision";
    return false;
  }
  if (p->m_max < 5 || p->m_max > MAX_M) {
    why = "m_max must be in [5, 61]";
    return false;
  }
  if (!(p->krylov_tol > 0.0)) {
    why = "krylov_tol must be positive";
    return false;
  }
  if (p->scheme < 0 || p->scheme > ETD_SCHEME_ETD3) {
    why = "unknown scheme";
    return false;
  }
  if ((p->scheme == ETD_SCHEME_ETD3RK || p->scheme == ETD_SCHEME_ETD4RK || p->scheme == ETD_SCHEME_ETD3) &&
      p->m_max > MAX_M - 1) {
    why = "ETD3RK, ETD4RK and ETD3 need m_max <= 60";
    return false;
  }
  if (p->reaction < 0 || p->reaction > 3 || (p->reaction == ETD_REACTION_COMPETITION && p->nspecies != 2)) {
    why = "unknown reaction, or competition without two species";
    return false;
  }
  for (int s = 0; s < p->nspecies; ++s) {
    if (!(p->beta[s] > 0.0)) {
      why = "beta must be positive";
      return false;
    }
  }
  return true;
}

size_t carve(const GridDev& g, const etd_params& p, char* base, etd_ctx* c) {
  Carver cv{base};
  const size_t G = (size_t)g.size;
  const bool f32 = p.precision == ETD_PRECISION_MIXED;
  const size_t s = f32 ? 4 : 8;
  DevStatus* st = cv.take<DevStatus>(1);
  StatsDev* stats = cv.take<StatsDev>(1);
  double* part = cv.take<double>(8 * MAX_BLOCKS);
  double* pout = cv.take<double>(2);
  int* tiles = cv.take<int>(init_scratch_ints(g.size) + 1);
  if (c) {
    c->st = st;
    c->stats = stats;
    c->part = part;
    c->pout = pout;
    c->tile_count = tiles;
  }
  for (int sp = 0; sp < p.nspecies; ++sp) {
    SpeciesBufs b;
    b.kind = cv.take<uint8_t>(G);
    b.idx = cv.take<int>(G);
    b.ncomp = cv.take<int>(1);
    b.diag = cv.take<double>(G);
    b.diagf = f32 ? cv.take<float>(G) : nullptr;
    b.Fprev = cv.take<double>(G);
    b.Fprev2 = p.scheme == ETD_SCHEME_ETD3 ? cv.take<double>(G) : nullptr;
    b.fvalid = cv.take<uint8_t>(G);
    b.V = cv.take<char>(s * G * (p.m_max + 1));
    b.Yg = cv.take<char>(s * G);
    b.W1g = cv.take<char>(s * G);
    b.Yc = cv.take<double>(G);
    b.V1c = cv.take<char>(s * G);
    b.V2c = cv.take<char>(s * G);
    b.Z[0] = cv.take<char>(s * G);
    b.Z[1] = cv.take<char>(s * G);
    b.V3c = cv.take<char>(s * G);
    b.W2g = cv.take<char>(s * G);
    if (p.scheme == ETD_SCHEME_ETD3RK || p.scheme == ETD_SCHEME_ETD4RK)
      for (int i = 0; i < 3; ++i) b.stg[i] = cv.take<double>(G);
    if (f32) {
      b.qidx = cv.take<int>(G / 4 + 1);
      b.qk = cv.take<int>(G / 4 + 1);
      b.qmeta = cv.take<int>(2);
    }
    if (c) c->sp[sp] = b;
  }
  LevelsetBufs lb = levelset_carve(g, [&](size_t bytes) { return cv.take<char>(bytes); });
  if (c) c->ls = lb;
  if (p.boundary_data) {
    const size_t slots = G * 2 * (size_t)g.ndim * (g.ndim == 2 ? 2 : 1);
    for (int sp = 0; sp < p.nspecies; ++sp) {
      double* bco = cv.take<double>(slots);
      double* bpts = cv.take<double>(slots * (size_t)g.ndim);
      if (c) {
        c->sp[sp].bco = bco;
        c->sp[sp].bpts = bpts;
      }
    }
  }
  if (p.adjoint) {
    for (int i = 0; i < 8; ++i) {
      double* b = cv.take<double>(G);
      if (c) c->adj[i] = b;
    }
    for (int i = 0; i < ADJ_NQ_MAX; ++i) {
      double* bm = cv.take<double>(G);
      double* by = cv.take<double>(G);
      if (c) {
        c->adj_mu[i] = bm;
        c->adj_y[i] = by;
      }
    }
    double* fw = cv.take<double>(G * 2 * (size_t)g.ndim);
    if (c) c->facew = fw;
  }
  cv.off = (cv.off + 255) & ~size_t(255);
  return cv.off;
}

etd_status fail(etd_ctx* c, etd_status code, const std::string& why) {
  if (c) c->err = why;
  return code;
}

etd_status cuda_fail(etd_ctx* c, cudaError_t e, const char* where) {
  return fail(c, ETD_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

etd_status read_status(etd_ctx* c) {
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "stream synchronise");
  int err = 0;
  e = cudaMemcpy(&err, &c->st->err, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(c, e, "status read");
  if (err == 0) return ETD_OK;
  int zero = 0;
  cudaMemcpy(&c->st->err, &zero, sizeof(int), cudaMemcpyHostToDevice);
  if (err & ERRF_TIMEOUT) return fail(c, ETD_ERR_TIMEOUT, "a bounded device wait timed out");
  if (err & ERRF_NONFINITE) return fail(c, ETD_ERR_NONFINITE, "non-finite value in a reduction");
  if (err & ERRF_DOMAIN) return fail(c, ETD_ERR_DOMAIN, "an inside node lies within 3 nodes of the box edge");
  if (err & ERRF_KRYLOV) return fail(c, ETD_ERR_KRYLOV, "Krylov tolerance not met at the smallest substep");
  if (err & ERRF_UNSUPPORTED)
    return fail(c, ETD_ERR_ARG, "nonzero boundary data at a case-3 ghost face is defined for N = 2 only");
  return fail(c, ETD_ERR_ARG, "a device list or trace outgrew its buffer");
}

etd_status copy_stats(etd_ctx* c, etd_step_stats* stats) {
  etd_status rs = read_status(c);
  StatsDev h;
  cudaError_t e = cudaMemcpy(&h, c->stats, sizeof(h), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(c, e, "stats read");
  memset(stats, 0, sizeof(*stats));
  for (int s = 0; s < c->last_nspecies; ++s) {
    const int so = c->last_species0 + s;
    int nc = 0;
    cudaMemcpy(&nc, c->sp[so].ncomp, sizeof(int), cudaMemcpyDeviceToHost);
    stats->ncomp[s] = nc;
    stats->substeps[s] = h.substeps[s];
    stats->rejections[s] = h.rejections[s];
    stats->krylov_iters[s] = h.iters[s];
    stats->trace_len[s] = h.trace_len[s];
    for (int i = 0; i < ETD_TRACE_MAX && i < TRACE_MAX; ++i) {
      stats->trace_m[s][i] = h.trace_m[s][i];
      stats->trace_tau[s][i] = h.trace_tau[s][i];
    }
  }
  return rs;
}

template <typename T>
SpeciesDev<T> species_dev(etd_ctx* c, int s, double* u, int stage = 0) {
  SpeciesBufs& b = c->sp[s];
  SpeciesDev<T> d;
  d.src = b.src[stage] ? b.src[stage] : b.src[0];
  d.bco = b.bco;
  d.bval = b.bval[stage] ? b.bval[stage] : b.bval[0];
  d.idx = b.idx;
  d.ncomp = b.ncomp;
  d.diag = b.diag;
  d.diagf = b.diagf;
  d.kind = b.kind;
  d.beta_field = b.beta_field;
  d.beta_c = c->par.beta[s];
  d.gersh = &c->st->gersh[s];
  d.u = u;
  d.Fprev = b.Fprev;
  d.Fprev2 = b.Fprev2;
  d.fvalid = b.fvalid;
  d.V = (T*)b.V;
  d.Yg = (T*)b.Yg;
  d.W1g = (T*)b.W1g;
  d.Yc = b.Yc;
  d.V1c = (T*)b.V1c;
  d.V2c = (T*)b.V2c;
  d.V3c = (T*)b.V3c;
  d.W2g = (T*)b.W2g;
  d.Z[0] = (T*)b.Z[0];
  d.Z[1] = (T*)b.Z[1];
  for (int i = 0; i < 3; ++i) d.stg[i] = b.stg[i];
  d.qidx = sizeof(T) == 4 ? b.qidx : nullptr;
  d.qk = sizeof(T) == 4 ? b.qk : nullptr;
  d.qmeta = sizeof(T) == 4 ? b.qmeta : nullptr;
  return d;
}

template <typename T>
etd_status run_phipm(etd_ctx* c, int mode, double dt, double* const* u, int species, const double* const* given,
                     etd_step_stats* stats, bool etd1 = false, bool keep_stats = false, int p = 2,
                     const StageDesc* stage = nullptr, int nq = 0, const double* tq = nullptr,
                     double* const* outs = nullptr) {
  PhipmArgs<T> a;
  memset(&a, 0, sizeof(a));
  a.g = c->g;
  a.mode = mode;
  a.m_max = c->par.m_max;
  a.dt = dt;
  a.cfac = dt / (c->g.h * c->g.h);
  a.tol = c->par.krylov_tol;
  a.reaction = c->par.reaction;
  for (int i = 0; i < 4; ++i) a.rp[i] = c->par.rp[i];
  a.etd1 = etd1 ? 1 : 0;
  a.ms3 = mode == MODE_ETD2 && c->par.scheme == ETD_SCHEME_ETD3 ? 1 : 0;
  a.p = a.ms3 ? 3 : p;
  if (stage) a.stage = *stage;
  a.nq = nq;
  for (int i = 0; i < nq; ++i) a.tq[i] = tq[i];
  const int nout = mode == MODE_ADJ_LAMBDA ? 3 + nq : mode == MODE_ADJ_Y ? nq : 0;
  for (int i = 0; i < nout; ++i) a.out[i] = outs[i];
  const bool all = mode == MODE_ETD2 || mode == MODE_RK2 || mode == MODE_STAGE;
  if (all) {
    a.nspecies = c->par.nspecies;
    for (int s = 0; s < a.nspecies; ++s) a.sp[s] = species_dev<T>(c, s, u[s], mode == MODE_RK2 ? 1 : 0);
  } else {
    a.nspecies = 1;
    a.sp[0] = species_dev<T>(c, species, u[0]);
    const int ng = mode == MODE_ADJ_LAMBDA ? 1 : mode == MODE_EXPLICIT || mode == MODE_ADJ_Y ? 2 : p + 1;
    for (int i = 0; i < ng; ++i) a.given[i] = given[i];
  }
  if (mode == MODE_EXPLICIT || mode == MODE_ADJ_Y) {
    a.reaction = c->par.reaction;
    for (int i = 0; i < 4; ++i) a.rp[i] = c->par.rp[i];
  }
  a.part = c->part;
  a.st = c->st;
  a.stats = c->stats;
  cudaError_t e = cudaSuccess;
  if (!keep_stats) {
    e = cudaMemsetAsync(c->stats, 0, sizeof(StatsDev), c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "stats reset");
  }
  // the 768-thread FP32 kernel when a species of this launch takes the
  // 4-node groups (its latest known point count; only the speed depends on it)
  bool wide = false;
  if (sizeof(T) == 4 && c->ncomp_host) {
    const int s0 = all ? 0 : species, s1 = all ? a.nspecies : species + 1;
    for (int s = s0; s < s1; ++s) {
      if (c->ncomp_pending[s] && cudaEventQuery(c->ncomp_ev[s]) == cudaSuccess) {
        c->ncomp_known[s] = c->ncomp_host[s];
        c->ncomp_pending[s] = false;
      }
      wide = wide || (c->ncomp_known[s] >= QUAD_MIN_POINTS && c->sp[s].beta_field == nullptr &&
                      c->g.n[c->g.ndim - 1] % 4 == 0);
    }
  }
  e = launch_phipm<T>(a, c->nblocks, c->stream, wide);
  if (e != cudaSuccess) return cuda_fail(c, e, "phipm launch");
  c->last_nspecies = a.nspecies;
  c->last_species0 = all ? 0 : species;
  if (!stats) return ETD_OK;
  return copy_stats(c, stats);
}

// ETD3RK and ETD4RK (Sec. 3.2) as a sequence of stage launches.  Each stage
// is one combination phi_0(h C) v_0 + h phi_1(h C) g_1 + h phi_2(h C) g_2
// + h phi_3(h C) g_3 with h = dt or dt / 2, v_0 = U_n or a_n, and g_j linear
// combinations of F(U_n), F(a_n), F(b_n), F(c_n) (U + h phi_1(h C) C U =
// phi_0(h C) U).  The paper's phi_3 (Eq. 3.7) is twice the standard phi_3
// that the kernel evaluates, so the tables hold the paper's phi_3
// coefficients times two.
struct RkStage {
  double dt_factor;
  int p;
  StageDesc d;
};
static const RkStage kEtd3rk[3] = {
    // a_n = U_n + dt/2 phi_1(dt C / 2)(F_n + C U_n)
    {0.5, 2, {0, 1, {{1, 0, 0, 0}, {0, 0, 0, 0}, {0, 0, 0, 0}}}},
    // b_n = U_n + dt phi_1(dt C)(C U_n + 2 F(a_n) - F_n)
    {1.0, 2, {0, 2, {{-1, 2, 0, 0}, {0, 0, 0, 0}, {0, 0, 0, 0}}}},
    // U_{n+1}: phi_1 (F_n), phi_2 (-3 F_n + 4 F(a_n) - F(b_n)), phi_3 2 x (2, -4, 2)
    {1.0, 3, {0, 0, {{1, 0, 0, 0}, {-3, 4, -1, 0}, {4, -8, 4, 0}}}}};
static const RkStage kEtd4rk[4] = {
    // a_n = U_n + dt/2 phi_1(dt C / 2)(F_n + C U_n)
    {0.5, 2, {0, 1, {{1, 0, 0, 0}, {0, 0, 0, 0}, {0, 0, 0, 0}}}},
    // b_n = U_n + dt/2 phi_1(dt C / 2)(F(a_n) + C U_n)
    {0.5, 2, {0, 2, {{0, 1, 0, 0}, {0, 0, 0, 0}, {0, 0, 0, 0}}}},
    // c_n = a_n + dt/2 phi_1(dt C / 2)(2 F(b_n) - F_n + C a_n)
    {0.5, 2, {1, 3, {{-1, 0, 2, 0}, {0, 0, 0, 0}, {0, 0, 0, 0}}}},
    // U_{n+1}: phi_1 (F_n), phi_2 (-3 F_n + 2 F(a_n) + 2 F(b_n) - F(c_n)),
    // phi_3 2 x (2, -2, -2, 2)
    {1.0, 3, {0, 0, {{1, 0, 0, 0}, {-3, 2, 2, -1}, {4, -4, -4, 4}}}}};

etd_status step_rk34(etd_ctx* c, int scheme, double dt, double* const* u, etd_step_stats* stats) {
  for (int s = 0; s < c->par.nspecies; ++s)
    if (c->sp[s].src[0] || c->sp[s].bval[0])
      return fail(c, ETD_ERR_ARG, "ETD3RK and ETD4RK take the reaction term only (no source, no boundary data)");
  const RkStage* tab = scheme == ETD_SCHEME_ETD3RK ? kEtd3rk : kEtd4rk;
  const int ns = scheme == ETD_SCHEME_ETD3RK ? 3 : 4;
  for (int i = 0; i < ns; ++i) {
    etd_step_stats* st = i == ns - 1 ? stats : nullptr;  // statistics of all stages
    const double h = tab[i].dt_factor * dt;
    etd_status r = c->fp32 ? run_phipm<float>(c, MODE_STAGE, h, u, 0, nullptr, st, false, i > 0, tab[i].p, &tab[i].d)
                           : run_phipm<double>(c, MODE_STAGE, h, u, 0, nullptr, st, false, i > 0, tab[i].p, &tab[i].d);
    if (r != ETD_OK) return r;
  }
  return ETD_OK;
}

}  // namespace

extern "C" {

size_t etd_workspace_bytes(const etd_grid* grid, const etd_params* params) {
  GridDev g;
  std::string why;
  if (!check_grid(grid, g, why) || !check_params(params, why)) return 0;
  return carve(g, *params, nullptr, nullptr);
}

etd_status etd_create(const etd_grid* grid, const etd_params* params, void* workspace, size_t workspace_bytes,
                      void* stream, etd_ctx** out) {
  if (!out) return ETD_ERR_ARG;
  *out = nullptr;
  etd_ctx* c = new etd_ctx();
  std::string why;
  if (!check_grid(grid, c->g, why) || !check_params(params, why)) {
    delete c;
    return ETD_ERR_ARG;
  }
  c->grid = *grid;
  c->par = *params;
  c->stream = (cudaStream_t)stream;
  c->fp32 = params->precision == ETD_PRECISION_MIXED;
  size_t need = carve(c->g, c->par, nullptr, nullptr);
  if (!workspace || workspace_bytes < need || ((uintptr_t)workspace & 255u)) {
    delete c;
    return ETD_ERR_WORKSPACE;
  }
  c->ws = (char*)workspace;
  c->ws_bytes = workspace_bytes;
  carve(c->g, c->par, c->ws, c);
  cudaError_t e = cudaMemsetAsync(c->ws, 0, need, c->stream);
  if (e != cudaSuccess) {
    delete c;
    return ETD_ERR_CUDA;
  }
  c->nblocks = phipm_max_blocks(c->g.ndim, c->fp32);
  if (c->nblocks <= 0 || c->nblocks > MAX_BLOCKS) {
    delete c;
    return ETD_ERR_CUDA;
  }
  if (c->fp32) {
    bool ok = cudaMallocHost(&c->ncomp_host, 2 * sizeof(int)) == cudaSuccess;
    for (int s = 0; s < 2 && ok; ++s) ok = cudaEventCreateWithFlags(&c->ncomp_ev[s], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
      delete c;
      return ETD_ERR_CUDA;
    }
  }
  *out = c;
  return ETD_OK;
}

void etd_destroy(etd_ctx* ctx) { delete ctx; }

const char* etd_last_error(const etd_ctx* ctx) { return ctx ? ctx->err.c_str() : "no context"; }

etd_status etd_init_domain(etd_ctx* c, int species, const double* phi, const double* beta_field) {
  Range range("etd_init_domain");
  if (!c) return ETD_ERR_ARG;
  if (species < 0 || species >= c->par.nspecies || !phi) return fail(c, ETD_ERR_ARG, "bad species or phi");
  SpeciesBufs& b = c->sp[species];
  b.beta_field = beta_field;
  ClassifyArgs ca;
  memset(&ca, 0, sizeof(ca));
  ca.g = c->g;
  ca.phi = phi;
  ca.kind = b.kind;
  ca.tile_count = c->tile_count;
  ca.st = c->st;
  ca.nzero = 5;
  if (c->fp32) {
    ca.zero_f32[0] = (float*)b.Yg;
    ca.zero_f32[1] = (float*)b.W1g;
    ca.zero_f32[2] = (float*)b.Z[0];
    ca.zero_f32[3] = (float*)b.Z[1];
    ca.zero_f32[4] = (float*)b.W2g;
    ca.basis_f32 = (float*)b.V;
  } else {
    ca.zero_f64[0] = (double*)b.Yg;
    ca.zero_f64[1] = (double*)b.W1g;
    ca.zero_f64[2] = (double*)b.Z[0];
    ca.zero_f64[3] = (double*)b.Z[1];
    ca.zero_f64[4] = (double*)b.W2g;
    ca.basis_f64 = (double*)b.V;
  }
  ca.nbasis = c->par.m_max + 1;
  MetaArgs ma;
  memset(&ma, 0, sizeof(ma));
  ma.g = c->g;
  ma.phi = phi;
  ma.kind = b.kind;
  ma.idx = b.idx;
  ma.ncomp = b.ncomp;
  ma.beta_field = beta_field;
  ma.beta_c = c->par.beta[species];
  ma.diag = b.diag;
  ma.diagf = b.diagf;
  ma.facew = species == 0 ? c->facew : nullptr;
  ma.bco = b.bco;
  ma.bpts = b.bpts;
  ma.gersh = &c->st->gersh[species];
  ma.st = c->st;
  cudaError_t e = cudaSuccess;
  // the Krylov kernel's 4-node group list belongs to the previous domain
  if (b.qmeta) e = cudaMemsetAsync(b.qmeta, 0, 2 * sizeof(int), c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "init_domain group list reset");
  e = launch_init_domain(ca, ma, c->tile_count, b.ncomp, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "init_domain launch");
  if (c->ncomp_host) {
    e = cudaMemcpyAsync(c->ncomp_host + species, b.ncomp, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaEventRecord(c->ncomp_ev[species], c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "point count copy");
    c->ncomp_pending[species] = true;
  }
  b.ready = true;
  return ETD_OK;
}

etd_status etd_step(etd_ctx* c, double dt, double* const* u, etd_step_stats* stats) {
  Range range("etd_step");
  if (!c) return ETD_ERR_ARG;
  if (!u || !(dt > 0.0)) return fail(c, ETD_ERR_ARG, "u missing or dt <= 0");
  for (int s = 0; s < c->par.nspecies; ++s) {
    if (!u[s]) return fail(c, ETD_ERR_ARG, "u[s] is NULL");
    if (!c->sp[s].ready) return fail(c, ETD_ERR_ARG, "etd_init_domain not called for every species");
  }
  const int scheme = c->par.scheme == 0 ? ETD_SCHEME_ETD2 : c->par.scheme;
  if (scheme == ETD_SCHEME_ETD3RK || scheme == ETD_SCHEME_ETD4RK) return step_rk34(c, scheme, dt, u, stats);
  if (scheme != ETD_SCHEME_ETD2RK) {
    const bool etd1 = scheme == ETD_SCHEME_ETD1;
    return c->fp32 ? run_phipm<float>(c, MODE_ETD2, dt, u, 0, nullptr, stats, etd1)
                   : run_phipm<double>(c, MODE_ETD2, dt, u, 0, nullptr, stats, etd1);
  }
  // ETD2RK: the ETD1 step gives a_n in u (and leaves F_n in F_{n-1}'s
  // store), then u += dt phi_2(dt C)(F(a_n) - F_n)
  etd_status r = c->fp32 ? run_phipm<float>(c, MODE_ETD2, dt, u, 0, nullptr, nullptr, true)
                         : run_phipm<double>(c, MODE_ETD2, dt, u, 0, nullptr, nullptr, true);
  if (r != ETD_OK) return r;
  return c->fp32 ? run_phipm<float>(c, MODE_RK2, dt, u, 0, nullptr, stats, false, true)
                 : run_phipm<double>(c, MODE_RK2, dt, u, 0, nullptr, stats, false, true);
}

etd_status etd_phi_combination(etd_ctx* c, int species, double dt, const double* v0, const double* v1,
                               const double* v2, double* y, etd_step_stats* stats) {
  Range range("etd_phi_combination");
  if (!c) return ETD_ERR_ARG;
  if (species < 0 || species >= c->par.nspecies || !v0 || !v1 || !v2 || !y || !(dt > 0.0))
    return fail(c, ETD_ERR_ARG, "bad arguments");
  if (!c->sp[species].ready) return fail(c, ETD_ERR_ARG, "etd_init_domain not called");
  const double* given[3] = {v0, v1, v2};
  double* out[1] = {y};
  return c->fp32 ? run_phipm<float>(c, MODE_GIVEN, dt, out, species, given, stats)
                 : run_phipm<double>(c, MODE_GIVEN, dt, out, species, given, stats);
}

etd_status etd_phi_combination3(etd_ctx* c, int species, double dt, const double* v0, const double* v1,
                                const double* v2, const double* v3, double* y, etd_step_stats* stats) {
  Range range("etd_phi_combination3");
  if (!c) return ETD_ERR_ARG;
  if (species < 0 || species >= c->par.nspecies || !v0 || !v1 || !v2 || !v3 || !y || !(dt > 0.0))
    return fail(c, ETD_ERR_ARG, "bad arguments");
  if (c->par.m_max > MAX_M - 1) return fail(c, ETD_ERR_ARG, "a phi_3 combination needs m_max <= 60");
  if (!c->sp[species].ready) return fail(c, ETD_ERR_ARG, "etd_init_domain not called");
  const double* given[4] = {v0, v1, v2, v3};
  double* out[1] = {y};
  return c->fp32 ? run_phipm<float>(c, MODE_GIVEN, dt, out, species, given, stats, false, false, 3)
                 : run_phipm<double>(c, MODE_GIVEN, dt, out, species, given, stats, false, false, 3);
}

etd_status etd_set_source(etd_ctx* c, int species, const double* src_n, const double* src_np1) {
  if (!c) return ETD_ERR_ARG;
  if (species < 0 || species >= c->par.nspecies) return fail(c, ETD_ERR_ARG, "bad species");
  c->sp[species].src[0] = src_n;
  c->sp[species].src[1] = src_np1;
  return ETD_OK;
}

etd_status etd_boundary_points(etd_ctx* c, int species, double* points, int* ncomp, int* slots) {
  if (!c || !ncomp || !slots) return ETD_ERR_ARG;
  if (species < 0 || species >= c->par.nspecies) return fail(c, ETD_ERR_ARG, "bad species");
  if (!c->par.boundary_data) return fail(c, ETD_ERR_ARG, "created without boundary_data");
  if (!c->sp[species].ready) return fail(c, ETD_ERR_ARG, "etd_init_domain not called");
  etd_status rs = read_status(c);
  if (rs != ETD_OK) return rs;
  int n = 0;
  cudaError_t e = cudaMemcpy(&n, c->sp[species].ncomp, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(c, e, "ncomp read");
  const int N = c->g.ndim;
  *ncomp = n;
  *slots = 2 * N * (N == 2 ? 2 : 1);
  if (points && n > 0) {
    e = cudaMemcpyAsync(points, c->sp[species].bpts, (size_t)n * (size_t)(*slots) * N * sizeof(double),
                        cudaMemcpyDeviceToDevice, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "boundary points copy");
    e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "stream synchronise");
  }
  return ETD_OK;
}

etd_status etd_set_boundary_values(etd_ctx* c, int species, const double* values_n, const double* values_np1) {
  if (!c) return ETD_ERR_ARG;
  if (species < 0 || species >= c->par.nspecies) return fail(c, ETD_ERR_ARG, "bad species");
  if (!c->par.boundary_data && (values_n || values_np1)) return fail(c, ETD_ERR_ARG, "created without boundary_data");
  c->sp[species].bval[0] = values_n;
  c->sp[species].bval[1] = values_np1;
  return ETD_OK;
}

etd_status etd_poisson_solve(etd_ctx* c, int species, const double* f, double* u, double tol, int max_iter,
                             int* iters, double* rel_resid) {
  Range range("etd_poisson_solve");
  if (!c) return ETD_ERR_ARG;
  if (species < 0 || species >= c->par.nspecies || !f || !u || !(tol > 0.0) || max_iter < 1)
    return fail(c, ETD_ERR_ARG, "bad arguments");
  if (c->fp32) return fail(c, ETD_ERR_ARG, "the Poisson solve needs an FP64 context");
  if (!c->sp[species].ready) return fail(c, ETD_ERR_ARG, "etd_init_domain not called");
  PoissonArgs a;
  memset(&a, 0, sizeof(a));
  a.g = c->g;
  a.S = species_dev<double>(c, species, u);
  a.S.src = nullptr;
  a.f = f;
  a.u = u;
  a.tol = tol;
  a.max_iter = max_iter;
  a.part = c->part;
  a.st = c->st;
  a.out = c->pout;
  cudaError_t e = launch_poisson(a, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "poisson launch");
  etd_status rs = read_status(c);
  double out[2] = {0.0, 0.0};
  e = cudaMemcpy(out, c->pout, sizeof(out), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(c, e, "poisson result read");
  if (iters) *iters = (int)out[0];
  if (rel_resid) *rel_resid = out[1];
  return rs;
}

etd_status etd_set_reaction(etd_ctx* c, int reaction, const double* rp) {
  if (!c) return ETD_ERR_ARG;
  if (reaction < 0 || reaction > 3 || !rp) return fail(c, ETD_ERR_ARG, "bad reaction");
  if (reaction == ETD_REACTION_COMPETITION && c->par.nspecies != 2) return fail(c, ETD_ERR_ARG, "competition needs 2 species");
  c->par.reaction = reaction;
  for (int i = 0; i < 4; ++i) c->par.rp[i] = rp[i];
  return ETD_OK;
}

etd_status etd_step_explicit(etd_ctx* c, int species, double dt, const double* u_n, const double* u_nm1,
                             double* u_out, etd_step_stats* stats) {
  Range range("etd_step_explicit");
  if (!c) return ETD_ERR_ARG;
  if (species < 0 || species >= c->par.nspecies || !u_n || !u_nm1 || !u_out || !(dt > 0.0) || u_out == u_n ||
      u_out == u_nm1)
    return fail(c, ETD_ERR_ARG, "bad arguments");
  if (c->par.reaction == ETD_REACTION_COMPETITION) return fail(c, ETD_ERR_ARG, "explicit step is single-species");
  if (!c->sp[species].ready) return fail(c, ETD_ERR_ARG, "etd_init_domain not called");
  const double* given[3] = {u_n, u_nm1, nullptr};
  double* out[1] = {u_out};
  return c->fp32 ? run_phipm<float>(c, MODE_EXPLICIT, dt, out, species, given, stats)
                 : run_phipm<double>(c, MODE_EXPLICIT, dt, out, species, given, stats);
}

static void gauss_legendre01(int n, double* t, double* w) {
  // roots of P_n by Newton from the Chebyshev-like initial guesses
  for (int i = 0; i < n; ++i) {
    double x = cos(3.14159265358979323846 * (i + 0.75) / (n + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = x;
      for (int k = 2; k <= n; ++k) {
        const double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (x * p1 - p0) / (x * x - 1.0);
      const double dx = p1 / dp;
      x -= dx;
      if (fabs(dx) < 1e-16) break;
    }
    {
      double p0 = 1.0, p1 = x;
      for (int k = 2; k <= n; ++k) {
        const double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (x * p1 - p0) / (x * x - 1.0);
    }
    t[i] = 0.5 * (x + 1.0);
    w[i] = 1.0 / ((1.0 - x * x) * dp * dp);  // half of the [-1, 1] weight
  }
}

etd_status etd_adjoint_step(etd_ctx* c, int species, double dt, const double* u_n, const double* u_nm1, int first,
                            double* lam, double* acc, double* grad_beta, double* grad_params, int nquad) {
  Range range("etd_adjoint_step");
  if (!c) return ETD_ERR_ARG;
  if (!c->par.adjoint || !c->facew) return fail(c, ETD_ERR_ARG, "context created without params.adjoint");
  if (species != 0 || !u_n || !u_nm1 || !lam || !acc || !grad_beta || !grad_params || !(dt > 0.0) || nquad < 1 ||
      nquad > ADJ_NQ_MAX)
    return fail(c, ETD_ERR_ARG, "bad arguments");
  if (c->par.reaction == ETD_REACTION_COMPETITION) return fail(c, ETD_ERR_ARG, "adjoint is single-species");
  if (!c->sp[0].ready) return fail(c, ETD_ERR_ARG, "etd_init_domain not called");
  double* P0 = c->adj[0];
  double* P1 = c->adj[1];
  double* P2 = c->adj[2];
  const double* Zero = c->adj[7];  // never written: zero since etd_create
  double t[ADJ_NQ_MAX], w[ADJ_NQ_MAX], s[ADJ_NQ_MAX];
  gauss_legendre01(nquad, t, w);
  for (int i = 0; i < nquad; ++i) s[i] = 1.0 - t[i];
  etd_status rs;
  // 1. One Krylov basis on lambda: Phi_k = phi_k(A) lambda (k = 0, 1, 2) and
  //    mu(t_i) = exp((1 - t_i) A) lambda.
  {
    double* outs[ADJ_NQ_MAX + 3] = {P0, P1, P2};
    for (int i = 0; i < nquad; ++i) outs[3 + i] = c->adj_mu[i];
    const double* given[1] = {lam};
    double* none[1] = {nullptr};
    rs = c->fp32 ? run_phipm<float>(c, MODE_ADJ_LAMBDA, dt, none, 0, given, nullptr, false, false, 2, nullptr, nquad, s,
                                    outs)
                 : run_phipm<double>(c, MODE_ADJ_LAMBDA, dt, none, 0, given, nullptr, false, false, 2, nullptr, nquad, s,
                                     outs);
    if (rs != ETD_OK) return rs;
  }
  int missed = 0;
  cudaError_t e = cudaMemcpyAsync(&missed, &c->stats->single_basis_missed, sizeof(int), cudaMemcpyDeviceToHost,
                                  c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "adjoint basis flag read");
  if (missed) {
    // m_max vectors do not reach the tolerance with one basis: each action
    // by its own time-stepped evaluation
    auto phi = [&](double sdt, const double* v0, const double* v1, const double* v2, double* out) {
      const double* given[3] = {v0, v1, v2};
      double* o[1] = {out};
      return c->fp32 ? run_phipm<float>(c, MODE_GIVEN, sdt, o, 0, given, nullptr)
                     : run_phipm<double>(c, MODE_GIVEN, sdt, o, 0, given, nullptr);
    };
    if ((rs = phi(dt, lam, Zero, Zero, P0)) != ETD_OK) return rs;
    if ((rs = phi(dt, Zero, lam, Zero, P1)) != ETD_OK) return rs;
    if ((rs = phi(dt, Zero, Zero, lam, P2)) != ETD_OK) return rs;
    for (int i = 0; i < nquad; ++i)
      if ((rs = phi(s[i] * dt, lam, Zero, Zero, c->adj_mu[i])) != ETD_OK) return rs;
  }
  // 2. y(t_i) of Eq. 3.10 (y' = A y + v_1 + t v_2, y(0) = u_n) at every
  //    quadrature time, from one time-stepped evaluation.
  {
    const double* given[2] = {u_n, u_nm1};
    double* none[1] = {nullptr};
    rs = c->fp32 ? run_phipm<float>(c, MODE_ADJ_Y, dt, none, 0, given, nullptr, false, false, 2, nullptr, nquad, t,
                                    c->adj_y)
                 : run_phipm<double>(c, MODE_ADJ_Y, dt, none, 0, given, nullptr, false, false, 2, nullptr, nquad, t,
                                     c->adj_y);
    if (rs != ETD_OK) return rs;
  }
  AdjointArgs a;
  memset(&a, 0, sizeof(a));
  a.g = c->g;
  a.idx = c->sp[0].idx;
  a.ncomp = c->sp[0].ncomp;
  a.kind = c->sp[0].kind;
  a.facew = c->facew;
  a.reaction = c->par.reaction;
  for (int i = 0; i < 4; ++i) a.rp[i] = c->par.rp[i];
  a.dt = dt;
  a.first = first ? 1 : 0;
  a.un = u_n;
  a.unm1 = u_nm1;
  a.P0 = P0;
  a.P1 = P1;
  a.P2 = P2;
  a.lam = lam;
  a.acc = acc;
  a.part = c->part;
  a.grad_params = grad_params;
  a.nq = nquad;
  for (int i = 0; i < nquad; ++i) {
    a.muq[i] = c->adj_mu[i];
    a.yq[i] = c->adj_y[i];
    a.wq[i] = w[i] * dt;
  }
  // 3. the beta contraction over all quadrature times, then 4. the
  //    pointwise combination (which overwrites lam)
  e = launch_beta_contract_multi(a, grad_beta, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "beta contraction");
  e = launch_adjoint_combine(a, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "adjoint combine");
  return ETD_OK;
}

etd_status etd_apply_operator(etd_ctx* c, int species, double dt, const double* x, double* y) {
  Range range("etd_apply_operator");
  if (!c) return ETD_ERR_ARG;
  if (species < 0 || species >= c->par.nspecies || !x || !y) return fail(c, ETD_ERR_ARG, "bad arguments");
  if (!c->sp[species].ready) return fail(c, ETD_ERR_ARG, "etd_init_domain not called");
  ApplyArgs a;
  a.g = c->g;
  a.idx = c->sp[species].idx;
  a.ncomp = c->sp[species].ncomp;
  a.diag = c->sp[species].diag;
  a.beta_field = c->sp[species].beta_field;
  a.beta_c = c->par.beta[species];
  a.cfac = dt / (c->g.h * c->g.h);
  a.x = x;
  a.y = y;
  cudaError_t e = launch_apply(a, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "apply launch");
  return ETD_OK;
}

etd_status etd_last_stats(etd_ctx* c, etd_step_stats* stats) {
  if (!c || !stats) return ETD_ERR_ARG;
  return copy_stats(c, stats);
}

etd_status etd_set_wait_limit(etd_ctx* c, double seconds) {
  if (!c) return ETD_ERR_ARG;
  if (!(seconds == seconds)) return fail(c, ETD_ERR_ARG, "wait limit is NaN");
  // 0 or less: the default; at most ~584 years in ns
  c->wait_ns = seconds <= 0.0 ? 0ull : (seconds >= 1.8e10 ? 18000000000000000000ull
                                                            : (unsigned long long)(seconds * 1e9 + 0.5));
  if (seconds > 0.0 && c->wait_ns == 0ull) c->wait_ns = 1ull;
  cudaError_t e = cudaMemcpyAsync(&c->st->wait_ns, &c->wait_ns, sizeof(c->wait_ns), cudaMemcpyHostToDevice,
                                  c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "wait limit write");
  e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "stream synchronise");
  return ETD_OK;
}

etd_status etd_selfcheck_round_f32(const double* x, float* lib, float* hw, long long n, void* stream) {
  if (n < 0 || (n > 0 && (!x || !lib || !hw))) return ETD_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  if (launch_round_check(x, lib, hw, n, st) != cudaSuccess) return ETD_ERR_CUDA;
  return cudaStreamSynchronize(st) == cudaSuccess ? ETD_OK : ETD_ERR_CUDA;
}

etd_status etd_sync(etd_ctx* c) {
  Range range("etd_sync");
  if (!c) return ETD_ERR_ARG;
  return read_status(c);
}

etd_status etd_read_domain(etd_ctx* c, int species, int* ncomp, int* nclamp, double* gersh, uint8_t* kind, int* idx,
                           double* diag, int cap) {
  if (!c) return ETD_ERR_ARG;
  if (species < 0 || species >= c->par.nspecies) return fail(c, ETD_ERR_ARG, "bad species");
  etd_status rs = read_status(c);
  SpeciesBufs& b = c->sp[species];
  int nc = 0;
  cudaError_t e = cudaMemcpy(&nc, b.ncomp, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(c, e, "read ncomp");
  if (ncomp) *ncomp = nc;
  if (nclamp) cudaMemcpy(nclamp, &c->st->nclamp, sizeof(int), cudaMemcpyDeviceToHost);
  if (gersh) cudaMemcpy(gersh, &c->st->gersh[species], sizeof(double), cudaMemcpyDeviceToHost);
  if (kind) cudaMemcpy(kind, b.kind, (size_t)c->g.size, cudaMemcpyDeviceToHost);
  const int n = nc < cap ? nc : cap;
  if (idx && n > 0) cudaMemcpy(idx, b.idx, sizeof(int) * n, cudaMemcpyDeviceToHost);
  if (diag && n > 0) cudaMemcpy(diag, b.diag, sizeof(double) * n, cudaMemcpyDeviceToHost);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(c, e, "read domain");
  return rs;
}

etd_status levelset_advance(etd_ctx* c, int species, double* phi, double* u, double dt, int do_reinit) {
  Range range("levelset_advance");
  if (!c) return ETD_ERR_ARG;
  if (species < 0 || species >= c->par.nspecies || !phi || !u || !(dt > 0.0))
    return fail(c, ETD_ERR_ARG, "bad arguments");
  if (!c->sp[species].ready) return fail(c, ETD_ERR_ARG, "etd_init_domain not called");
  cudaError_t e = launch_levelset_advance(c->g, c->ls, c->st, c->sp[species].kind, phi, u, dt, c->par.mu[species],
                                          do_reinit != 0, c->fp32, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "levelset launch");
  return ETD_OK;
}

etd_status levelset_last_stats(etd_ctx* c, int* info) {
  if (!c || !info) return ETD_ERR_ARG;
  etd_status rs = read_status(c);
  cudaError_t e = cudaMemcpy(info, c->ls.info, 8 * sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(c, e, "levelset stats read");
  return rs;
}

etd_status levelset_prepare(etd_ctx* c, double* phi, int do_reinit) {
  Range range("levelset_prepare");
  if (!c) return ETD_ERR_ARG;
  if (!phi) return fail(c, ETD_ERR_ARG, "phi is NULL");
  cudaError_t e = launch_levelset_prepare(c->g, c->ls, c->st, phi, do_reinit != 0, c->fp32, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "levelset launch");
  return ETD_OK;
}

}  // extern "C"
