// Kernel argument blocks and host-side launch entry points shared by the
// translation units of the library.
#pragma once
#include "common.cuh"

namespace etd {

struct ClassifyArgs {
  GridDev g;
  const double* phi;
  uint8_t* kind;
  int* tile_count;
  DevStatus* st;
  // stencil-input vectors whose entries must be zero off the computational set
  int nzero;
  double* zero_f64[4];
  float* zero_f32[4];
  int nbasis;
  double* basis_f64;
  float* basis_f32;
};

struct MetaArgs {
  GridDev g;
  const double* phi;
  const uint8_t* kind;
  int* idx;  // written by the compaction, read by the metadata pass
  const int* ncomp;
  const double* beta_field;  // node field or nullptr
  double beta_c;
  double* diag;
  float* diagf;  // nullptr unless FP32 vectors are in use
  double* gersh;
  DevStatus* st;
};

int scan_tiles(long long size);
cudaError_t launch_init_domain(const ClassifyArgs& ca, const MetaArgs& ma, int* tile_count, int* ncomp_dev,
                               cudaStream_t stream);

// ---------------------------------------------------------------- Krylov
constexpr int TRACE_MAX = 64;

struct StatsDev {
  int substeps[2];
  int rejections[2];
  int iters[2];
  int trace_len[2];
  int trace_m[2][TRACE_MAX];
  double trace_tau[2][TRACE_MAX];
};

template <typename T>
struct SpeciesDev {
  const int* idx;
  const int* ncomp;
  const double* diag;
  const float* diagf;
  const uint8_t* kind;
  const double* beta_field;
  double beta_c;
  const double* gersh;
  // caller's field (full grid, FP64); other species' field for coupling
  double* u;
  // F_{n-1} on the grid and its validity flags
  double* Fprev;
  uint8_t* fvalid;
  // full-grid stencil inputs (zero off the computational set)
  T* V;   // m_max + 1 slots, slot stride = grid size
  T* Yg;  // y(t_k) copy in T
  T* W1g; // w_1
  // compact per-ordinal vectors
  double* Yc;
  T* V1c;
  T* V2c;
  T* Z[2];  // full grid: A V_j of the last two basis vectors (unnormalised)
};

// mode of the phi-combination kernel
enum : int {
  MODE_ETD2 = 0,   // v0 = u, v1 = dt F(u), v2 = dt (F(u) - F_prev); writes u
  MODE_GIVEN = 1,  // v0, v1, v2 given on the grid (Yg/Yc preset by the host path); writes Yc
};

template <typename T>
struct PhipmArgs {
  GridDev g;
  int nspecies;
  int mode;
  int m_max;
  double dt;
  double cfac;  // dt / h^2
  double tol;
  int reaction;
  double rp[4];
  SpeciesDev<T> sp[2];
  const double* given[3];  // MODE_GIVEN: v0, v1, v2 on the grid (species 0)
  double* part;
  DevStatus* st;
  StatsDev* stats;
};

template <typename T>
cudaError_t launch_phipm(const PhipmArgs<T>& a, int nblocks, cudaStream_t stream);
int phipm_max_blocks(int ndim, bool fp32);

// y = A x on the computational set (x, y full grid FP64), for parity tests
struct ApplyArgs {
  GridDev g;
  const int* idx;
  const int* ncomp;
  const double* diag;
  const double* beta_field;
  double beta_c;
  double cfac;
  const double* x;
  double* y;
};
cudaError_t launch_apply(const ApplyArgs& a, cudaStream_t stream);

}  // namespace etd
