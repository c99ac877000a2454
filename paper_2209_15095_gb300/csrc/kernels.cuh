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
  double* zero_f64[5];
  float* zero_f32[5];
  int nbasis;
  double* basis_f64;
  float* basis_f32;
};

struct MetaArgs {
  GridDev g;
  const double* phi;
  const uint8_t* kind;
  int* idx;  // written by the compaction, read by the metadata pass
  int* ncomp;  // written by the compaction, read by the metadata pass
  const double* beta_field;  // node field or nullptr
  double beta_c;
  double* diag;
  float* diagf;  // nullptr unless FP32 vectors are in use
  double* facew; // nullptr, or per point and face: 1 - w on ghost faces, 0 otherwise
  double* bco;   // nullptr, or per point, face and slot (2 slots for N = 2, else 1):
  double* bpts;  //   boundary-data coefficient and point (N doubles)
  double* gersh;
  DevStatus* st;
};

// ints of per-CTA counts and word scratch of the set-up kernel
constexpr int init_scratch_ints(long long size) { return MAX_BLOCKS + 2 * (int)((size + 31) / 32); }
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
  int single_basis_missed;  // MODE_ADJ_LAMBDA: tolerance not met by one basis of m_max vectors
  int pad;
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
  // F_{n-1} (and, for multistep ETD3, F_{n-2}) on the grid, and their
  // validity bits (bit 0: F_{n-1}, bit 1: F_{n-2})
  double* Fprev;
  double* Fprev2;
  uint8_t* fvalid;
  // full-grid stencil inputs (zero off the computational set)
  T* V;   // m_max + 1 slots, slot stride = grid size
  T* Yg;  // y(t_k) copy in T
  T* W1g; // w_1
  // compact per-ordinal vectors
  double* Yc;
  T* V1c;
  T* V2c;
  T* V3c;   // v_3 (phi_3 combinations only)
  T* W2g;   // full grid: w_2 (phi_3 combinations only; zero off the computational set)
  T* Z[2];  // full grid: A V_j of the last two basis vectors (unnormalised);
            // on the 4-node groups u_j = A v_j - beta_j v_{j-1} (quad_pass_1)
  // stage fields a, b, c of the Runge-Kutta schemes (full grid, FP64; only
  // the computational points are written and read)
  double* stg[3];
  // FP32 contexts: the aligned groups of 4 nodes along the last axis that
  // hold computational points ("quads"; group index = node >> 2), in order,
  // and the list index of each group's first computational point (size /
  // 4 + 1 entries each; nullptr: no quad path)
  int* qidx;
  int* qk;
  // qmeta[0] = 1 when qidx / qk hold the list of the current domain (the
  // host zeroes it with every domain set-up), qmeta[1] = the list length;
  // nullptr: the list is built by every launch
  int* qmeta;
  // caller's source (full grid) and boundary data for this launch: F gains
  // src[p] + sum over the point's face slots of bco * bval (nullptr: none)
  const double* src;
  const double* bco;
  const double* bval;
};

// mode of the phi-combination kernel
enum : int {
  MODE_ETD2 = 0,      // v0 = u, v1 = dt F(u), v2 = dt (F(u) - F_prev) (0 with etd1);
                      // F_prev <- F(u); writes u
  MODE_GIVEN = 1,     // v0, v1, v2 given on the grid; writes the output field
  MODE_EXPLICIT = 2,  // given[0] = u_n, given[1] = u_{n-1}: v0 = u_n, v1 = dt F(u_n),
                      // v2 = dt (F(u_n) - F(u_{n-1})); writes the output field
  MODE_RK2 = 3,       // second ETD2RK stage: v0 = v1 = 0, v2 = dt (F(u) - F_prev);
                      // u <- u + result
  MODE_STAGE = 4,     // a stage of ETD3RK / ETD4RK (StageDesc); reaction term only
  MODE_ADJ_LAMBDA = 5,  // one Krylov basis on given[0] = lambda: out[0..2] = phi_0..2(A) lambda,
                        // out[3 + i] = exp(tq[i] A) lambda; no time stepping (flags
                        // single_basis_missed if m_max vectors do not reach the tolerance)
  MODE_ADJ_Y = 6,       // as MODE_EXPLICIT, writing y(tq[i]) of Eq. 3.10 to out[i] (no u output)
};

constexpr int ADJ_NQ_MAX = 32;  // quadrature times of the adjoint modes

// One stage of ETD3RK / ETD4RK: fields 0 = u, 1..3 = the stage fields a, b, c.
// v_0 = field v0_field; v_j = dt sum_i coef[j-1][i] F(field i), j = 1..3;
// the result goes to field out_field.
struct StageDesc {
  int v0_field;
  int out_field;
  double coef[3][4];
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
  const double* given[4];  // MODE_GIVEN: v0 .. v_p on the grid (species 0)
  int etd1;                // MODE_ETD2: v2 = 0 (the ETD1 step)
  int p;                   // highest phi index of the combination: 2 or 3
  int ms3;                 // MODE_ETD2: multistep ETD3 (Eq. 3.8b, s = 3; p = 3)
  StageDesc stage;         // MODE_STAGE
  int nq;                  // MODE_ADJ_*: number of times tq
  double tq[ADJ_NQ_MAX];   // MODE_ADJ_LAMBDA: exponent factors s_i; MODE_ADJ_Y: output times t_i
  double* out[ADJ_NQ_MAX + 3];  // MODE_ADJ_*: output fields (full grid FP64, computational points)
  double* part;
  DevStatus* st;
  StatsDev* stats;
};

template <typename T>
cudaError_t launch_phipm(const PhipmArgs<T>& a, int nblocks, cudaStream_t stream, bool wide = false);
// FP32 problems from this many computational points run the Krylov basis on
// the 4-node groups (with a constant beta and the last axis a multiple of 4);
// `wide` picks the 768-thread FP32 kernel for them
constexpr int QUAD_MIN_POINTS = 1 << 18;
int phipm_max_blocks(int ndim, bool fp32);
// The Krylov kernels of one precision and CTA size (krylov_impl.cuh):
// fn[ndim - 2][adjoint instantiation], threads per CTA, the adjoint
// instantiation's dynamic shared memory, and the loader of the unit's
// constant table.
struct PhipmKernels {
  void* fn[3][2];
  int nt;
  size_t adj_smem;
  cudaError_t (*load_consts)();
};

// Embedded-boundary Poisson solve by conjugate gradients (FP64)
struct PoissonArgs {
  GridDev g;
  SpeciesDev<double> S;  // domain, beta, boundary data; Yg, Yc, V1c, V2c as CG vectors
  const double* f;       // full grid: right-hand side
  double* u;             // full grid: initial guess in, solution out (computational points)
  double tol;            // relative residual |r| / |b - f|
  int max_iter;
  double* part;
  DevStatus* st;
  double* out;           // device, 2 doubles: iterations, final relative residual
};
cudaError_t launch_poisson(const PoissonArgs& a, cudaStream_t stream);

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
cudaError_t launch_round_check(const double* x, float* lib, float* hw, long long n, cudaStream_t stream);

// ---------------------------------------------------------------- adjoint
struct AdjointArgs {
  GridDev g;
  const int* idx;
  const int* ncomp;
  const uint8_t* kind;
  const double* facew;
  int reaction;
  double rp[4];
  double dt;
  int first;
  const double* un;
  const double* unm1;
  const double* P0;
  const double* P1;
  const double* P2;
  double* lam;   // in: dL/du_{n+1}; out: dL/du_n
  double* acc;   // in: contribution to dL/du_n from the later step; out: to dL/du_{n-1}
  double* part;  // per-block partial sums of the alpha gradient
  double* grad_params;
  // the beta contraction over the quadrature times: mu(t_i), y(t_i), weights
  int nq;
  const double* muq[ADJ_NQ_MAX];
  const double* yq[ADJ_NQ_MAX];
  double wq[ADJ_NQ_MAX];
};
cudaError_t launch_adjoint_combine(const AdjointArgs& a, cudaStream_t stream);
// v1 = dt F(u_n), v2 = dt (F(u_n) - F(u_{n-1})) scaled by (s1, s2) on the computational set
cudaError_t launch_adjoint_rhs(const AdjointArgs& a, double s1, double s2, double* v1, double* v2, cudaStream_t stream);
// grad_beta += coef * d(mu^T C y)/d beta (node field, face mean)
cudaError_t launch_beta_contract(const AdjointArgs& a, const double* mu, const double* y, double coef,
                                 double* grad_beta, cudaStream_t stream);
// grad_beta += sum_i wq[i] d(mu_i^T C y_i)/d beta over the quadrature times (one launch)
cudaError_t launch_beta_contract_multi(const AdjointArgs& a, double* grad_beta, cudaStream_t stream);

}  // namespace etd
