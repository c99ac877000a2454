/*
 * etd_gb300.h -- C ABI of the GB300 (sm_103a) library for exponential time
 * differencing (ETD2) of reaction-diffusion systems on embedded-boundary
 * domains with a level-set free boundary, after Liu & Liu, "Integration
 * factor combined with level set method for reaction-diffusion systems with
 * free boundary in high spatial dimensions" (arXiv 2209.15095).
 *
 * Problem (Eq. free): u_t = div(beta grad u) + f(u) in Omega(t), u = 0 outside,
 * boundary normal speed mu |grad u| (Stefan condition, Sec. 4.3), on a node
 * grid x_i = lo + i h (Sec. 2), Omega = {phi < 0}.
 *
 * Conventions for every entry point
 *   - Grids are row-major (C order), the last axis fastest, 2 <= ndim <= 4,
 *     the same spacing h on every axis, at most 2^31 - 1 nodes.
 *   - Field arguments (phi, u, beta, x, y, v0..v2) are DEVICE pointers to
 *     full-grid FP64 arrays owned by the caller; the library never frees or
 *     keeps them beyond the call, except beta_field, which must stay valid
 *     until the next etd_init_domain of that species.
 *   - The workspace is a caller-owned device buffer of etd_workspace_bytes()
 *     bytes, 256-byte aligned; the library allocates no device memory.
 *   - Calls are asynchronous on the stream given to etd_create unless they
 *     take a host output (stats, etd_read_domain, etd_sync), which
 *     synchronise that stream.  Errors raised on the device (domain too close
 *     to the box, Krylov tolerance not met, non-finite values, a device wait
 *     that timed out) are reported by the next synchronising call.
 *   - Return value: ETD_OK or a negative etd_status; etd_last_error() gives a
 *     message.  On an error the output fields are unspecified.
 */
#ifndef ETD_GB300_H
#define ETD_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  ETD_OK = 0,
  ETD_ERR_ARG = -1,        /* invalid argument, or call out of order          */
  ETD_ERR_CUDA = -2,       /* a CUDA runtime call failed                      */
  ETD_ERR_WORKSPACE = -3,  /* workspace missing, misaligned or too small      */
  ETD_ERR_KRYLOV = -4,     /* Krylov tolerance not met at the smallest substep */
  ETD_ERR_DOMAIN = -5,     /* an inside node within 3 nodes of the box edge   */
  ETD_ERR_NONFINITE = -6,  /* NaN or Inf met in a reduction                   */
  ETD_ERR_TIMEOUT = -7     /* a bounded device wait (grid barrier) gave up    */
} etd_status;

/* Node grid (Sec. 2: x_ij = (x_L + (i-1) h, y_L + (j-1) h), generalised to ndim
 * axes): n[d] nodes on [lo[d], hi[d]]; entries beyond ndim are ignored. */
typedef struct {
  int ndim;
  int n[4];
  double lo[4];
  double hi[4];
} etd_grid;

enum { ETD_REACTION_NONE = 0, ETD_REACTION_LOGISTIC = 1, ETD_REACTION_LOGISTIC_AK = 2, ETD_REACTION_COMPETITION = 3 };
enum { ETD_PRECISION_FP64 = 0, ETD_PRECISION_MIXED = 1 };
enum {
  ETD_SCHEME_ETD1 = 1,
  ETD_SCHEME_ETD2 = 2,
  ETD_SCHEME_ETD2RK = 3,
  ETD_SCHEME_ETD3RK = 4,
  ETD_SCHEME_ETD4RK = 5,
  ETD_SCHEME_ETD3 = 6
};

/* Method parameters.
 *   nspecies    1 or 2
 *   precision   ETD_PRECISION_FP64: every vector and reduction in FP64.
 *               ETD_PRECISION_MIXED: Krylov vectors and the stencil in FP32,
 *               dot products / norms and the basis combination accumulated
 *               error-free in FP32 pairs and summed across the grid in FP64;
 *               H, the small exponential, the controller, u and F stay FP64.
 *               From 2^18 computational points (constant beta, last axis a
 *               multiple of 4) the basis is built by the one-pass form of the
 *               symmetric Lanczos recurrence (C is symmetric), its sums per
 *               group of 4 nodes in FP32 and accumulated error-free.
 *               In the level set, phi, u and the RK updates stay FP64; the
 *               HJ-WENO5/Godunov arithmetic is FP32 for the advection and,
 *               beyond h from the interface, for the reinitialisation; the
 *               extension sweeps and the Stefan speed's interpolation run in
 *               FP32 (the extended u off the interior differs from FP64 by
 *               rounding, within 1e-5 of max |u|).
 *   krylov_tol  relative tolerance of the adaptive Krylov evaluation
 *   m_max       largest Krylov basis, 5 <= m_max <= 61
 *   reaction    f(u):  NONE 0;  LOGISTIC u(1-u);  LOGISTIC_AK rp[0] u (1 - u/rp[1]);
 *               COMPETITION (species 0, 1) = (u(1-u-rp[0] v), rp[2] v (1-v-rp[1] u))
 *   mu[s]       Stefan coefficient of species s (boundary speed mu |grad u|)
 *   beta[s]     constant diffusion coefficient of species s, used when no
 *               beta field is given to etd_init_domain
 *   adjoint     1 to reserve the workspace of etd_adjoint_step (species 0)
 *   scheme      time integrator of etd_step (Sec. 3.1-3.2): ETD_SCHEME_ETD1,
 *               ETD_SCHEME_ETD2 (also selected by 0), ETD_SCHEME_ETD2RK,
 *               ETD_SCHEME_ETD3RK, ETD_SCHEME_ETD4RK (these two need
 *               m_max <= 60, reserve three more full-grid FP64 fields per
 *               species, and step the reaction term only: no source, no
 *               boundary data) or ETD_SCHEME_ETD3 (multistep, third order;
 *               m_max <= 60, one more full-grid FP64 field per species)
 *   boundary_data  1 to reserve the workspace of nonzero Dirichlet data
 *               (etd_boundary_points / etd_set_boundary_values) */
typedef struct {
  int nspecies;
  int precision;
  double krylov_tol;
  int m_max;
  int reaction;
  double rp[4];
  double mu[2];
  double beta[2];
  int adjoint;
  int scheme;
  int boundary_data;
} etd_params;

#define ETD_TRACE_MAX 64

/* Per-call statistics of the adaptive Krylov evaluation (decision trace). */
typedef struct {
  int ncomp[2];                       /* computational points per species    */
  int substeps[2];                    /* accepted substeps                   */
  int rejections[2];                  /* rejected step sizes                 */
  int krylov_iters[2];                /* basis vectors built, all substeps   */
  int trace_len[2];
  int trace_m[2][ETD_TRACE_MAX];      /* basis size of each accepted substep */
  double trace_tau[2][ETD_TRACE_MAX]; /* step of each accepted substep       */
} etd_step_stats;

typedef struct etd_ctx etd_ctx;

/* Bytes of device workspace needed for this grid and parameter set. */
size_t etd_workspace_bytes(const etd_grid* grid, const etd_params* params);

/* Create a context on the current device.  `workspace` (device, >= the size
 * above, 256-byte aligned) is zeroed on `stream` (a cudaStream_t, NULL for
 * the legacy default stream) and carved into the library's buffers; the
 * caller keeps ownership and must keep it alive until etd_destroy. */
etd_status etd_create(const etd_grid* grid, const etd_params* params, void* workspace, size_t workspace_bytes,
                      void* stream, etd_ctx** out);

/* Release the host-side context (the workspace is the caller's). */
void etd_destroy(etd_ctx* ctx);

/* Domain set-up for `species` from the level set phi (Sec. 2): classifies
 * nodes (inside phi < 0; ghost: inside with an axis neighbour outside;
 * computational: inside with all 2N neighbours inside), lists the
 * computational points in grid order and packs per-row metadata: the
 * diagonal D_p = sum_faces beta_f - sum_ghost faces beta_f w_f, with w_f the
 * ghost weight of case 2 (Eq. DirichletLineByLine) or case 3 (Eq. rbf_ubp),
 * clamped to [0, 1].  beta_field: NULL for the constant params->beta[species],
 * else a full-grid node field (face value = mean of the two nodes). */
etd_status etd_init_domain(etd_ctx* ctx, int species, const double* phi, const double* beta_field);

/* One time step of every species on the current domains, by the scheme of
 * params->scheme:
 *   ETD2   (Sec. 3.1)  U_{n+1} = phi_0(dt C) U_n + dt phi_1(dt C) F_n
 *                                + dt phi_2(dt C)(F_n - F_{n-1});
 *   ETD1   (Sec. 3.1)  the same without the phi_2 term;
 *   ETD2RK (Sec. 3.2)  a_n = phi_0(dt C) U_n + dt phi_1(dt C) F_n (the ETD1 step),
 *                      U_{n+1} = a_n + dt phi_2(dt C)(F(a_n) - F_n): two Krylov
 *                      evaluations, the second with v_0 = v_1 = 0;
 *   ETD3RK, ETD4RK (Sec. 3.2)  the stages a_n, b_n (and c_n) with dt / 2 or
 *                      dt, then U_{n+1} by one combination up to phi_3: three
 *                      and four Krylov evaluations.  The paper's phi_3 is that
 *                      of Eq. 3.7, twice the standard phi_3;
 *   ETD3 (Eq. 3.8b, s = 3)  U_{n+1} = phi_0 U_n + dt phi_1 F_n
 *                      + dt phi_2 (3/2 F_n - 2 F_{n-1} + 1/2 F_{n-2})
 *                      + dt phi_3 (F_n - 2 F_{n-1} + F_{n-2}) (standard phi_k);
 *                      where a point lacks F_{n-2} the step is ETD2 there,
 *                      and where it also lacks F_{n-1}, ETD1.
 * Each phi-combination (Eq. 3.9) is evaluated by adaptive Krylov
 * time-stepping of the ODE of Eq. 3.10.  u[s] (device, full grid, in/out):
 * read at the computational points of species s; on return it holds U_{n+1}
 * there and 0 at every other node.  F_{n-1} (ETD2) is kept by the context;
 * where a point was not computational at the previous step (and at the first
 * step) F_{n-1} = F_n.  stats: NULL for an asynchronous call, else filled
 * after synchronising; for the Runge-Kutta schemes the counts add all
 * evaluations and the trace lists their substeps in order. */
etd_status etd_step(etd_ctx* ctx, double dt, double* const* u, etd_step_stats* stats);

/* The phi-combination alone (Sec. 3.3, Eq. 3.9 with p = 2):
 *   y = phi_0(dt C) v0 + phi_1(dt C) v1 + phi_2(dt C) v2
 * on the computational points of `species`; v0, v1, v2, y are device full-grid
 * FP64 arrays; y is 0 off the computational set. */
etd_status etd_phi_combination(etd_ctx* ctx, int species, double dt, const double* v0, const double* v1,
                               const double* v2, double* y, etd_step_stats* stats);

/* The phi-combination with p = 3 (Eq. 3.9, standard phi_k):
 *   y = phi_0(dt C) v0 + phi_1(dt C) v1 + phi_2(dt C) v2 + phi_3(dt C) v3,
 * arguments as etd_phi_combination.  Needs m_max <= 60 (ETD_ERR_ARG
 * otherwise). */
etd_status etd_phi_combination3(etd_ctx* ctx, int species, double dt, const double* v0, const double* v1,
                                const double* v2, const double* v3, double* y, etd_step_stats* stats);

/* Embedded-boundary Poisson solve (Sec. 2: div(beta grad u) = f with
 * Dirichlet data; Sec. 4.1): at the computational points of `species`,
 * C u + b = f, with C the operator of etd_init_domain (dt = 1) and b the
 * boundary-data term of etd_set_boundary_values (values_n; none set: zero
 * data).  Conjugate gradients on -C (symmetric positive definite, Sec. 2) in
 * FP64.  f (device, full grid) is read at the computational points; u
 * (device, full grid, in/out) holds the initial guess there and receives the
 * solution (other nodes unchanged).  Stops when |r| <= tol |b - f|; after
 * max_iter iterations without that, returns ETD_ERR_KRYLOV.  iters,
 * rel_resid (host, optional): iterations and |r| / |b - f|.  Synchronises.
 * FP64 contexts only (ETD_ERR_ARG otherwise). */
etd_status etd_poisson_solve(etd_ctx* ctx, int species, const double* f, double* u, double tol, int max_iter,
                             int* iters, double* rel_resid);

/* Additive source term of F for `species` (Sec. 3, Eq. 3.2: F(U, t) = f(U) +
 * sources): src_n (device, full grid FP64, caller-owned, read at the
 * computational points) enters F_n in every following etd_step; src_np1 is
 * the source at t_n + dt, read by the second ETD2RK stage (NULL: src_n).
 * Both pointers must stay valid while steps that use them run; NULL clears.
 * The stored F_{n-1} of ETD2 includes the source of its step. */
etd_status etd_set_source(etd_ctx* ctx, int species, const double* src_n, const double* src_np1);

/* Nonzero Dirichlet data u = u_Gamma on the boundary (Sec. 2: the ghost
 * value of case 2 (Eq. DirichletLineByLine) is w u_p + g_Gamma u_Gamma at the
 * crossing point, of case 3 in 2D (Eq. rbf_ubp) w u_p + c_1 u(Gamma1) +
 * c_2 u(Gamma2); the boundary part goes to the right-hand side).  Needs
 * params->boundary_data.  After etd_init_domain, returns the number of
 * computational points (*ncomp) and of boundary slots per point (*slots =
 * 2N faces x J, J = 2 for N = 2, else 1) and, if `points` (device, at least
 * ncomp * slots * N doubles, caller-owned) is not NULL, copies the slot
 * points there: slot (k, f, j) of computational point k (index-list order),
 * face f (axis f / 2, side f % 2: -1, +1) at points[((k * 2N + f) * J + j) * N
 * + 0..N-1]; slots without a boundary point hold NaN.  Synchronises.  A
 * case-3 face in N >= 3 has no boundary reading: ETD_ERR_ARG. */
etd_status etd_boundary_points(etd_ctx* ctx, int species, double* points, int* ncomp, int* slots);

/* Boundary values u_Gamma at the slot points, in the slot order above
 * (device, ncomp * slots doubles, caller-owned; NaN slots are ignored):
 * values_n enter F_n of every following etd_step, values_np1 (t_n + dt,
 * NULL: values_n) the second ETD2RK stage.  They must stay valid while steps
 * that use them run; NULL clears. */
etd_status etd_set_boundary_values(etd_ctx* ctx, int species, const double* values_n, const double* values_np1);

/* Replace the reaction kind and parameters of the context (as in
 * etd_params; rp: host, 4 doubles). */
etd_status etd_set_reaction(etd_ctx* ctx, int reaction, const double* rp);

/* One ETD2 step (Sec. 3.1) of `species` on its current domain from both
 * time levels given explicitly (no state kept in the context):
 *   u_out = phi_0(dt C) u_n + dt phi_1(dt C) F(u_n) + dt phi_2(dt C)(F(u_n) - F(u_nm1));
 * pass u_nm1 = u_n for the first step.  u_n, u_nm1, u_out: device full-grid
 * FP64, read at / written to the computational points, u_out = 0 elsewhere;
 * u_out may alias neither input. */
etd_status etd_step_explicit(etd_ctx* ctx, int species, double dt, const double* u_n, const double* u_nm1,
                             double* u_out, etd_step_stats* stats);

/* Adjoint of one etd_step_explicit step on a frozen domain (species 0; needs
 * params->adjoint).  A = dt C is symmetric (Sec. 2), so with
 * lambda = dL/du_{n+1} and Phi_k = phi_k(A) lambda:
 *   lam  <- Phi_0 + dt F'(u_n)(Phi_1 + Phi_2) + acc        (dL/du_n)
 *   acc  <- -dt F'(u_nm1) Phi_2                              (to dL/du_{n-1})
 *   grad_params[0] += dt <Phi_1 + Phi_2, dF/dalpha(u_n)> - dt <Phi_2, dF/dalpha(u_nm1)>
 *   grad_beta += int_0^1 d(mu(t)^T A y(t))/d beta dt,  mu(t) = e^{(1-t)A} lambda,
 *                y(t) = phi_0(tA) u_n + phi_1(tA) t v_1 + phi_2(tA) t^2 v_2
 * (the step is y(1) of y' = A y + v_1 + t v_2, Eq. 3.10; v_1 = dt F(u_n),
 * v_2 = dt (F(u_n) - F(u_nm1))), by nquad-point Gauss-Legendre in t and the
 * face contraction of the symmetric stencil (node field beta, face value the
 * mean of the two nodes; ghost nodes included).  Two Krylov evaluations per
 * step: Phi_0, Phi_1, Phi_2 and every mu(t_i) from one basis of the Krylov
 * space of A and lambda (grown until the estimate of exp(A) lambda meets
 * krylov_tol; if m_max vectors do not, each action is evaluated by its own
 * time-stepped Krylov evaluation instead), and every y(t_i) from one
 * time-stepped evaluation of Eq. 3.10, written as its substeps pass the t_i.  first = 1 for the first step, where u_nm1 = u_n and acc is
 * folded into lam.  u_n, u_nm1 (in), lam, acc (in/out), grad_beta (accumulated):
 * device full-grid FP64, zero off the computational set except grad_beta;
 * grad_params: device, 1 double, accumulated (alpha of ETD_REACTION_LOGISTIC_AK).
 * 1 <= nquad <= 32. */
etd_status etd_adjoint_step(etd_ctx* ctx, int species, double dt, const double* u_n, const double* u_nm1, int first,
                            double* lam, double* acc, double* grad_beta, double* grad_params, int nquad);

/* y = dt C x on the computational points (Sec. 2 operator, matrix-free);
 * y is written at computational points only.  FP64. */
etd_status etd_apply_operator(etd_ctx* ctx, int species, double dt, const double* x, double* y);

/* Level-set step of the free-boundary algorithm (Sec. 4.3, Steps 1-2) for
 * `species`, on the domain last given to etd_init_domain:
 *   1. extend u from the computational points into the tube around the
 *      interface by quadratic extrapolation along the normal (Aslam 2004);
 *   2. Stefan speed V = mu |grad u| at the interface, carried to the tube
 *      along the normal (closest-point extension);
 *   3. advect phi_t + V |grad phi| = 0 (Godunov HJ-WENO5, TVD-RK3, CFL substeps);
 *   4. if do_reinit, reinitialise phi_t + S(phi_0)(|grad phi| - 1) = 0;
 *   5. clamp phi to [-6h, 6h] (local level set: only the tube |phi| < 6h,
 *      grown by one node, is updated).
 * phi (in/out) and u (in/out, extended on return) are device full-grid FP64. */
etd_status levelset_advance(etd_ctx* ctx, int species, double* phi, double* u, double dt, int do_reinit);

/* Clamp phi to [-6h, 6h] and, if do_reinit, reinitialise it (as step 4 above). */
etd_status levelset_prepare(etd_ctx* ctx, double* phi, int do_reinit);

/* Synchronise and report the work of the last levelset_advance /
 * levelset_prepare (for throughput accounting): info[0] work-list length and
 * info[1] update-set (tube) size of the advection, info[2] advection
 * substeps, info[3] and info[4] the same two sizes for the
 * reinitialisation, info[5] 1 if it reinitialised.  info: host, 8 ints. */
etd_status levelset_last_stats(etd_ctx* ctx, int* info);

/* Synchronise and copy the statistics of the last etd_step or
 * etd_phi_combination of this context (what a non-NULL stats argument of
 * that call would have received). */
etd_status etd_last_stats(etd_ctx* ctx, etd_step_stats* stats);

/* Limit of every bounded device wait (the grid barriers of the cooperative
 * kernels) in this context's later launches, in seconds; 0 or less restores
 * the default of 1 s.  A wait that reaches it stops its kernel (every CTA
 * returns) and the next synchronising call returns ETD_ERR_TIMEOUT; the
 * outputs of that launch are unspecified and the context stays usable.  For
 * failure-detection tests and for callers that want an early timeout.
 * Synchronises the stream. */
etd_status etd_set_wait_limit(etd_ctx* ctx, double seconds);

/* Wait for the stream and report any error raised on the device since the
 * last report. */
etd_status etd_sync(etd_ctx* ctx);

/* Synchronise and copy domain data of `species` to host memory: the number
 * of computational points and of clamped ghost weights, the Gershgorin bound
 * max_p sum_q |C_pq|, and optionally (non-NULL) the node kinds (grid size
 * bytes: 0 outside, 1 ghost, 2 computational), the computational points' grid
 * indices and their diagonals D_p (cap entries each). */
etd_status etd_read_domain(etd_ctx* ctx, int species, int* ncomp, int* nclamp, double* gersh, uint8_t* kind,
                           int* idx, double* diag, int cap);

/* Message for the last error of this context (static storage of the ctx). */
const char* etd_last_error(const etd_ctx* ctx);

/* Largest problem etd_phi_combination_noalloc accepts, and the size of the
 * fixed device array it works in. */
#define ETD_NOALLOC_MAX_NODES 32768
#define ETD_NOALLOC_MAX_M 30
#define ETD_NOALLOC_SCRATCH_BYTES (10u << 20)

/* The paper has no counterpart to this entry point; it exists for callers
 * that may not allocate device memory at all: a host that owns every byte of
 * the GPU through its own allocator and hands a plug-in only its inputs and
 * outputs, or a deployment that forbids allocation once it is running.  It
 * computes the same result as etd_init_domain(phi, constant beta) followed by
 * etd_phi_combination in FP64:
 *   y = phi_0(dt C) v0 + phi_1(dt C) v1 + phi_2(dt C) v2
 * on the computational points of {phi < 0}, y = 0 elsewhere.  grid, phi, v0,
 * v1, v2 and y are as for the context calls (device, full grid, FP64, owned by
 * the caller); stream is a cudaStream_t (NULL: legacy default stream) of the
 * current device (a stream of another device: ETD_ERR_ARG).
 * Scratch: one file-scope device array of ETD_NOALLOC_SCRATCH_BYTES (10 MiB)
 * that every GPU which loads the library holds until the process exits; no
 * cudaMalloc, cudaFree or other allocating call is made.  Limits: at most
 * ETD_NOALLOC_MAX_NODES grid nodes and m_max <= ETD_NOALLOC_MAX_M, else
 * ETD_ERR_WORKSPACE; the largest such problem fits the array (checked when
 * the library is compiled).  The first call on a device looks up the array's
 * device address (cudaGetSymbolAddress, with that device current) and keeps
 * it for later calls; make that first call before any stream capture.  The
 * kept address belongs to the device's primary context: after a
 * cudaDeviceReset (or any reset of that context) the process must not call
 * this entry point on that device again.  Every call clears the part of the array it
 * uses, then works in it; calls that overlap on the GPU (two streams, or two
 * host threads) share the array and race.  The call synchronises `stream` and
 * returns any device-side error. */
etd_status etd_phi_combination_noalloc(const etd_grid* grid, const double* phi, double beta, double dt,
                                       const double* v0, const double* v1, const double* v2, double* y,
                                       double krylov_tol, int m_max, void* stream);

/* Self-check of the library's FP64 -> FP32 rounding (round to nearest, ties
 * to even), which the FP32-mixed contexts use on the integer pipe for the
 * FP32 copies of y, v_1, v_2 and v_3: for i < n, lib[i] = that rounding of
 * x[i] and hw[i] = the hardware conversion of x[i].  x, lib and hw are device
 * pointers of n elements (caller-owned); stream is a cudaStream_t (NULL: the
 * default stream).  Synchronises the stream; ETD_ERR_ARG for n < 0 or a NULL
 * pointer with n > 0, ETD_ERR_CUDA for a launch failure. */
etd_status etd_selfcheck_round_f32(const double* x, float* lib, float* hw, long long n, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* ETD_GB300_H */
