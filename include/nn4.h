/*
 * nn4.h - C ABI of the GB300 pressure-multigrid library (Q1 finite elements on vertex grids).
 *
 * The library implements the pressure-correction multigrid of Chen, Heaney, Gomes, Matar and
 * Pain, "Solving the discretised multiphase flow equations with interface capturing on
 * structured grids using machine learning libraries" (arXiv 2401.06755), Section 2.4, together
 * with the explicit Petrov-Galerkin volume-fraction and momentum residuals that feed it
 * (Sections 2.3.1, 2.3.2, 2.3.4 and 2.3.5).  All compute runs in CUDA kernels on one GPU.
 *
 * Conventions shared by every call
 *   - A field on a grid with n = (nx, ny, nz) nodes is a device array with x fastest, then y,
 *     then z.  Element (i, j, k) lives at offset i + pitch * (j + ny * k); `pitch` is given in
 *     elements by the nn4_grid passed with the array, must be >= nx, and pitch * sizeof(elem)
 *     must be a multiple of 16 bytes.  nn4_row_pitch() returns the pitch the library uses for
 *     its own arrays (a multiple of 128 bytes).  Padding elements are never read or written.
 *   - Node i of an axis sits at i * h; the grid covers the closed box [0, (n-1) h].
 *   - Each of the six faces (x-, x+, y-, y+, z-, z+) is Dirichlet (nodes on it are stored
 *     values that never change; their residual and correction are zero) or natural (the
 *     zero-derivative condition of Section 2.3.3, realised by finite-element truncation).
 *   - A is the weak form of -laplacian assembled from Q1 elements (the paper's w_lap filter,
 *     Section 2.2.4, with a positive diagonal).  With a coefficient field k it is Eq. k-T:
 *     A_k x = 1/2 [ L(k x) + k L x - x L k ].
 *   - Calls are asynchronous on the given stream (a cudaStream_t passed as void*, NULL for the
 *     legacy default stream) unless stated otherwise.  Argument errors are detected on the host
 *     before anything is launched.  Pointers are never freed by the library.
 *   - Every function returns an nn4_status; nn4_last_error() gives a message for the calling
 *     thread.  Device-side failures of bounded waits are latched in a device word that
 *     nn4_device_error() reads and clears.
 */
#ifndef NN4_H
#define NN4_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  NN4_OK = 0,
  NN4_EINVAL = -1,        /* bad argument (sizes, pointers, alignment, dtype) */
  NN4_ECUDA = -2,         /* a CUDA runtime or driver call failed */
  NN4_ENOMEM = -3,        /* device allocation failed (plan creation only) */
  NN4_ENOCONV = -4,       /* iteration cap reached before the tolerance */
  NN4_ENONFINITE = -5,    /* a residual norm was NaN or infinite */
  NN4_ETIMEOUT = -6,      /* a bounded device-side wait gave up */
  NN4_EBOUNDS = -7,       /* a checked index was out of range (bounds-check builds) */
  NN4_EUNSUPPORTED = -8   /* valid but unsupported request (e.g. coarsest level too large) */
} nn4_status;

typedef enum { NN4_F64 = 0, NN4_F32 = 1, NN4_BF16 = 2 } nn4_dtype;

typedef enum { NN4_BC_DIRICHLET = 0, NN4_BC_NATURAL = 1 } nn4_bc;

/* Vertex grid: n nodes per axis, spacing h, one nn4_bc per face (x-, x+, y-, y+, z-, z+),
 * and the row pitch (in elements) of the arrays passed together with this descriptor. */
typedef struct {
  int32_t n[3];
  double h[3];
  int32_t bc[6];
  int64_t pitch;
} nn4_grid;

/* Row pitch in elements for nx values of dtype dt: nx rounded up to a multiple of 128 bytes.
 * Returns -1 for a bad argument. */
int64_t nn4_row_pitch(int32_t nx, nn4_dtype dt);

/* ----------------------------------------------------------------- single multigrid steps */

/* y = A x at every node (Dirichlet nodes included: the assembled row with natural truncation).
 * Section 2.2.2 (filter application), Section 2.2.4 (w_lap), Eq. k-T when k != NULL.
 * x, k, y: device arrays of dtype dt on grid g (k may be NULL).  y must not alias x or k.
 * Errors: NN4_EINVAL for a null x/y, a grid with fewer than 2 nodes on an axis, or a bad pitch. */
int nn4_stencil_apply(const nn4_grid* g, nn4_dtype dt, const void* x, const void* k, void* y,
                      void* stream);

/* r = b - A x at free nodes and r = 0 at Dirichlet nodes (the pressure residual of Eq. ph_disc
 * and Eq. ph_disc2 with the sign convention of A above).  If norm2 != NULL it is a device
 * double that is overwritten with sum r^2 (accumulated in FP64).  r must not alias b, x or k. */
int nn4_residual(const nn4_grid* g, nn4_dtype dt, const void* b, const void* x, const void* k,
                 void* r, double* norm2, void* stream);

/* r_coarse = R r_fine with R = P^T (weights prod_d (1/2)^|offset_d|, stride 2), and
 * r_coarse = 0 at coarse Dirichlet nodes.  The coarse grid has (n+1)/2 nodes per axis (every
 * n must be odd and >= 3) and its array uses pitch nn4_row_pitch((nx+1)/2, dt).  Section 2.4
 * (the sawtooth multigrid: stride-2 restriction). */
int nn4_restrict(const nn4_grid* fine, nn4_dtype dt, const void* r_fine, void* r_coarse,
                 void* stream);

/* r_coarse = R (b - A x): the residual of nn4_residual restricted as by nn4_restrict, in one
 * pass that does not store the fine residual (the start of every V-cycle whose correction is not
 * zero; Section 2.4 and Eq. ph_disc).  If norm2 != NULL it is a device double overwritten with
 * sum over fine nodes of (b - A x)^2 (FP64 across blocks).  Grids, pitches and k as for
 * nn4_residual and nn4_restrict; every n must be odd and >= 3.  The fine residual is computed in
 * FP32 for F32 / BF16 storage and rounded to the storage type once, on the coarse value, so its
 * result can differ from nn4_residual followed by nn4_restrict by that rounding.  r_coarse must
 * not alias b, x or k. */
int nn4_residual_restrict(const nn4_grid* fine, nn4_dtype dt, const void* b, const void* x,
                          const void* k, void* r_coarse, double* norm2, void* stream);

/* e_fine = P e_coarse (accumulate = 0) or e_fine += P e_coarse (accumulate != 0), P the
 * trilinear interpolation (injection at even nodes, averages of 2, 4 or 8 coarse nodes
 * elsewhere); fine Dirichlet nodes are set to 0 (accumulate = 0) or left unchanged.  Coarse
 * array pitch as for nn4_restrict.  Section 2.4 (prolongation in the U-Net decoder). */
int nn4_prolong(const nn4_grid* fine, nn4_dtype dt, const void* e_coarse, void* e_fine,
                int accumulate, void* stream);

/* One weighted-Jacobi sweep x_out = x_in + omega D^-1 (b - A x_in) at free nodes; Dirichlet
 * nodes are copied.  D is the exact diagonal of A (boundary rows included).  Section 1.1 (the
 * multigrid solver smooths with Jacobi iterations).  x_out must not alias x_in. */
int nn4_jacobi_smooth(const nn4_grid* g, nn4_dtype dt, const void* b, const void* k,
                      const void* x_in, void* x_out, double omega, void* stream);

/* ----------------------------------------------------------------- plans and solves */

typedef enum {
  NN4_OUTER_CYCLES = 0,  /* x += (inner_cycles V-cycles on A e = b - A x): the paper's repeated
                            cycles, in defect-correction form */
  NN4_OUTER_FCG = 1      /* flexible CG with the V-cycles as preconditioner (not in the paper;
                            needed for large density ratios) */
} nn4_outer;

typedef struct {
  nn4_dtype inner;       /* storage type of the multigrid hierarchy: F64 = the plain method;
                            F32 / BF16 = mixed precision (FP32 arithmetic, FP64 outer loop) */
  int32_t inner_cycles;  /* V-cycles per outer iteration, >= 1 */
  int32_t outer;         /* nn4_outer */
  double omega;          /* Jacobi weight, 2/3 in the paper's setting */
  int32_t use_graph;     /* capture each outer iteration as a CUDA graph (1) or launch eagerly */
  int32_t check_every;   /* read the residual norm back every this many outer iterations (>=1) */
  int32_t profile;       /* 1: launch eagerly and time every kernel with CUDA events (see
                            nn4_plan_profile); for measurement only */
  int32_t inner_krylov;  /* 0: the preconditioner is inner_cycles V-cycles.  n > 0: it is n
                            iterations of flexible CG in FP32 vectors on A e = r, each
                            preconditioned by inner_cycles V-cycles (mixed precision only) */
  int32_t coarse_tail;   /* 1: run the coarse levels in one launch (see coarse_entry_nodes; same
                            arithmetic as the per-level kernels); 0: one launch per step */
  int32_t autotune;      /* 1: time the compiled tile shapes, pipeline depths and z-march depths
                            of every stencil pass at plan creation and keep the fastest (cached
                            per process by grid size); 0: fixed defaults */
  int32_t coarse_entry_nodes; /* with coarse_tail: levels with at most this many nodes (0: 40000)
                            run in one cooperative launch over all SMs when the first of them has
                            more than 800 nodes */
  int32_t fused_prolong; /* 1: in a cycle that starts from e = 0, the level-0 Jacobi sweep forms
                            the prolonged correction itself from coarse tiles (no separate
                            prolongation launch); 0 (default): separate launch, measured faster
                            on GB300 (the in-tile build adds a synchronised phase to an
                            issue-bound sweep) */
  int32_t pass_shape;    /* -1: tile shapes autotuned (autotune = 1) or the defaults.  0 ..
                            nn4_pass_shapes() - 1: that compiled tile shape for every stencil pass
                            that has it (overrides autotune; shapes compiled for FP64 only leave
                            the FP32/BF16 passes at their default).  For verification */
} nn4_plan_opts;

/* Number of compiled stencil-pass tile shapes (the range of nn4_plan_opts.pass_shape).  The
   paper has no counterpart: tiling is an implementation choice.  Never fails. */
int32_t nn4_pass_shapes(void);

/* Fills o with the defaults: F64, 1 cycle, NN4_OUTER_CYCLES, omega 2/3, graphs on, check 1,
 * profile off, no inner Krylov loop, coarse tail on, autotuning on. */
void nn4_plan_opts_default(nn4_plan_opts* o);

typedef struct nn4_plan_s* nn4_plan;

/* Builds the multigrid hierarchy of grid g (g->pitch is the pitch of the FP64 arrays b, x
 * and k used with this plan).  k: device FP64 coefficient field on g, or NULL for the constant
 * coefficient.  Coarsening halves every axis ((n+1)/2) while all axes are odd and >= 5; the
 * coarsest level is solved with a dense inverse computed here (pseudo-inverse when no face is
 * Dirichlet).  With k, coarse operators are Galerkin products P^T A P formed on the device.
 * The plan owns every workspace array; this is the only call that allocates.
 * Errors: NN4_EINVAL, NN4_ENOMEM, NN4_EUNSUPPORTED (coarsest level above 1024 free nodes). */
int nn4_plan_create(const nn4_grid* g, const double* k, const nn4_plan_opts* o, nn4_plan* out);

int nn4_plan_destroy(nn4_plan p);

/* One sawtooth V(0,1) cycle on A x = b, in place on x (Section 2.4): residual on the finest
 * level, restriction down to the coarsest level, exact coarsest solve, then on every level on
 * the way up prolongation followed by one Jacobi sweep.  b and x are device arrays of the
 * plan's inner dtype on the fine grid with pitch nn4_row_pitch(nx, inner). */
int nn4_vcycle(nn4_plan p, const void* b, void* x, void* stream);

typedef struct {
  int32_t iterations;    /* outer iterations done */
  int32_t cycles;        /* V-cycles done */
  double rel_res;        /* final ||b - A x|| / ||b|| (free nodes), recomputed in FP64 */
  double* history;       /* caller-owned host array or NULL: relative residual after each
                            outer iteration, history[0] for the initial x */
  int32_t history_len;   /* capacity of history */
  int64_t kernels;       /* kernels launched by the call (graph kernel nodes included) */
} nn4_solve_info;

/* Solves A x = b (FP64 device arrays on the plan's grid, pitch g->pitch) from the x given,
 * until ||b - A x||_2 / ||b||_2 <= rtol or max_iters outer iterations.  Synchronises the stream.
 * Returns NN4_ENOCONV (with info filled) when the cap is reached, NN4_ENONFINITE for a
 * non-finite norm.  Section 2.4, Stages 1 and 3 (the pressure residual driven to zero by the
 * U-Net multigrid). */
int nn4_pressure_solve(nn4_plan p, const double* b, double* x, double rtol, int32_t max_iters,
                       nn4_solve_info* info, void* stream);

/* The same solve with host arrays: b_host and x_host are dense [nz][ny][nx] FP64 arrays in
 * host memory (pinned for full copy speed); they are copied in and the solution copied out
 * through plan-owned device buffers inside the call. */
int nn4_pressure_solve_host(nn4_plan p, const double* b_host, double* x_host, double rtol,
                            int32_t max_iters, nn4_solve_info* info, void* stream);

/* Per-kernel timing of a plan created with profile = 1: for every kernel category launched since
 * the last call (or plan creation), its name, launch count and summed device time in ms, taken
 * from CUDA events recorded on the launching stream around each launch.  Writes up to `cap`
 * entries and returns how many categories exist (or a negative status).  Synchronises. */
typedef struct {
  char name[32];
  int64_t launches;
  double total_ms;
} nn4_kernel_time;

int nn4_plan_profile(nn4_plan p, nn4_kernel_time* out, int32_t cap);

/* Static facts of a plan: number of levels and node counts per level (up to 16). */
typedef struct {
  int32_t levels;
  int32_t n[16][3];
  int32_t coarsest_free;
  int64_t device_bytes;  /* device memory owned by the plan */
} nn4_plan_info;

int nn4_plan_query(nn4_plan p, nn4_plan_info* out);

/* ----------------------------------------------------------------- batched solves */

typedef struct nn4_batch_s* nn4_batch;

/* A batch of `count` independent constant-coefficient pressure systems on grids of uneven sizes
 * (grids[i]: node counts, spacing (equal on the three axes), faces, and the pitch of that
 * instance's FP64 arrays).  Options as for nn4_plan_create: `inner` storage type and
 * `inner_cycles` V-cycles per outer FP64 defect-correction iteration (Section 2.4's repeated
 * cycles); `check_every` sets how often the host reads the per-instance convergence flags.  Every
 * step of the cycle is one launch over the work items of all instances (the batching form; not
 * in the paper).  With `autotune` (default on) the Jacobi launch of every level step is timed here
 * for each compiled tile shape and z-march depth cap and the fastest kept (nn4_batch_query);
 * `pass_shape` in 0 .. 3 forces one shape.  Allocates all workspace here.  Errors: NN4_EINVAL, NN4_EUNSUPPORTED (unequal
 * spacings, fewer than two levels, coarsest level above 1024 free nodes), NN4_ENOMEM. */
int nn4_batch_create(const nn4_grid* grids, int32_t count, const nn4_plan_opts* opts, nn4_batch* out);

int nn4_batch_destroy(nn4_batch b);

/* What the batch's autotuner chose for the Jacobi launch of each level step (level 0 = the finest
 * level of every instance; levels that join the one-CTA coarse tails have no such launch).  Not in
 * the paper: tile shapes and z-march depths are implementation choices.  shape: index of the
 * compiled tile shape (0 .. 3, the first four of nn4_pass_shapes()); zmax: the cap on output planes
 * per work item; jacobi_us: the launch's measured time at creation (0 when not timed: a forced or
 * default shape); items: work items of the launch; nodes: nodes it covers over all instances. */
typedef struct {
  int32_t levels;
  int32_t shape[16];
  int32_t zmax[16];
  float jacobi_us[16];
  int32_t items[16];
  int64_t nodes[16];
} nn4_batch_info;

int nn4_batch_query(nn4_batch b, nn4_batch_info* info);

/* Solves every instance from its x (bs[i], xs[i]: host arrays of device pointers to FP64 arrays)
 * until its own relative residual <= rtol or max_iters outer iterations; converged instances stop
 * early (their work items are skipped).  infos (host, count entries, nullable) receives each
 * instance's iterations and final relative residual; latency_ms (host, nullable) the time from the
 * start of the solve to the instance's convergence, from device %globaltimer stamps (-1 if it did
 * not converge).  Synchronises the stream.  Returns NN4_ENOCONV if any instance hit the cap,
 * NN4_ENONFINITE if any residual was not finite. */
int nn4_pressure_solve_batched(nn4_batch b, const double* const* bs, double* const* xs, double rtol,
                               int32_t max_iters, nn4_solve_info* infos, float* latency_ms, void* stream);

/* ----------------------------------------------------------------- explicit multiphase terms */

/* Constants of the compressive Petrov-Galerkin volume-fraction scheme (Sections 2.3.5-2.3.6). */
typedef struct {
  double dt;         /* time step */
  double alpha_a;    /* Eq. a_psi: 2 */
  double eps_k;      /* Eq. k-abs: 1e-7 */
  double K_plus;     /* weight w+: 300 */
  double K_minus;    /* weight w-: 300 */
  double beta;       /* Eq. negativek: 0.1 */
  double eps_x;      /* Eqs. negativek, normalisation: 1e-4 */
  double K_pos;      /* Eq. positivek: 3 */
  double alpha_min;  /* Eq. alpha_min_and_max: 1e-4 */
  double alpha_max;  /* Eq. alpha_min_and_max: 0.05 */
  double detect_hi;  /* detector override C > 0.95 */
  double detect_lo;  /* detector override C < 0.05 */
  int32_t p;         /* polynomial order (1: linear filters) */
  int32_t compute;   /* NN4_F64 (default): FP64 arithmetic.  NN4_F32: FP32 arithmetic on the FP64
                        state (C, u, v, w, s_C, C_next stay FP64 in memory; the detector override
                        is decided on the FP64 C; C_next = C - dt m^-1 s_C adds the FP32 increment
                        in FP64).  Not in the paper: a precision form of this library. */
} nn4_vof_params;

/* Fills p with the paper's constants and the given time step. */
void nn4_vof_params_default(nn4_vof_params* p, double dt);

/* Bytes of device workspace nn4_vof_advect_residual needs for grid g (the three directional
 * diffusion coefficient fields k^x, k^y, k^z, sized as FP64), or -1. */
int64_t nn4_vof_workspace_bytes(const nn4_grid* g);

/* One explicit volume-fraction step (Stage 4 of Section 2.4): s_C of Eq. Petrov-Cs (advection
 * with the first-derivative filters plus the compressive directional Petrov-Galerkin diffusion
 * of Section 2.3.6 in the form of Eq. k-Txx) and, if C_next != NULL, C_next = C - dt m^-1 s_C
 * (Eq. transport-indicator-1, m the lumped nodal volume).  C, u, v, w (q^{n+1}), s_C, C_next:
 * FP64 device arrays on g; workspace: nn4_vof_workspace_bytes(g) bytes of device memory owned by
 * the caller (contents overwritten).  Natural faces for C; the oscillation detector uses the
 * copy-halo of Section 2.3.3 at walls.  Arithmetic in p->compute (FP64 by default).
 * Two launches: the coefficients k^d (Eqs. a_psi to alpha_min_and_max) into the workspace, then
 * s_C and C_next.  Errors: NN4_EINVAL for a bad grid, parameter or pointer, or outputs aliasing C. */
int nn4_vof_advect_residual(const nn4_grid* g, const nn4_vof_params* p, const double* C, const double* u,
                            const double* v, const double* w, double* s_C, double* C_next, void* workspace,
                            void* stream);

/* The same volume-fraction step for callers that cannot allocate device memory: hosts that hand
 * out all device memory from their own pool or fixed budget, and loops in which the implicit
 * device synchronisation of cudaMalloc / cudaFree is not acceptable.  The paper has no
 * counterpart; this is a deployment variant of nn4_vof_advect_residual.
 * It takes no workspace: its scratch (the three coefficient fields) is a fixed device array
 * inside the library (18 MiB, held by every GPU that loads the library until the process exits)
 * and it calls no allocating routine.  Grids need pitch * ny * nz <= 786432 (e.g. 129 x 65 x 65 with the FP64
 * pitch); larger grids return NN4_EINVAL with the limit in nn4_last_error().
 * The first call on each device looks up the array's device address (cudaGetSymbolAddress) with
 * that device current; make that first call before any stream capture.  Every call, on every
 * stream, shares the one array: calls that overlap on the GPU race on it and give wrong
 * results, so serialise them (one stream, or events).  Each call writes every scratch element
 * it reads, so no state carries over from the previous call.  Arguments and results as for
 * nn4_vof_advect_residual. */
int nn4_vof_advect_residual_static(const nn4_grid* g, const nn4_vof_params* p, const double* C, const double* u,
                                   const double* v, const double* w, double* s_C, double* C_next, void* stream);

/* *out (device FP64) = sum_i m_i C_i with m the lumped nodal volume: the C(t) of the mass
 * diagnostic (Section 3, mass conservation), accumulated in FP64. */
int nn4_mass_sum(const nn4_grid* g, const double* C, double* out, void* stream);

/* Physical constants and scheme settings of a multiphase run (Sections 2.1-2.4). */
typedef struct {
  double dt;                 /* time step */
  double rho_l, rho_g;       /* densities of liquid (C = 1) and gas */
  double mu_l, mu_g;         /* viscosities; mu = mu_l C + mu_g (1 - C) */
  double sigma_t;            /* surface tension coefficient */
  double g;                  /* gravity magnitude, acting along -z */
  double alpha_a;            /* Eq. a_psi: 2 */
  double eps_k;              /* Eqs. k-abs, h_Psi, k-square: 1e-7 */
  int32_t p;                 /* polynomial order (1) */
  int32_t momentum_iters;    /* Stage 2 predictor iterations (2) */
  int32_t correction_iters;  /* Stage 3 pressure-velocity corrections N_I (2) */
  int32_t pressure_cycles;   /* outer iterations per pressure solve when pressure_rtol <= 0 (20) */
  double pressure_rtol;      /* > 0: solve each pressure equation to this relative residual */
  int32_t compute;           /* NN4_F64 (default) or NN4_F32: the arithmetic of the explicit terms
                                (sources, right-hand sides, velocity correction, predictor and the
                                volume-fraction step); state stays FP64 in memory.  Not in the
                                paper: a precision form of this library. */
} nn4_flow_params;

void nn4_flow_params_default(nn4_flow_params* p, double dt);

/* Momentum sources (Eqs. surface-tension-uvw, surface-tension-k, gravity): s_d = sigma_t kappa
 * C_d, and s_z -= g rho, with C_d the pointwise gradient m^-1 f(C; w_d), normals C_d / (eps_t +
 * |grad C|), eps_t = 1e-7 / min(h), kappa = m^-1 sum_d f(n_d; w_d).  s0, s1, s2: outputs; kappa:
 * optional output; workspace: unused (may be NULL; the normals are formed in shared memory).  FP64
 * device arrays on g; arithmetic in fp->compute. */
int nn4_momentum_sources(const nn4_grid* g, const nn4_flow_params* fp, const double* C, double* s0, double* s1,
                         double* s2, double* kappa, double* workspace, void* stream);

/* Stage-1 right-hand side (Eq. ph_disc, continuum signs): b = sum_d G_d^T s_d, G_d the assembled
 * first-derivative filter w_d, 0 on the Dirichlet faces of g (the pressure faces). */
int nn4_pressure_rhs_hs(const nn4_grid* g, const double* s0, const double* s1, const double* s2, double* b,
                        void* stream);
/* The same with the arithmetic in `compute` (NN4_F64 or NN4_F32; arrays stay FP64). */
int nn4_pressure_rhs_hs_ex(const nn4_grid* g, int compute, const double* s0, const double* s1, const double* s2,
                           double* b, void* stream);

/* Stage-3 right-hand side (Eq. ph_disc2): b = -(1/dt) sum_d [ f(rho u~_d; w_d) - u~_d f(rho; w_d) ],
 * rho from C (formed in shared memory); 0 on the Dirichlet faces of g.  rho_ws: unused (may be
 * NULL).  Arithmetic in fp->compute. */
int nn4_pressure_rhs_nh(const nn4_grid* g, const nn4_flow_params* fp, const double* C, const double* u,
                        const double* v, const double* w, double* b, double* rho_ws, void* stream);

/* Eq. vel-cor and the Stage-3 updates: (u, v, w) += -dt m^-1 f(dp; w_d) / rho except on the
 * Dirichlet (no-slip) faces of g, and p_nh += dp (p_nh may be NULL). */
int nn4_velocity_correct(const nn4_grid* g, const nn4_flow_params* fp, const double* C, const double* dp, double* u,
                         double* v, double* w, double* p_nh, void* stream);

/* One Stage-2 predictor iteration for the three components (Eqs. Petrov-u/v/w, k_Psi-n, k-abs,
 * k-square, max-k, velocity-1 with sigma = 0): from u^n (un), the current u^{n+1/2} (uh), the total
 * pressure p = p_hs + p_nh and the sources s (from nn4_momentum_sources), writes u~ (ut) and, if
 * uh_next != NULL, the next u^{n+1/2} = (u^n + u~)/2 (uh_next).  un, uh, ut, uh_next, s: arrays of
 * three device pointers; ut and uh_next must not alias any input (the filters read uh around each
 * node).  Dirichlet faces of g are no-slip walls.  workspace: nn4_momentum_workspace_bytes(g)
 * bytes (the three coefficient fields k_Psi).  Arithmetic in fp->compute. */
int64_t nn4_momentum_workspace_bytes(const nn4_grid* g);
int nn4_momentum_predict(const nn4_grid* g, const nn4_flow_params* fp, const double* C, const double* const* un,
                         const double* const* uh, double* const* ut, double* const* uh_next, const double* p,
                         const double* const* s, void* workspace, void* stream);

/* A multiphase time stepper: Stage 1 (hydrostatic + surface-tension pressure), Stage 2 (momentum
 * predictor), Stage 3 (N_I non-hydrostatic pressure corrections), Stage 4 (volume fraction) of
 * Section 2.4, with the pressure solves of a plan created with popts.  vel_grid: the node grid
 * with the no-slip faces as Dirichlet; p_grid: the same nodes with the pressure faces (Dirichlet
 * where p = 0).  All workspace is allocated here. */
typedef struct nn4_flow_s* nn4_flow;

typedef struct {
  double mass;          /* sum_i m_i C_i after the step */
  double c_min, c_max;  /* range of C after the step */
  int32_t hs_iters;     /* outer iterations of the Stage-1 solve */
  int32_t nh_iters;     /* outer iterations of the last Stage-3 solve */
  double hs_rel, nh_rel;
} nn4_flow_stats;

int nn4_flow_create(const nn4_grid* vel_grid, const nn4_grid* p_grid, const nn4_flow_params* fp,
                    const nn4_plan_opts* popts, nn4_flow* out);
int nn4_flow_destroy(nn4_flow f);

/* Advances the caller's device state (FP64, vel_grid pitch) by one step in place: C, u, v, w at
 * level n -> n+1, p_hs and p_nh updated.  stats: host, nullable.  Synchronises the stream. */
int nn4_flow_step(nn4_flow f, double* C, double* u, double* v, double* w, double* p_hs, double* p_nh,
                  nn4_flow_stats* stats, void* stream);

/* ----------------------------------------------------------------- diagnostics */

const char* nn4_last_error(void);

/* Reads and clears the device error word: NN4_OK, NN4_ETIMEOUT or NN4_EBOUNDS. Synchronises. */
int nn4_device_error(void);

const char* nn4_version(void);

#ifdef __cplusplus
}
#endif

#endif /* NN4_H */
