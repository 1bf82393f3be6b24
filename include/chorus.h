/*
 * chorus.h - C ABI of the GB300 spectral-difference (SD) residual library.
 *
 * The library evaluates the semi-discrete residual of the compressible
 * Navier-Stokes equations for a stratified, rotating spherical shell (gravity
 * g = -GM r_hat / r^2, Coriolis force about +z; paper Section 2, Eqs. 1-9)
 * discretised by the spectral difference method on curved 20-node hexahedra
 * (Section 3, Eqs. 10-19), with impenetrable stress-free walls (Section 5),
 * and advances it with the three-stage SSP Runge-Kutta scheme.
 *
 * Conventions shared by every call
 *  - p is the polynomial degree, N = p + 1 solution points per direction,
 *    N^3 solution points per element.  2 <= p <= 5.
 *  - State layout: Q[e][v][i + N*j + N*N*k] (element-major, then the five
 *    conserved variables rho, rho u, rho v, rho w, E, then the solution point
 *    with i along xi fastest).  Solution points are the Chebyshev-Gauss points
 *    of Eq. 13 in each direction of the reference cube [0,1]^3.
 *  - Precision:
 *      CHORUS_FP64       Q holds the total conserved state, double.
 *      CHORUS_FP32_PERT  Q holds the perturbation q' = Q - Q0 from the
 *                        polytropic background Q0 (Eqs. 25-27 at rest), float.
 *                        The background residual R(Q0) and the background
 *                        tables are kept in FP64-derived form by the library.
 *    Residuals R are dQ/dt in the same precision as Q (total, not
 *    perturbation, for both precisions).
 *  - Device pointers (Q, R, workspace) are caller-owned, contiguous, 16-byte
 *    aligned device allocations.  Host pointers are marked "host".
 *  - stream is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    Calls are asynchronous on that stream except where stated.
 *  - Errors: arguments are validated before any launch (CHORUS_EINVAL,
 *    CHORUS_EMESH); a CUDA error from a launch or copy returns CHORUS_ECUDA;
 *    a device-side timeout of a bounded wait is reported as CHORUS_ETIMEOUT
 *    by the next call that synchronises (chorus_reduce, chorus_check), which
 *    then clears the flag.  A kernel whose wait ran out writes none of its
 *    outputs, so check before using a result when timeouts are possible.
 *    No call aborts the process or traps the GPU.
 */
#ifndef CHORUS_H
#define CHORUS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct chorus_mesh_s* chorus_mesh;

typedef enum {
  CHORUS_OK = 0,
  CHORUS_EINVAL = 1,      /* bad argument */
  CHORUS_ENOMEM = 2,      /* device or host allocation failed */
  CHORUS_ECUDA = 3,       /* CUDA runtime error */
  CHORUS_EMESH = 4,       /* invalid connectivity, non-manifold face, |J| <= 0, stray boundary */
  CHORUS_ENAN = 5,        /* non-finite value found by a reduction */
  CHORUS_ETIMEOUT = 6,    /* a bounded device-side wait ran out */
  CHORUS_EUNSUPPORTED = 7 /* order or mode not built */
} chorus_status;

typedef enum { CHORUS_FP64 = 0, CHORUS_FP32_PERT = 1 } chorus_precision;

/* Physical parameters (paper Section 2, Eq. 24, Section 4.2, Section 5), nondimensional.
 * gamma, R_gas: ideal gas (Eq. 22); GM: gravity g = GM/r^2; Omega: rotation about +z;
 * nu: kinematic viscosity (mu = rho nu, Eq. 9); kappa: entropy diffusivity; kappa_r: thermal
 * (radiative) diffusivity (f = -kappa rho T grad S - kappa_r rho C_p grad T); poly_n, N_rho, rho_c:
 * polytrope of Eqs. 25-27 (beta = r_inner / r_outer from the mesh); bottom_flux: f.r_hat
 * imposed on the inner wall (L / (4 pi R_i^2)); T_top: temperature imposed on the outer wall,
 * NaN meaning the polytrope temperature at r_outer; kappa_r1, kappa_r2: a radial profile of the
 * radiative diffusivity, kappa_r(r) = kappa_r + kappa_r1 r + kappa_r2 r^2 (the solar benchmark's
 * quadratic, Section 7.2); 0, 0 for a constant.  A varying profile enters the fluxes as its values
 * at the solution points interpolated to the flux points (Eq. 17), like the solution itself, and
 * must be non-negative at both walls (else CHORUS_EINVAL). */
typedef struct {
  double gamma, R_gas, GM, Omega;
  double nu, kappa, kappa_r;
  double poly_n, N_rho, rho_c;
  double bottom_flux, T_top;
  double kappa_r1, kappa_r2;
} chorus_params;

/* Build a mesh handle from 20-node hexahedra (Section 3 iso-parametric map, Section 5 20-node
 * elements).  node_xyz: host [n_nodes][3] double.  hex20: host [n_elem][20] int64, 0-based,
 * local node order: corners (0,0,0) (1,0,0) (1,1,0) (0,1,0) (0,0,1) (1,0,1) (1,1,1) (0,1,1),
 * then the mid-edge nodes of edges 0-1, 1-2, 2-3, 3-0, 4-5, 5-6, 6-7, 7-4, 0-4, 1-5, 2-6, 3-7
 * (reference axes xi, eta, zeta).  Faces are paired by their corner nodes; unpaired faces must lie
 * on the sphere r_inner (inner wall) or r_outer (outer wall) to a relative 1e-6, else
 * CHORUS_EMESH.  metric_mode 0: conservative curl-form metrics (freestream preserving for every
 * p; for p >= 3 the curl form equals the cofactor rows exactly and is evaluated in that form, with
 * less rounding); 1: analytic cofactors of the 20-node map (freestream preserving for p >= 3).
 * The Jacobian and the metrics are formed from node coordinates measured from each element's node
 * centroid (a translation, which leaves them unchanged but avoids cancellation in FP64).  The library
 * copies what it needs; the caller keeps ownership of its arrays.  Synchronises the stream. */
chorus_status chorus_mesh_create(int64_t n_nodes, const double* node_xyz, int64_t n_elem,
                                 const int64_t* hex20, int p, double r_inner, double r_outer,
                                 int metric_mode, void* stream, chorus_mesh* out);
chorus_status chorus_mesh_destroy(chorus_mesh mesh);

/* n_dof = n_elem * N^3 (Eq. 19); n_faces = interior faces + wall faces; h_min = shortest
 * corner-to-corner element edge; volume = sum of w_i w_j w_k |J| (host outputs, any may be NULL). */
chorus_status chorus_mesh_info(chorus_mesh mesh, int64_t* n_dof, int64_t* n_faces, double* h_min,
                               double* volume);

/* Build the per-parameter background tables (polytropic Q0, its FP64 residual R(Q0), lifted
 * background density gradient, background face traces, gravity vectors).  Must be called before
 * FP32_PERT residual/rk calls and before chorus_state_init; calling again with other parameters
 * rebuilds them.  Allocates device memory owned by the mesh handle. */
chorus_status chorus_prepare(chorus_mesh mesh, const chorus_params* params, void* stream);

/* Background from a radial profile instead of the polytrope: rho0, p0 host double[n] (n >= 4) on the
 * uniform grid r_j = r0 + j (r1 - r0)/(n - 1), at rest; the solution-point values come from cubic
 * Lagrange interpolation on the four nearest nodes.  The grid must cover the radii of all solution
 * points - 20-node elements can place some slightly outside the spherical walls, so take a margin
 * of a few percent of the shell thickness - and be fine enough that the interpolation error is
 * negligible (16,385 nodes give about 1e-15 relative for the workloads).  Builds the same tables as
 * chorus_prepare; a later chorus_prepare with the same params keeps this background.  Non-positive
 * or non-finite entries, n < 4 or r1 <= r0 > 0: CHORUS_EINVAL.  Synchronises. */
chorus_status chorus_prepare_profile(chorus_mesh mesh, const chorus_params* params, int64_t n, double r0, double r1,
                                     const double* rho0, const double* p0, void* stream);

/* The almost-flux-balance stratification of Section 4.3 on the uniform grid above (host; no GPU):
 * target entropy gradient Gamma(r) = -(L/(4 pi r^2) + rho_a C_p kappa_r(r) dT_a/dr) / (rho_a T_a kappa)
 * (the thermal balance of Section 4.1 integrated with outward luminosity L; superadiabatic)
 * with L = 4 pi r_inner^2 bottom_flux and the polytrope rho_a, T_a of params and the shell radii,
 * then drho0/dr = -rho0 (Gamma/C_p + g rho0/(gamma p0)), dp0/dr = -rho0 g (g = GM/r^2), integrated
 * with classical RK4 (16 substeps per grid interval) outward and inward from the middle radius
 * (r_inner + r_outer)/2, where rho0 and p0 take the polytrope's values (the paper starts its solve
 * from the polytrope; the anchoring point is this library's reading).  The grid [r0, r1] may extend
 * beyond the walls (the equations continue there).  n >= 2, kappa > 0; rho0, p0: host double[n]
 * outputs.  CHORUS_ENAN if the stratification leaves positive density or pressure. */
chorus_status chorus_afb_profile(const chorus_params* params, double r_inner, double r_outer, double r0, double r1,
                                 int64_t n, double* rho0, double* p0);

/* Seeded initial state (Section 4): the prepared background at rest with an entropy perturbation
 * S'/C_p = A xi, xi in [-1,1) from SplitMix64(seed XOR g) at global solution point
 * g = e N^3 + (i + N j + N^2 k); pressure kept, rho = rho_a exp(-A xi).  Q: device, layout above,
 * in the given precision (total state for FP64, perturbation for FP32_PERT). */
chorus_status chorus_state_init(chorus_mesh mesh, const chorus_params* params, uint64_t seed,
                                double entropy_amp, chorus_precision prec, void* Q, void* stream);

/* dQ/dt of the SD discretisation at the solution points (Sections 3 and 5).  Q, R: device.
 * Needs chorus_rk_workspace_bytes() of scratch, passed as workspace. */
chorus_status chorus_residual(chorus_mesh mesh, const chorus_params* params, chorus_precision prec,
                              const void* Q, void* R, void* workspace, void* stream);

/* The fixed explicit time step of the workloads (the paper states only a CFL condition, Section 7.5):
 * dt = 0.25 h_min / ((2p + 1) c_max), capped by 0.25 h_min^2 / ((2p + 1)^2 max(nu, kappa)), with
 * c_max = sqrt(gamma R T_a(r_inner)) the largest sound speed of the polytrope at rest of params
 * (Eqs. 25-27; T_a peaks at the inner wall).  h / ((2p + 1) c) is the one-dimensional limit of the
 * degree-p SD operator; elements with comparable edges share it among three directions, hence 0.25.
 * chorus_stable_dt_rule takes the order and the shortest element edge h_min (host computation, no
 * GPU); chorus_stable_dt takes them from the mesh (chorus_mesh_info's h_min).  dt: host double.
 * Bad arguments: CHORUS_EINVAL; a non-finite or non-positive result: CHORUS_ENAN. */
chorus_status chorus_stable_dt_rule(int p, double h_min, double r_inner, double r_outer,
                                    const chorus_params* params, double* dt);
chorus_status chorus_stable_dt(chorus_mesh mesh, const chorus_params* params, double* dt);

/* Measured fused multiply-add rate of the current GPU, for rooflines (a measurement helper with no
 * counterpart in the paper): 8 independent FMA chains per thread on 8 CTAs of 256 threads per SM,
 * timed with CUDA events on `stream` over a launch sized to about 20 ms, 2 flops per FMA.
 * prec CHORUS_FP64: double; CHORUS_FP32_PERT: float.  flops_per_s: host double.  Allocates and frees
 * a small output buffer (stream-ordered) and synchronises the stream. */
chorus_status chorus_fma_rate(int prec, void* stream, double* flops_per_s);

/* Bytes of device scratch needed by chorus_residual and chorus_rk_step. */
size_t chorus_rk_workspace_bytes(chorus_mesh mesh, chorus_precision prec);

/* n_steps SSP-RK3 steps of size dt, in place on Q (Shu-Osher form:
 * u1 = u + dt L(u); u2 = 3/4 u + 1/4 (u1 + dt L(u1)); u^{n+1} = 1/3 u + 2/3 (u2 + dt L(u2))). */
chorus_status chorus_rk_step(chorus_mesh mesh, const chorus_params* params, chorus_precision prec,
                             void* Q, void* workspace, double dt, int64_t n_steps, void* stream);

/* chorus_rk_step on a state held in host memory: copies Q_host (host, the state layout, pinned for
 * full copy bandwidth) to Q_dev (device, caller-owned, same size), takes n_steps SSP-RK3 steps there,
 * copies the result back into Q_host and synchronises the stream.  workspace as for chorus_rk_step.
 * This is the end-to-end form of a step for callers whose state lives on the host.  In the FP32 form
 * the state is copied in by eight element ranges (on a stream of the mesh's own, after the work
 * already queued on `stream`), each range's face traces computed as soon as it has arrived, and the
 * last stage's residual runs on the same ranges, each range's new state copied back while the next is
 * computed; the result equals chorus_rk_step's bit for bit.  Calls on one mesh must not overlap. */
chorus_status chorus_rk_step_host(chorus_mesh mesh, const chorus_params* params, chorus_precision prec,
                                  void* Q_host, void* Q_dev, void* workspace, double dt, int64_t n_steps,
                                  void* stream);

/* n_steps steps of an explicit SSP scheme, in place on Q.  scheme 0: the SSP-RK3 of
 * chorus_rk_step; scheme 1: the five-stage fourth-order SSP-RK(5,4) of Spiteri and Ruuth that the
 * paper integrates with (Section 7.4; Shu-Osher form u1 = u + b10 dt L(u), ...,
 * u^{n+1} = a52 u2 + a53 u3 + b53 dt L(u3) + a54 u4 + b54 dt L(u4), published coefficients).
 * Workspace as for chorus_rk_step. */
chorus_status chorus_rk_step_scheme(chorus_mesh mesh, const chorus_params* params, chorus_precision prec,
                                    int scheme, void* Q, void* workspace, double dt, int64_t n_steps,
                                    void* stream);

/* FP64 volume integrals of Q (total state): out[0] mass, out[1] total energy, out[2] kinetic
 * energy sum |m|^2/(2 rho), out[3] |L| with L = integral of x cross (rho u) (Section 6, Eq. 32).
 * out: host double[4].  Synchronises the stream; returns CHORUS_ENAN on non-finite results. */
chorus_status chorus_reduce(chorus_mesh mesh, const chorus_params* params, chorus_precision prec,
                            const void* Q, double* out, void* stream);

/* Angular-momentum correction (Section 6): L = integral of x cross (rho u) (Eq. 32), moments of
 * inertia I_x = integral of rho (y^2 + z^2) etc., delta Omega_i = L_i / I_i (Eq. 33), and the
 * velocity update of Eq. 34 (u -= delta Omega x r) at every solution point, in place on Q; density
 * and pressure are kept (the total energy takes the new kinetic energy).  Integrals in FP64 with
 * the solution-point quadrature.  domega: host double[3] receiving delta Omega (the call then
 * synchronises the stream) or NULL (fully asynchronous).  FP32_PERT needs chorus_prepare. */
chorus_status chorus_am_correct(chorus_mesh mesh, const chorus_params* params, chorus_precision prec,
                                void* Q, double* domega, void* stream);

/* ---- Learned subgrid closure for coarse (p = 2) runs.
 * The paper names subgrid-scale modelling as future work (Section 8); the closure is a workload
 * extension.  Per element, the p = 2 state's departure from the background, q' (27 points x 5
 * variables, in the state layout, i.e. index v*27 + pt), divided by in_scale[v], feeds a network
 * 135 -> 128 (SiLU) -> 128 (SiLU) -> 135; its output times out_scale[v] is added to dQ/dt.
 * Record (device, caller-owned, chorus_closure_bytes() bytes): BF16 W1 [128][135], W2 [128][128],
 * W3 [135][128] (row-major, output index first), FP32 b1 [128], b2 [128], b3 [135], in_scale [5],
 * out_scale [5].  Arithmetic accumulates in FP32. */
size_t chorus_closure_bytes(void);

/* Seeded initial record: weights uniform in +-sqrt(3/fan_in) (output layer x 0.1), zero biases,
 * the given scales (host float[5] each, > 0).  Synchronises the stream. */
chorus_status chorus_closure_init(void* weights, uint64_t seed, const float* in_scale, const float* out_scale,
                                  void* stream);

/* Overwrite the input and output scales of a record (host float[5] each, > 0), keeping its weights:
 * scaling out_scale by a factor relaxes the correction.  Synchronises the stream. */
chorus_status chorus_closure_set_scales(void* weights, const float* in_scale, const float* out_scale, void* stream);

/* Per-element L2 projection from `fine` to `coarse` (same elements, lower order) in the reference
 * cube, one direction at a time (P = M_c^-1 B with exact Gauss-Legendre integrals).  kind 0: a
 * state in the given precision (for FP32_PERT the fine background is added before and the coarse
 * one subtracted after, both meshes prepared with the same parameters); kind 1: any 5-variable
 * field such as a residual.  Qf, Qc: device, state layout of each mesh. */
chorus_status chorus_project(chorus_mesh fine, chorus_mesh coarse, chorus_precision prec, int kind, const void* Qf,
                             void* Qc, void* stream);

/* Network forward pass on n samples: X, Y device [n][135] FP32, FP32 activations (the training
 * arithmetic). */
chorus_status chorus_closure_forward(const void* weights, const float* X, float* Y, int64_t n, void* stream);

/* The same forward pass on the tensor cores (tcgen05, 128-sample tiles, persistent CTAs): each
 * layer's input is rounded to BF16 (nearest even), products accumulate in FP32, bias and SiLU in
 * FP32.  This is the arithmetic of the closure inside the residual and the RK stages
 * (chorus_closure_apply / chorus_closure_attach). */
chorus_status chorus_closure_forward_tc(const void* weights, const float* X, float* Y, int64_t n, void* stream);

/* Gradient of L = sum (y - t)^2 / (2 * 135 n) with respect to the parameters (FP32 device vector of
 * W1, W2, W3, b1, b2, b3 in that order, 51,335 entries, overwritten) and the loss (host).
 * Synchronises the stream. */
chorus_status chorus_closure_grad(const void* weights, const float* X, const float* Y, int64_t n, float* grad,
                                  double* loss, void* stream);

/* Training pairs of one coarse state: X = q'_c / in_scale, Y = (P R_fine - R_coarse) / out_scale per
 * element (X, Y device [E][135] FP32; Qc, PRf, Rc device in the mesh's state layout and precision). */
chorus_status chorus_closure_make_pairs(chorus_mesh coarse, chorus_precision prec, const void* weights,
                                        const void* Qc, const void* PRf, const void* Rc, float* X, float* Y,
                                        void* stream);

typedef struct {
  int64_t epochs, batch;        /* passes over the pairs, samples per Adam step */
  double lr, beta1, beta2, eps; /* Adam (Kingma and Ba) */
  uint64_t seed;                /* reserved */
} chorus_train_cfg;

/* Adam training of the record in place on n_pairs pairs (X, Y device [n][135] FP32, taken in order
 * in batches; shuffle beforehand).  FP32 master weights live in a temporary device workspace; the
 * record's BF16 weights are rewritten after every step.  losses: host double[epochs] receiving the
 * mean batch loss of each epoch, or NULL.  Synchronises the stream. */
chorus_status chorus_closure_train(const float* X, const float* Y, int64_t n_pairs, void* weights,
                                   const chorus_train_cfg* cfg, double* losses, void* stream);

/* R += closure(Q) for a p = 2 mesh (FP64 needs chorus_prepare for the background). */
chorus_status chorus_closure_apply(chorus_mesh coarse, chorus_precision prec, const void* weights, const void* Q,
                                   void* R, void* stream);

/* Attach a record to a p = 2 mesh: chorus_residual and every RK stage then add the closure to
 * dQ/dt.  NULL detaches.  The record must stay valid while attached. */
chorus_status chorus_closure_attach(chorus_mesh coarse, const void* weights);

/* Kernel timing for measurement.  While enabled, every kernel that chorus_residual and
 * chorus_rk_step launch is bracketed by a pair of CUDA events recorded on the call's stream (the
 * kernels themselves are unchanged).  chorus_timing_read synchronises the stream and returns, per
 * kernel class (0: face traces, 1: lifted gradients / one-sided viscous fluxes / wall fluxes,
 * 2: residual and RK update, 3: common fluxes of the interior faces), the summed device
 * milliseconds and launch counts recorded since the last read, then clears them.  ms, counts: host
 * arrays of 4.  enable = 0 stops recording. */
chorus_status chorus_timing_enable(chorus_mesh mesh, int enable);
chorus_status chorus_timing_read(chorus_mesh mesh, void* stream, double* ms, int64_t* counts);

/* chorus_residual without any device allocation by the caller or the library.  The paper has no
 * counterpart: this is a library convenience.  Some callers cannot allocate device memory when they
 * need a residual - for example an application that has handed all device memory to its own pool
 * allocator, or a latency-critical loop that must not call cudaMalloc (which can synchronise the
 * device).  They pass only the state Q and the output R (device, layout above); the scratch (face
 * traces, one-sided viscous face fluxes, gradient record, common face fluxes) lives in one fixed
 * 32 MiB device array
 * inside the library, which every GPU that loads the library holds until the process exits.
 *  - Size limit: E * (6 * 14 * N^2 + 12 * N^3) words of the chosen precision must fit in 32 MiB
 *    (FP32 p = 3: up to 3,971 elements; FP64 p = 3: up to 1,985).  Larger meshes return
 *    CHORUS_EINVAL before any launch; use chorus_residual with a workspace for them.
 *  - Set-up: the first call on a device looks up the array's device address with that device
 *    current; make that first call before any stream capture.  Call with the mesh's device current.
 *  - Sharing: all calls share the one array and it keeps the previous call's contents (every call
 *    overwrites all it reads, nothing needs to start at zero).  Calls that overlap on the GPU (other
 *    streams, other threads) race on it and must be serialised by the caller.
 *  - FP32_PERT needs chorus_prepare with the same params first, as chorus_residual does.
 *  - An attached closure (chorus_closure_attach) is added as chorus_residual adds it; its output
 *    buffer was allocated by the attach call.  FP64 with a closure needs chorus_prepare.
 *  - A radial kappa_r(r) (kappa_r1 or kappa_r2 non-zero) needs its flux-point table, which
 *    chorus_prepare (or any call with a workspace) builds for the mesh; without it this call returns
 *    CHORUS_EINVAL instead of allocating. */
chorus_status chorus_residual_noalloc(chorus_mesh mesh, const chorus_params* params, chorus_precision prec,
                                      const void* Q, void* R, void* stream);

/* ---- Batched independent shells -------------------------------------------------------------
 * Many independent shell instances of different resolution and order advanced together, for
 * ensembles and parameter studies (the paper runs one shell at a time; this is a throughput mode
 * of the same discretisation, Sections 3-5).  All shells share the radii and the physical
 * parameters; each has its own mesh, order and seeded perturbation.
 *  - Shells of one order form one internal mesh (their disjoint union), so each kernel of an RK
 *    stage is one launch per order present; the orders run concurrently on forked streams or one
 *    after another, and one RK step of the whole batch is captured once as a CUDA graph and
 *    replayed.  A third schedule runs every order in one persistent cooperative launch per RK
 *    stage: its CTAs take (order, tile) work items of each phase (traces, lifting, face fluxes,
 *    residual; the orders' tiles in one list) from a counter and meet at bounded grid barriers
 *    between the phases (a barrier that runs out of polls sets CHORUS_ETIMEOUT; nothing spins
 *    unbounded).  chorus_batch_schedule sets it; the autotuner times all three.
 *  - State: FP32 perturbation form (CHORUS_FP32_PERT) only.  One caller-owned device array holds
 *    every shell; shell s occupies [state_offset[s], state_offset[s] + n_elem_s * 5 * N_s^3)
 *    floats, in the single-mesh layout of its own order.
 *  - A shell of the batch computes bit for bit what a single mesh of that shell computes with the
 *    same tile shape (the union adds no coupling: shells share no faces). */
typedef struct chorus_batch_s* chorus_batch;

typedef struct {
  int64_t n_nodes;
  const double* node_xyz; /* host [n_nodes][3] */
  int64_t n_elem;
  const int64_t* hex20;   /* host [n_elem][20], 0-based, order as in chorus_mesh_create */
  int p;                  /* 2..5 */
  uint64_t seed;          /* perturbation seed (as chorus_state_init) */
  double entropy_amp;     /* perturbation amplitude (as chorus_state_init), 0 <= amp < 1 */
} chorus_shell_desc;

/* Build the batch: one mesh per order present (curl-form metrics), its background for params
 * (as chorus_prepare) and the forked streams.  Synchronises. */
chorus_status chorus_batch_create(int n_shells, const chorus_shell_desc* shells, double r_inner, double r_outer,
                                  const chorus_params* params, void* stream, chorus_batch* out);
chorus_status chorus_batch_destroy(chorus_batch batch);

/* state_offset: host int64[n_shells] (float offsets, see above) or NULL; n_state: total floats;
 * workspace_bytes: bytes of the workspace chorus_batch_rk_step needs; n_groups: orders present;
 * group_p, group_h_min: host arrays of 4 receiving, per order present (ascending), the order and
 * the shortest element edge chord of its shells (for the caller's time-step choice), or NULL.
 * Any output may be NULL. */
chorus_status chorus_batch_layout(chorus_batch batch, int64_t* state_offset, int64_t* n_state,
                                  size_t* workspace_bytes, int* n_groups, int* group_p, double* group_h_min);

/* Seeded perturbation of every shell (shell s as chorus_state_init of its own mesh with its seed). */
chorus_status chorus_batch_init(chorus_batch batch, float* Q, void* stream);

/* n_steps SSP-RK3 steps of size dt for every shell.  The step graph is captured on the first call
 * for (Q, workspace, dt) and replayed; a call with other pointers or dt captures again (the
 * persistent schedule launches directly, three launches a step).  launches: host int64 receiving
 * the kernel launches per step, or NULL. */
chorus_status chorus_batch_rk_step(chorus_batch batch, float* Q, void* workspace, double dt, int64_t n_steps,
                                   void* stream, int64_t* launches);

/* chorus_batch_rk_step on a batch state held in host memory (Q_host: host, the batch layout, pinned
 * for full copy bandwidth; Q_dev: device, caller-owned, n_state floats): each order's state is copied
 * in, stepped n_steps times and copied back, the orders pipelined (the copy in of one order and the
 * copy out of another overlap the steps of a third; the smallest state first) on copy streams of
 * the batch's own; the kernels are the per-order ones, one order after another, so the result
 * equals chorus_batch_rk_step's with the serial schedule bit for bit.  Synchronises; calls on one
 * batch must not overlap. */
chorus_status chorus_batch_rk_step_host(chorus_batch batch, float* Q_host, float* Q_dev, void* workspace, double dt,
                                        int64_t n_steps, void* stream);

/* Per-shell FP64 reductions of the total state as chorus_reduce: out host double[n_shells][4]
 * (mass, total energy, kinetic energy, |L|).  Synchronises. */
chorus_status chorus_batch_reduce(chorus_batch batch, const float* Q, double* out, void* stream);

/* Autotuner: for each order, times n_trials RK steps with every built tile shape (elements per CTA)
 * of the FP32 kernels on this batch's own meshes and keeps the fastest; then times n_trials replays
 * of the captured step with the orders on concurrent streams and with the orders one after another,
 * and n_trials persistent steps where available, keeps the fastest schedule, and drops the
 * captured graph.  Q and workspace are scratch (their
 * contents are overwritten).  choice: host int[4] receiving the chosen elements per CTA for
 * p = 2..5 (0 where the order is absent), or NULL.  Synchronises. */
chorus_status chorus_batch_autotune(chorus_batch batch, float* Q, void* workspace, double dt, int n_trials,
                                    void* stream, int* choice);

/* Schedule of the orders within a batch step: set 1 = concurrent streams, 0 = one after another,
 * 2 = one persistent launch per RK stage (CHORUS_EUNSUPPORTED without cooperative launch or with a
 * radial kappa_r(r)), any other value leaves it; concurrent: host int receiving the schedule in
 * force (0, 1 or 2), or NULL. */
chorus_status chorus_batch_schedule(chorus_batch batch, int set, int* concurrent);

/* chorus_set_wait_limit on every mesh of the batch.  The persistent schedule's grid barriers poll
 * with the same limit (0: a barrier gives up at once, sets the error flag, and the launch ends
 * without computing; chorus_batch_reduce then reports CHORUS_ETIMEOUT).  Synchronous. */
chorus_status chorus_batch_set_wait_limit(chorus_batch batch, int64_t polls);

/* Well-balanced perturbation residual (FP32_PERT only; a library option the paper has no
 * counterpart for).  The residual of Q0 + q' becomes R(Q0 + q') - R(Q0): the discrete residual of the
 * polytropic background at rest, which is not zero but of truncation size (the discretised
 * hydrostatic balance, Section 4), is left out, so the background is an exact steady state and q'
 * evolves only under its own dynamics.  Used to compare runs of different orders, whose background
 * truncation errors differ.  enable = 0 restores the plain residual.  Applies to chorus_residual and
 * chorus_rk_step / chorus_rk_step_scheme in the FP32 perturbation form. */
chorus_status chorus_set_well_balanced(chorus_mesh mesh, int enable);

/* Synchronise the stream and report a pending device-side error flag (CHORUS_ETIMEOUT) of the
 * mesh's kernels, then clear it. */
chorus_status chorus_check(chorus_mesh mesh, void* stream);

/* Limit of the bounded device-side waits with which the residual and lifting kernels of this mesh
 * wait for the bulk copies that stage each element's state, background and gradient blocks in shared
 * memory: after `polls` polls the wait gives up, the kernel sets the mesh's error flag, waits (with
 * the default limit) for its copies still in flight and returns without computing or storing
 * anything; chorus_check then reports CHORUS_ETIMEOUT.  polls < 0 restores the default (2^24 polls
 * with back-off, about a second); 0 makes every wait give up at once, so the failure path can be
 * exercised without a fault.  polls >= 2^32 - 1: CHORUS_EINVAL.  Synchronous. */
chorus_status chorus_set_wait_limit(chorus_mesh mesh, int64_t polls);

const char* chorus_strerror(chorus_status status);

#ifdef __cplusplus
}
#endif
#endif /* CHORUS_H */
