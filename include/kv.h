/*
 * kv.h -- C ABI of libkv: the B300 (sm_103a) hot path of the reduced
 * Kelvin-Voigt shear-wave method (explicit FDTD time stepping of
 * rho u_tt = mu lap(u) + eta lap(u_t) + f_S, with the body force projected
 * onto its solenoidal part by a matrix-free conjugate-gradient Poisson solve).
 *
 * Paper: "A reduced viscoelastic FDTD formulation for ultrasound-driven shear
 * wave propagation in soft tissue". Sections cited below:
 *   Sec. 2.3 reduced shear equation (Eq. shear_reduced_kv)
 *   Sec. 3.1 explicit leapfrog update, 7-point Laplacian, eta = 0 CFL bound
 *   Sec. 3.2 solenoidal projection, masked CG (recurrences, stop rule, guards)
 *   Sec. 3.3 pre-computed projection for separable forces f = b0(x) g(t)
 *   Sec. 3.5 Dirichlet outer layer, curl-based initial velocity
 *   Sec. 4   sensor traces (displacement at fixed nodes every step)
 *
 * Conventions shared by every call
 * --------------------------------
 * Grid      nx*ny*nz nodes at spacing dx on every axis, x fastest. A dense
 *           field is nx*ny*nz contiguous values at index (k*ny + j)*nx + i.
 *           The outer node layer is the Dirichlet layer (u = 0 there).
 * Precision KV_FP32: state, coefficients and force in float; every inner
 *           product and residual norm of the CG, and the potential phi, in
 *           double. KV_FP64: everything in double (a check mode).
 * Pointers  Inputs are described by kv_field: a scalar, a host pointer or a
 *           device pointer (the current CUDA device). The caller owns every
 *           pointer it passes; libkv copies what it needs into its own device
 *           memory (allocated in kv_create, freed in kv_destroy) and never
 *           keeps a caller pointer after a call returns.
 * Streams   Every call is asynchronous on the handle's stream except those
 *           documented as synchronising (kv_create, kv_set_medium,
 *           kv_project_force, kv_read_*, kv_sync). Host inputs are copied
 *           before the call returns, so the caller may reuse them. Device
 *           inputs and output buffers are accessed on the handle's stream
 *           only: the caller must have completed (or ordered before that
 *           stream) any work of its own that writes them, e.g. by creating
 *           the handle on its own stream or synchronising its stream first.
 * Errors    Every call returns a kv_status and never aborts. A CUDA error, a
 *           device-side timeout or a non-finite CG puts the handle in an
 *           error state; kv_last_error() gives a one-line description.
 *           Asynchronous CUDA errors surface on the next synchronising call.
 */
#ifndef KV_H_
#define KV_H_

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    KV_OK = 0,
    KV_ERR_ARG = 1,          /* invalid argument (size, pointer, enum) */
    KV_ERR_CUDA = 2,         /* a CUDA runtime or driver call failed */
    KV_ERR_OOM = 3,          /* device allocation failed */
    KV_ERR_UNSTABLE_DT = 4,  /* dt above the stability limit (kv_stable_dt) */
    KV_ERR_NONFINITE = 5,    /* NaN/Inf in an input or in a CG residual */
    KV_CG_BREAKDOWN = 6,     /* p.Ap non-finite or <= 0 (Sec. 3.2.3 guard) */
    KV_CG_MAXITER = 7,       /* tolerance not met within max_iter iterations */
    KV_ERR_TIMEOUT = 8,      /* a bounded device-side wait gave up */
    KV_ERR_STATE = 9,        /* call out of order or handle in an error state */
    KV_ERR_UNSUPPORTED = 10  /* option not available in this build */
} kv_status;

typedef enum { KV_FP32 = 0, KV_FP64 = 1 } kv_precision;

typedef enum { KV_SCALAR = 0, KV_HOST = 1, KV_DEVICE = 2 } kv_where;

/* Spatial operator of the shear-wave equation in a heterogeneous medium.
 * KV_OP_POINTWISE   (G/rho) L u + (eta/rho) L udot with the 7-point Laplacian L
 *                   (Sec. 3.1, Eq. of the reduced Kelvin-Voigt model).
 * KV_OP_DIVERGENCE  (1/rho) div(G grad u) + (1/rho) div(eta grad udot): the
 *                   flux form for spatially varying moduli, each of the six
 *                   face fluxes using the mean of the two nodes' moduli.
 * The two coincide in a homogeneous medium. */
typedef enum { KV_OP_POINTWISE = 0, KV_OP_DIVERGENCE = 1 } kv_operator;

/* A scalar or a dense nx*ny*nz float field on the host or the device. */
typedef struct {
    const float *data; /* dense field (KV_HOST / KV_DEVICE), else ignored */
    double value;      /* the value when where == KV_SCALAR */
    int where;         /* kv_where */
} kv_field;

/* Statistics of one projection solve (Sec. 3.2.3). */
typedef struct {
    int iters;                /* CG iterations (all refinement cycles) */
    int refinements;          /* true-residual evaluations after the first */
    int status;               /* kv_status of the solve */
    double rel_res_true;      /* ||b - A phi||_2 / ||b||_2, evaluated in FP64 */
    double rel_res_recursive; /* last recursive ||r|| / ||b|| */
    double ms;                /* wall time of the call */
} kv_cg_stats;

typedef struct kv_handle kv_handle;

/*
 * Stability limit of the explicit update (Sec. 3.1; extended to eta > 0).
 * For frozen coefficients a Laplacian mode follows
 *   c_{n+1} = (2 - (a+b) lam) c_n - (1 - b lam) c_{n-1},
 * a = dt^2 G/rho, b = dt eta/rho, lam <= 12/dx^2, which is stable iff
 * dt^2 c^2 + 2 dt nu <= dx^2/3 with c^2 = G/rho, nu = eta/rho. *dt_max gets the
 * positive root minimised over nodes; at eta = 0 it is the paper's bound
 * dt <= (1/c)(3/dx^2)^(-1/2). Synchronising. Fields as in kv_create.
 */
kv_status kv_stable_dt(int nx, int ny, int nz, double dx, kv_field G, kv_field rho,
                       kv_field eta, double *dt_max);

/* Stability limit for an operator (kv_operator). KV_OP_POINTWISE is
 * kv_stable_dt. KV_OP_DIVERGENCE bounds the spectrum of the flux operator by
 * Gershgorin's theorem: at every interior node the pointwise formula is
 * evaluated with G and eta replaced by the mean of the six face values
 * (6 G_i + sum of the six neighbours' G) / 12, and rho by the node's own rho.
 * Boundary nodes are only checked for valid values. Synchronising. */
kv_status kv_stable_dt_op(int nx, int ny, int nz, double dx, kv_field G, kv_field rho,
                          kv_field eta, int op, double *dt_max);

/*
 * Create a solver for one grid (Sec. 3.1, 3.5). G (shear modulus mu, Pa),
 * rho (kg/m^3), eta (Pa s) are scalars or dense fields; all three scalar gives
 * the homogeneous kernels. dt must not exceed kv_stable_dt (else
 * KV_ERR_UNSTABLE_DT). stream: a cudaStream_t, or NULL for a stream the
 * handle creates and owns. Allocates all device memory the handle needs
 * (state, coefficients, force, CG vectors). Synchronising.
 */
kv_status kv_create(kv_handle **out, int nx, int ny, int nz, double dx, double dt, kv_field G,
                    kv_field rho, kv_field eta, int precision, void *stream);

/* Re-fold a new medium into an existing handle (Sec. 3.1 coefficients
 * A = dt^2 G/rho, B = dt eta/rho, S = dt^2/rho). The homogeneous/heterogeneous
 * choice must match kv_create's. Synchronising (it checks dt). */
kv_status kv_set_medium(kv_handle *h, kv_field G, kv_field rho, kv_field eta);

/* Select the spatial operator (kv_operator) and fold the medium for it. The
 * handle's dt must not exceed kv_stable_dt_op for that operator (else
 * KV_ERR_UNSTABLE_DT and nothing changes). The divergence form stores three
 * coefficient fields (dt^2 G/dx^2, dt eta/dx^2, 1/rho) instead of two; the
 * two-step kernels (kv_set_step_config variants 2 to 4) support only the pointwise
 * operator (KV_ERR_UNSUPPORTED). The state and traces are kept. A kv_create
 * handle starts with KV_OP_POINTWISE. Synchronising. */
kv_status kv_set_operator(kv_handle *h, int op, kv_field G, kv_field rho, kv_field eta);

/* How the FP32 step reads a heterogeneous medium (Sec. 3.1 folded
 * coefficients: A' = dt^2 G/(rho dx^2), B' = dt eta/(rho dx^2) for the
 * pointwise operator; m = dt^2 G/dx^2, e = dt eta/dx^2, 1/rho for the flux form).
 * KV_MEDIUM_AUTO (the default): after each fold the handle counts the
 * distinct coefficient tuples on the device; if there are at most 256 (a
 * segmented medium: background and inclusions, layers), it stores one class
 * byte per node and a table of the FP32 tuples, and the TMA step kernel
 * (variant 0) reads the byte and the table instead of the FP32 fields: 49
 * instead of 56 (pointwise) or 60 (flux form) bytes per node and step, with
 * results bit for bit those of the fields. More tuples, a flux-form medium
 * where (m, e) does not fix 1/rho, FP64 handles, the other step variants and
 * batches read the fields. KV_MEDIUM_FIELDS always reads the fields.
 * The class bytes take nx_pitched * ny * nz bytes of device memory.
 * Synchronising; the state and traces are kept. KV_ERR_ARG for another value. */
typedef enum { KV_MEDIUM_AUTO = 0, KV_MEDIUM_FIELDS = 1 } kv_medium_encoding;
kv_status kv_set_medium_encoding(kv_handle *h, int encoding);
/* Number of medium classes the step reads (0: it reads the fields; -1: h is NULL). */
int kv_medium_classes(kv_handle *h);

/* Temporal envelope g(t_n), n = 0..n-1 (Sec. 3.3, Eq. separable_force); g = 0
 * beyond the table. g: float table on the host or device (where). */
kv_status kv_set_envelope(kv_handle *h, const float *g, int n, int where);

/* Sensors (Sec. 4): host array of n (i, j, k) node triples, every node inside
 * the grid. capacity: steps of trace storage ([capacity][n][3] values).
 * Resets the trace record. */
kv_status kv_set_sensors(kv_handle *h, const int *ijk, int n, int capacity);

/* Zero the displacement state, the step counter and the trace record. */
kv_status kv_reset(kv_handle *h);

/* Failure-path check (no counterpart in the paper): launches one block that
 * waits, with the bounded wait every step and CG kernel uses (about a second of
 * SM clocks), on an mbarrier that nothing completes. The wait gives up, sets
 * the device error flag, and the call returns KV_ERR_TIMEOUT with the handle in
 * the error state, exactly as a timed-out step or CG kernel would leave it.
 * Nothing faults and the CUDA context stays usable. Synchronising. */
kv_status kv_selftest_wait(kv_handle *h);

/* Checkpoint and resume (no counterpart in the paper). The state of a step is
 * the two fields u^n and d^n = u^n - u^{n-1} in the handle's own layout: six
 * component planes [6][nz][ny][px] of float (KV_FP32) or double (KV_FP64),
 * rows padded to px = nx rounded up to 32, kv_state_bytes(h) bytes in all.
 * kv_save_state copies it to buf (host or device memory, per where) and
 * returns the step index; kv_load_state copies a buffer saved from a handle of
 * the same grid and precision back and sets the step index, after which
 * kv_step continues bit for bit as the saved run did (same medium, force,
 * envelope and sensors). The outer node layer must hold zeros; the row padding
 * is never read into a result. Synchronising. */
long long kv_state_bytes(kv_handle *h);
kv_status kv_save_state(kv_handle *h, void *buf, int where, long long *step);
kv_status kv_load_state(kv_handle *h, const void *buf, int where, long long step);

/* Initial velocity v0 (Sec. 3.5 curl-based start): u^0 = 0, u^{-1} = -dt v0,
 * applied on interior nodes. Resets the step counter and traces. */
kv_status kv_set_initial_velocity(kv_handle *h, kv_field vx, kv_field vy, kv_field vz);

/*
 * Pre-computed solenoidal projection of a force pattern b0 (Sec. 3.2, 3.3):
 *   b   = -(D- . b0) on interior nodes (backward differences),
 *   A phi = b with A = -L (7-point), phi = 0 on the outer layer, by masked CG
 *         from phi = 0, stopped when ||b - A phi|| / ||b|| < tol (true residual,
 *         evaluated in FP64),
 *   f_S0 = b0 - D+ phi (forward differences) on every node,
 * and stores F = (dt^2/rho) f_S0 for the time step. fx, fy, fz: dense fields.
 * max_iter <= 0 selects 20 * max(nx, ny, nz). mode: 0 = zero initial guess,
 * 1 = learned initial guess from the net attached with kv_attach_net, scaled
 * by the minimal-residual factor alpha = (A phi0).b / |A phi0|^2 (its residual
 * is never larger than the zero start's; the stopping rule is the same);
 * 3 = start from the potential of the previous projection on this handle
 * (zero if there is none); 4 = zero start, CG preconditioned by one symmetric
 * multigrid V(1,1)-cycle (damped Jacobi smoothing, trilinear prolongation,
 * its transpose as restriction; not in the paper: the same system and the
 * same stopping rule, far fewer iterations; FP32 handles only, and the first
 * mode-4 call allocates the level arrays, about 2.3 floats per node);
 * 5 = the learned initial guess of mode 1, then the preconditioned CG of
 * mode 4; 2 = flexible CG with the attached net as preconditioner (z = Net(r)
 * each iteration, Polak-Ribiere beta; FP64 vectors, allocated on the first
 * mode-2 call, 5 doubles per node; not in the paper: same system and stopping
 * rule, checked on the true residual); modes 1, 2 and 5 without an attached
 * net that fits the grid: KV_ERR_STATE; other values KV_ERR_UNSUPPORTED.
 * fs_out: NULL, or a device
 * pointer to 3*nx*ny*nz floats (component-major) that receives f_S0.
 * stats: NULL or filled. Returns KV_OK, KV_CG_MAXITER, KV_CG_BREAKDOWN or
 * KV_ERR_NONFINITE (the stats say which). A zero right-hand side gives
 * phi = 0, f_S0 = b0 and 0 iterations. Synchronising.
 */
kv_status kv_project_force(kv_handle *h, kv_field fx, kv_field fy, kv_field fz, double tol,
                           int max_iter, int mode, float *fs_out, kv_cg_stats *stats);

/*
 * The projection of kv_project_force without any device allocation. The paper
 * has no counterpart: this entry point exists for callers that cannot call
 * cudaMalloc or cudaFree -- code whose device memory is owned by another
 * allocator (a framework's caching allocator that has already reserved the
 * pool, or a fixed memory budget) and code on a latency-critical stream that
 * cannot afford the device-wide synchronisation cudaFree implies. No handle is
 * needed. fx, fy, fz: device pointers to dense nx*ny*nz float fields. fs_out:
 * device pointer to 3*nx*ny*nz floats (component-major) that receives
 * f_S0 = b0 - D+ phi, as kv_project_force's fs_out does (FP32 vectors, FP64
 * reductions, same stopping rule). tol, max_iter and stats as in
 * kv_project_force. stream: a cudaStream_t or NULL (the legacy default stream).
 *
 * The working set lives in one static device array of about 11 MB that every
 * GPU which loads libkv holds until the process exits. Limit: rows are padded
 * to a multiple of 32 nodes and the padded grid ((nx rounded up to 32) * ny * nz)
 * may have at most 262144 nodes (64^3 fits); larger grids are rejected with
 * KV_ERR_ARG and a message in kv_last_error(NULL). The first call on a device
 * looks up the array's device address (cudaGetSymbolAddress), so make that
 * first call before any stream capture. Every call shares the array and it
 * keeps the last call's contents: each call clears what must start at zero,
 * and calls that overlap on the GPU (other streams, other host threads) race
 * on it. Errors are reported in kv_last_error(NULL). Synchronising.
 */
kv_status kv_project_force_noalloc(int nx, int ny, int nz, double dx, const float *fx,
                                   const float *fy, const float *fz, double tol, int max_iter,
                                   float *fs_out, kv_cg_stats *stats, void *stream);

/*
 * One application of the preconditioner of projection modes 4 and 5: z = M r
 * with M the symmetric multigrid V(1,1)-cycle for A = -L (the 7-point
 * Laplacian of Sec. 3.2.3 with phi = 0 on the outer layer) on the handle's
 * grid: damped Jacobi smoothing (omega = 6/7), cell-centred coarsening of the
 * interior nodes (coarse cell I covers fine cells 2I-1 and 2I), trilinear
 * prolongation P, restriction P^T / 8, 32 damped Jacobi sweeps on the
 * coarsest level (at most 4096 cells with the ghost layer); a grid too small
 * to coarsen gets M = omega dx^2 / 6 (diagonal scaling). The paper has no
 * counterpart (its CG is unpreconditioned); this entry point exposes the
 * operator the mode-4 CG applies every iteration, for checks and reuse.
 * nx, ny, nz: the handle's grid (KV_ERR_ARG if they differ). r, z: device
 * pointers to dense nz*ny*nx floats (x fastest), the caller's; only r's
 * interior nodes are read, z is written on every node (0 on the outer layer).
 * rz: NULL or receives r.z over the interior (FP64 sum of float-float
 * partials; 0 when r is 0). FP32 handles only (KV_ERR_UNSUPPORTED otherwise);
 * the first call allocates the level arrays (as the first mode-4 projection
 * does). Uses the handle's CG scratch and control block, so it must not run
 * while a projection of the same handle is in flight. Synchronising.
 */
kv_status kv_apply_preconditioner(kv_handle *h, int nx, int ny, int nz, const float *r, float *z,
                                  double *rz);

/*
 * Learned warm start of the projection. A small 3D U-Net (BF16 tensor-core
 * convolutions with FP32 accumulation, trained on the GPU by these calls)
 * maps the Poisson right-hand side b = -(D- . f) to an approximation of phi;
 * kv_project_force(mode = 1) on a handle with an attached net starts the CG
 * from that phi and stops on the same true residual as the zero start, so
 * the result meets the same tolerance whatever the net predicts.
 * Architecture: `levels` resolution levels with channels[l] in {16, 32, 64};
 * per level two 3x3x3 conv + ReLU, 2x average pooling down, nearest 2x
 * upsampling + conv + ReLU + skip addition + conv + ReLU up, a final conv.
 * The input is b scaled to unit RMS; the target phi * s / dx^2 with the same
 * scale s; the loss (Adam on FP32 master weights) is chosen by kv_net_set_loss:
 * KV_LOSS_MSE (default), the mean squared error of the potential, or
 * KV_LOSS_RESIDUAL, the mean squared residual of the prediction,
 * |L^(y - t)|^2 / V with L^ the unscaled 7-point Laplacian on interior nodes,
 * i.e. |s (b - A phi_hat)|^2 / V (Sec. 3.2.3: A phi = b is what the CG solves;
 * this loss weights the error as the CG's stopping test does). Neither is in
 * the paper, whose projection has no learned part.
 * kv_net_create allocates activations for grids up to max_n* (each axis);
 * b, phi: dense nx*ny*nz float device arrays. stream: cudaStream_t or NULL.
 * kv_net_get/set_params: kv_net_num_params floats on the host.
 * kv_attach_net: use net for mode 1 of h (NULL detaches; the net must
 * outlive its use). Errors are reported in kv_last_error(NULL).
 */
typedef struct kv_net kv_net;
kv_status kv_net_create(kv_net **out, int levels, const int *channels, int max_nx, int max_ny,
                        int max_nz, void *stream);
kv_status kv_net_destroy(kv_net *n);
long long kv_net_num_params(kv_net *n);
kv_status kv_net_init(kv_net *n, unsigned long long seed);
enum { KV_LOSS_MSE = 0, KV_LOSS_RESIDUAL = 1 };
kv_status kv_net_set_loss(kv_net *n, int kind);
kv_status kv_net_get_params(kv_net *n, float *host);
kv_status kv_net_set_params(kv_net *n, const float *host);
kv_status kv_net_train_step(kv_net *n, int nx, int ny, int nz, double dx, const float *b,
                            const float *phi, double lr, double *loss);
kv_status kv_net_predict(kv_net *n, int nx, int ny, int nz, double dx, const float *b, float *phi);
kv_status kv_attach_net(kv_handle *h, kv_net *net);

/*
 * Layer operations of the net (exposed for tests): channel-last BF16 tensors
 * [nz][ny][nx][C], C in {16, 32, 64}; W[t][ci][co] BF16 with tap
 * t = (dz+1)*9 + (dy+1)*3 + (dx+1), zero padding of one voxel.
 *   kv_nn_conv3d_fwd: out = bias + conv(x, W) (ReLU if relu), BF16 or FP32 out.
 *   kv_nn_conv3d_flip: Wt[t][co][ci] = W[26-t][ci][co] (input gradient =
 *     kv_nn_conv3d_fwd of the output gradient with Wt, cin/cout swapped).
 *   kv_nn_conv3d_bwd_weight: gW[t][ci][co] += sum_v x[v+d(t)][ci] g[v][co],
 *     gb[co] += sum_v g[v][co] (FP32, accumulating with atomics, so the sum
 *     order and the last bits vary from call to call; gb may be NULL).
 * x, g, W and gW are device pointers, 16-byte aligned (KV_ERR_ARG otherwise);
 * the calls are asynchronous on `stream`.
 */
kv_status kv_nn_conv3d_fwd(int nx, int ny, int nz, int cin, int cout, const void *x, const void *W,
                           const float *bias, void *out, int out_f32, int relu, void *stream);
kv_status kv_nn_conv3d_flip(int cin, int cout, const void *W, void *Wt, void *stream);
kv_status kv_nn_conv3d_bwd_weight(int nx, int ny, int nz, int cin, int cout, const void *x,
                                  const void *g, float *gW, float *gb, void *stream);

/* Drop the projected force (the step then runs unforced). */
kv_status kv_clear_force(kv_handle *h);

/*
 * Advance n time steps (Sec. 3.1 with Sec. 3.3's f_S^n = g(t_n) f_S0):
 *   u^{n+1} = 2u^n - u^{n-1} + dt^2 [ (G/rho) L u^n + (eta/rho) L (u^n-u^{n-1})/dt
 *                                     + g(t_n) f_S0 / rho ]
 * on interior nodes, computed in the equivalent increment form
 *   d^{n+1} = d^n + A' L^ u^n + B' L^ d^n + g_n F,  u^{n+1} = u^n + d^{n+1},
 * d = u^n - u^{n-1}, L^ the unscaled 7-point stencil, A' = A/dx^2, B' = B/dx^2.
 * After each step the sensors record u^{n+1}. Asynchronous.
 */
kv_status kv_step(kv_handle *h, int n);

/*
 * General per-step projection (Sec. 3.2: a different body force at each time
 * step, each projected on its own): project this step's force f^n (fields as
 * in kv_project_force; mode 0: the CG starts from zero, as the paper's general
 * solver; mode 3: from the previous step's potential; mode 4: from zero,
 * preconditioned by the multigrid V-cycle (FP32 only); all stop on tol), then
 * advance one step with f_S^n (envelope 1 for this step). The projected force
 * stays stored afterwards. stats: NULL or the projection's statistics.
 * Synchronising.
 */
kv_status kv_step_force(kv_handle *h, kv_field fx, kv_field fy, kv_field fz, double tol, int max_iter,
                        int mode, kv_cg_stats *stats);

/* Steps taken since the last reset (host-side count). */
long long kv_steps_taken(kv_handle *h);

/* Copy the trace record [n_written][n_sensors][3] (float for KV_FP32, double
 * for KV_FP64) to out (host or device per where). *n_written = steps recorded
 * (at most the capacity). Synchronising. */
kv_status kv_read_traces(kv_handle *h, void *out, int where, int *n_written);

/*
 * Copy one dense field out (element type as for traces; phi always double):
 *   which 0: u^n component comp     which 1: d^n = u^n - u^{n-1}, component comp
 *   which 2: phi (comp ignored)     which 3: F = dt^2 f_S0 / rho, component comp
 *   which 4: b = -(D- . f) of the last projection (double, comp ignored)
 * out: nx*ny*nz elements on the host or device (where). Synchronising.
 */
kv_status kv_read_field(kv_handle *h, int which, int comp, void *out, int where);

/* Wait for all work on the handle's stream; report device-side errors. */
kv_status kv_sync(kv_handle *h);

/* Kernel selection and launch shape of the FP32 step (autotuning and tests).
 * variant 0: TMA-staged z-march kernel (default); 1: plain per-node kernel;
 * 2: two steps per z sweep (temporal blocking, pointwise operator only;
 * tiles 32x4, 32x8, 64x4, 64x8, 128x4 with ns in {4, 6});
 * 3: two steps per z sweep with one displacement component per block (the
 * pointwise operator couples the components only through the shared
 * coefficients; pointwise operator only; tiles 32x8, 32x16, 64x4, 64x8,
 * 64x16, 128x4, 128x8 with ns in {4, 6});
 * 4: as 3 with a tx x 14 tile whose intermediate step takes one group of four
 * nodes per thread plus one warp for the two halo columns (tx in {32, 64, 128},
 * ty = 14, ns in {2, 3, 4, 6}; with 2 stages the copy of plane k + 3 is
 * issued once plane k + 1 is consumed and three 64 x 14 blocks share an SM).
 * Variants 2 to 4 read the coefficient fields,
 * never class bytes, and give bit for bit the result of two single steps.
 * Variants 0 and 1: tx in {32, 64, 128}, ty in {2, 4, 8, 16} with tx*ty/4 in
 * [64, 512]; zc >= 1 planes per block; ns in {4, 6, 8} shared-memory stages
 * (ns - 3 planes in flight per block). Values <= 0 keep the current choice. A shape
 * whose stages exceed the shared memory of a block is refused (KV_ERR_ARG)
 * and the previous configuration is kept. */
kv_status kv_set_step_config(kv_handle *h, int variant, int tx, int ty, int zc, int ns);

/* Current step configuration: cfg[5] = {variant, tx, ty, zc, ns}. */
kv_status kv_get_step_config(kv_handle *h, int *cfg);

/* Autotuner of the FP32 step: times trial_steps steps of every supported
 * (variant, tile, stage count, z chunk; z chunks 16, 32, 64, and for variant 4
 * 32, 64, 128 and a third, a half and all of the interior depth, 3 stages) on this
 * handle's grid with CUDA events
 * on its stream, times the four fastest (and the fastest one-step candidate)
 * again over 4 x trial_steps steps and keeps the fastest of those, a two-step
 * variant only if it is more than 3 % faster than the best one-step kernel,
 * then resets the state (kv_reset). *best_ms:
 * mean milliseconds per step of the choice (NULL allowed). Synchronising. */
kv_status kv_autotune_step(kv_handle *h, int trial_steps, double *best_ms);

/* Launch shape of the FP32 CG passes (Sec. 3.2.3 iteration): zc planes per
 * block of the TMA z-march (0: the default, about one wave of blocks:
 * 148 x 4 blocks of 64 x 8 columns over the grid, between 8 and 128 planes). A value giving more blocks than
 * the handle's reduction buffer holds is refused (KV_ERR_ARG). The arithmetic
 * and its order do not depend on zc except through the order of the block
 * partial sums. kv_get_cg_config: the current zc. */
kv_status kv_set_cg_config(kv_handle *h, int zc);
kv_status kv_get_cg_config(kv_handle *h, int *zc);

/* Autotuner of the FP32 CG passes: runs the projection of (fx, fy, fz) for
 * iters iterations (twice) with each z chunk in {8, 16, 24, 32, 48, 64, 96,
 * 128} that fits the grid and each shared-memory stage count of the passes
 * (8 or 4 planes per block's ring), keeps the fastest and reports its wall time in
 * *best_ms (NULL allowed). The trial projections stop early, so the force
 * must be projected again (kv_project_force) before stepping. No-op for
 * FP64 handles. Synchronising. */
kv_status kv_autotune_cg(kv_handle *h, kv_field fx, kv_field fy, kv_field fz, int iters,
                         double *best_ms);

/* Number of kernel launches libkv has issued on this handle. */
long long kv_launch_count(kv_handle *h);

kv_status kv_destroy(kv_handle *h);

/*
 * Batched time stepping (parameter sweeps, Sec. 3.1 applied to many media at
 * once). A batch refers to n existing FP32 handles -- all homogeneous, all
 * heterogeneous with the pointwise operator or all with the divergence-form
 * operator, all created on the same stream -- of any grid sizes. Each
 * kv_batch_step(b, n) advances every case by n steps with one kernel launch
 * per step covering the tile grids of all cases (blocks of 32 steps replay
 * from a CUDA graph); each case keeps its own state, coefficients, envelope,
 * sensors, traces and step count, readable through its handle as usual. The
 * cases must be at the same step parity (e.g. all freshly reset). The batch
 * holds a device table of its cases (allocated in kv_batch_create, freed in
 * kv_batch_destroy) and rebuilds it when a case's parameters change.
 * kv_batch_set_config: tile (tx, ty), z chunk zc and stage count ns as in
 * kv_set_step_config. kv_batch_autotune: times every supported configuration
 * over trial_steps and keeps the fastest, then resets every case.
 * kv_batch_get_config: cfg[4] = {tx, ty, zc, ns}. The handles must outlive the
 * batch. Errors are reported in kv_last_error(NULL).
 */
typedef struct kv_batch kv_batch;
kv_status kv_batch_create(kv_batch **out, int n, kv_handle *const *cases);
kv_status kv_batch_set_config(kv_batch *b, int tx, int ty, int zc, int ns);
kv_status kv_batch_get_config(kv_batch *b, int *cfg);
kv_status kv_batch_autotune(kv_batch *b, int trial_steps, double *best_ms);
kv_status kv_batch_step(kv_batch *b, int n);
long long kv_batch_launch_count(kv_batch *b);
kv_status kv_batch_destroy(kv_batch *b);

/*
 * Reuse one projection for another handle on the same grid (Sec. 3.3: the
 * solenoidal projection depends on the force pattern only, not on the medium):
 * dst's projected force becomes (dt_dst^2/rho_dst) f_S0 with f_S0 taken from
 * src's stored F = (dt_src^2/rho_src) f_S0. Both FP32, same nx, ny, nz;
 * src must hold a projected force. Synchronising.
 */
kv_status kv_share_force(kv_handle *dst, kv_handle *src);

/* One-line description of the last error on h (or of the last failed
 * kv_create when h is NULL). Never NULL. */
const char *kv_last_error(kv_handle *h);

/* Name of a status code. */
const char *kv_status_string(int status);

#ifdef __cplusplus
}
#endif

#endif /* KV_H_ */
