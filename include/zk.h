/*
 * zk.h - C ABI of the B300 Zakharov / HOS wave step.
 *
 * The library advances the canonical Zakharov pair (eta, psi) of
 * "Hamiltonian Two-Way Coupling of Nonlinear Waves and 3D Flows"
 * (Sec. 3.1, Eqs. 4-5) on a doubly periodic grid over finite depth h. The
 * Dirichlet-Neumann operator G(eta) is the order-M truncated series of
 * Sec. 3.2 (Eq. 9; M = number of retained terms G_0 .. G_{M-1}, so the
 * paper's HOS-3 is M = 3), evaluated with the 3/2-rule de-aliasing and the
 * super-Gaussian taper of Sec. 6.1, the nonlinear Bernoulli term of
 * Eqs. 10-11, the state filter of Eq. 17, and classical RK4 or the
 * integrating-factor AB2 of Sec. 3.4 (Eqs. 15-16) as time integrator.
 *
 * Conventions shared by every entry point
 *  - Physical arrays are row-major [nz][nx], x fastest, element (iz, ix) at
 *    x = ix * Lx/nx, z = iz * Lz/nz. Their element type is given by a dtype
 *    argument (ZK_F32 or ZK_F64), independent of the context's compute
 *    precision; on_device = 1 means the pointer is device memory of the
 *    context's current device, 0 means host memory (pageable or pinned).
 *  - The caller owns every buffer it passes; the library copies inputs in and
 *    results out and keeps no pointer after the call returns.
 *  - The context owns all device memory it uses (allocated in zk_create,
 *    freed in zk_destroy) and launches on the stream given in zk_options
 *    (NULL = the legacy default stream).
 *  - Functions return a zk_status and never abort. A CUDA error seen during a
 *    call is returned as ZK_ECUDA; an asynchronous device error is reported
 *    by the next call that synchronises (zk_sync, zk_get_state, zk_energy).
 *  - A context is used by one host thread at a time.
 */
#ifndef ZK_H
#define ZK_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct zk_ctx zk_ctx;

typedef enum {
    ZK_OK = 0,
    ZK_EINVAL = 1,        /* bad argument (size, pointer, dtype, option value) */
    ZK_ENOMEM = 2,        /* device or host allocation failed */
    ZK_ECUDA = 3,         /* a CUDA runtime call or kernel launch failed */
    ZK_ENONFINITE = 4,    /* the state holds NaN or Inf (checked by zk_energy) */
    ZK_ETIMEOUT = 5,      /* a bounded device-side wait ran out */
    ZK_EUNSUPPORTED = 6,  /* valid request this build does not implement */
    ZK_ESTATE = 7         /* call out of order (e.g. step before set_state) */
} zk_status;

enum { ZK_F32 = 0, ZK_F64 = 1 };               /* element types of I/O arrays and of the compute path */
enum { ZK_RK4 = 0, ZK_IFRK4 = 1, ZK_IFAB2 = 2 };   /* time integrators */

typedef struct {
    double eps;        /* nonlinear-amplitude parameter of Eqs. 9-11, in [0, 1]; default 1 */
    int integrator;    /* ZK_RK4 (default), ZK_IFRK4 (RK4 on the rotation of Eq. 14) or ZK_IFAB2 (Sec. 3.4, Eqs. 15-16) */
    int taper;         /* 1 (default): taper exp[-(|k|/kc)^8] on nonlinear products (Sec. 6.1) */
    int filter;        /* 1 (default): state filter A(k) of Eq. 17 once per step */
    void *stream;      /* cudaStream_t for all launches; NULL = legacy default stream */
} zk_options;

/* Create a context for an nx x nz grid of extent Lx x Lz over depth h, gravity g,
 * with M retained DNO terms (1 <= M <= ZK_MAX_ORDER) and compute precision
 * ZK_F32 or ZK_F64. nx, nz: powers of two in [16, 2048] (FP64: [16, 1024]).
 * Allocates all device buffers on the current device. Options start at their
 * defaults. Errors: ZK_EINVAL (sizes, M, precision, non-positive lengths),
 * ZK_ENOMEM, ZK_ECUDA. *out is NULL on error. */
#define ZK_MAX_ORDER 8
zk_status zk_create(zk_ctx **out, int nx, int nz, double Lx, double Lz,
                    double h, double g, int M, int precision);

/* zk_create with a choice of padded grid for the nonlinear products:
 * ZK_PAD_3_2 is the 3/2 rule of Sec. 6.1 (what zk_create uses): exact for
 * quadratic products only. ZK_PAD_3 pads to 3 nx x 3 nz, which makes every
 * product of up to five band-limited factors exact - all products of the
 * order-M series for M <= 5 - the de-aliasing fitted to the higher-order terms
 * that Sec. 9 lists as future work (the Bernoulli term, a quotient, stays
 * approximate). ZK_PAD_3 costs about 4x the transform work and needs FP32
 * and nx, nz <= 1024 (ZK_EUNSUPPORTED otherwise; series sums stay FP32).
 * Other values of pad: ZK_EINVAL. */
#define ZK_PAD_3_2 0
#define ZK_PAD_3 1
zk_status zk_create_ex(zk_ctx **out, int nx, int nz, double Lx, double Lz,
                       double h, double g, int M, int precision, int pad);

/* Release every device buffer and the context (NULL is accepted). */
void zk_destroy(zk_ctx *ctx);

/* Replace the options (copied). ZK_EINVAL if eps is outside [0, 1] or a flag is unknown. */
zk_status zk_set_options(zk_ctx *ctx, const zk_options *opt);
zk_status zk_get_options(const zk_ctx *ctx, zk_options *opt);

/* Load the state from physical eta, psi [nz][nx]. The library forms their
 * spectra and sets the Nyquist mode of each axis to zero (the paper does not
 * say; this is the reading every spectral operator here uses). Resets the
 * integrator history (the next IF-AB2 step bootstraps with IF-Euler). */
zk_status zk_set_state(zk_ctx *ctx, const void *eta, const void *psi, int dtype, int on_device);

/* Copy the current state out as physical eta, psi [nz][nx]. Synchronises. */
zk_status zk_get_state(zk_ctx *ctx, void *eta, void *psi, int dtype, int on_device);

/* Asynchronous state I/O with pinned host buffers (same layouts as
 * zk_set_state / zk_get_state, host pointers only). The copies run on two copy
 * streams of the context (uploads, downloads) through two staging slots per
 * direction, so the
 * upload of the next state and the download of the last one overlap the
 * context's kernels on its stream; neither call waits. zk_set_state_async:
 * the host arrays must stay unchanged until the upload is done (zk_sync).
 * zk_get_state_async: the host arrays hold the state as of the call once
 * zk_sync has returned. zk_io_join makes the context's stream wait for every
 * copy issued so far (no host wait), e.g. before recording a timing event.
 * Host memory that is not page-locked makes the copies synchronous. Errors as
 * for zk_set_state / zk_get_state; the first call allocates the staging slots. */
zk_status zk_set_state_async(zk_ctx *ctx, const void *eta, const void *psi, int dtype);
zk_status zk_get_state_async(zk_ctx *ctx, void *eta, void *psi, int dtype);
zk_status zk_io_join(zk_ctx *ctx);

/* Checkpoint and resume of a single context (library addition; the paper's
 * integrator, Sec. 3.4, Eqs. 15-16, carries the previous step's nonlinear forcing
 * F_{n-1}, so resuming from the state alone would restart with an IF-Euler step).
 * A checkpoint holds the compact state spectra eta_hat, psi_hat and the IF-AB2
 * history (F_{n-1} of both equations, the dt it was taken at, whether it is
 * valid) plus the order the context steps at, in the context's precision.
 * zk_checkpoint_size: bytes of a checkpoint of this context (header included).
 * zk_checkpoint_save: waits for the context's stream, then copies the checkpoint
 *   to host memory `buf` (caller-owned, at least zk_checkpoint_size bytes).
 * zk_checkpoint_load: restores a checkpoint into a context created with the same
 *   grid, order, precision and padding (the header is checked: ZK_EINVAL on a
 *   mismatch or a short buffer; ZK_ESTATE if `buf` holds no state). Options are
 *   not part of the checkpoint. After a load, stepping continues bitwise
 *   identically to the uninterrupted run. */
zk_status zk_checkpoint_size(const zk_ctx *ctx, size_t *bytes);
zk_status zk_checkpoint_save(zk_ctx *ctx, void *buf, size_t bytes);
zk_status zk_checkpoint_load(zk_ctx *ctx, const void *buf, size_t bytes);

/* Right-hand side of Eqs. 4 and 10 at the current state, as physical fields
 * [nz][nx]: d eta/dt = G(eta) psi (mean set to zero), d psi/dt. Synchronises. */
zk_status zk_rhs(zk_ctx *ctx, void *deta_dt, void *dpsi_dt, int dtype, int on_device);

/* Forward DNO map of Eq. 18, v = G(eta) psi with M terms, physical [nz][nx]
 * (mean set to zero). Synchronises. */
zk_status zk_dno(zk_ctx *ctx, void *v, int dtype, int on_device);

/* Reflecting walls by even extension (Sec. 3.3, Eq. 12). The context's grid
 * (nx, nz, Lx, Lz) is the doubled computational grid; the caller's arrays are
 * the tank of (nx/2) x (nz/2) cell-centred samples over Lx/2 x Lz/2. set mirrors
 * the tank across each wall (sample i -> 2m-1-i) into the doubled periodic
 * field; the even symmetry is kept by every step (all operators commute with
 * the reflection), so get returns the (0:nz/2, 0:nx/2) corner. set resets the
 * integrator history like zk_set_state; get synchronises. */
zk_status zk_set_state_tank(zk_ctx *ctx, const void *eta, const void *psi, int dtype, int on_device);
zk_status zk_get_state_tank(zk_ctx *ctx, void *eta, void *psi, int dtype, int on_device);

/* Inverse DNO map of Eq. 19 (Sec. 3.5): replace psi so that G(eta) psi = v at
 * the current eta, for physical v [nz][nx]. psi(0) = G0^{-1} v, then `iters`
 * fixed-point updates psi <- G0^{-1}(v - [G(eta) - G0] psi) (the paper uses 8);
 * the k = 0 mode of psi (its mean, which G0 does not see) keeps its value.
 * Used to start from a physically specified (eta, v) pair. Synchronises. */
zk_status zk_dno_inverse(zk_ctx *ctx, const void *v, int dtype, int on_device, int iters);

/* Relaxation source of Sec. 5 after a wave step (Alg. 2 steps 7-9): keep
 * v = G(eta) psi of the current state, relax eta pointwise toward eta_target
 * with rate sigma [nz][nx] (1/s) by the exact decay of Eq. 34,
 * eta <- eta_t + (eta - eta_t) exp(-sigma dt), then recompute psi from the
 * relaxed eta and v by the inverse map (Eq. 35 via Eq. 19, `iters` updates).
 * sigma >= 0 and eta_target are physical arrays of the given dtype (a box
 * footprint ramp as in Eq. 33 is the caller's choice). The IF-AB2 history is
 * kept, as in the paper's substep loop. Synchronises. */
zk_status zk_relax(zk_ctx *ctx, const void *sigma, const void *eta_target, int dtype, int on_device,
                   double dt, int iters);

/* Advance n steps of size dt with the selected integrator (each followed by
 * the state filter when enabled). Asynchronous on the context's stream; the
 * launch sequence of one step is captured once in a CUDA graph and replayed.
 * ZK_RK4 evaluates the right-hand side four times per step. ZK_IFAB2 (Sec. 3.4)
 * evaluates it once: the linear part is rotated exactly per mode (Eq. 14) and
 * the nonlinear forcing enters through Eqs. 15-16 with F* = 3/2 F_n - 1/2 F_{n-1};
 * the first step after zk_set_state, after an option change, or with a dt
 * different from the previous step's uses F* = F_n (IF-Euler bootstrap).
 * ZK_IFRK4 evaluates it four times: integrating-factor RK4 in Lawson's form,
 * the linear rotation of Eq. 14 applied exactly over h/2 and h, classical RK4
 * stages on the nonlinear part in the rotating frame (fourth order, exact
 * linear dispersion; needs no history).
 * ZK_ESTATE before zk_set_state. */
zk_status zk_step(zk_ctx *ctx, double dt, int n);

/* Hamiltonian of Eq. 1 by Parseval, reduced in FP64 on the device in a fixed
 * order: H = kin + pot, kin = 1/2 int psi G(eta) psi, pot = 1/2 g int eta^2,
 * mean_eta = spatial mean of eta. Any pointer may be NULL. Synchronises.
 * ZK_ENONFINITE if the state holds NaN/Inf. */
zk_status zk_energy(zk_ctx *ctx, double *H, double *kin, double *pot, double *mean_eta);

/* Wait for all work of the context; returns a pending asynchronous error. */
zk_status zk_sync(zk_ctx *ctx);

/* Bytes of device memory the context holds. */
zk_status zk_device_bytes(const zk_ctx *ctx, size_t *bytes);

/* Number of kernel launches one zk_step(dt, 1) issues. */
zk_status zk_launches_per_step(const zk_ctx *ctx, int *n);

/* Kernel classes reported by zk_profile_step. */
enum { ZK_K_COL_STATE = 0, ZK_K_ROW_ROUND = 1, ZK_K_COL_PHI = 2, ZK_K_ROW_FINAL = 3, ZK_K_COL_FINAL = 4 };

/* Run nsteps steps of size dt eagerly (no graph) with a CUDA event recorded
 * on the context's stream before every launch and after the last one, and
 * add each launch's device time in milliseconds to ms[slot] (slot = launch
 * index within one step, in launch order; ms must hold *nslots entries, at
 * most cap). For every slot, kind[slot] is its kernel class and
 * bytes[slot] the algorithmic global-memory bytes it must move (each input
 * field read once, each output written once); kind and bytes may be NULL.
 * The state advances exactly as with zk_step. Synchronises. */
zk_status zk_profile_step(zk_ctx *ctx, double dt, int nsteps, double *ms, int *kind, double *bytes,
                          int cap, int *nslots);

/* ---- Allocation-free DNO (the paper has no counterpart; library addition) ----
 *
 * zk_dno_static computes the same v = G(eta) psi as zk_dno, but without a
 * context and without allocating device memory, for callers that cannot
 * call cudaMalloc: code embedded in a host application that owns the device
 * memory pool (a raw cudaMalloc bypasses the pool's accounting or fails once
 * the pool has reserved the memory), and loops with latency limits that
 * forbid allocation after start-up (cudaMalloc may synchronise the device).
 *
 * All intermediates live in one fixed device array of ZK_STATIC_SCRATCH_BYTES
 * inside the library, which every GPU that loads the library holds until the
 * process exits. eta, psi (inputs) and v (output) are device pointers to
 * FP32 [nz][nx] arrays owned by the caller. nx, nz: powers of two in
 * [16, 256]; 1 <= M <= ZK_MAX_ORDER; eps in [0, 1]; taper 0/1. Sizes whose
 * intermediates would not fit the array (256 x 256 with M = 8) are rejected
 * with ZK_EINVAL before any GPU work; 256 x 256 fits up to M = 7 and 128 x 128
 * every M. The work is queued on `stream` (cudaStream_t, NULL = legacy default)
 * and the call returns without waiting; synchronise before reading v.
 * The first call in each CUDA context (per device, and again after a
 * cudaDeviceReset) looks up the array's device address in that context, which
 * may load the library's device code; make that first call before any stream
 * capture. Every call on a device shares the array and overwrites what it
 * needs, so calls whose GPU work overlaps (other streams or host threads on
 * the same device) race and must be serialised by the caller. */
#define ZK_STATIC_SCRATCH_BYTES (16u * 1024u * 1024u)
zk_status zk_dno_static(const float *eta, const float *psi, float *v, int nx, int nz,
                        double Lx, double Lz, double h, double g, int M, double eps, int taper,
                        void *stream);

/* Precision form for FP32 contexts: with on = 1 the series sums of the
 * right-hand side run in FP64 - the Taylor sums in eta inside each order's W(m)
 * and Phi(m) (Sec. 4.2 recursion), the accumulation of sum_m eps^m G_m over the
 * orders (Eq. 9) and the assembly of G_nl, W and N_psi (Eqs. 10-11) - while the
 * transforms and the stored fields stay FP32. on = 0 restores the FP32 sums.
 * FP64 contexts ignore the call (ZK_OK). ZK_EINVAL for other values of on. */
zk_status zk_set_series_fp64(zk_ctx *ctx, int on);

/* Split-precision DFT-GEMM stages (the precision form of the padded
 * transforms; the paper computes in FP32 on the GPU, Sec. 4.3, and names mixed-precision
 * FFT pipelines as future work, Sec. 9). mode ZK_DFT_F32 (default): every
 * stage of the padded line transforms is an FP32 butterfly. ZK_DFT_BF16X3 /
 * ZK_DFT_FP16X3: the innermost radix-8 stage of every padded row and column
 * transform of the right-hand side is a matrix product with the length-8 DFT
 * matrix (as the real 16 x 16 matrix [[Fr, -Fi], [Fi, Fr]]) on the tensor
 * cores, each FP32 operand split into a 16-bit high and low part (BF16, or
 * FP16 with a power-of-two scale per 8-point block) and three products
 * summed in FP32. The other stages, the
 * unpadded state transforms and all pointwise arithmetic stay FP32. Needs an
 * FP32 context with the 3/2 rule, FP32 series sums and padded lengths 1536 or
 * 3072 on both axes (nx, nz in {1024, 2048}), else ZK_EUNSUPPORTED;
 * ZK_EINVAL for other modes. While a split mode is set, zk_set_series_fp64(1)
 * returns ZK_EUNSUPPORTED. */
enum { ZK_DFT_F32 = 0, ZK_DFT_BF16X3 = 1, ZK_DFT_FP16X3 = 2 };
zk_status zk_set_dft_precision(zk_ctx *ctx, int mode);

/* Adaptive order (the adaptive-order scheme Sec. 9 lists as future work, in
 * its global form): the context keeps its order M as the maximum. Every
 * check_every steps, before the step, it evaluates the order-M right-hand side
 * f_M at the current state and then f_m for m = m_min, m_min + 1, ... and
 * steps at the first m with |f_m - f_M| <= tol |f_M| (L2 over both spectra,
 * FP64 sums), or at M if none qualifies. zk_rhs, zk_dno and zk_energy use the
 * chosen order too; a change of order restarts the IF-AB2 history (IF-Euler). Checks synchronise the stream and cost up to
 * M - m_min + 1 right-hand sides. check_every = 0 switches it off (order M
 * again). ZK_EINVAL for m_min outside [1, M] or tol < 0; ZK_EUNSUPPORTED while
 * a closure is attached. */
zk_status zk_set_adaptive_order(zk_ctx *ctx, int m_min, double tol, int check_every);
/* order: the order in use; checks made; err[m-1] (ZK_MAX_ORDER entries): the
 * relative difference measured for order m at the last check (0 for M, -1 when
 * not evaluated). */
zk_status zk_adaptive_status(const zk_ctx *ctx, int *order, int *checks, double *err);

/* ---- Batched tiles (many independent seas advanced together) ----
 *
 * A batch holds ntiles independent periodic tiles; tile t has grid
 * nx[t] x nz[t] over Lx[t] x Lz[t], depth h[t] and order M[t] (limits as in
 * zk_create), all with gravity g and one precision. Each tile is the same
 * problem as a zk_ctx of its own (Sec. 3.2 right-hand side, Sec. 3.4 or RK4
 * integration, Eq. 17 filter); the batch only changes how launches are made.
 * Tiles with equal (nx, nz, Lx, Lz, M) form a group whose buffers are laid
 * out tile after tile, and every pass of a group is one launch over all its
 * tiles; zk_batch_step replays one captured graph in which the groups are
 * independent branches, so the GPU runs the groups' launches concurrently.
 * Results are bitwise equal to stepping each tile in its own context with the
 * same launch shape (same kernels, same arithmetic order).
 *
 * Status: ZK_EINVAL for bad arguments or a tile index out of range;
 * ZK_ESTATE when a tile without state is stepped, read or tuned; ZK_ENOMEM,
 * ZK_ECUDA as elsewhere. The batch owns all its device memory. */
typedef struct zk_batch zk_batch;
zk_status zk_batch_create(zk_batch **out, int ntiles, const int *nx, const int *nz, const double *Lx,
                          const double *Lz, const double *h, double g, const int *M, int precision);
void zk_batch_destroy(zk_batch *b);
/* Options for every tile (as zk_set_options); the stream is the batch's. */
zk_status zk_batch_set_options(zk_batch *b, const zk_options *opt);
/* Per-tile state I/O and energy: as zk_set_state / zk_get_state / zk_energy
 * for tile `tile` (arrays [nz[tile]][nx[tile]]). Setting any tile's state
 * restarts the IF-AB2 history of the whole batch (next step is IF-Euler). */
zk_status zk_batch_set_state(zk_batch *b, int tile, const void *eta, const void *psi, int dtype, int on_device);
zk_status zk_batch_get_state(zk_batch *b, int tile, void *eta, void *psi, int dtype, int on_device);
zk_status zk_batch_energy(zk_batch *b, int tile, double *H, double *kin, double *pot, double *mean_eta);
/* Advance every tile by n steps of dt, asynchronously on the batch stream. */
zk_status zk_batch_step(zk_batch *b, double dt, int n);
zk_status zk_batch_sync(zk_batch *b);
/* Number of groups, kernel launches per step (all groups) and device bytes. */
zk_status zk_batch_info(const zk_batch *b, int *ngroups, int *launches_per_step, size_t *device_bytes);
/* Group gi: its grid, order, tile count and launch shape. The launch shape is
 * plan_v (FFT plan variant of the padded lines: 0 = default radices, 1 = the
 * radix-16 alternative of lines 768, 1536, 3072), col_ci (columns per column-
 * kernel block: 0 / 1 / 2 = half / default / double; FP32 lines >= 192 only)
 * and row_occ (row-kernel blocks per SM, 0 = all that fit). */
zk_status zk_batch_group(const zk_batch *b, int gi, int *nx, int *nz, int *M, int *ntiles, int *plan_v,
                         int *col_ci, int *row_occ);
zk_status zk_batch_set_shape(zk_batch *b, int gi, int plan_v, int col_ci, int row_occ);
/* Autotuner: for each group, time one step (mean of 3 after a warm-up) under
 * every launch shape and keep the fastest; shapes that cannot launch are
 * skipped. The tiles' states and IF-AB2 histories are restored afterwards
 * (the next IF-AB2 step is IF-Euler). With cache_path non-NULL, a group whose
 * key (device name, grid, order, precision, tile count) is in the JSON cache
 * takes the stored shape without timing, and new results are written back.
 * tuned / cached (may be NULL) receive how many groups were timed / looked up.
 * Blocks until done. */
zk_status zk_batch_autotune(zk_batch *b, double dt, const char *cache_path, int *tuned, int *cached);

/* ---- Learned closure (library addition; the paper has no learned component) ----
 *
 * A small network corrects the order-b right-hand side towards the order-M
 * one of the same context (Sec. 3.2 series, Eq. 9, truncated at b and M
 * terms): f_closure = f_b + R_hat, where R is the network's prediction of the
 * physical residual f_M - f_b of both equations (Eqs. 4 and 10) and R_hat its
 * spectrum with the Nyquist modes zero, the taper of the nonlinear terms
 * applied and the mean of d eta / dt kept at zero.
 *
 * Network (zk_net): x [B][6][H][W] -> 3x3 conv 6->32, tanh -> 3x3 conv 32->32,
 * tanh -> 3x3 conv 32->32, tanh -> 1x1 conv 32->2 -> y [B][2][H][W]; periodic
 * convolutions (cross-correlation, wrap-around at the edges); weights and the
 * activations entering each convolution rounded to FP16, FP32 arithmetic.
 * Parameters: one FP32 vector W1 b1 W2 b2 W3 b3 W4 b4, weights [out][in][k][k]
 * (20322 values). H, W: multiples of 16. All tensors are device FP32 arrays
 * owned by the caller; the network keeps its own activations for one
 * backward pass. Work is queued on `stream` (cudaStream_t, NULL = legacy
 * default); calls that return a host value synchronise it. */
typedef struct zk_net zk_net;
/* cin, width, cout must be 6, 32, 2 (ZK_EUNSUPPORTED otherwise); parameters start at zero. */
zk_status zk_net_create(zk_net **out, int cin, int width, int cout);
void zk_net_destroy(zk_net *n);
zk_status zk_net_param_count(const zk_net *n, int *count);
/* Replace the parameters (host or device FP32 vector); resets the Adam moments. */
zk_status zk_net_set_params(zk_net *n, const float *theta, int on_device);
zk_status zk_net_get_params(zk_net *n, float *theta, int on_device);
/* y = net(x) for `batch` samples of nz x nx; y may be NULL. Keeps what backward needs. */
zk_status zk_net_forward(zk_net *n, const float *x, float *y, int batch, int nz, int nx, void *stream);
/* Given dL/dy of the last forward pass: dL/dtheta into grad (device, may be NULL:
 * kept inside for zk_net_adam) and dL/dx into dx (may be NULL). ZK_ESTATE
 * before any forward pass. */
zk_status zk_net_backward(zk_net *n, const float *dy, float *grad, float *dx, void *stream);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected) with the
 * given device gradient, or the one the last backward pass kept (grad NULL). */
zk_status zk_net_adam(zk_net *n, const float *grad, double lr, void *stream);
/* forward, mean-squared error against target (same shape as y), backward and
 * one Adam step; *loss (may be NULL) receives the loss before the update. */
zk_status zk_net_train_step(zk_net *n, const float *x, const float *target, int batch, int nz, int nx, double lr,
                            double *loss, void *stream);
/* Data preparation of the closure's training set (the network's per-channel input and output
 * scales). x: device FP32 array [n][c][hw] (n samples, c <= 64 channels of hw values each).
 * zk_net_channel_rms: rms[ch] = sqrt(mean over samples and positions of x^2), into host memory
 * rms[c]; FP64 sums in a fixed order (the same result on every call).
 * zk_net_scale_channels: x[smp][ch][:] *= mul[ch] in place, mul a host array of c factors.
 * Both queue on `stream` and synchronise it before returning; their few scratch bytes come
 * from the stream-ordered allocator. ZK_EINVAL for bad sizes or NULL pointers, ZK_ENOMEM,
 * ZK_ECUDA. */
zk_status zk_net_channel_rms(const float *x, long long n, int c, int hw, float *rms, void *stream);
zk_status zk_net_scale_channels(float *x, long long n, int c, int hw, const float *mul, void *stream);
/* Inference engine of the network (used by zk_net_predict and by an attached
 * closure): mode 0 = the FP32 SIMT kernels above; mode 1 (the default) = 5th-generation
 * tensor cores (tcgen05 MMAs with FP32 accumulators in TMEM; the same FP16
 * rounding of weights and layer inputs, FP32 sums, so results agree with mode 0
 * to summation order). Every wait of a tensor-core block on its MMAs is bounded; a
 * block whose wait runs out frees its TMEM and flags the call, which then returns
 * ZK_ETIMEOUT. mode 2 = self-test of that path: the tensor-core kernels issue no MMA,
 * so every wait runs out after a short limit and zk_net_predict returns ZK_ETIMEOUT
 * with the network and the device still usable (its output is meaningless).
 * ZK_EINVAL for other modes. */
zk_status zk_net_set_inference(zk_net *n, int mode);
/* y [2][nz][nx] = net(x [6][nz][nx]) for one sample with the current engine
 * (device arrays; nz, nx multiples of 16). Synchronises the stream;
 * ZK_ETIMEOUT if a tensor-core block gave up waiting for its MMAs (the output
 * is then invalid). */
zk_status zk_net_predict(zk_net *n, const float *x, float *y, int nz, int nx, void *stream);
/* Training pair at the context's current state (FP32 contexts): feat [6][nz][nx]
 * = eta, d_x eta, d_z eta, G0 psi, (d eta/dt)_b - G0 psi, (d psi/dt)_b + g eta,
 * each divided by in_scale[c] (NULL: 1); target [2][nz][nx] (may be NULL) =
 * f_M - f_b divided by out_scale (NULL: 1). 1 <= b < M. Device outputs; syncs. */
zk_status zk_closure_features(zk_ctx *ctx, int base_order, const float *in_scale, const float *out_scale, float *feat,
                              float *target);
/* Attach net (NULL detaches) to an FP32 context with the scales it was trained
 * with. From then on zk_step (RK4 only; ZK_EUNSUPPORTED for IF-AB2 and IF-RK4), zk_rhs and
 * zk_dno use f_closure. Every check_every steps (0 = never), before the step,
 * the context computes f_M and f_b at the current state and the relative L2
 * error of the predicted residual against f_M - f_b; above check_tol the
 * closure is switched off for good and the context steps at order M (the
 * fallback). Checks synchronise the stream. The caller keeps net alive while
 * attached. */
zk_status zk_closure_set(zk_ctx *ctx, zk_net *net, int base_order, const float *in_scale, const float *out_scale,
                         int check_every, double check_tol);
/* How often the closure's network is evaluated in an RK4 step: on = 0 (default) at every
 * stage's state; on = 1 at the first stage only, its residual spectrum then applied again at
 * stages 2-4 (a quarter of the network's cost; the correction lags the stage states by up to
 * one step). The base-order right-hand side is still evaluated at every stage. ZK_EINVAL for
 * other values. */
zk_status zk_closure_set_once_per_step(zk_ctx *ctx, int on);
/* active: 1 while the closure is in use; checks made; the step count at which
 * it fell back (-1: never); the error of the last check (-1: none yet). */
zk_status zk_closure_status(const zk_ctx *ctx, int *active, int *checks, long long *fallback_step, double *last_err);

/* Static text for a status code. */
const char *zk_strerror(zk_status s);

/* Library version string. */
const char *zk_version(void);

#ifdef __cplusplus
}
#endif

#endif /* ZK_H */
