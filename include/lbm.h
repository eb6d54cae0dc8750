/*
 * lbm.h -- C ABI of the GB300 D2Q9 generalized Onsager-regularised lattice
 * Boltzmann library (liblbm.so).
 *
 * Method: arXiv 2602.21242 ("Generalized Onsager-Regularized Lattice Boltzmann
 * Method for error-free Navier-Stokes models on standard lattices"). One time
 * step is the lattice Boltzmann equation, Eq. 1: collide every node,
 *   f*_i = f^eq_i + (1 - 1/tau) g_i                                  (Eq. 1a)
 * then propagate f*_i(x, t) -> f_i(x + c_i, t + 1)                   (Eq. 1b)
 * on a doubly periodic nx x ny D2Q9 grid (velocities numbered as in Fig. 1a),
 * with f^eq the guided equilibrium (Eq. 10) and g chosen by the model:
 *   LBM_LBGK           g = f - f^eq                         (Eq. 1a, Sec. 1)
 *   LBM_OREG           g = f^OReg                            (Eq. 2)
 *   LBM_OREG_PARTIAL   g = f^OReg + Psi^P                    (Eqs. 7, 14)
 *   LBM_OREG_COMPLETE  g = f^OReg + Psi^C, with Pi~ from Eqs. 11b and 12 (Eqs. 7, 15)
 *   LBM_OREG_COMPLETE_NEQ  as LBM_OREG_COMPLETE with Eq. 12's strain estimate taken
 *                      from f^neq instead of f^OReg (pref = -N_d / (2 theta^2)), with
 *                      which the corrected stress equals Pi^NS exactly (Eq. 7)
 *   LBM_LBGK_POLY      g = f - f^eq with f^eq the second-order polynomial equilibrium
 *                      rho w_i [1 + c.u/theta + ((c.u)^2 - theta u^2)/(2 theta^2)],
 *                      w_i = W(c_ix) W(c_iy), W(0) = 1 - theta, W(+-1) = theta/2: a second
 *                      reading of Sec. 5.1's "standard Lattice-BGK" (the paper does not
 *                      print its equilibrium); at theta = 1/3 the textbook D2Q9 BGK. Not
 *                      differentiable through lbm_vjp (LBM_EINVAL).
 *
 * Conventions shared by every call:
 *   - Fields are row-major [y][x] (x fastest), nx * ny doubles, unpadded.
 *     Population arrays are [i][y][x], 9 * nx * ny doubles, i in Fig. 1a order:
 *     c0=(0,0) c1=(1,0) c2=(0,1) c3=(-1,0) c4=(0,-1) c5=(1,1) c6=(-1,1) c7=(-1,-1) c8=(1,-1).
 *   - The STATE of a lattice at time t is its pre-collision populations f(x, t).
 *     lbm_init sets f(x, 0) = f^eq(rho0(x), u0(x)); lbm_step advances t.
 *   - theta is the reduced lattice temperature, tau the relaxation time. The
 *     lattice viscosity is nu = theta (tau - 1/2): the paper prints tau = nu/theta
 *     (Sec. 1); the 1/2 follows from the (1 - dt/2tau) factors of Eq. 5 at dt = 1.
 *   - Pointers named d_* are DEVICE pointers, h_* are HOST pointers; all are
 *     owned by the caller and must stay valid until the call's work completes
 *     on the lattice's stream (calls are asynchronous unless stated).
 *   - Every call returns an lbm_status. On failure, lbm_last_error(ctx) holds a
 *     one-line message. A call that fails leaves the lattice's state unchanged
 *     unless stated otherwise.
 *   - A lattice is bound to the CUDA device that was current at creation; call
 *     with the same device current. Calls on one lattice are not thread-safe.
 */
#ifndef LBM_H
#define LBM_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_ctx lbm_ctx;

/* Collision models (Sec. 4; model 4 is the f^neq variant of Eq. 12's prefactor,
 * model 5 the polynomial-equilibrium reading of Sec. 5.1's LBGK). */
enum lbm_model {
  LBM_LBGK = 0,
  LBM_OREG = 1,
  LBM_OREG_PARTIAL = 2,
  LBM_OREG_COMPLETE = 3,
  LBM_OREG_COMPLETE_NEQ = 4,
  LBM_LBGK_POLY = 5
};

/* Storage / arithmetic forms.
 *   LBM_F64        populations stored in FP64, all arithmetic in FP64.
 *   LBM_F32_SHIFT  stored as deviations f_i - rho_ref w_i(theta) in FP32, where
 *                  w_i(theta) is the rest GEq (Eq. 10 at u = 0) and rho_ref = 1;
 *                  collision arithmetic in FP32, reductions in FP64.
 *   LBM_F16_SHIFT  as LBM_F32_SHIFT with the deviations stored in IEEE FP16.
 *   LBM_F64_DF     populations stored in FP64 (the LBM_F64 layout), collision
 *                  arithmetic in double-float: each value the unevaluated sum of
 *                  two FP32 numbers (about 48 significant bits, FP32 exponent
 *                  range; magnitudes below 1.2e-38 become zero), built from
 *                  error-free transformations on the FP32 pipes. Same results
 *                  as LBM_F64 to about 1e-13 relative per step. Step launches
 *                  of at most 256 threads a block; lbm_vjp runs its adjoint in
 *                  double-float too; not available to the batched form. */
enum lbm_prec {
  LBM_F64 = 0,
  LBM_F32_SHIFT = 1,
  LBM_F16_SHIFT = 2,
  LBM_F64_DF = 3
};

enum lbm_status {
  LBM_OK = 0,
  LBM_EINVAL = -1,     /* an argument is out of range or a pointer is NULL      */
  LBM_ENOMEM = -2,     /* device or host allocation failed                       */
  LBM_ECUDA = -3,      /* a CUDA runtime call or kernel launch failed            */
  LBM_ENONFINITE = -4, /* a diagnostics pass found non-finite populations        */
  LBM_ETIMEOUT = -5,   /* a bounded device-side wait gave up                     */
  LBM_ESTATE = -6      /* call out of order (e.g. stepping before lbm_init)      */
};

/* Library version, (major << 16) | minor (no counterpart in the paper). */
int lbm_version(void);

/*
 * Device memory layout of one population buffer for (nx, ny, prec) (no
 * counterpart in the paper, which fixes no storage; the planes hold the nine
 * f_i of Eq. 1 in Fig. 1a's order): each of the 9 planes has ny rows of *pitch elements (pitch >= nx, rows 128-byte aligned) and
 * planes are *plane elements apart (256-byte aligned). *state_bytes is the size
 * of ONE buffer; a lattice holds two (ping-pong). Any output pointer may be NULL.
 * Errors: LBM_EINVAL for nx, ny < 1, sizes whose buffers exceed 2^40 bytes, or an
 * unknown prec.
 */
int lbm_layout(int nx, int ny, int prec, long long* pitch, long long* plane,
               long long* state_bytes);

/*
 * Create a lattice for the problem of Sec. 1 / Eq. 1: nx x ny periodic grid,
 * temperature theta, relaxation time tau and collision model (enum lbm_model),
 * FP64 storage, on the legacy default stream, library-owned buffers.
 * Errors: LBM_EINVAL unless nx, ny >= 1, 0 < theta < 1, tau > 1/2 and model in
 * range; LBM_ENOMEM; LBM_ECUDA (e.g. no device). *out is set only on success.
 */
int lbm_create(int nx, int ny, double theta, double tau, int model, lbm_ctx** out);

/*
 * As lbm_create (Sec. 1 / Eq. 1) with a storage form (enum lbm_prec), a CUDA stream (a
 * cudaStream_t cast to void*, NULL = legacy default stream) and, optionally,
 * caller-owned population memory: d_pop_buffers, if not NULL, is a device
 * pointer to 2 * state_bytes bytes (see lbm_layout), 256-byte aligned, that the
 * caller keeps alive until lbm_destroy; the library never frees it.
 */
int lbm_create_ex(int nx, int ny, double theta, double tau, int model, int prec,
                  void* stream, void* d_pop_buffers, lbm_ctx** out);

/* Release the lattice and the device memory it owns (no counterpart in the paper).
 * NULL is accepted. Synchronises its stream. */
int lbm_destroy(lbm_ctx* ctx);

/*
 * Rebind the lattice to another stream (no counterpart in the paper;
 * cudaStream_t as void*, NULL = legacy default). Work already enqueued for the lattice (steps on the old stream and
 * the fused diagnostics' final sums joined into it) is ordered before anything
 * later enqueued on the new stream: the new stream waits for an event recorded
 * on the old one. Does not synchronise the host.
 */
int lbm_set_stream(lbm_ctx* ctx, void* stream);

/*
 * Initial state f(x, 0) = f^eq(rho0(x), u0(x)), the guided equilibrium of Eq. 10,
 * at every node; resets the step counter to 0. d_rho, d_ux, d_uy: device arrays
 * of nx * ny doubles. GEq populations are positive only where
 * 1 - theta - u^2 > 0 and theta + u^2 > |u| per axis; the call does not check.
 */
int lbm_init(lbm_ctx* ctx, const double* d_rho, const double* d_ux, const double* d_uy);

/*
 * Advance the state by n >= 0 time steps of Eq. 1 (fused pull-stream + collide).
 * Asynchronous. If a diagnostics interval M > 0 is set, every step whose start
 * time t is a multiple of M also reduces the diagnostics of f(x, t) (see
 * lbm_diagnostics) on the device; lbm_sync / lbm_step_diagnostics report them.
 * The final sums of those reductions run on a second stream that the context
 * owns, beside the following steps; before returning, the call makes the
 * context's stream wait for them, so work queued on that stream afterwards sees
 * every result of the call.
 * Errors: LBM_ESTATE before lbm_init or lbm_set_state; LBM_EINVAL for n < 0.
 */
int lbm_step(lbm_ctx* ctx, int n);

/* Fused diagnostics interval M (0 = off, the default): the reductions of
 * lbm_diagnostics taken inside lbm_step (no counterpart in the paper). */
int lbm_set_diagnostics_interval(lbm_ctx* ctx, int every);

/*
 * Fullway bounce-back walls (the wall treatment of Sec. 5.2's shocktube). h_mask:
 * HOST array of nx * ny bytes, row-major [y][x]; a nonzero byte makes that node
 * a wall: in every later step (lbm_step, lbm_run_host, the forward and reverse
 * sweeps of lbm_vjp) the node does not collide but returns each population the
 * way it came, f*_i = f_ibar with c_ibar = -c_i. NULL removes all walls (the
 * default: doubly periodic). Wall nodes keep populations; moments, state copies
 * and diagnostics cover them like any node (bounce-back conserves each node's
 * mass, so total mass stays conserved; momentum does not). *h_count (may be
 * NULL) receives the number of wall nodes. Synchronous: waits for the lattice's
 * stream, then uploads the list. The mask is copied; the caller keeps it.
 * Errors: LBM_ENOMEM, LBM_ECUDA; the previous walls are gone after a failure.
 */
int lbm_set_walls(lbm_ctx* ctx, const unsigned char* h_mask, long long* h_count);

/*
 * Latest diagnostics reduced inside lbm_step (no counterpart in the paper): h_out5 as in lbm_diagnostics,
 * *h_time = the time t they describe (-1 if none yet). Synchronises the stream.
 * Returns LBM_ENONFINITE if any fused pass so far met a non-finite population.
 */
int lbm_step_diagnostics(lbm_ctx* ctx, double* h_out5, long long* h_time);

/*
 * Moments of the current state (Sec. 1): rho = sum_i f_i and u = sum_i c_i f_i / rho,
 * written to device arrays of nx * ny doubles. 1 / rho is formed as in the step
 * (within an ulp or two of the quotient); a node whose density lies outside
 * [2^-126, 2^126) gets non-finite velocities.
 */
int lbm_moments(lbm_ctx* ctx, double* d_rho, double* d_ux, double* d_uy);

/*
 * Global diagnostics of the current state (the moments of Sec. 1 summed over
 * the grid: mass, momentum and kinetic energy, which Eq. 1a's collision
 * conserves or the model's viscosity dissipates), reduced on the device in a fixed
 * order (deterministic for a given size) in FP64, written to the HOST array
 * h_out5 = { sum rho, sum rho u_x, sum rho u_y, sum rho |u|^2 / 2,
 * number of nodes with a non-finite population } (sums skip those nodes).
 * Synchronises. Returns LBM_ENONFINITE when out5[4] > 0 (out5 is still written).
 */
int lbm_diagnostics(lbm_ctx* ctx, double* h_out5);

/* Copy the state f(x, t) (the populations of Eq. 1 at time t) to / from a device
 * array of 9 * nx * ny doubles ([i][y][x]). */
int lbm_get_state(lbm_ctx* ctx, double* d_f);
int lbm_set_state(lbm_ctx* ctx, const double* d_f);

/*
 * Slab split of one periodic lattice along y (Eq. 1's streaming across the faces
 * between slabs; no counterpart in the paper, which runs one lattice). A context
 * of nx x ny nodes created for rows [y0, y0 + ny) of an nx x NY lattice is
 * initialised from those rows (lbm_init, lbm_set_state; they need no exchange)
 * and advanced one step at a time: after every step (lbm_step(ctx, 1)) each
 * slab calls lbm_halo_pack, sends the two face buffers to its neighbours (`up`
 * to the slab above, y0 + ny, `down` to the slab below, y0 - 1, both taken
 * periodically) and calls lbm_halo_unpack with the buffers it received from
 * the slab below and the slab above. The context then describes its rows of
 * the whole lattice: the next step pulls across the faces, and lbm_moments,
 * lbm_get_state, lbm_diagnostics and the fused diagnostics of the next step
 * cover exactly its rows (summed over the slabs they give the whole
 * lattice's). With one slab the exchange returns each buffer to its sender and
 * changes nothing. Between a step and its exchange the context's state is not
 * that of the whole lattice. Walls, lbm_run_host and lbm_vjp act on the
 * context alone.
 *
 * lbm_halo_bytes: *h_bytes = bytes of each face buffer, 3 * nx storage elements
 * (8 bytes each for LBM_F64 and LBM_F64_DF, 4 for LBM_F32_SHIFT, 2 for
 * LBM_F16_SHIFT; values move bit for bit in the storage form, so every slab must
 * use the same form, theta and tau).
 * lbm_halo_pack: d_up receives the populations with c_y = +1 (i = 2, 5, 6, in
 * that order, each nx values, x fastest) that leave through the top face, d_down
 * those with c_y = -1 (i = 4, 7, 8) that leave through the bottom face.
 * lbm_halo_unpack: the slab below's d_up (d_from_below) and the slab above's
 * d_down (d_from_above) take their places.
 * Buffers: device memory of lbm_halo_bytes each, aligned to the storage element,
 * owned by the caller, not overlapping the context's buffers or each other.
 * Asynchronous on the context's stream. Errors: LBM_EINVAL for NULL or
 * misaligned pointers; LBM_ESTATE before lbm_init / lbm_set_state, for a pack
 * unless exactly one step has run since the last unpack, lbm_init or
 * lbm_set_state, and for an unpack without a pack since the last step.
 */
int lbm_halo_bytes(const lbm_ctx* ctx, long long* h_bytes);
int lbm_halo_pack(lbm_ctx* ctx, void* d_up, void* d_down);
int lbm_halo_unpack(lbm_ctx* ctx, const void* d_from_below, const void* d_from_above);

/*
 * Reverse-mode derivative (vector-Jacobian product) of n steps of Eq. 1 started
 * from the guided equilibrium f(x, 0) = f^eq(rho0(x), u0(x)) (Eq. 10), with
 * respect to the initial fields. Given the cotangents g_rho, g_ux, g_uy of the
 * final moments (rho, u)(x, n) (device arrays of nx * ny doubles; any may be
 * NULL = 0), writes the cotangents of (rho0, u0) to g_rho0, g_ux0, g_uy0 (device,
 * nx * ny doubles; any may be NULL to skip).
 * Method: a forward pass from d_rho0, d_ux0, d_uy0 (device) storing a checkpoint
 * every ckpt_every steps, then per segment, last first, a recomputation of its
 * states and the adjoint steps lambda(t) = J_C(f(t))^T S^T lambda(t + 1), where S^T
 * reads lambda_i(t + 1) at x + c_i and J_C^T is the hand-derived transposed
 * Jacobian of the model's collision. FP64, double-float and FP32 storage (the
 * adjoint runs in the form's arithmetic: FP64, double-float pairs, FP32);
 * LBM_EINVAL for FP16. Device work memory of
 * (ceil(n / ckpt_every) + ckpt_every + 2) population buffers is kept by the
 * lattice. Asynchronous; on return the lattice holds f(x, n) of this run.
 */
int lbm_vjp(lbm_ctx* ctx, int n, int ckpt_every, const double* d_rho0, const double* d_ux0,
            const double* d_uy0, const double* g_rho, const double* g_ux, const double* g_uy,
            double* g_rho0, double* g_ux0, double* g_uy0);

/*
 * The forward pass of lbm_vjp on its own (no counterpart in the paper): lbm_init
 * from d_rho0, d_ux0, d_uy0 (device, nx * ny doubles), then n steps, keeping the
 * checkpoints (every ckpt_every steps) and the states of the last segment in the
 * lattice's work memory; the lattice then holds f(x, n), as after lbm_init +
 * lbm_step(n) without fused diagnostics. A following lbm_vjp_ex with flag
 * LBM_VJP_REUSE_FORWARD and the same n and ckpt_every skips its own forward pass,
 * as long as no call changed the lattice in between (lbm_init, lbm_set_state,
 * lbm_step, lbm_set_walls, lbm_vjp*). Errors and forms as lbm_vjp. Asynchronous.
 */
int lbm_vjp_forward(lbm_ctx* ctx, int n, int ckpt_every, const double* d_rho0, const double* d_ux0,
                    const double* d_uy0);

#define LBM_VJP_REUSE_FORWARD 1

/*
 * lbm_vjp with flags: 0 is lbm_vjp; LBM_VJP_REUSE_FORWARD uses the checkpoints of
 * the preceding lbm_vjp_forward (d_rho0, d_ux0, d_uy0 must be the fields it ran
 * from: the derivative through Eq. 10 is taken at them) and returns LBM_ESTATE,
 * with nothing done, when they no longer describe the lattice. LBM_EINVAL for
 * other flags.
 */
int lbm_vjp_ex(lbm_ctx* ctx, int n, int ckpt_every, const double* d_rho0, const double* d_ux0,
               const double* d_uy0, const double* g_rho, const double* g_ux, const double* g_uy,
               double* g_rho0, double* g_ux0, double* g_uy0, int flags);

/* Current time t of Eq. 1 (steps since lbm_init / lbm_set_state). */
int lbm_time(const lbm_ctx* ctx, long long* h_t);

/*
 * End-to-end call on HOST memory (no counterpart in the paper; Eq. 10's
 * initial state and n steps of Eq. 1): copy rho0, u0 (host, nx * ny doubles each;
 * page-locked memory recommended) to the device, lbm_init, run n steps, copy the
 * final moments to h_rho, h_ux, h_uy (host, may be NULL to skip) and the final
 * diagnostics to h_diag5 (host, may be NULL). Synchronous. Device staging
 * memory is allocated on the first call and kept by the lattice.
 */
int lbm_run_host(lbm_ctx* ctx, const double* h_rho0, const double* h_ux0, const double* h_uy0,
                 int n, double* h_rho, double* h_ux, double* h_uy, double* h_diag5);

/*
 * Launch shape of the fused step kernel (no counterpart in the paper): blocks of
 * bx x by threads (bx a multiple of 32, bx * by <= 512; <= 256 for LBM_F64_DF),
 * each thread updating `rows` nodes (node pairs for the shifted forms when nx
 * is even) of one column (1 <= rows <= 64). Results do not depend on the
 * shape except for the order of the diagnostics sums. Each storage form starts
 * from a default measured on GB300; lbm_set_launch may reallocate the small
 * diagnostics buffer (it then synchronises the stream). Errors: LBM_EINVAL.
 */
int lbm_set_launch(lbm_ctx* ctx, int bx, int by, int rows);
int lbm_get_launch(const lbm_ctx* ctx, int* bx, int* by, int* rows);

/*
 * Step-kernel selection (no counterpart in the paper). kind 0: the column kernel
 * of lbm_set_launch. kind 1 (shifted FP32/FP16 forms and FP64, any nx; not
 * LBM_F64_DF): a producer warp streams each output row's nine plane segments
 * into a shared-memory ring with TMA bulk copies and mbarrier transaction
 * counts while consumer warps collide node pairs (FP64: single nodes); the
 * lattice is cut into tiles of 256 (FP32), 512 (FP16) or 128 (FP64) columns by
 * `rows` rows (1..4096); bx = 0 launches one CTA per tile, bx = k > 0 (shifted
 * forms only; LBM_EINVAL for FP64) a persistent grid of k
 * CTAs per SM (capped at the resident count) whose CTAs take the next tile from
 * a counter in device memory that the context owns (by ignored). Its waits are
 * bounded: a wait that gives up makes lbm_sync and lbm_step_diagnostics return
 * LBM_ETIMEOUT. Same results as kind 0 for even nx (FP32 rounding may differ in
 * the last bit for odd nx, where kind 0 updates single nodes) except the
 * diagnostics' summation order. Default for the shifted forms on lattices at
 * least 32 columns wide: FP32 kind 2 below on 24-row tiles (48 from 8192^2); FP16 one CTA
 * per tile with the height in {48, 40, 32, 24, 16} that best fills the last
 * wave of CTAs (halved further on small lattices).
 * kind 2 (shifted FP32/FP16 forms; bx = 0, by ignored): two steps per launch
 * (temporal blocking of Eq. 1): each CTA computes step t's post-collision values
 * on its tile of 254 (FP32) or 510 (FP16) columns by `rows` rows plus a
 * one-node border, rounds them to the storage type in a shared-memory window
 * and computes step t + 1 from there, so the state is read and written once per
 * two steps. Results are bit-identical to two single steps (the diagnostics'
 * summation order aside). It applies where two steps of a call follow each
 * other and no walls are set (any nx); other steps (the last of an odd
 * count) take kind 1 with one CTA per tile of the same height.
 */
int lbm_set_launch_ex(lbm_ctx* ctx, int kind, int bx, int by, int rows);
int lbm_get_launch_ex(const lbm_ctx* ctx, int* kind, int* bx, int* by, int* rows);

/* ------------------------------------------------------------------------
 * Batched form: many independent doubly periodic lattices of uneven size,
 * each with its own theta and tau, sharing one collision model and storage
 * form, advanced together (Eq. 1 per domain). Domain k's fields are packed
 * one after another (domain 0 first), each row-major [y][x] with nx[k] * ny[k]
 * doubles. The ABI conventions above apply.
 * ------------------------------------------------------------------------ */
typedef struct lbm_batch lbm_batch;

/*
 * The batched form advances many domains by one persistent launch captured in a
 * CUDA graph. The two modes read that design two ways:
 *   LBM_BATCH_GRAPH      the graph: every step is one launch of the tile kernel
 *                        over all domains, and the n launches of a call are
 *                        captured once into a CUDA graph and replayed as one
 *                        graph launch (fused diagnostics as a parallel branch).
 *   LBM_BATCH_PERSISTENT the persistent launch in a graph: one cooperative
 *                        launch runs all n steps, a grid barrier with a bounded
 *                        wait between steps; it is captured with the barrier's
 *                        reset into a CUDA graph once per n and buffer parity
 *                        and replayed; the call then reads the barrier's status
 *                        back and synchronises.
 * Measured on GB300 over 256 uneven Taylor-Green domains (FP32): with single
 * steps both reach about 88 % of HBM; with two steps a launch (kind 2) graph
 * mode 113 and persistent mode 106 GLUPS, 1.2 and 1.13 x the single-step roof.
 */
enum lbm_batch_mode {
  LBM_BATCH_GRAPH = 0,      /* one tile-kernel launch per step, n steps captured into one CUDA graph */
  LBM_BATCH_PERSISTENT = 1  /* one cooperative launch for all n steps, bounded-wait grid barrier per step */
};

/* Create n >= 1 domains (arrays of length n), each the problem of Sec. 1 / Eq. 1
 * (the batched form itself has no counterpart in the paper). Errors: LBM_EINVAL for a domain
 * outside the lbm_create ranges; LBM_ENOMEM; LBM_ECUDA. Message: lbm_last_error(NULL). */
int lbm_batch_create(int n, const int* nx, const int* ny, const double* theta, const double* tau,
                     int model, int prec, void* stream, lbm_batch** out);
int lbm_batch_destroy(lbm_batch* b);

/* Tile shape (no counterpart in the paper), launch kind 0 (the column routine): blocks of bx x by threads (bx a
 * multiple of 32, bx * by <= 512) updating tiles of bx (node pairs: 2 bx) columns x
 * by * rows rows. Rebuilds the tile list (synchronous). */
int lbm_batch_set_launch(lbm_batch* b, int bx, int by, int rows);
int lbm_batch_get_launch(const lbm_batch* b, int* bx, int* by, int* rows, int* ntiles);

/* Launch kind and tile shape (no counterpart in the paper). kind 0: as lbm_batch_set_launch. kind 1 (the shifted
 * forms only; the FP16 default): the bulk-copy pipeline of the single-lattice
 * kind-1 kernel, one CTA of bx consumer threads (+ one producer warp) per tile of
 * 2 bx columns x rows rows (1..4096), any domain width; bx = 32, 64 or 128 (FP32),
 * 64, 128 or 256 (FP16), 0 = 128 (FP32) / 256 (FP16); narrower tiles waste less
 * of a strip on narrow domains. by is ignored. A domain's results equal those of
 * a single lattice stepped with the same launch kind. kind 2 (shifted forms, bx =
 * 0; the FP32 default, 32 rows): two steps a launch (the two-step tile routine
 * of the single-lattice kind 2 on tiles of 254 (FP32) or 510 (FP16) columns x
 * rows rows of every domain, any width): in graph mode n / 2 two-step launches,
 * in persistent mode one cooperative launch looping over n / 2 pairs of steps;
 * an odd last step uses the kind 1 tiles of the same height (in persistent mode
 * a second cooperative launch captured in the same graph); results equal kind 1
 * bit for bit.
 * Errors: LBM_EINVAL (kinds 1 and 2 on FP64 storage, bx or rows out of range).
 * lbm_batch_get_launch_ex also reports the kind (and, for kind 2, the two-step
 * tile count). */
int lbm_batch_set_launch_ex(lbm_batch* b, int kind, int bx, int by, int rows);
int lbm_batch_get_launch_ex(const lbm_batch* b, int* kind, int* bx, int* by, int* rows, int* ntiles);
/* Batch mode, enum lbm_batch_mode; default LBM_BATCH_GRAPH (no counterpart in the paper). */
int lbm_batch_set_mode(lbm_batch* b, int mode);
/* Fused per-domain diagnostics every M steps in LBM_BATCH_GRAPH mode (0 = off; no
 * counterpart in the paper). */
int lbm_batch_set_diagnostics_interval(lbm_batch* b, int every);

/* f(x, 0) = f^eq(rho0, u0) (Eq. 10) for every domain, from packed device fields. */
int lbm_batch_init(lbm_batch* b, const double* d_rho, const double* d_ux, const double* d_uy);
/* Domain k's state f(x, t) (Eq. 1's populations at time t) to / from a device array of 9 * nx[k] * ny[k] doubles ([i][y][x]). */
int lbm_batch_get_state(lbm_batch* b, int k, double* d_f);
int lbm_batch_set_state(lbm_batch* b, int k, const double* d_f);
/* Moments (Sec. 1) of every domain into packed device fields (asynchronous). */
int lbm_batch_moments(lbm_batch* b, double* d_rho, double* d_ux, double* d_uy);

/*
 * Advance every domain by n steps of Eq. 1. LBM_BATCH_GRAPH: asynchronous; the n launches
 * are captured once into a graph (re-captured when n, the buffer parity or the
 * diagnostics phase changes) and replayed; each diagnosed step's final sum is a
 * parallel branch of the graph. LBM_BATCH_PERSISTENT: one cooperative launch
 * replayed from a CUDA graph (captured once per n and buffer parity), without
 * fused diagnostics (lbm_batch_diagnostics reduces the state after it);
 * synchronises and returns LBM_ETIMEOUT if a grid barrier waited longer than
 * about a second (the state is then undefined).
 */
int lbm_batch_step(lbm_batch* b, int n);
/* Latest fused diagnostics (no counterpart in the paper), h_out[5 * k + j] as lbm_diagnostics for domain k; *h_time
 * the time they describe (-1 if none). Synchronises; LBM_ENONFINITE if any pass met one. */
int lbm_batch_step_diagnostics(lbm_batch* b, double* h_out, long long* h_time);
/* Diagnostics of every domain's current state (the moments of Sec. 1 summed per
 * domain, as lbm_diagnostics) into h_out[5 * n] (host). Synchronises. */
int lbm_batch_diagnostics(lbm_batch* b, double* h_out);
/* Total nodes, bytes of the population arena, current time; waiting for the
 * batch's stream; the last error message (no counterpart in the paper). */
int lbm_batch_info(const lbm_batch* b, long long* total_nodes, long long* arena_bytes, long long* t);
int lbm_batch_sync(lbm_batch* b);
const char* lbm_batch_last_error(const lbm_batch* b);

/* Wait for the lattice's stream (no counterpart in the paper); report a pending CUDA error (LBM_ECUDA) or a
 * non-finite population seen by a fused diagnostics pass (LBM_ENONFINITE). */
int lbm_sync(lbm_ctx* ctx);

/*
 * Measured arithmetic ceiling of the current device (no counterpart in the
 * paper; used as the roofline denominator of ALU-bound kernels): kind 0 = FP64,
 * kind 1 = FP32, kind 2 = packed FP32 (fma.rn.f32x2, two FMAs per instruction),
 * as FLOP/s of fused multiply-adds (2 FLOP each) from independent
 * FMA chains on 8 blocks per SM, best of 3 timed launches. Synchronous, runs on
 * the legacy default stream and allocates a small scratch buffer.
 */
int lbm_measure_peak(int kind, double* h_flops);

/*
 * One fused FP64 step with diagnostics that allocates no device memory (no
 * counterpart in the paper). For callers that cannot call cudaMalloc: code
 * whose device memory must all come from its own pool or arena, or loops where
 * an allocation's implicit synchronisation would stall the GPU. It needs no
 * lattice object: the caller passes every input
 * and output, and the only scratch, the per-block diagnostics sums, lives in a
 * fixed static device array of 320 KiB (8192 blocks x 5 doubles) that every
 * GPU which loads the library holds until the process exits.
 *
 *   d_src   device buffer in the FP64 layout of lbm_layout(nx, ny, LBM_F64)
 *           holding the state at time t as the library keeps it: plane i, node y
 *           holds f_i(y + c_i, t) (periodic), the population that node y + c_i
 *           pulls from y; read only.
 *   d_dst   a second such buffer; receives the state at t + 1 in the same
 *           convention.
 *   d_diag5 device array of 5 doubles: mass, momentum x, y and kinetic energy of
 *           f(x, t) as in lbm_diagnostics, and in element 4 the number of nodes
 *           whose populations do not sum to a finite value (left out of the
 *           sums). The call never returns LBM_ENONFINITE: callers check
 *           element 4 themselves.
 *   stream  cudaStream_t as void* (NULL = legacy default stream).
 *
 * d_src, d_dst and d_diag5 must not share a byte (LBM_EINVAL otherwise).
 * Asynchronous. The first call on a device, and the first after that device's
 * context was reset or re-created, resolves the scratch array's device address
 * (a cudaGetSymbolAddress on that device, which must be current); make that
 * first call before any stream capture. All calls on a device share the
 * scratch: calls whose work overlaps on the GPU race on it. Lattices that need
 * more than 8192 blocks of 32 x 8 threads with up to 64 rows per thread (for
 * example a 16384 x 16384 grid; 8192 x 8192 fits) are rejected with LBM_EINVAL.
 * On failure, lbm_last_error(NULL) describes the error.
 */
int lbm_step_noalloc(int nx, int ny, double theta, double tau, int model, const double* d_src,
                     double* d_dst, double* d_diag5, void* stream);

/*
 * Self-test of the bounded device-side waits (no counterpart in the paper):
 * which = 0 waits on an mbarrier phase that never completes (the wait routine of
 * the kind-1 step kernel), which = 1 on a grid barrier one block never reaches
 * (the routine of the persistent batched kernel). Each wait gives up after about
 * a second; the call returns LBM_ETIMEOUT and the elapsed host time in
 * *h_seconds, and the context stays usable. Synchronous (cudaDeviceSynchronize).
 */
int lbm_selftest_timeout(int which, double* h_seconds);

/*
 * Self-test of the FP64 arithmetic helpers the FP64 step kernel runs on the
 * integer pipe (no counterpart in the paper): applies helper `op` on the GPU to
 * the n host values h_x and writes the results to h_out (host, n doubles,
 * caller-owned). op = 0, 1, 2: the exact scaling x * k for k = 1/2, -1/2, 1/4
 * (exponent-field arithmetic; exact for x and x k in FP64's normal range, zeros,
 * infinities and NaNs as x k); op = 3: the reciprocal used for 1/rho (FP32 seed
 * of x truncated to FP32, one cubic Newton step; within an ulp or two of 1/x for
 * 2^-126 <= |x| < 2^126, non-finite for every other x); op = 4: x truncated to FP32 and widened back
 * (integer conversions; zero below FP32's normal range, infinity above it and
 * for infinities and NaNs). Synchronous.
 * Returns LBM_EINVAL for another op, n < 0 or null pointers with n > 0.
 */
int lbm_selftest_fp64(int op, const double* h_x, long long n, double* h_out);

/*
 * Self-test of the integer-pipe binary64 arithmetic of the FP64 form (no
 * counterpart in the paper; IEEE 754 round to nearest, ties to even): for the n
 * host operand pairs (h_a[k], h_b[k]) writes the integer-pipe result to h_emu[k]
 * and the FP64 instruction's result to h_fp64[k] (host, n doubles each,
 * caller-owned); op = 0 the sum, op = 1 the product. The two agree bit for bit
 * for every input (NaNs as NaNs). Synchronous. Returns LBM_EINVAL for another
 * op, n < 0 or null pointers with n > 0.
 */
int lbm_selftest_fp64_emu(int op, const double* h_a, const double* h_b, long long n, double* h_emu,
                          double* h_fp64);

/*
 * Self-test of the FP64 collision (Eq. 1a with the model's f^OReg and
 * corrections; no counterpart in the paper beyond that): collides the n nodes
 * of h_f (host, n x 9 doubles, populations in the order of Fig. 1a) on the GPU
 * twice, with the FP64 kernels' arithmetic and with every product on the FP64
 * pipe (never contracted into an FMA), and writes per node the nine
 * post-collision populations and m0, j_x, j_y, u_x, u_y (14 doubles) to h_emu
 * and h_ref (host, n x 14 doubles each, caller-owned). mode selects the
 * products the kernels' arithmetic starts with: 0 the integer pipes, 1 the
 * integer pipes with zero operands on their fast path, 2 the FP64 pipe (the
 * kernels step a warp from 0 to 1 to 2 each time one of its nodes needs a redo
 * on FP64 products). The two agree bit for bit. Coefficients from theta and tau
 * (rho_ref = 1). Synchronous. Returns LBM_EINVAL for an unknown model or mode,
 * n < 0, theta outside (0, 1), tau <= 1/2 or null pointers with n > 0.
 */
int lbm_selftest_collide_f64(int model, int mode, double theta, double tau, const double* h_f, long long n,
                             double* h_emu, double* h_ref);

/* Message of the last failed call on ctx ("" if none); a static string if ctx is NULL
 * (no counterpart in the paper). */
const char* lbm_last_error(const lbm_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* LBM_H */
