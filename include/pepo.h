/*
 * libpepo -- C ABI of the GB300 (sm_103a) implementation of the
 * Heisenberg-picture operator-network (PEPO) evolution of the 2D
 * transverse-field Ising model.
 *
 * Method (paper arxiv 2606.30985):
 *   Sec. 2.1  Eq. 1       H = -J sum X_i X_j - h sum Z_i (or the ZZ/X gate set)
 *   Sec. 2.2  Eq. 4       C(t) = Tr[Z_c(t) Z_c] / 2^N
 *   Sec. 2.3              Pauli-basis network, site tensor chi^deg x 4
 *   Sec. 2.4  Eq. 5, 6    Trotter step O -> U^dagger O U, four-colour bonds
 *   Sec. 2.5  Alg. 1      bond update: absorb, QR, RR, gate, SVD, truncate,
 *                         reconstruct, deabsorb, Vidal normalisation
 *   Sec. 4.2  Eq. 10       hybrid QR (Cholesky-QR for tall n > 150, m/n > 150)
 *   Sec. 4.2  Eq. 11, 12   truncation and lambda = s / ||s||
 *   Sec. 4.2  Eq. 13, 14  BP message update and stopping rule
 *   Sec. 6.3  Eq. 19      damped BP
 *   Sec. 2.6  Eq. 7-9   Bethe value of C(t) in log space with signs
 *   Sec. 3.1              zero-malloc workspace / IsingState
 *   Sec. 5    Eq. 15-17   analytic memory model
 *
 * Conventions shared by every entry point
 *   - Sites: (x, y), x = column in [0, Lx), y = row in [0, Ly), origin top
 *     left; site index v = y * Lx + x.
 *   - Bonds: horizontal bond (x,y)-(x+1,y) has id y*(Lx-1) + x; vertical bond
 *     (x,y)-(x,y+1) has id Ly*(Lx-1) + y*Lx + x.  The "first" site of a bond
 *     is the left / upper one.  Colour of a horizontal bond = x % 2, of a
 *     vertical bond = 2 + y % 2 (Sec. 2.4 four-colour partition).
 *   - Site tensors in the canonical host layout: legs [U, D, L, R] (absent
 *     legs skipped), then the Pauli index p in {I, X, Y, Z} = {0,1,2,3},
 *     row-major (Pauli fastest), real coefficients.  Element type double.
 *   - Directed messages: message of bond b in direction dir (0: first site ->
 *     second site, 1: second -> first) is the environment of the receiving
 *     site's leg on b; chi x chi, row-major, real symmetric.
 *   - Ownership: the caller owns the device arena, the CUDA stream and every
 *     host array.  After pepo_init the library never allocates device memory
 *     (Sec. 3.1 zero-malloc rule); it carves everything from the arena.
 *   - Errors: every call returns a pepo_status and never aborts.  On an error
 *     pepo_last_error(ctx) returns a message.  BP non-convergence is a
 *     reported outcome (sweeps == max), not an error.
 *   - Threading: calls on one context must not run concurrently.
 *   - Asynchrony: pepo_trotter_step only enqueues work on the stream; calls
 *     that return host values synchronise the stream.
 */
#ifndef PEPO_H
#define PEPO_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pepo_ctx pepo_ctx;

typedef enum {
  PEPO_OK = 0,
  PEPO_E_INVALID = 1,   /* bad argument or configuration */
  PEPO_E_OOM = 2,       /* arena smaller than pepo_required_bytes */
  PEPO_E_CUDA = 3,      /* a CUDA runtime call failed */
  PEPO_E_NUMERIC = 4,   /* reserved: numerical trouble is reported in pepo_diag.flags */
  PEPO_E_STATE = 5      /* a call out of order: warm-start weights without a warm_start
                           instance, or a call that needs whole steps while a step is
                           partly applied (pepo_trotter_colour) */
} pepo_status;

typedef enum {
  PEPO_GATES_ZZ_X = 0,  /* exp(-i J dt ZZ) bonds, exp(-i h dt X) sites */
  PEPO_GATES_XX_Z = 1   /* the paper's Eq. 1 / Eq. 6 convention */
} pepo_gateset;

typedef enum {
  PEPO_FP64 = 0,        /* site tensors and all arithmetic in double */
  PEPO_FP32 = 1,        /* site tensors float; small linear algebra double */
  PEPO_TF32X3 = 2,      /* site tensors float; absorb, BP and reconstruct contractions on
                           tcgen05 as three TF32 products (hi*hi + hi*lo + lo*hi, FP32
                           accumulation); factorisations in double.  chi_max > 128
                           runs the FP32 (CUDA-core) kernels instead */
  PEPO_BF16X3 = 3       /* not built: refused with PEPO_E_INVALID by pepo_required_bytes and
                           pepo_init (a BF16 split needs six BF16 products for FP32-level
                           accuracy, twice the tensor time of the three TF32 products) */
} pepo_precision;

typedef struct {
  int Lx, Ly;              /* grid; Lx * Ly >= 2 */
  double J, h, dt;         /* couplings and Trotter step */
  int trotter_order;       /* 1: site gates then bonds; 2: symmetric split */
  int obs_x, obs_y;        /* observable site */
  int obs_pauli;           /* 1 = X, 2 = Y, 3 = Z */
  int chi_max;             /* bond-dimension cap, >= 1 */
  double eps_cut;          /* Eq. 11 relative singular-value cut (1e-11) */
  double bp_alpha;         /* Eq. 19 damping (1 = undamped) */
  double bp_tol;           /* Eq. 14 tolerance on the message diagonals */
  int bp_max_sweeps;       /* sweep budget (100) */
  int qr_n_thresh;         /* Eq. 10 branch: Cholesky-QR if n > qr_n_thresh ... */
  double qr_ratio_thresh;  /* ... and m / n > qr_ratio_thresh (150, 150).  A Cholesky-QR
                              site whose Gram has an accepted pivot keeping less than
                              1e-4 (FP32 storage) / 1e-10 (FP64) of its own column's
                              diagonal is factored by Householder instead (Sec. 4.2's
                              fallback; counted by pepo_qr_branch_counts) */
  double pinv_rel;         /* rank threshold for message square roots (1e-12) */
  int gates;               /* pepo_gateset */
  int prec;                /* pepo_precision */
  int warm_start;          /* 1: pepo_bp_converge applies the learned warm start once
                              weights are set (pepo_set_warmstart_weights); 0: plain BP */
  int inflight_sites;      /* sites updated concurrently (scratch slabs), 0 = auto */
} pepo_config;

/* Per-instance measurement record (Table 1 diagnostics). */
typedef struct {
  double C;                /* Eq. 9 / Bethe ratio: C_proj / sqrt(norm) */
  double C_proj;           /* single-layer Bethe value (with site scales) */
  double log_norm;         /* log of the double-layer Bethe value ("Bethe norm") */
  double gate_err;         /* Table 1: discarded weight summed over the last step */
  int bp_sweeps;           /* double-layer sweeps of the last pepo_bp_converge */
  double bp_delta;
  int bp1_sweeps;          /* single-layer sweeps */
  double bp1_delta;
  double entropy_frac_max; /* Table 1: max over bonds of S_e / log chi_e */
  int trap_type1;          /* sweeps >= 30 and delta < tol (Sec. 6.3) */
  int trap_type2;          /* sweeps == max */
  int norm_exploded;       /* exp(log_norm) >= 2 */
  int flags;               /* bit 0: rank-deficient message met (env projector
                              skipped), bit 1: non-finite value seen,
                              bit 2: a Jacobi SVD hit its sweep cap,
                              bit 3: gate rank above the bound (init only) */
  int steps;               /* Trotter steps taken so far */
  int core_sweeps32_max;   /* max FP32 (preconditioning) Jacobi sweeps of a bond core, last step */
  int core_sweeps64_max;   /* max FP64 Jacobi sweeps of a bond core, last step */
  int c_drop;              /* Sec. 6.3 remediation check: |C| fell below half of the previous
                              layer's with no jump of gate_err (pepo_c_drop); with trap_type1
                              it marks a trapped layer.  0 without a previous layer measured
                              since the last state upload or restore */
} pepo_diag;

/* Sec. 6.3 (trap remediation, second check): 1 if |C| < |C_prev| / 2 while
 * the discarded weight did not jump, gate_err <= 2 max(gate_err_prev, 1e-12);
 * 0 otherwise or when an argument is not finite.  Pure host function. */
int pepo_c_drop(double C_prev, double gate_err_prev, double C, double gate_err);

/* Fill *cfg with the paper's defaults (Sec. 6: eps_cut 1e-11, tol 1e-5,
 * 100 sweeps, thresholds 150/150) and the ZZ_X gate set, 3x3 grid. */
void pepo_config_default(pepo_config* cfg);

/* Bytes of device memory pepo_init needs for n_inst instances (array cfgs).
 * Returns 0 if a configuration is invalid.  Follows the analytic memory model
 * (Eq. 15-17) adapted to this implementation: site tensors at chi_max, two
 * scratch slabs per in-flight site, messages and small workspaces. */
size_t pepo_required_bytes(const pepo_config* cfgs, int n_inst);

/* Create a context.  cfgs: n_inst configurations (host, copied).  dev_arena:
 * device pointer, 256-byte aligned, at least pepo_required_bytes bytes, owned
 * by the caller and kept alive until pepo_destroy.  cuda_stream: a
 * cudaStream_t (NULL = legacy default stream).  Initialises every instance to
 * the Sec. 2.3 initial state (observable Pauli at the chosen site, identity
 * elsewhere, all chi = 1, all messages [[1]]).  Errors: PEPO_E_INVALID,
 * PEPO_E_OOM, PEPO_E_CUDA; *out is NULL on error. */
pepo_status pepo_init(const pepo_config* cfgs, int n_inst, void* dev_arena,
                      size_t arena_bytes, void* cuda_stream, pepo_ctx** out);

/* Enqueue n_steps Trotter steps (Eq. 6 schedule, Alg. 1 per bond) on every
 * instance.  Asynchronous.  Errors: PEPO_E_INVALID (NULL context,
 * n_steps < 0), PEPO_E_CUDA (a launch or a graph capture failed; message in
 * pepo_last_error).  Numerical trouble (a rank-deficient environment, a
 * non-finite value, a Jacobi sweep cap) does not fail the call: it is
 * reported in pepo_diag.flags by pepo_correlator. */
pepo_status pepo_trotter_step(pepo_ctx* ctx, int n_steps);

/* Enqueue the bond gates of one colour class (0..3, Sec. 2.4 four-colour
 * partition) of the current Trotter step on every instance: the colours of a
 * step are applied in the order 0, 1, 2, 3, and the four calls together do
 * exactly what one pepo_trotter_step does (the site gates of Eq. 6 are folded
 * into the first and last bond gate of each site, so they travel with the
 * colour that holds that bond).  The step counter advances after colour 3.
 * Used to inspect the state in the middle of a step (pepo_get_site,
 * pepo_get_spectrum, pepo_get_message): between the calls, every call that needs
 * whole steps (pepo_trotter_step, BP, the correlator, state uploads,
 * snapshots, the warm start) fails with PEPO_E_STATE.  Launches directly
 * (no graph).  Asynchronous.  Errors: PEPO_E_INVALID (NULL context, colour
 * outside 0..3), PEPO_E_STATE (colour out of order), PEPO_E_CUDA. */
pepo_status pepo_trotter_colour(pepo_ctx* ctx, int colour);

/* Run damped double-layer BP (Eq. 13-19) to tolerance or the sweep budget.
 * sweeps_out / delta_out: host arrays of n_inst entries (may be NULL).
 * Synchronises the stream.  Errors: PEPO_E_INVALID (NULL context),
 * PEPO_E_CUDA (a launch or read-back failed, or a tensor-core pipeline wait
 * ran out of time: the kernels return instead of hanging and the call fails
 * with that message). */
pepo_status pepo_bp_converge(pepo_ctx* ctx, int* sweeps_out, double* delta_out);

/* Single-layer BP on the pinned network and the Bethe value of C(t)
 * (Eq. 7-9).  Uses the current double-layer messages (call
 * pepo_bp_converge first).  C_out: n_inst doubles; diag_out: n_inst records
 * (either may be NULL).  Synchronises the stream.  Errors as
 * pepo_bp_converge. */
pepo_status pepo_correlator(pepo_ctx* ctx, double* C_out, pepo_diag* diag_out);

/* Per-site Pauli weights of the last pepo_correlator call (Sec. 6.4 and
 * Appendix A.3: the non-identity weight n(r, t) is 1 - out[4 v + 0]): for
 * every site v the Hilbert-Schmidt weights of the Pauli components I, X, Y, Z
 * of its tensor with the converged double-layer messages contracted on every
 * leg, normalised to sum 1 per site.  out: host array of 4 * Lx * Ly doubles,
 * site-major.  Synchronises the stream.  Errors: PEPO_E_INVALID (bad
 * instance, NULL array), PEPO_E_CUDA.  Zero rows before the first
 * correlator call. */
pepo_status pepo_pauli_weights(pepo_ctx* ctx, int inst, double* out);

/* Vidal-normalised singular values of a bond (Eq. 12) from its last update.
 * lam_out: at least chi_max doubles; *chi_out receives the live chi. */
pepo_status pepo_get_spectrum(pepo_ctx* ctx, int inst, int bond, double* lam_out,
                              int* chi_out);

/* Copy a site tensor to the host in the canonical layout, multiplied by its
 * stored scale exp(sigma_v).  dims_out: 4 ints, the live chi of legs U, D, L,
 * R (0 for absent legs).  out: host doubles, capacity `count`. */
pepo_status pepo_get_site(pepo_ctx* ctx, int inst, int site, double* out, size_t count,
                          int* dims_out);

/* Overwrite the state of one instance: every site tensor (canonical layout,
 * concatenated in site order), every bond's chi and lambda, and every
 * directed message.  chi: nbonds ints; lam: nbonds * chi_max doubles (first
 * chi[b] used); msgs: nbonds * 2 * chi_max * chi_max doubles (row-major
 * chi[b] x chi[b] block at the start of each chi_max^2 slot).  Used to start
 * from a synthetic saturated state.  Synchronises the stream. */
pepo_status pepo_set_state(pepo_ctx* ctx, int inst, const double* sites, size_t count,
                           const int* chi, const double* lam, const double* msgs);

/* Set every bond's chi, lambda and both directed messages of one instance
 * (formats as in pepo_set_state).  Call before pepo_set_site when the bond
 * dimensions change.  Synchronises the stream. */
pepo_status pepo_set_bonds(pepo_ctx* ctx, int inst, const int* chi, const double* lam,
                           const double* msgs);

/* Overwrite one site tensor from host data in the canonical layout; dtype 0 =
 * float, 1 = double; count must equal 4 * prod(live chi of its legs).  The data
 * is staged in a scratch slab and permuted into the stored layout on the device
 * (the paper's tensor permutation, Sec. 4.1).  Resets the site's log-scale.
 * Synchronises the stream. */
pepo_status pepo_set_site(pepo_ctx* ctx, int inst, int site, const void* data, int dtype,
                          size_t count);

/* Snapshot of one instance's state (site tensors at their slab capacity,
 * live bond dimensions, lambda, double- and single-layer messages,
 * log-scales, discarded weights) for restarting from the same state.
 * dev_buf: device memory owned by the caller, at least pepo_state_bytes
 * bytes.  Device-to-device copies on the context's stream (asynchronous after
 * one synchronising read of the site pointers).  Not a step of the paper's
 * method. */
size_t pepo_state_bytes(const pepo_ctx* ctx, int inst);
pepo_status pepo_save_state(pepo_ctx* ctx, int inst, void* dev_buf, size_t bytes);
pepo_status pepo_load_state(pepo_ctx* ctx, int inst, const void* dev_buf, size_t bytes);

/* Checkpoint of one instance to host memory and restart from it (the
 * paper's long runs, Appendix A; not a step of the method): the same layout
 * as pepo_save_state (pepo_state_bytes bytes), copied between the device
 * state and the caller's host array host_buf (page-locked memory copies
 * fastest).  *steps_out receives the instance's step count, which
 * pepo_load_state_host restores from `steps` (the measurement history used
 * by the Sec. 6.3 C-drop check starts afresh).  Both synchronise the stream.
 * Errors: PEPO_E_INVALID (NULL context or buffer, bad instance, a buffer
 * smaller than pepo_state_bytes, steps < 0), PEPO_E_STATE (a step partly
 * applied), PEPO_E_CUDA. */
pepo_status pepo_save_state_host(pepo_ctx* ctx, int inst, void* host_buf, size_t bytes, int* steps_out);
pepo_status pepo_load_state_host(pepo_ctx* ctx, int inst, const void* host_buf, size_t bytes, int steps);

/* pepo_set_site without any memory allocation (the paper has no counterpart:
 * it is an interface variant, not a step of the method).  Same arguments and
 * result as pepo_set_site, but the host data is staged in a fixed 16 MiB
 * device buffer compiled into the library instead of the arena's scratch
 * slab, and dtype must be the storage type (0 = float for FP32 / TF32X3
 * contexts, 1 = double for FP64).  For callers that may not allocate or touch
 * the arena's scratch (device memory fully committed to the arena, or a
 * latency-bound loop where an allocation would synchronise the device).
 * Limit: 4 * prod(chi) * sizeof(storage) <= 16 MiB, else PEPO_E_INVALID with
 * the sizes in pepo_last_error.  The first call on each device looks up the
 * buffer's device address (call it with that device current, once, before
 * any stream capture).  Nothing in the buffer needs to start at zero.  Calls
 * that overlap in time share the buffer and race: serialise them.
 * Synchronises the stream. */
pepo_status pepo_set_site_static(pepo_ctx* ctx, int inst, int site, const void* data, int dtype,
                                 size_t count);

/* ---- Learned BP warm start ------------------------------------------------
 * The paper has no learned part (it motivates one by BP's sweep counts and
 * fixed-point traps, Sec. 6.3); this is an extension of the method.  Rows are (bond b, direction dir, Schmidt index k < chi_b)
 * in bond order, dir 0 = first site -> second site; pepo_ws_rows gives their
 * number (sum of 2 chi_b).  A row has PEPO_WS_FEATURES floats:
 *   log lam_k, k / chi_b, S_b / log chi_b, deg(src) / 4, deg(dst) / 4,
 *   |src - obs|_1 / (Lx + Ly), |dst - obs|_1 / (Lx + Ly), t = steps * dt, h,
 *   J, mean and max of S_e / log chi_e over the source site's other bonds.
 * The MLP maps a row to y = predicted log M_e[k, k] of the converged message
 * (trace-1 normalised, in the bond's Schmidt basis): widths 12 -> 256 -> 256
 * -> 1, exact (erf) GELU, weights and activations rounded to BF16 with FP32
 * accumulation, mean squared error, Adam (0.9, 0.999, 1e-8) on an FP32 master
 * copy.  Parameters are one float vector: W1 [12 x 256 row-major], b1 [256],
 * W2 [256 x 256], b2 [256], W3 [256], b3 [1] (pepo_mlp_num_params floats).
 * All *_dev pointers are device memory owned by the caller; calls are
 * asynchronous on the stream given at init unless stated otherwise. */
#define PEPO_WS_FEATURES 12
#define PEPO_WS_WIDTH 256
typedef struct pepo_mlp pepo_mlp;
long long pepo_mlp_num_params(void);
/* Device bytes for a network that trains / predicts up to max_rows rows. */
size_t pepo_mlp_required_bytes(int max_rows);
/* dev_buf: 256-byte aligned, pepo_mlp_required_bytes(max_rows) bytes, owned
 * by the caller.  params: host floats (initial weights).  Synchronises.
 * Errors: PEPO_E_INVALID, PEPO_E_OOM, PEPO_E_CUDA. */
pepo_status pepo_mlp_init(void* dev_buf, size_t bytes, int max_rows, const float* params,
                          void* cuda_stream, pepo_mlp** out);
/* FP32 master weights to the host.  Synchronises. */
pepo_status pepo_mlp_get_params(pepo_mlp* mlp, float* params_out);
/* y_dev[rows] = MLP(X_dev[rows x 12]). */
pepo_status pepo_mlp_forward(pepo_mlp* mlp, const float* X_dev, int rows, float* y_dev);
/* Forward + backward of the mean squared error against t_dev; keeps the
 * gradient for pepo_mlp_adam_step; loss_out / grad_host (num_params floats)
 * may be NULL.  Synchronises. */
pepo_status pepo_mlp_gradient(pepo_mlp* mlp, const float* X_dev, const float* t_dev, int rows,
                              float* loss_out, float* grad_host);
/* One Adam update with the last gradient. */
pepo_status pepo_mlp_adam_step(pepo_mlp* mlp, float lr);
void pepo_mlp_destroy(pepo_mlp* mlp);
/* The warm start inside pepo_bp_converge: dev_weights holds the network's
 * pepo_mlp_num_params FP32 parameters (layout above; device memory owned by
 * the caller, copied during the call).  From then on every pepo_bp_converge
 * first writes, for each instance created with warm_start = 1, the blended
 * start (1 - 0.25) d / sum d + 0.25 exp(y) / sum exp(y) into its messages
 * (features, forward pass and writer as pepo_ws_features / pepo_mlp_forward
 * / pepo_ws_apply); damped BP then runs to its tolerance as usual.  The arena
 * holds the workspace only when some instance has warm_start = 1.  Errors:
 * PEPO_E_INVALID (bytes != pepo_mlp_num_params * 4, NULL weights),
 * PEPO_E_STATE (no instance has warm_start = 1), PEPO_E_CUDA.  Synchronises
 * the stream. */
pepo_status pepo_set_warmstart_weights(pepo_ctx* ctx, const void* dev_weights, size_t bytes);
/* Row count of instance inst (-1 on error).  Synchronises. */
int pepo_ws_rows(pepo_ctx* ctx, int inst);
/* Feature rows of the current state into X_dev (rows beyond max_rows dropped). */
pepo_status pepo_ws_features(pepo_ctx* ctx, int inst, float* X_dev, int max_rows);
/* Training targets: log of the diagonal of the current (converged) messages. */
pepo_status pepo_ws_targets(pepo_ctx* ctx, int inst, float* t_dev, int max_rows);
/* Warm start: overwrite every message of the instance with the diagonal
 * (1 - gamma) d / sum d + gamma exp(y) / sum exp(y), d = the current diagonal
 * (diag(lambda) right after a Trotter step); gamma in [0, 1] (1 = the
 * prediction alone).  y_dev has pepo_ws_rows entries. */
pepo_status pepo_ws_apply(pepo_ctx* ctx, int inst, const float* y_dev, float gamma);

/* Change the BP settings of instance inst (-1: every instance) between
 * calls: damping alpha of Eq. 19 in (0, 1], tolerance tol > 0 of Eq. 14 and
 * the sweep budget (>= 1), for the following pepo_bp_converge and
 * pepo_correlator calls.  Used by the Sec. 6.3 trap remediation (retry BP
 * with another damping).  Synchronises the stream.  Errors: PEPO_E_INVALID
 * (a value out of range, a bad instance), PEPO_E_CUDA. */
pepo_status pepo_set_bp_params(pepo_ctx* ctx, int inst, double alpha, double tol, int max_sweeps);

/* All double-layer messages of instance inst as stored: 2 * num_bonds
 * messages of chi_max x chi_max doubles (message 2 b + dir, row-major, zero
 * outside the live chi x chi block).  pepo_get_messages copies them to the
 * host array out; pepo_set_messages replaces them from msgs (same layout),
 * e.g. to restart BP from the messages a snapshot holds.  Both synchronise
 * the stream.  Errors: PEPO_E_INVALID (bad instance, NULL array),
 * PEPO_E_CUDA. */
pepo_status pepo_get_messages(pepo_ctx* ctx, int inst, double* out);
pepo_status pepo_set_messages(pepo_ctx* ctx, int inst, const double* msgs);

/* Copy one directed message (chi x chi, row-major) to the host. */
pepo_status pepo_get_message(pepo_ctx* ctx, int inst, int bond, int dir, double* out,
                             int* chi_out);

/* Number of bonds of instance inst (0 on a bad argument). */
int pepo_num_bonds(const pepo_ctx* ctx, int inst);

/* Kernel-class timing (off by default).  When enabled, every launch is
 * bracketed by CUDA events on the context's stream and credited with its
 * algorithmic bytes and FLOPs, computed from the live bond dimensions read at
 * the start of each call (exact whenever chi does not change inside the call,
 * e.g. in the saturated regime).  The Householder class ("householder_tsqr")
 * is the exception: which sites take that branch is decided on the device,
 * so its FLOPs (2 m n^2 - 2 n^3 / 3 per factored m x n matrix) and bytes (one
 * read of it) are counted there, whether timing is on or not, and reset by
 * pepo_reset_timing.  Classes are numbered 0 .. pepo_timing_classes()-1. */
pepo_status pepo_set_timing(pepo_ctx* ctx, int enable);

int pepo_timing_classes(void);
const char* pepo_timing_class_name(int kclass);
/* Totals since the last reset: launches, milliseconds, algorithmic bytes and
 * FLOPs of one class.  Synchronises the stream. */
pepo_status pepo_get_timing(pepo_ctx* ctx, int kclass, long long* launches, double* ms,
                            double* bytes, double* flops);
pepo_status pepo_reset_timing(pepo_ctx* ctx);

/* Launch shapes of a context (batching and autotuning; the paper has no
 * counterpart).  The K range of a Gram is cut into splits reduced in FP64
 * afterwards: more splits fill more SMs when few Grams run at once, fewer
 * splits mean less partial traffic.  Results differ only in the rounding of
 * the split sums.  A field of 0 selects the default (free-leg Gram 64, row
 * Gram 32).  May be called at any time: a change synchronises the context's
 * stream and drops its captured CUDA graphs (captured again at their next
 * use).  PEPO_E_INVALID for a value outside 1..128 (gram_leg_splits) or
 * 1..64 (gram_rows_splits), PEPO_E_CUDA if the synchronisation fails; the
 * context is unchanged on error.  The tuning belongs to the caller-owned
 * struct only for the duration of the call. */
typedef struct {
  int gram_leg_splits;    /* free-leg Gram of a BP message (Eq. 13) / the absorb step */
  int gram_rows_splits;   /* Cholesky-QR Gram cv^T cv of the bond update (Eq. 10) */
} pepo_tuning;
pepo_status pepo_set_tuning(pepo_ctx* ctx, const pepo_tuning* tuning);
pepo_status pepo_get_tuning(const pepo_ctx* ctx, pepo_tuning* tuning);

/* Limit of every pipeline wait inside the tensor-core (PEPO_TF32X3) kernels,
 * in seconds, 1e-9 .. 60 (default 4).  A wait that runs longer makes its
 * kernel leave its loops, let its own MMAs and copies in flight finish
 * (bounded), free its tensor memory and return instead of hanging; the next
 * call that reads results (pepo_bp_converge, pepo_correlator) fails with
 * PEPO_E_CUDA and clears the kernel error word, so the context stays usable,
 * but its state is undefined until restored (pepo_load_state) or uploaded
 * again.  A change synchronises the stream and drops captured graphs.
 * Errors: PEPO_E_INVALID (value out of range), PEPO_E_CUDA.  Not a step of
 * the paper's method: failure handling of this implementation. */
pepo_status pepo_set_wait_limit(pepo_ctx* ctx, double seconds);

/* Sites factored by each branch of the hybrid QR (Sec. 4.2, Eq. 10) since the
 * last reset, over all instances: out[0] Householder by the branch rule,
 * out[1] Cholesky-QR, out[2] Cholesky-QR sites handed to Householder because
 * a pivot of their Gram kept too small a share of its column's diagonal.
 * `out` is host memory of 3 values; reset != 0 zeroes the counters after the
 * read.  Synchronises the stream.  Errors: PEPO_E_INVALID (null), PEPO_E_CUDA. */
pepo_status pepo_qr_branch_counts(pepo_ctx* ctx, long long* out, int reset);

/* Number of kernel launches enqueued by this context so far. */
long long pepo_launch_count(const pepo_ctx* ctx);

/* Last error message of the context (static string if ctx is NULL). */
const char* pepo_last_error(const pepo_ctx* ctx);

/* Release host-side resources.  Does not free the arena (the caller owns it). */
void pepo_destroy(pepo_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* PEPO_H */
