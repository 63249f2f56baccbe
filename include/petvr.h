/*
 * petvr.h -- C ABI of the GB300 (sm_103a) library for penalised PET
 * reconstruction by (variance-reduced) stochastic EM.
 *
 * The method is the one of Kereta, Twyman, Arridge, Thielemans and Jin,
 * "Stochastic EM methods with Variance Reduction for Penalised PET
 * Reconstructions": maximise Phi(f) = L(f) - beta R(f) over f >= 0 (§3,
 * Eq. (PET-MAP)) with the Poisson log-likelihood L of §2.1
 * (Eq. (log_likelihood)) split over ordered subsets of the sinogram rows
 * (§2.1, Eq. (subobjective)), by OSEM (§2.2, Eq. (Mstep)), SVREM (§2.3,
 * Eq. (tempsvrem), with the surrogate M-step of §3, Eq. (svrsurder)), and
 * preconditioned proximal SAGA / SVRG (§4, Eq. (saga_update),
 * Eq. (svrg_update)).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Pointers named d_* are CUDA device pointers (or managed memory) on the
 *   current device; pointers named h_* are host pointers.  The caller owns
 *   every buffer it passes; the library never frees them.  Objects created
 *   here (plan, problem, state) own only the device tables they allocate and
 *   borrow the caller's buffers, which must outlive them.
 * - Images are float32, nz independent slices of nx*ny pixels, laid out
 *   [iy][ix][z] (slice index innermost; nz = 1 is a plain [iy][ix] image).
 *   Sinograms are float32 [view][bin][z].  A "subset sinogram" holds only the
 *   views of one subset, in increasing view order ([view-in-subset][bin][z]).
 * - `stream` is a cudaStream_t (0 = the legacy default stream).  Every call
 *   is asynchronous on that stream unless documented as synchronising.
 * - Every call returns a pet_status.  Argument errors are detected on the
 *   host and returned immediately, with nothing enqueued.  CUDA launch or
 *   allocation errors return PET_ERR_CUDA / PET_ERR_OOM.  Numeric problems
 *   found by a kernel (a nonpositive expected count with positive data) are
 *   latched in a device status word and returned by the next synchronising
 *   call (pet_objective, pet_state_sync).  No call aborts the process.
 *   pet_last_error() gives a message for the calling thread's last failure.
 */
#ifndef PETVR_H
#define PETVR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PET_OK = 0,
    PET_ERR_INVALID = 1, /* bad argument, size or object                    */
    PET_ERR_OOM = 2,     /* device allocation failed                         */
    PET_ERR_CUDA = 3,    /* a CUDA runtime call or kernel launch failed      */
    PET_ERR_TIMEOUT = 4, /* reserved: a bounded device wait gave up          */
    PET_ERR_NUMERIC = 5, /* latched device-side numeric error                */
    PET_ERR_STATE = 6    /* call not valid for this object's algorithm/state */
} pet_status;

/* Algorithms (pet_state_create). */
enum { PET_ALGO_OSEM = 0, PET_ALGO_SVREM = 1, PET_ALGO_SAGA = 2, PET_ALGO_SVRG = 3,
       PET_ALGO_SGA = 4, PET_ALGO_SEM = 5, PET_ALGO_SAGAEM = 6 };
/* SAGA gradient-table storage (pet_state_create). */
enum { PET_TABLE_FP32 = 0, PET_TABLE_BF16 = 1 };
/* Preconditioner of SAGA and SVRG (pet_state_set_preconditioner). */
enum { PET_PRECOND_CONSTANT = 0, PET_PRECOND_ITERATE = 1 };
/* How pet_batch_epoch runs a batch's updates (pet_batch_set_mode). */
enum { PET_BATCH_PHASES = 0, PET_BATCH_DATAFLOW = 1, PET_BATCH_STREAMS = 2 };
/* Potentials of the pairwise penalty (Table 1, t = f_n - f_j, delta > 0):
 * quadratic t^2/2; Huber t^2/2 for |t| <= delta else delta|t| - delta^2/2;
 * log cosh delta^2 log cosh(t/delta); hyperbola delta^2 (sqrt(1+(t/delta)^2) - 1)
 * (the form whose derivative is Table 1's t / sqrt(1+(t/delta)^2)). */
enum { PET_POT_QUADRATIC = 0, PET_POT_HUBER = 1, PET_POT_LOGCOSH = 2, PET_POT_HYPERBOLA = 3 };

/* 2-D parallel-beam geometry (optionally a stack of nz independent slices).
 * Pixel (ix, iy) is the half-open square [x_min + ix d, x_min + (ix+1) d) x
 * [y_min + iy d, ...) with x_min = -nx d / 2, y_min = -ny d / 2, d = pixel_mm.
 * View i is at theta_i = i pi / n_angles; bin j at s_j = (j - (n_bins-1)/2)
 * bin_mm (bin_mm <= 0 means bin_mm = pixel_mm).  Ray (i, j) is the line
 * x cos(theta_i) + y sin(theta_i) = s_j and a_mn is its length (mm) inside
 * pixel n: the exact Siddon intersection length (the paper's forward model is
 * a Radon transform, §5.1; A is any nonnegative system matrix, §2.1).
 * Limits: nx, ny <= 16384, n_angles <= 1024, nx*ny*nz and n_angles*n_bins*nz
 * below 2^31.
 *
 * n_rings = 0: nz independent slices (a stack of 2-D problems), sinograms
 * [view][bin][z].  n_rings >= 1: a multi-ring scanner with fully 3-D lines
 * of response (the torso data of §5.3 come from 2 rings).  The image is a
 * volume of nz layers, each slice_mm thick, centred on z = 0; voxel
 * (ix, iy, iz) is half-open in z as in x and y, stored [iy][ix][iz].  Ring r
 * sits at z_r = (r - (n_rings-1)/2) ring_mm on a detector cylinder of radius
 * radius_mm, which must exceed every |s_j|.  Line (i, j, r1, r2) is ray
 * (i, j) in the transaxial plane, meeting the cylinder at t = -T on ring r1
 * and t = +T on ring r2 (t the transaxial arc length, T = sqrt(R^2 - s_j^2)),
 * so z(t) = (z_r1 + z_r2)/2 + t (z_r2 - z_r1) / (2T); a_mn is its 3-D length
 * inside voxel n.  Sinograms are [view][bin][pair], pair = r1 n_rings + r2
 * (every ordered pair), and the penalty couples the two axial neighbours
 * too (6-neighbourhood).  n_rings <= 4.  Fields after bin_mm are ignored when
 * n_rings = 0, so a zero-initialised tail selects the stacked 2-D mode. */
typedef struct {
    int32_t nx, ny, nz;
    double pixel_mm;
    int32_t n_angles, n_bins;
    double bin_mm;
    int32_t n_rings;
    double ring_mm, radius_mm, slice_mm;
} pet_geometry;

/* Ordered subsets (§2.1): scheme 0 = angle-interleaved, view i belongs to
 * subset i mod n_subsets (1 <= n_subsets <= n_angles). */
typedef struct {
    int32_t n_subsets;
    int32_t scheme;
} pet_subsets;

/* Penalty beta R(f), R = 1/2 sum_n sum_{j in N4(n)} rho(f_n - f_j) (§3). */
typedef struct {
    int32_t potential; /* PET_POT_* */
    float beta;        /* >= 0 */
    float delta;       /* > 0; unused by the quadratic potential */
} pet_penalty;

typedef struct pet_plan pet_plan;
typedef struct pet_problem pet_problem;
typedef struct pet_state pet_state;
typedef struct pet_batch pet_batch;

/* ---- plan: geometry tables and sensitivities ---------------------------- */

/* Build the per-view and per-ray geometry tables on the current device and
 * the subset sensitivities sens_t = A_t^T 1 and sens = A^T 1 (the
 * denominators of §2.2, Eq. (Mstep)).  Synchronises the legacy stream once.
 * *out is set on success and must be released with pet_plan_destroy. */
pet_status pet_plan_create(const pet_geometry *geom, const pet_subsets *subsets, pet_plan **out);
void pet_plan_destroy(pet_plan *plan);

/* Number of views in subset t (t in [0, n_subsets)), or of all views for
 * t = -1; the subset sinogram of t has n_views * n_bins * nz floats. */
pet_status pet_plan_subset_views(const pet_plan *plan, int32_t t, int32_t *h_n_views);

/* Number of nonzeros of A_t (t >= 0) or of A (t = -1) for one slice: the
 * (ray, pixel) pairs with a positive intersection length, counted on the
 * device when the plan is built.  This is the algorithmic work of one
 * projection (one multiply-add per nonzero). */
pet_status pet_plan_nnz(const pet_plan *plan, int32_t t, int64_t *h_nnz);

/* Launch shapes of the single-slice kernels: band chunks per ray in the
 * forward projector (8, 16 or 32; 0 = size-based default) and pixels per run
 * in the tiled back projector (4 or 8).  The chunk count is the one of subset
 * projections; full-data forward passes (objectives, anchor ratios, all-view
 * projections) of images large enough to fill the GPU several times over use
 * half as many, but not fewer than 16.  Results are identical up to the FP32
 * summation order.  Set them before creating states: captured epochs keep the
 * shapes they were captured with. */
pet_status pet_plan_set_tuning(pet_plan *plan, int32_t fwd_chunks, int32_t back_run);
pet_status pet_plan_get_tuning(const pet_plan *plan, int32_t *h_fwd_chunks, int32_t *h_back_run);

/* Autotuner: times every forward chunk count and back-projection run length
 * on this plan's own geometry (all subsets, best of three passes on a
 * private stream, synchronising), keeps the fastest of each, and reports them
 * (either pointer may be NULL).  Allocates and frees scratch images.  Slice
 * stacks have nothing to tune. */
pet_status pet_plan_autotune(pet_plan *plan, int32_t *h_fwd_chunks, int32_t *h_back_run);

/* Device bytes a plan holds, and the bytes pet_problem_create would
 * allocate for a problem on it (with a background sinogram if has_bg): the
 * admission figures of a serving loop, beside pet_state_create's query. */
pet_status pet_plan_bytes(const pet_plan *plan, size_t *h_bytes);
pet_status pet_problem_bytes(const pet_plan *plan, int32_t has_bg, size_t *h_bytes);
/* The bytes pet_state_create would allocate for `algo` on any problem of plan. */
pet_status pet_plan_state_bytes(const pet_plan *plan, int32_t algo, int32_t table_dtype, size_t *h_bytes);

/* Copy sens_t (t >= 0) or sens (t = -1), nx*ny floats, into d_out. */
pet_status pet_plan_sensitivity(const pet_plan *plan, int32_t t, float *d_out, void *stream);

/* ---- projectors ----------------------------------------------------------- */

/* Forward projection y = A_t f + w (§2.1, Eq. (voxel_td)).  subset = -1
 * projects every view into a full sinogram; subset = t writes the subset
 * sinogram of t.  d_bg (same layout as d_sino) may be NULL, then the scalar
 * bg is added to every ray.  d_img and d_sino must not overlap. */
pet_status pet_forward(const pet_plan *plan, const float *d_img, const float *d_bg, float bg,
                       int32_t subset, float *d_sino, void *stream);

/* Back projection b = A_t^T y (the adjoint of pet_forward without the
 * background; used in every update of §2.2-§4).  d_sino is the subset
 * sinogram of t (full sinogram for subset = -1); d_img receives b. */
pet_status pet_back(const pet_plan *plan, const float *d_sino, int32_t subset, float *d_img,
                    void *stream);

/* ---- problem: data, background and penalty -------------------------------- */

/* Bind counts g (full sinogram, float32, [view][bin][z]), background w
 * (full sinogram, or NULL for the scalar bg) and the penalty.  The data are
 * copied into subset-major device order, so d_counts / d_bg may be freed
 * after the call returns and the stream has drained. */
pet_status pet_problem_create(const pet_plan *plan, const float *d_counts, const float *d_bg,
                              float bg, const pet_penalty *pen, pet_problem **out, void *stream);
void pet_problem_destroy(pet_problem *problem);

/* Replace the counts (and background) of an existing problem in place, with
 * the same layouts and rules as pet_problem_create; nothing is allocated.
 * d_bg must be non-NULL exactly when the problem was created with a
 * background sinogram.  States of this problem keep working: a new scalar
 * background makes them re-capture their cached epoch graphs at their next
 * call (new counts need no re-capture). */
pet_status pet_problem_update(pet_problem *problem, const float *d_counts, const float *d_bg, float bg,
                              void *stream);

/* Warm start (every method of §5.1 starts from one OSEM epoch): write the constant
 * image f_u = sum_m max(g_m - w_m, 0) / sum_n (A^T 1)_n into d_img, then run
 * one unpenalised OSEM epoch in cyclic subset order on it.  Its scratch is the
 * problem's own, so warm starts of one problem must be ordered on one stream
 * (pet_run_to_gap warm-starts its workers with their states' own scratch). */
pet_status pet_warm_start(const pet_problem *problem, float *d_img, void *stream);

/* Objective Phi(f) = sum_m (g_m log yhat_m - yhat_m) - beta R(f), with
 * yhat = A f + w, reduced in FP64 (§2.1, Eq. (log_likelihood); §3,
 * Eq. (PET-MAP)).  Synchronising: returns after *h_phi is written.  Returns
 * PET_ERR_NUMERIC if some yhat_m <= 0 with g_m > 0; *h_phi is then -inf (the
 * log-likelihood of a nonpositive mean with positive data). */
pet_status pet_objective(const pet_problem *problem, const float *d_img, double *h_phi, void *stream);

/* The same objective, enqueued only: d_phi (device, 3 doubles) receives
 * {Phi, L, R} when the stream reaches it.  Numeric errors are latched and
 * reported by the next synchronising call.  Calls on one problem share its
 * reduction scratch, so they must be ordered on one stream. */
pet_status pet_objective_async(const pet_problem *problem, const float *d_img, double *d_phi, void *stream);

/* Objective {Phi, L, R} of d_img into d_phi (device, 3 doubles) without any
 * device allocation, for callers that cannot call cudaMalloc: code whose
 * device memory is owned by a framework or serving allocator (a caching
 * allocator or a fixed pool that must account for every byte) and code on a
 * latency path that cannot take cudaMalloc's implicit synchronisation.  The
 * paper has no counterpart; it is an interface convenience.
 * Inputs as for pet_problem_create (counts and optional background as full
 * sinograms in view order, [view][bin][z]) plus the quadratic penalty weight
 * beta; no problem object is needed.  The reduction scratch is a fixed
 * 1 MiB array (131072 doubles) in this library's device memory, which every
 * device that loads the library holds until the process exits.  Sizes that
 * need more block partials than that (roughly more than 1M rays x 32 lanes or
 * 33M pixels) are rejected with PET_ERR_INVALID and a message.  The first
 * call on each device looks the array's device address up (with that device
 * current), so make that first call before any stream capture.  All calls
 * share the array and every call overwrites the partials it uses, so calls
 * that overlap on the GPU (different streams, or different threads) race:
 * order them on one stream.  A ray with a nonpositive expected count and
 * positive data makes Phi and L come out -inf (their true value); this entry
 * point has no status word to latch it in (pet_objective also returns
 * PET_ERR_NUMERIC for it).  The current device must be the plan's device
 * (else PET_ERR_INVALID).  Every ray's expected count is the one
 * pet_objective computes; only the FP64 summation order of the per-ray terms
 * differs.  Multi-ring plans are rejected with PET_ERR_INVALID (their penalty
 * couples layers; use pet_objective_async).  Enqueued only. */
pet_status pet_objective_noalloc(const pet_plan *plan, const float *d_img, const float *d_counts,
                                 const float *d_bg, float bg, float beta, double *d_phi, void *stream);

/* ---- state: one running reconstruction ------------------------------------ */

/* Create the state of `algo` on the image d_img_inout (borrowed: every epoch
 * call reads the current iterate from it and leaves the new one there).
 * SAGA and SVRG freeze the preconditioner d = N_s f^(0) / A^T 1 at this
 * image (§4: constant d = d(f^(0))); SAGA also fills its gradient table with
 * grad Phi_t(f^(0)) for every t (one full pass), enqueued on `stream`.
 * If out == NULL only *bytes_needed (device bytes this state would
 * allocate) is computed: an admission query that allocates nothing. */
pet_status pet_state_create(const pet_problem *problem, int32_t algo, int32_t table_dtype,
                            float *d_img_inout, size_t *bytes_needed, pet_state **out,
                            void *stream);
pet_status pet_state_destroy(pet_state *state);

/* Restart the state from the image currently in its d_img_inout buffer, as
 * pet_state_create would (update counter to 0, SAGA table / SVRG and SAGA
 * preconditioner recomputed, SVREM statistic re-initialised at the next
 * anchor), without allocating: a slot can serve a new reconstruction.
 * Enqueued on `stream`. */
pet_status pet_state_reset(pet_state *state, void *stream);

/* Preconditioner of a SAGA or SVRG state's updates (§4).
 * PET_PRECOND_CONSTANT (the default): d = N_s f^(0) / A^T 1, frozen at the
 *   state's starting image (§4: the remedy of freezing the preconditioner;
 *   0 where A^T 1 = 0).
 * PET_PRECOND_ITERATE: d_t(f^k) = f^k / A_t^T 1 of Eq. (preconditioners),
 *   recomputed at every update from the current iterate and the subset's
 *   sensitivity, as Eqs. (saga_update) and (svrg_update) print it (0 where
 *   A_t^T 1 = 0).
 * Takes effect from the next update; the SAGA table and the SVRG anchor are
 * left as they are.  Returns PET_ERR_INVALID for another algorithm or kind.
 * Host-side only (no stream work). */
pet_status pet_state_set_preconditioner(pet_state *state, int32_t kind);

/* n_iter updates (an epoch is n_iter = n_subsets) with subset indices
 * h_subset_seq[0..n_iter-1], each in [0, n_subsets).  The update counter k
 * persists across calls; anchors are refreshed when k mod (eta N_s) == 0.
 *
 * OSEM  (§2.2, Eq. (Mstep) with the penalised surrogate of §3):
 *       f <- root(a = f . A_t^T(g_t / yhat_t), sens_t, beta / N_s).
 * SVREM (§2.3, Eq. (tempsvrem); §3 M-step with sens and beta):
 *       s <- (1-alpha) s + alpha (tau_t(f) - tau_t(f_anc) + s_anc).
 * SAGA  (§4, Eq. (saga_update)): f <- P>=0(f + alpha d (q_new - q_t + mean q)).
 * SVRG  (§4, Eq. (svrg_update)):
 *       f <- P>=0(f + alpha d (grad Phi_t(f) - grad Phi_t(f_anc) + q~)).
 * Returns PET_ERR_STATE if the state was created for another algorithm.
 *
 * The subset sequence is copied to the device first; the launches of an
 * epoch are captured once into a CUDA graph (keyed by n_iter, alpha, eta and
 * where anchors fall) and replayed on later calls with the same key, so the
 * first call with a new key costs a capture.  All calls on one state must be
 * ordered on one stream, and a state's first call with a new key should not
 * come while `stream` is itself being captured.  A state (and a batch) keeps
 * at most 64 captured graphs; past that the least recently launched one is
 * destroyed (freed by the driver once any launch of it completes).  Setting
 * the environment variable PETVR_NO_GRAPHS=1 issues the launches directly
 * instead. */
pet_status pet_osem_epoch(pet_state *state, const int32_t *h_subset_seq, int32_t n_iter, void *stream);
pet_status pet_svrem_epoch(pet_state *state, float alpha, int32_t eta, const int32_t *h_subset_seq,
                           int32_t n_iter, void *stream);
pet_status pet_saga_epoch(pet_state *state, float alpha, const int32_t *h_subset_seq, int32_t n_iter,
                          void *stream);
pet_status pet_svrg_epoch(pet_state *state, float alpha, int32_t eta, const int32_t *h_subset_seq,
                          int32_t n_iter, void *stream);

/* Objective {Phi, L, R} of the state's current image into d_phi (device,
 * 3 doubles), enqueued only, using the state's own reduction scratch (so
 * states of one problem may evaluate it on different streams). */
pet_status pet_state_objective_async(pet_state *state, double *d_phi, void *stream);

/* ---- batches: many reconstructions per launch ------------------------------ */

/* Group n existing states (any algorithms; single-slice plans of any sizes;
 * each state at most once) so that their updates run together (the batched
 * form of the reconstructions, with per-member geometry, data and subset
 * indices).  Every update of pet_batch_epoch runs as persistent phases: one
 * resident grid, sized to the GPU, claims the forward-projection work items
 * of every member (ray blocks of the member's current subset, and of all its
 * views where its anchor pass is due); then one resident grid per potential
 * class claims the back-projection + update items (16 x 16 tiles, and the
 * anchor passes' (subset, tile) items).  An update with anchors due runs the
 * anchor back projections beside the other members' updates, then the anchor
 * finishes, then the anchored members' updates.  Each member's result is
 * bit-identical to running its own epoch call with the same subset sequence
 * (each work item is one block of the member's own launch).  The batch
 * borrows the states, which must outlive it; a state in a batch may still be
 * used on its own between batch calls. */
pet_status pet_batch_create(pet_state *const *states, int32_t n, pet_batch **out);
pet_status pet_batch_destroy(pet_batch *batch);

/* Whether pet_batch_epoch captures and replays CUDA graphs (default on).
 * A batch whose membership changes every few calls (a serving loop) is
 * cheaper without: each new batch would otherwise pay one capture. */
pet_status pet_batch_set_graphs(pet_batch *batch, int32_t on);

/* n_iter updates of every member: h_subset_seqs is row-major [n][n_iter]
 * (member j's subset indices), h_alpha[j] and h_eta[j] its step size and
 * anchor period (ignored where the algorithm has none).  Anchor passes are
 * due per member as in the single-state calls.  Captured into a CUDA graph
 * keyed by n_iter and the anchor pattern, like pet_*_epoch. */
pet_status pet_batch_epoch(pet_batch *batch, const int32_t *h_subset_seqs, int32_t n_iter, const float *h_alpha,
                           const int32_t *h_eta, void *stream);

/* Objectives {Phi, L, R} of every member's current image into d_phi
 * (device, [n][3] doubles), enqueued only. */
pet_status pet_batch_objective_async(pet_batch *batch, double *d_phi, void *stream);

/* How pet_batch_epoch runs the updates (the same results either way, bit for
 * bit, and the same as each member's own epoch calls):
 *   PET_BATCH_PHASES (default): per update, persistent phases separated by
 *     kernel boundaries (see pet_batch_create);
 *   PET_BATCH_DATAFLOW: one launch for the whole call.  Its resident grid
 *     claims the stages of every update of every member from one work list in
 *     which each stage waits only for the earlier stages of its own member
 *     (the previous update's back projection, its own forward projection, the
 *     anchor pass when due), so the members' phases overlap instead of meeting
 *     at a kernel boundary after every phase.  The waits are bounded (see
 *     pet_batch_set_wait_limit).  Applies when every member uses the same
 *     potential class (quadratic, or edge-preserving); otherwise the batch
 *     runs in phases;
 *   PET_BATCH_STREAMS: every member's own epoch call (and objective call),
 *     its captured graphs, member j on stream j mod k of k <= 8 streams the
 *     batch creates on first use, which wait for `stream` and which `stream`
 *     then waits for. */
pet_status pet_batch_set_mode(pet_batch *batch, int32_t mode);

/* PET_BATCH_DATAFLOW only: how many times a block polls (with a short sleep
 * between polls: a few seconds at the default 2^22) for a stage it waits for
 * before it gives up: the kernel then latches PET_ERR_TIMEOUT in the batch's
 * status word, the remaining work items skip their work and the launch ends;
 * the members' iterates are then not valid.  0 fails any wait that is not
 * already satisfied (a way to exercise that path).  polls < 0 is refused. */
pet_status pet_batch_set_wait_limit(pet_batch *batch, int64_t polls);

/* Synchronise `stream` and read the batch's status word: PET_ERR_TIMEOUT if a
 * dependency wait ran out since the last call (the word is then cleared),
 * PET_OK otherwise. */
pet_status pet_batch_sync(pet_batch *batch, void *stream);

/* The paper's non-variance-reduced baselines on the same kernels (§5.1),
 * with step alpha_k = alpha0 / (decay k + 1), k the state's update counter:
 * SGA   (§4, Eq. (sga)): f <- P>=0(f + alpha_k (f / A_t^T 1) . grad Phi_t(f));
 *       decay = 0, alpha0 = 1 is SGA; decay = 0.001 is the subset-dependent
 *       BSREM of §5.1.  State algorithm PET_ALGO_SGA.
 * SEM   (§2.3, Eq. (tempsem)): s <- (1 - alpha_k) s + alpha_k tau_t(f), then
 *       the M-step of §3 with A^T 1 and beta; s starts at s(f^(0)) (one full
 *       pass on the first call).  State algorithm PET_ALGO_SEM. */
pet_status pet_sga_epoch(pet_state *state, float alpha0, float decay, const int32_t *h_subset_seq,
                         int32_t n_iter, void *stream);
pet_status pet_sem_epoch(pet_state *state, float alpha0, float decay, const int32_t *h_subset_seq,
                         int32_t n_iter, void *stream);

/* SAGA on the EM statistic (§2.3, the remark after Eq. (tempsvrem)):
 * s <- (1-alpha) s + alpha (tau_t(f) - T_t + mean_t T_t), the M-step of §3,
 * then T_t <- tau_t(f) for the subset just used; the table starts at
 * tau_t(f^(0)) (one full pass at state creation).  PET_ALGO_SAGAEM. */
pet_status pet_sagaem_epoch(pet_state *state, float alpha, const int32_t *h_subset_seq, int32_t n_iter,
                            void *stream);

/* n_iter updates of the state's own algorithm with the objective inside:
 * the updates of the epoch call of that algorithm (the same sequence rules,
 * anchors and update counter; step alpha_k = alpha / (decay k + 1) for every
 * algorithm that takes a step, ignored by OSEM; eta used by SVREM and SVRG
 * only), and, when objective_every > 0, after every objective_every-th update
 * of this call the objective {Phi, L, R} (§3, Eq. (PET-MAP)) of the
 * iterate then reached, written to d_phi[3 j], d_phi[3 j + 1], d_phi[3 j + 2]
 * for the j-th such point (j from 0; device, 3 * floor(n_iter /
 * objective_every) doubles, owned by the caller).  The results are those of
 * the epoch calls with pet_state_objective_async between them, bit for bit.
 *
 * Where an objective's iterate is the anchor of the next update (SVREM and
 * SVRG at k mod (eta N_s) == 0, inside this call), that anchor's full-data
 * ratios g / (A f + w) are the objective's own forward projection: one
 * forward pass serves both, and the anchor pass starts from its back
 * projection.  Across calls nothing is shared (the image may change between
 * calls).  Graph capture as for the epoch calls (keyed also by
 * objective_every and d_phi).  objective_every < 0, or objective_every > 0
 * with d_phi null, is refused with PET_ERR_INVALID; eta < 1 for SVREM/SVRG
 * and non-finite alpha or decay (decay < 0) as in the epoch calls. */
pet_status pet_state_run(pet_state *state, const int32_t *h_subset_seq, int32_t n_iter, float alpha, float decay,
                         int32_t eta, int32_t objective_every, double *d_phi, void *stream);

/* Executor: n_jobs reconstructions of one problem and method, each run to a
 * relative objective gap (phi_star - Phi(f)) / |phi_star| <= gap (§5.1, the
 * paper's convergence measure, with phi_star the caller's reference optimum)
 * or to max_epochs epochs, up to n_workers at a time.  The workers are
 * distinct states of one problem and algorithm, each with its own image; each
 * runs on a CUDA stream of its own that the call creates.  Job j takes the
 * next free worker: the warm start of pet_warm_start into the worker's image
 * (with the worker's own scratch), the state's reset (pet_state_reset), then
 * epochs of the worker's algorithm (the epoch calls' updates, step alpha_k =
 * alpha / (decay k + 1) where the algorithm takes one, eta for SVREM and
 * SVRG), the j-th subset sequence h_seqs[j * max_epochs * N_s ...] (host,
 * max_epochs * N_s indices per job), each epoch followed by its objective,
 * which the host reads before it launches the job's next epoch or retires it.
 * The workers start after the work already enqueued on `stream`; the call
 * returns when every job is done (synchronising).
 *
 * Per job (host arrays of n_jobs): h_epochs[j] the epochs run, h_gap[j] the
 * relative gap after the last one, h_ms[j] the host time from the job's start
 * (its warm start enqueued) to the host reading its last objective.  With
 * d_results (device, n_jobs times the image size, or null) each job's final
 * image is copied there.  A job's results are those of the same warm start,
 * reset, epoch calls and objective calls on one stream, bit for bit.  SAGA and
 * SAGA-EM resets fill their tables through the problem's scratch and run one
 * after another.  Refused with PET_ERR_INVALID before any CUDA call: no or
 * null workers, workers of different problems or algorithms, repeated workers
 * or images, n_jobs < 0, max_epochs < 1, null host arrays (n_jobs > 0), a
 * non-finite or zero phi_star, a negative or non-finite gap, alpha/decay/eta
 * as in the epoch calls, a subset index outside [0, N_s).  A device-side
 * numeric error latched meanwhile is returned at the end (PET_ERR_NUMERIC). */
pet_status pet_run_to_gap(pet_state *const *workers, int32_t n_workers, int32_t n_jobs, const int32_t *h_seqs,
                          int32_t max_epochs, float alpha, float decay, int32_t eta, double phi_star, double gap,
                          float *d_results, int32_t *h_epochs, double *h_gap, double *h_ms, void *stream);

/* The executor for reconstructions that each have their own state (any
 * problems, plans and algorithms, e.g. a batch of independent
 * reconstructions): job j runs on states[j] (which keeps its final image)
 * with its own subset sequence h_seqs[j] (host, max_epochs * N_s indices of
 * its plan), step h_alpha[j] / (h_decay[j] k + 1), anchor period h_eta[j]
 * (as the epoch calls take them) and reference optimum h_phi_star[j], up to
 * n_streams jobs at a time, each on a stream the call creates; otherwise as
 * pet_run_to_gap (warm start, reset, epochs with the objective after each
 * until the gap or max_epochs; outputs h_epochs, h_gap, h_ms per job;
 * synchronising).  Refused with PET_ERR_INVALID: null arrays, states or
 * sequences, repeated states or images, n_streams < 1, and the argument
 * checks of pet_run_to_gap per job. */
pet_status pet_run_jobs_to_gap(pet_state *const *states, const int32_t *const *h_seqs, const float *h_alpha,
                               const float *h_decay, const int32_t *h_eta, const double *h_phi_star, int32_t n_jobs,
                               int32_t n_streams, int32_t max_epochs, double gap, int32_t *h_epochs, double *h_gap,
                               double *h_ms, void *stream);

/* pet_run_jobs_to_gap for jobs that arrive over time: job j may start only
 * once h_arrival_s[j] seconds (finite, >= 0, nondecreasing in j) have passed
 * since the call, and jobs start in index order on the first free stream.
 * Outputs per job: h_epochs, h_gap as above, and h_start_ms[j], h_done_ms[j]:
 * when it started and when the host read its last objective, in milliseconds
 * since the call (its latency is h_done_ms[j] - 1000 h_arrival_s[j]).  The host
 * loop sleeps while no job runs and the next is more than 2 ms away, and spins
 * otherwise.  Argument errors as for
 * pet_run_jobs_to_gap, and bad arrival times, with PET_ERR_INVALID. */
/* A request of pet_serve_requests (host data; the plan is the caller's). */
typedef struct {
    const pet_plan *plan;
    const float *h_counts;   /* host float32 counts, the plan's sinogram layout (as pet_problem_create) */
    float bg;                /* uniform background per bin */
    pet_penalty penalty;
    int32_t algo, table_dtype;
    const int32_t *h_seq;    /* max_epochs * N_s subset indices of the plan */
    float alpha, decay;      /* step alpha / (decay k + 1), as the epoch calls take it */
    int32_t eta;             /* SVREM / SVRG anchor period */
    double phi_star;         /* reference optimum of the request's objective */
    double arrival_s;        /* seconds after the call; nondecreasing over the requests */
    float *h_image;          /* host, the plan's image size: the result; or null */
} pet_request;

/* What pet_serve_requests did with its device-memory budget. */
typedef struct {
    size_t peak_bytes;       /* most bytes its slots held at once */
    int32_t slots_created, slots_reused, slots_evicted, admissions_deferred;
} pet_serve_stats;

/* A request stream served to the objective gap with admission by a device
 * memory budget, the whole loop in C++: request j is admitted once
 * arrival_s seconds have passed since the call, a stream of the n_streams the
 * call creates is free, and a slot fits the budget; a slot is a problem
 * (pet_problem_create on the request's counts, uploaded through a staging
 * buffer), a state (pet_state_create) and an image, and is kept after the
 * request ends for the next request of the same plan, algorithm, table and
 * penalty (pet_problem_update with the new counts and background), or freed,
 * least recently used first, when an admission needs its bytes.  A slot's
 * bytes are pet_problem_bytes + pet_plan_state_bytes + its staging and image.
 * While the next request does not fit, it and those after it wait (in order)
 * for a running request to end.  Each request then runs as a job of
 * pet_serve_jobs (warm start, reset, epochs with the objective after each,
 * until the gap or max_epochs) and its final image is copied to h_image.
 * Outputs per request: h_epochs, h_gap, h_start_ms, h_done_ms as for
 * pet_serve_jobs; *stats for the call.  Synchronising.  Refused with
 * PET_ERR_INVALID before any CUDA call: null arrays, a request with a null
 * plan, counts or sequence, an unknown algorithm or table type, a non-finite
 * background, a non-finite or zero phi_star, bad arrival times, alpha/decay/
 * eta as in the epoch calls, a subset index out of range, or a request whose
 * slot alone exceeds the budget.  A numeric error latched by a request's
 * problem is returned when its slot is freed or at the end. */
pet_status pet_serve_requests(const pet_request *reqs, int32_t n, int32_t n_streams, size_t budget_bytes,
                              int32_t max_epochs, double gap, int32_t *h_epochs, double *h_gap, double *h_start_ms,
                              double *h_done_ms, pet_serve_stats *stats, void *stream);

pet_status pet_serve_jobs(pet_state *const *states, const int32_t *const *h_seqs, const float *h_alpha,
                          const float *h_decay, const int32_t *h_eta, const double *h_phi_star,
                          const double *h_arrival_s, int32_t n_jobs, int32_t n_streams, int32_t max_epochs, double gap,
                          int32_t *h_epochs, double *h_gap, double *h_start_ms, double *h_done_ms, void *stream);

/* Synchronise `stream` and return any latched device-side error. */
pet_status pet_state_sync(pet_state *state, void *stream);

/* Number of kernels this library has launched in this process (all threads),
 * kernels replayed from its captured graphs included. */
uint64_t pet_kernel_launches(void);

/* Optional per-kernel timing for profiling: while enabled, every forward and
 * back-projection launch is bracketed by two CUDA events on its stream.
 * pet_profile_read synchronises those events and returns, for kernel kind
 * `kind` (0 forward projection of an update's subset, 1 back projection with
 * update epilogue, 2 multi-subset back projection of an anchor pass or table
 * fill, 3 forward projection of all rays or an API call), the number of launches
 * and their summed duration in ms since the last reset.  Not thread-safe
 * with respect to concurrent launches from several host threads. */
pet_status pet_profile_enable(int32_t on);
pet_status pet_profile_reset(void);
pet_status pet_profile_read(int32_t kind, int64_t *h_launches, double *h_total_ms);

/* Message for the calling thread's most recent failed call ("" if none). */
const char *pet_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* PETVR_H */
