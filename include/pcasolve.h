/*
 * pcasolve.h -- C ABI of the GB300 (sm_103a) single-projection PCA lung-motion
 * solver: Li et al., "3D tumor localization through real-time volumetric x-ray
 * imaging for lung cancer radiotherapy", arXiv:1102.1712.
 *
 * The method (Sec. II.A and Appendix): a reference CT f0 is deformed by the
 * PCA motion model x = xbar + U w (Eq. 1), projected to a digitally
 * reconstructed radiograph P f, and w is fitted to one measured cone-beam
 * projection y by minimising J = ||P f - a y - b||^2 (Eq. 2), alternating the
 * intensity fit (Eq. A.1) with normalised gradient steps under Armijo
 * backtracking (Eq. A.2).  The tumour is then located by inverting the DVF at
 * its reference centroid (Sec. II.A, fixed point of Chen et al.).
 *
 * Conventions shared by every call
 * --------------------------------
 * Memory.  Pointers documented "device" are CUDA device pointers owned by the
 *   caller; pointers documented "host" are ordinary host memory.  No call
 *   allocates device memory: calls that need scratch take a caller-provided
 *   device workspace sized by pcas_workspace_bytes().
 * Streams.  `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *   stream).  Calls whose outputs are device arrays only enqueue work and
 *   return; calls with host outputs (marked "synchronous") block until those
 *   outputs are ready.
 * Volumes.  float32, layout [nz][ny][nx] (x fastest), voxel (i,j,k) centred
 *   at (ox + i sx, oy + j sy, oz + k sz) mm.  Values outside the grid are 0.
 *   Size limits (PCAS_ERR_INVALID_ARG beyond them): ny, nz <= 65535,
 *   (m + 10)(m + 4)(nz + 4) < 2^31 with m = max(nx, ny), and
 *   (nx + 6)(ny + 6)(nz + 6) < 2^31.
 * Motion model.  mean: [3][N] float32 mm (may be NULL = zero mean field);
 *   U: [K][3][N] float32 mm, component 0 = x (lateral), 1 = y (AP),
 *   2 = z (SI), N = nx ny nz; 1 <= K <= PCAS_KMAX.
 * Images.  float32, layout [nv][nu] (u fastest).
 * Geometry (a reading; the paper does not state axes).  Gantry rotation about
 *   z through the world origin; source S = (sad sin a, -sad cos a, 0); the
 *   detector plane is normal to the central ray at distance sdd from S; pixel
 *   (iu,iv) centre = S + sdd ew + ((iu - (nu-1)/2) du + off_u) eu
 *   + ((iv - (nv-1)/2) dv + off_v) ev, ew = (-sin a, cos a, 0),
 *   eu = (cos a, sin a, 0), ev = (0, 0, 1).  The whole support box of the
 *   volume must lie in front of the source (else PCAS_ERR_INVALID_ARG).
 * Projector P (a reading; the paper only says P projects f, Eq. 2).  Pixel
 *   value = step * sum_i f(S + i step dhat) over the integers i whose sample
 *   lies in the support box [-1, n_c] (voxel units) of the trilinear
 *   interpolant (Eq. A.5): a source-anchored ray march, so P and P^T visit
 *   exactly the same (ray, sample) pairs.
 * Errors.  Every call returns a pcas_status; pcas_last_error() returns a
 *   message for the calling thread's last failure.  Arguments are checked
 *   before any work is enqueued; a failed check leaves outputs untouched.
 */
#ifndef PCASOLVE_H
#define PCASOLVE_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PCAS_KMAX 8
#define PCAS_VERSION 1

typedef enum {
    PCAS_OK = 0,
    PCAS_ERR_INVALID_ARG = 1,   /* bad pointer, size, geometry or workspace   */
    PCAS_ERR_SINGULAR = 2,      /* Y^T Y of Eq. (A.1) singular (constant y)   */
    PCAS_ERR_CUDA = 3,          /* a CUDA runtime call or launch failed        */
    PCAS_NOT_CONVERGED = 4,     /* informational: iteration cap reached        */
    PCAS_ERR_TIMEOUT = 5        /* reserved: bounded device wait expired       */
} pcas_status;

typedef struct { int nx, ny, nz; double sx, sy, sz, ox, oy, oz; } pcas_vol;
typedef struct { double sad, sdd; int nu, nv; double du, dv, off_u, off_v, angle_rad; } pcas_cb;

/* Appendix, after Eq. (A.2): mu0 = 2, alpha = 0.1, beta = 0.5, stop when mu
 * < 0.1 or after 10 iterations, for w preconditioned to standard deviation
 * 10.  For O(1) coefficients use mu0 = 0.2, mu_min = 0.01.  max_trials caps
 * the backtracking steps of one iteration; step_mm is the ray-march step. */
typedef struct { double mu0, alpha, beta, mu_min; int max_iter, max_trials; double step_mm; } pcas_params;

/* iters: completed iterations; evals: DRR evaluations (1 + trials);
 * J0: cost at the first iteration; J, a, b: cost and intensity scaling at the
 * end; mu_last: last step size tried; status: pcas_status of the solve. */
typedef struct { int iters, evals, status; double J0, J, a, b, mu_last; } pcas_stats;

const char* pcas_last_error(void);
int pcas_version(void);

/* Bytes of device workspace needed by cost_grad / solve_projection for this
 * volume, view and K (0 if the arguments are invalid).  Pass a 256-byte
 * aligned buffer of at least this size. */
size_t pcas_workspace_bytes(const pcas_vol* vol, const pcas_cb* cb, int K);

/* Eq. (1): dvf[c][v] = mean[c][v] + sum_k w[k] U[k][c][v].
 * mean, U, dvf: device; w: host, K doubles.  Asynchronous. */
int pca_dvf(const float* mean, const float* U, int K, const double* w, const pcas_vol* vol,
            float* dvf, void* stream);

/* Eq. (A.3)/(A.5): f(i,j,k) = f0 trilinearly sampled at
 * (i + dvf[0]/sx, j + dvf[1]/sy, k + dvf[2]/sz), zero outside the grid.
 * f0, dvf ([3][N] mm), f: device.  Asynchronous. */
int warp_volume(const float* f0, const float* dvf, const pcas_vol* vol, float* f, void* stream);

/* Eq. (2), the projector P: p = P f (definition in the header comment).
 * f, p: device.  step_mm > 0.  Asynchronous. */
int drr_forward(const float* f, const pcas_vol* vol, const pcas_cb* cb, double step_mm,
                float* p, void* stream);

/* Siddon's exact radiological path, the projector Sec. II.B simulates its
 * measured projections with: p(ray) = the integral along the ray from the
 * source through the pixel centre of the piecewise-constant volume (voxel
 * (i,j,k) = f on the cube of side (sx, sy, sz) centred on it, zero outside).
 * Used to render measured images without the inverse crime of projecting
 * with the solver's own P; not on the solver path.  Voxel traversal and the
 * sum in double precision, p rounded to float.  f, p: device.  Asynchronous.
 * Errors: PCAS_ERR_INVALID_ARG for a NULL pointer, an invalid volume or
 * view, or a volume not entirely in front of the source. */
int drr_siddon(const float* f, const pcas_vol* vol, const pcas_cb* cb, float* p, void* stream);

/* P^T, the exact transpose of drr_forward (gradient formula below Eq. A.2),
 * computed in gather form without atomics: g[v] = step sum over rays and
 * samples of img(ray) times the trilinear weight of voxel v.
 * img, g: device; g is overwritten.  Asynchronous. */
int drr_adjoint(const float* img, const pcas_vol* vol, const pcas_cb* cb, double step_mm,
                float* g, void* stream);

/* One evaluation at w: (a, b) by Eq. (A.1) on P f(w), J by Eq. (2) and
 * dJ/dw = 2 U^T (df/dx) P^T (P f - a y - b) (gradient below Eq. A.2, warp
 * Jacobian of Eq. A.8) with (a, b) held.  f0, mean, U, y, ws: device;
 * w (K), J (1), dJdw (K), ab (2): host.  Synchronous.
 * Returns PCAS_ERR_SINGULAR if y is constant. */
int cost_grad(const float* f0, const float* mean, const float* U, int K, const double* w,
              const float* y, const pcas_vol* vol, const pcas_cb* cb, double step_mm,
              double* J, double* dJdw, double* ab, void* ws, size_t ws_bytes, void* stream);

/* Differentiation of Eq. (2) with respect to w and the reference CT.
 * J*(w, f0) = min over (a, b) of J is evaluated with (a, b) from Eq. (A.1);
 * since (a, b) minimise J, the gradients of J* are the partial derivatives at
 * that (a, b): dJ/dw as in cost_grad, and dJ/df0 = W^T (2 P^T r) with W the
 * trilinear warp of Eq. (A.5) at x(w) (the chain rule below Eq. A.2 stopped at
 * f instead of x).  The warped volume is recomputed on every call, never kept.
 * dJdw (K, host) may be NULL: then only J and (a, b) are computed.  dJdf0
 * (N floats, device) may be NULL; if given, dJdw must be given too.  The
 * scatter of W^T accumulates in 64-bit fixed point (deterministic).
 * Workspace: pcas_workspace_bytes_f0 (device, 256-byte aligned).  Synchronous. */
size_t pcas_workspace_bytes_f0(const pcas_vol* vol, const pcas_cb* cb, int K);
int cost_grad_f0(const float* f0, const float* mean, const float* U, int K, const double* w,
                 const float* y, const pcas_vol* vol, const pcas_cb* cb, double step_mm,
                 double* J, double* dJdw, double* ab, float* dJdf0, void* ws, size_t ws_bytes,
                 void* stream);

/* cost_grad without a caller workspace: the paper has no counterpart.  For
 * callers that cannot allocate device memory -- real-time loops where an
 * allocation could stall the frame, or host programs (a treatment-machine
 * controller, an embedding framework) whose own allocator owns all device
 * memory and hands none to libraries.  The scratch
 * is a file-scope __device__ array of PCAS_STATIC_SCRATCH_BYTES (16 MiB) in
 * the library, which every GPU that loads the library holds until exit; no
 * call here allocates.  Volumes and detectors whose scratch
 * (pcas_workspace_bytes) exceeds that size are rejected with
 * PCAS_ERR_INVALID_ARG (e.g. 72x72x40 voxels with a 192x144 detector and
 * K = 3 fit; 256x256x100 does not).  The first call on each device looks
 * up the array's device address (cudaGetSymbolAddress, which also loads the
 * library's device code there): make that first call before any stream
 * capture.  All calls on a device share the array and it keeps the last
 * call's contents; each call clears what must start at zero.  Calls that
 * overlap on the GPU (other streams, other host threads) race on it.
 * Arguments, outputs and errors as cost_grad.  Synchronous: it waits for its
 * work on `stream` and returns J, dJdw and ab on the host. */
#define PCAS_STATIC_SCRATCH_BYTES (16 * 1024 * 1024)
int cost_grad_static(const float* f0, const float* mean, const float* U, int K, const double* w,
                     const float* y, const pcas_vol* vol, const pcas_cb* cb, double step_mm,
                     double* J, double* dJdw, double* ab, void* stream);

/* Appendix: alternate Eq. (A.1) and Eq. (A.2) from w_init.  Each iteration
 * refits (a, b), takes d = -G/||G|| and tries mu = mu0, beta mu0, ... while
 * mu >= mu_min and at most max_trials times, accepting the first mu with
 * J(w + mu d) <= J(w) - alpha mu ||G||; if none passes, no step is taken and
 * the solve ends.  It also ends after max_iter iterations or at G = 0.
 * f0, mean, U, y, ws: device; w_init, w_out (K), params, stats: host.
 * The backtracking candidates are evaluated up to five at a time (one warp and
 * one projection pass for all of them; two when the previous iteration took
 * its first step size) and tested in schedule order, so the accepted step is
 * the one the one-at-a-time rule would take; stats->evals counts evaluations
 * as that rule would.  Synchronous (one host read of a
 * 4-byte flag per batch of candidates). */
int solve_projection(const float* f0, const float* mean, const float* U, int K, const float* y,
                     const pcas_vol* vol, const pcas_cb* cb, const double* w_init,
                     const pcas_params* params, double* w_out, pcas_stats* stats, void* ws,
                     size_t ws_bytes, void* stream);

/* Sec. II.A: the DVF is a pull-back field (new-image point c maps to
 * c + x(c) in the reference), so the tumour position solves c + x(c) = c_ref;
 * iterate y <- -x(c_ref + y) from y = 0 (x trilinear in mm, zero outside the
 * grid) until the update is below tol_mm or max_iter is reached; c = c_ref + y.
 * mean, U: device; w (K), c_ref, c_out: host.  Synchronous.  Returns
 * PCAS_NOT_CONVERGED (with c_out set) if the cap was reached. */
int localize_tumor(const float* mean, const float* U, int K, const double* w,
                   const pcas_vol* vol, const double c_ref[3], int max_iter, double tol_mm,
                   double c_out[3], void* stream);

/* ------------------------------------------------------------------------
 * Device-driven solves (the Appendix loop without host round trips).
 * A pcas_solver captures solve_projection for one reference CT, motion model
 * and detector shape as a CUDA graph whose iteration and backtracking loops
 * are conditional WHILE nodes driven by the device state; solving a
 * projection is one graph launch.  Results equal solve_projection's (same
 * kernels, same order of operations).
 *
 * pcas_solver_create: f0, mean, U (storage dtype as the *_typed calls) and
 *   the workspace (pcas_solver_workspace_bytes, device, 256-byte aligned) are
 *   owned by the caller and must stay valid until destroy; cb gives the
 *   detector shape (its angle and offsets are per-solve); params are fixed.
 *   Allocates pinned host staging buffers, a stream for the localisations
 *   of runs and one for the uploads of their host images, and builds the
 *   graph; not for use inside stream capture.  pcas_solver_destroy waits for
 *   those streams before it frees them.
 * pcas_solver_solve: y (device, [nv][nu]) is copied into the solver's image
 *   buffer unless it is that buffer (pcas_solver_y_buffer) or NULL; the view
 *   is the creation view with this angle and these detector offsets.
 *   w_init, w_out (K), stats: host.  Synchronous.  One solver must not be
 *   used by two host threads at once.
 * pcas_batch_create: one graph holding the solves of n solvers as independent
 *   branches (uneven sizes allowed), each preceded by a copy from y_src[i]
 *   (device, may be NULL: the solver's own buffer is used).
 * pcas_batch_solve: one graph launch for all n; angle_rad[i] per solve;
 *   w_init and w_out are n x PCAS_KMAX host arrays (row i, first K_i
 *   entries); stats[i] per solve (status set per solve).  Synchronous. */
typedef struct pcas_solver_s* pcas_solver;
typedef struct pcas_batch_s* pcas_batch;
size_t pcas_solver_workspace_bytes(const pcas_vol* vol, const pcas_cb* cb, int K);
int pcas_solver_create(pcas_solver* out, const void* f0, const void* mean, const void* U, int dtype,
                       int K, const pcas_vol* vol, const pcas_cb* cb, const pcas_params* params,
                       void* ws, size_t ws_bytes, void* stream);
float* pcas_solver_y_buffer(pcas_solver solver);
int pcas_solver_solve(pcas_solver solver, const float* y, double angle_rad, double off_u, double off_v,
                      const double* w_init, double* w_out, pcas_stats* stats, void* stream);
int pcas_solver_destroy(pcas_solver solver);

/* Fixed-angle fluoroscopy (Sec. IV: with the gantry held still the projection
 * matrix is constant).  A solver can keep the constant part of P^T for one
 * view -- the solver's detector at angle_rad with its creation offsets -- in
 * a caller-provided device cache: for every voxel its footprint on the
 * detector and the weight of each footprint ray in the gather of the
 * gradient (the sum over the ray's samples of the voxel's trilinear weight).
 * Solves staged at exactly that angle and those offsets (pcas_solver_solve,
 * runs, batches) then read these weights instead of recomputing them; the
 * sums keep their order, so results are bitwise those of the uncached solver.
 * pcas_solver_fixed_view_bytes: device bytes of the cache for angle_rad (0 if
 *   the solver or the view is invalid, or a detector side exceeds 32767
 *   pixels).  Counts on the device on `stream`; synchronous.
 * pcas_solver_fix_view: builds the cache (cache: device, 256-byte aligned,
 *   at least pcas_solver_fixed_view_bytes; owned by the caller, valid until
 *   the solver is destroyed or the cache is replaced); cache = NULL turns it
 *   off.  Synchronous.  Both calls use the solver's own scratch: not while a
 *   solve of this solver is in flight on another stream. */
size_t pcas_solver_fixed_view_bytes(pcas_solver solver, double angle_rad, void* stream);
int pcas_solver_fix_view(pcas_solver solver, double angle_rad, void* cache, size_t cache_bytes, void* stream);

/* Runs of consecutive projections on one solver (a breathing sequence): the
 * warm start of Eq. (3) runs inside the graph, from the solutions the run
 * keeps on the device, and the tumour localisation of Sec. II.A follows each
 * solve on a stream the solver owns (ordered after the solve by an event; the
 * next projection's solve does not wait for it), so projections can be
 * queued back to back with no host round trip in between.
 * pcas_solver_seq_begin: starts a run.  lp_coef: host K x L (c[k][l] as
 *   lp_fit, 1 <= L <= 8); c_ref: tumour centroid in the reference CT (mm);
 *   loc_max_iter, loc_tol_mm: as localize_tumor; w_hist: host n_hist x K
 *   solutions preceding the run, latest first (0 <= n_hist <= 8; NULL when
 *   0).  Synchronous.
 * pcas_solver_seq_enqueue: queues one projection on the stream and returns
 *   its ticket.  y: [nv][nu] floats, device or (pinned) host memory, copied
 *   into the solver's buffer; a host image is uploaded on a stream the solver
 *   owns, beside the solves queued before it (keep it unchanged until the
 *   ticket's result has been read); the view is the creation view at
 *   angle_rad.
 *   The start is w_first (host, K doubles, NULL = zeros) while the run has
 *   no solution yet, then the latest solution while it has fewer than L,
 *   then the Eq. (3) prediction from the last L (the same arithmetic as
 *   lp_predict).  Returns before the solve runs; at most 64 projections of a
 *   solver may be in flight (the call waits for a free slot).
 * pcas_solver_seq_result: waits for the projection of a ticket and returns
 *   its solution, centroid and statistics (host); valid for the last 64
 *   tickets of the solver.  Returns PCAS_ERR_SINGULAR for a constant image
 *   (the run goes on from the unchanged start).
 * Within a run the reference CT is read once, by the run's first projection
 * (its halo copy is kept for the rest): it must not change during a run.
 * A pcas_solver_solve or batch solve in between ends the run. */
typedef struct {
    double w[PCAS_KMAX];      /* solution (first K entries) */
    double c[3];              /* tumour centroid, mm */
    int loc_converged;        /* 1 if the localisation converged */
    pcas_stats stats;
} pcas_seq_result;
int pcas_solver_seq_begin(pcas_solver solver, const double* lp_coef, int L, const double* c_ref,
                          int loc_max_iter, double loc_tol_mm, const double* w_hist, int n_hist, void* stream);
int pcas_solver_seq_enqueue(pcas_solver solver, const void* y, double angle_rad, const double* w_first,
                            long long* ticket, void* stream);
int pcas_solver_seq_result(pcas_solver solver, long long ticket, pcas_seq_result* out);
int pcas_batch_create(pcas_batch* out, const pcas_solver* solvers, const float* const* y_src, int n,
                      void* stream);
int pcas_batch_solve(pcas_batch batch, const double* angle_rad, const double* w_init, double* w_out,
                     pcas_stats* stats, void* stream);
int pcas_batch_destroy(pcas_batch batch);

/* ------------------------------------------------------------------------
 * Storage precision of the reference CT and the motion model.  The *_typed
 * calls take f0, mean and U as float (PCAS_F32), bfloat16 (PCAS_BF16) or half
 * (PCAS_F16) arrays with the layouts above; every value is widened to float
 * on load, so interpolation, DVF synthesis, projection and accumulation stay
 * float32, and the cross-block reductions and scalar updates FP64 (Appendix
 * arithmetic unchanged).  The plain calls are the PCAS_F32 case.  Halves the
 * model and CT traffic of the warp and Jacobian passes. */
typedef enum { PCAS_F32 = 0, PCAS_BF16 = 1, PCAS_F16 = 2 } pcas_dtype;
int cost_grad_typed(const void* f0, const void* mean, const void* U, int dtype, int K,
                    const double* w, const float* y, const pcas_vol* vol, const pcas_cb* cb,
                    double step_mm, double* J, double* dJdw, double* ab, void* ws, size_t ws_bytes,
                    void* stream);
int solve_projection_typed(const void* f0, const void* mean, const void* U, int dtype, int K,
                           const float* y, const pcas_vol* vol, const pcas_cb* cb,
                           const double* w_init, const pcas_params* params, double* w_out,
                           pcas_stats* stats, void* ws, size_t ws_bytes, void* stream);
int localize_tumor_typed(const void* mean, const void* U, int dtype, int K, const double* w,
                         const pcas_vol* vol, const double c_ref[3], int max_iter, double tol_mm,
                         double c_out[3], void* stream);

/* Eq. (3): per coefficient k, least-squares fit over t = L..T-1 of
 * trace[t][k] ~ sum_{l=1..L} c[k][l-1] trace[t-l][k].  trace: host T x K;
 * c: host K x L.  Needs T > 2L.  Host only. */
int lp_fit(const double* trace, int T, int K, int L, double* c);

/* Eq. (3): w0[k] = sum_l c[k][l-1] hist[l-1][k], hist[l-1] = w*(t-l) (host). */
int lp_predict(const double* hist, const double* c, int K, int L, double* w0);

/* ---------------------------------------------------------------- autotuner
 * Launch shapes of the solver kernels, kept per size bucket (volume extents
 * in steps of 32, 32, 16 voxels, detector extents in steps of 64 pixels, K,
 * storage type).  No counterpart in the paper; they change speed only.
 *   ray_lw1           log2 of a warp's patch width on the detector (2..4) of
 *                     the one-volume projector: (1 << lw) x (32 >> lw) pixels
 *   chunk1            sample indices per shared-memory chunk of the one-volume
 *                     projector (even, 0..128; 0 = no staging, reads via L1)
 *   voxel_tile        voxel tile of the gradient pass: 0 = 8x8x4, 1 = 16x4x4,
 *                     2 = 32x4x2, 3 = 16x8x2, 4 = 32x8x1, 5 = 64x4x1
 *   gather_per_sm     blocks of the gradient gather per SM (1..26)
 *   skip_empty        empty-space skipping of the solver projectors (0 or 1):
 *                     the warp kernels mark the 8x8x8-voxel bricks holding
 *                     non-zero voxels, and each ray's samples are cut to the
 *                     span from its first to its last sample whose cell lies
 *                     in a marked brick.  Exact: the samples left out
 *                     interpolate eight zero voxels, so every sum is bitwise
 *                     the same either way
 * and per 22.5-degree bin of the gantry angle modulo 180 degrees (bin b is
 * centred on 22.5 b degrees):
 *   ray_lw4[b]        patch width of the batch projector (2..4)
 *   chunk[b]          its sample indices per shared-memory chunk (even, 2..64)
 *   swap[b]           layout of the solver volumes: 0 = x fastest,
 *                     1 = y fastest
 * Every call takes the entry of its bucket, or the defaults (3, 0, 0, 8, 1;
 * per bin 3, 16, y fastest in bins 3..5) when there is none; a device-driven
 * solver takes the entry in force when it is created (the per-bin shapes
 * follow the angle of each solve).  Other shapes reorder floating-point sums:
 * results can differ by rounding between shapes, and are reproducible for a
 * fixed table. */
typedef struct {
    int ray_lw1, chunk1, voxel_tile, gather_per_sm, skip_empty;
    unsigned char ray_lw4[8], chunk[8], swap[8];
} pcas_tuning;

/* Measures shapes on this problem and stores the fastest in its bucket:
 * trial solves (solve_projection with max_iter capped at 3, from w_init, at
 * the centre angle of a bin), every kernel timed with CUDA events: empty-
 * space skipping on or off, then per bin the layout, then per bin the patch
 * width and chunk of the five-candidate projector, then the one-volume
 * projector's width and chunk, the voxel tile and the gather size, each
 * chosen by the time of the kernels it drives (about 150 trial solves); a
 * shape replaces the one in place (default or earlier choice) only when it
 * is more than 1.5 % faster, and among the shapes within 1.5 % of the
 * fastest the first in a fixed candidate order is taken, so that timing
 * noise does not flip choices (which can change the rounding of results)
 * between runs.  f0, mean, U, y,
 * ws: device, as solve_projection
 * (ws of pcas_workspace_bytes); w_init: host, K doubles or NULL (zeros);
 * out (host, may be NULL) receives the stored entry.  Synchronous.  Bins
 * whose view is invalid (volume not in front of the source) keep their
 * layouts.  Call it from one thread, outside stream capture. */
int pcas_autotune(const void* f0, const void* mean, const void* U, int dtype, int K,
                  const pcas_vol* vol, const pcas_cb* cb, const pcas_params* params,
                  const double* w_init, const float* y, void* ws, size_t ws_bytes,
                  pcas_tuning* out, void* stream);
/* The entry in force for a problem's bucket (the defaults if none). */
int pcas_tuning_get(const pcas_vol* vol, const pcas_cb* cb, int K, int dtype, pcas_tuning* out);
/* Stores an entry (validated: PCAS_ERR_INVALID_ARG when a field is out of range). */
int pcas_tuning_set(const pcas_vol* vol, const pcas_cb* cb, int K, int dtype, const pcas_tuning* t);
/* Forgets every stored entry. */
int pcas_tuning_clear(void);

/* ------------------------------------------------------------------------
 * Benchmark instrumentation (the paper has no counterpart).  The library
 * counts every kernel it launches, per kernel class.  pcas_profile(1) resets
 * the counts and, until pcas_profile(0), also brackets each launch with a
 * pair of CUDA events recorded on the launch stream (events come from a pool
 * created on the first pcas_profile(1); up to 65536 launches are timed).
 * pcas_profile_read() returns the launches and the summed event time in ms
 * of one class since the last reset; it waits for the recorded events.
 * These calls are host-side and thread-safe. */
enum {
    PCAS_K_WARP_PCA = 0,     /* fused Eq. (1) + (A.5) into the solver volume   */
    PCAS_K_DRR_SOLVER = 1,   /* solver P with fused moments / Armijo test      */
    PCAS_K_RESID = 2,        /* Eq. (A.1) + residual + J                        */
    PCAS_K_ADJ_GRAD = 3,     /* fused P^T, Eq. (A.8) and dJ/dw reduction        */
    PCAS_K_DRR = 4,          /* drr_forward                                     */
    PCAS_K_ADJ = 5,          /* drr_adjoint                                     */
    PCAS_K_PCA_DVF = 6,      /* pca_dvf                                         */
    PCAS_K_WARP_DVF = 7,     /* warp_volume                                     */
    PCAS_K_LOCALIZE = 8,     /* localize_tumor                                  */
    PCAS_K_INIT = 9,         /* solver state reset                              */
    PCAS_K_WARP_BATCH = 10,  /* five line-search candidates warped at once      */
    PCAS_K_DRR_BATCH = 11,   /* five candidates projected and tested at once    */
    PCAS_K_GRAD_F0 = 12,     /* dJ/df0: full backprojection + warp transpose    */
    PCAS_K_GRAPH = 13,       /* kernels run inside device-driven (graph) solves  */
    PCAS_K_SIDDON = 14,      /* drr_siddon                                      */
    PCAS_K_COUNT = 15
};
int pcas_profile(int on);
int pcas_profile_read(int kind, long long* launches, double* total_ms);

#ifdef __cplusplus
}
#endif
#endif /* PCASOLVE_H */
