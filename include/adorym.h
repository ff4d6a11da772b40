/*
 * adorym.h -- C ABI of the GB300 loss-and-gradient engine for the multislice ptychography
 * forward model of Adorym (Du et al., arXiv 2012.12686).
 *
 * The engine evaluates, for a minibatch of probe positions, the forward model y = F(x, theta)
 * (Sec. 1, Eq. forward_model) of Algorithm 1 -- Fourier-shifted probe (Eq. fourier_shift),
 * multislice propagation through the refractive-index object (Eqs. ri_modulation,
 * fresnel_prop, paraxial_kernel), far-field (Eq. fraunhofer) or near-field Fresnel
 * propagation to the detector, incoherent sum over probe modes (Eq. multimode) -- the data
 * mismatch L (Eq. loss_function, in the forms of Eq. lsq_loss or Eq. poisson_loss), and the
 * gradient of L with respect to the object (delta, beta), the probe and the probe positions
 * (Sec. 2.3.2 "refinable parameters": probe position, and for holography the per-hologram
 * translation of Eq. affine_transform).
 *
 * Conventions
 *   - Object volumes are planar FP32, slice-major [Lz][Ly][Lx] (z along the beam).  The
 *     paper's [Ly][Lx][Lz][2] layout (Sec. 2.1, ObjectFunction) maps to two such arrays.
 *   - Complex arrays are interleaved (re, im) FP32 pairs, row-major [..][N][N].
 *   - Positions are (y, x) in pixels of the object grid; the patch corner is
 *     floor(pos + 1/2) and the residual is applied as a Fourier shift of the probe.
 *   - Far-field patterns are in unshifted FFT order (DC at [0][0]); the far field is the
 *     unitary transform with a positive exponent (negative phase convention, Sec. 2.2).
 *   - Complex gradients are returned as dL/dRe + i dL/dIm.
 *   - Every call is stream-ordered on the context's CUDA stream.
 *
 * Pointers
 *   Array arguments may be device pointers or host pointers (pinned or pageable), except the
 *   registered object volumes and the object-gradient volumes, which must be device memory.
 *   Host inputs are copied to device staging inside the call; host outputs are copied back
 *   and the call then waits for the stream.  With only device pointers (and a device
 *   loss_out) the call is asynchronous.  The caller owns every array; the library owns its
 *   workspace, twiddle/propagator tables, checkpoints and CUDA graphs.
 *
 * Errors
 *   Every entry point returns ADORYM_OK or an error code and never aborts; the message of the
 *   last error of a context is returned by adorym_last_error().  Kernels index the object only
 *   after bounds checks (pixels outside the volume read as vacuum and their gradients are
 *   dropped) and clamp patch corners to +-2^24 px, so no input can make them access memory out
 *   of range.  Data that only the device sees (positions, hologram shifts) are checked while the
 *   call runs: a non-finite or huge value sets the call's device status word, reported as
 *   ADORYM_EDATA by calls with host outputs, by adorym_check and by adorym_poll.  No kernel
 *   traps; the one device-side wait (a column tile's TMA copy) is bounded and reports a timeout
 *   through the same status word.
 */
#ifndef ADORYM_H
#define ADORYM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ADORYM_OK 0
#define ADORYM_EINVAL 1      /* invalid argument (sizes, pointers, unsupported configuration) */
#define ADORYM_ENOMEM 2      /* device memory could not be obtained / admission refused       */
#define ADORYM_ETIMEDOUT 3   /* adorym_poll: the request did not finish within the timeout    */
#define ADORYM_EDEVICE 4     /* a CUDA error was reported (message in adorym_last_error)      */
#define ADORYM_ENOENT 5      /* unknown object id or ticket                                    */
#define ADORYM_ETOOBIG 6     /* adorym_loss_grad_noalloc: the problem needs more scratch than
                                ADORYM_NOALLOC_SCRATCH_BYTES                                   */
#define ADORYM_EDATA 7       /* a kernel found invalid input data in device memory (a position
                                that is not finite or lies beyond +-2^24 px); reported through
                                the call's device status word, see adorym_check              */
#define ADORYM_ECANCELED 8   /* adorym_poll: the request was cancelled before it was admitted   */

#define ADORYM_LOSS_LSQ 0     /* Eq. lsq_loss: mean (sqrt(I+eps) - sqrt(I_meas+eps))^2        */
#define ADORYM_LOSS_POISSON 1 /* Eq. poisson_loss: mean (I - I_meas log(I+eps))               */

typedef struct adorym_ctx adorym_ctx;

/* One loss/gradient problem (the paper's reconstruct_ptychography parameters that reach the
 * forward model, Sec. 2.7 "User interface", reduced to dimensionless pixel units). */
typedef struct adorym_problem {
  int N;              /* tile (probe / detector) side in pixels: a power of two in 8..1024
                         (8..128: one fused kernel per call; 256..1024: two-pass path)     */
  int L;              /* slices each wave traverses                                        */
  int M;              /* incoherent probe modes (Eq. multimode)                            */
  int B;              /* far field: positions in the minibatch; near field: problems        */
  int Ly, Lx, Lz;     /* object dims; must equal the registered object's.  Far field:
                         Lz == L.  Near field: Ly == Lx == N and Lz == B * L (problem b uses
                         slices [b L, (b+1) L)).                                           */
  double kdz;         /* k * dz, k = 2 pi / lambda (Eq. ri_modulation)                      */
  double lambda_dz_over_px2; /* lambda dz / dx^2: slice-to-slice paraxial step (Eq. paraxial_kernel) */
  int farfield;       /* 1: far-field ptychography (Eq. fraunhofer); 0: near-field holography */
  int n_dist;         /* near field: number of sample-detector distances (1..4)              */
  double nf[4];       /* near field: Fresnel numbers dx^2 / (lambda z) of the distances       */
  int loss;           /* ADORYM_LOSS_LSQ or ADORYM_LOSS_POISSON                              */
  double eps;         /* eps of the loss terms (added to I and I_meas in LSQ, inside the log) */
  int tomo;           /* 1: sample the object rotated by theta about y (Eq. rotation_transform) */
  double theta;       /* tilt angle in radians                                              */
  int checkpoint_every; /* adjoint checkpoint spacing in slices; 0 = ceil(sqrt(L))          */
  const double* gaps; /* sparse / variable multislice (Sec. 2.2): NULL for equal spacing, else a
                         host array of L-1 values lambda dz_j / dx^2 for the Fresnel step from
                         slice j to j+1 (read during the call; replaces lambda_dz_over_px2)     */
} adorym_problem;

/* Create a context on CUDA device `device`, enqueueing on `cuda_stream` (a cudaStream_t; NULL =
 * the legacy default stream).  *ctx receives the context.  Returns EINVAL / EDEVICE on failure. */
int adorym_create(adorym_ctx** ctx, int device, void* cuda_stream);

/* Wait for the context's work, release its workspace, graphs and serving threads. */
void adorym_destroy(adorym_ctx* ctx);

/* Message of the most recent error on this context ("" if none).  Owned by the context. */
const char* adorym_last_error(adorym_ctx* ctx);

/* Device status word of the most recent adorym_forward / adorym_loss_grad(_ext) call of ctx.
 * Kernels never trap: input data that only the device sees (positions / hologram shifts) are
 * checked while the call runs, and an invalid value sets a bit in a per-call status word instead
 * (the call's results are then meaningless but no memory outside the object and the workspace is
 * touched: patch corners are clamped).  Calls that return host outputs wait for the GPU and
 * report ADORYM_EDATA themselves; for asynchronous calls this function waits for the context's
 * stream and returns ADORYM_OK or ADORYM_EDATA (message in adorym_last_error).  Serving
 * requests report it through adorym_poll. */
int adorym_check(adorym_ctx* ctx);

/* Number of kernels this library has launched in the process so far (kernels recorded into a
 * serving graph count once, at capture).  Accounting only (no counterpart in the paper):
 * differences around a region give the kernels that region launched. */
uint64_t adorym_kernel_launches(void);

/* Test hook for the bounded device-side waits (no counterpart in the paper).  Three waits exist:
 * a position waiting for a checkpoint segment that a recompute helper is working on (default
 * about 2^28 SM cycles, then the position recomputes the segment itself), a helper waiting for a
 * position's checkpoint (about 2^24 cycles, then the helper stops), and a two-pass column kernel
 * waiting for its tile's TMA copy (about 2^31 cycles, then the call's status word reports
 * ADORYM_EDATA "wait timed out", and the CTA waits for its copies with the default limit before it
 * leaves).  Each argument is a limit in SM clock cycles (>= 0), ADORYM_WAIT_DEFAULT to restore the
 * default, or for tile copies ADORYM_WAIT_GIVE_UP to report the timeout without waiting.  The
 * limits are process-wide and apply to calls enqueued afterwards (serving graphs keep the limits
 * of their capture).  Results do not depend on the first two limits; a tile-copy timeout makes
 * the call's results meaningless.  Returns ADORYM_OK or ADORYM_EINVAL. */
#define ADORYM_WAIT_DEFAULT (-1)
#define ADORYM_WAIT_GIVE_UP (-2)
int adorym_set_wait_limits(int64_t segment_cycles, int64_t checkpoint_cycles, int64_t tile_copy_cycles);

/* Measured FP32 fused-multiply-add throughput of `device` in TFLOP/s (2 flops per FMA): a
 * throughput kernel of independent FMA chains on several CTAs per SM, best of four timed runs
 * after one warm-up.  Measurement only (no counterpart in the paper): the denominator against
 * which the FP32-bound kernels' roofline fraction can be read.  Allocates a small buffer, runs
 * about 20 ms, synchronizes; returns ADORYM_OK or an error code. */
int adorym_fp32_peak(int device, double* tflops);

/* Register a resident object volume: delta, beta device pointers to FP32 [Lz][Ly][Lx]
 * (Sec. 2.1 refractive-index representation n = 1 - delta - i beta).  The memory stays owned
 * by the caller and must outlive the registration; its contents may change between calls
 * (an optimiser updating the object in place).  *obj_id receives the handle. */
int adorym_register_object(adorym_ctx* ctx, const float* delta, const float* beta, int Lz, int Ly, int Lx,
                           int* obj_id);

/* Drop a registration.  Host-side only: work already enqueued keeps the volume pointers it was
 * given, so the caller keeps the memory alive until that work has completed. */
int adorym_unregister_object(adorym_ctx* ctx, int obj_id);

/* Forward model only: predicted intensities y = F(x, theta) (Eq. forward_model, Algorithm 1).
 *   probe  complex [M][N][N]: far field the probe modes; near field the illumination.
 *   pos    far field [B][2] (y, x); near field per-hologram shifts [B][n_dist][2].
 *   I_out  far field [B][N][N]; near field [B][n_dist][N][N] (FP32, overwritten). */
int adorym_forward(adorym_ctx* ctx, const adorym_problem* p, int obj_id, const float* probe, const float* pos,
                   float* I_out);

/* Loss and gradients (Eq. loss_function with Eq. lsq_loss / Eq. poisson_loss, averaged over the
 * batch's detector pixels; adjoint with sqrt(L) checkpointing).
 *   I_meas   measured intensities, same shape as I_out of adorym_forward.
 *   loss_out one double (host or device), overwritten.  May be NULL.
 *   g_delta, g_beta  device FP32 [Lz][Ly][Lx]; the gradient is ADDED (+=).  NULL skips both.
 *   g_probe  complex [M][N][N]; ADDED (+=).  NULL skips it.
 *   g_pos    far field [B][2] dL/dpos; near field [B][n_dist][2] dL/dshift; OVERWRITTEN.
 *            NULL skips it.
 *   I_out    optional predicted intensities (overwritten), or NULL. */
int adorym_loss_grad(adorym_ctx* ctx, const adorym_problem* p, int obj_id, const float* probe, const float* pos,
                     const float* I_meas, double* loss_out, float* g_delta, float* g_beta, float* g_probe,
                     float* g_pos, float* I_out);

/* Outputs of adorym_loss_grad_ext (NULL members are skipped). */
typedef struct adorym_grads {
  double* loss;     /* one double (host or device), overwritten                                  */
  float* g_delta;   /* device FP32 [Lz][Ly][Lx], added (+=)                                      */
  float* g_beta;
  float* g_probe;   /* complex [M][N][N], added                                                  */
  float* g_pos;     /* far [B][2] / near [B][n_dist][2], overwritten                              */
  float* g_nf;      /* near field only: [B][n_dist] dL/dN_F, the gradient w.r.t. each problem's
                       Fresnel numbers (free-propagation distance refinement, Sec. 2.3.2;
                       N_F = dx^2 / (lambda z), so dL/dz = -dL/dN_F * N_F / z), overwritten   */
  float* I_out;     /* predicted intensities, overwritten                                        */
  float* g_gaps;    /* with variable spacing: [L-1] dL/d(lambda dz_j / dx^2), the slice-position
                       gradient (Sec. 2.3.2), summed over the batch, overwritten                  */
  float* g_offset;  /* far field only: [2] (y, x) gradient w.r.t. one position offset shared by
                       every position of the batch -- the per-angle probe-position offset of
                       ptychotomography (Sec. 2.3.2 "Probe position offset"), for a batch that
                       holds the positions of one angle.  Sum over the batch of the per-position
                       gradients, taken in FP64 in a fixed order; overwritten.                   */
} adorym_grads;

/* adorym_loss_grad with its outputs in a struct, including the near-field distance gradient. */
int adorym_loss_grad_ext(adorym_ctx* ctx, const adorym_problem* p, int obj_id, const float* probe, const float* pos,
                         const float* I_meas, const adorym_grads* out);

/* Regularizers of Table regularizers (refractive-index form), added to the data term as in
 * Eq. tikhonov:  R = (1/N_o) [ sum a_d W_d|delta| + a_b W_b|beta|
 *                              + gamma sum over x, y, z of (|grad delta| + |grad beta|) ],
 * N_o = Lz Ly Lx, forward differences with no term past the last index, subgradient 0 at 0. */
typedef struct adorym_reg {
  double alpha_delta;     /* l1 weight on delta (alpha_1)                                         */
  double alpha_beta;      /* l1 weight on beta (alpha_2)                                          */
  const float* w_delta;   /* reweighted l1: device [Lz][Ly][Lx] weights W_1, or NULL (plain l1)   */
  const float* w_beta;    /* W_2, or NULL                                                         */
  double gamma_tv;        /* total-variation weight gamma (0: no TV term)                         */
} adorym_reg;

/* R and its gradient for a registered object: *loss_out = R (host or device double, may be NULL);
 * g_delta, g_beta (device [Lz][Ly][Lx], may be NULL together) receive dR/ddelta, dR/dbeta added
 * (+=). */
int adorym_regularize(adorym_ctx* ctx, int obj_id, const adorym_reg* r, double* loss_out, float* g_delta,
                      float* g_beta);

/* Reweighted-l1 weights from a snapshot object: W = max|C| / (|C| + eps) for C = delta and beta,
 * written to device arrays w_delta, w_beta [Lz][Ly][Lx] (treated as constants by adorym_regularize). */
int adorym_l1_weights(adorym_ctx* ctx, int obj_id, double eps, float* w_delta, float* w_beta);

/* A loss/gradient request for the serving loop: the arguments of adorym_loss_grad. */
typedef struct adorym_request {
  adorym_problem problem;
  int obj_id;
  const float* probe;
  const float* pos;
  const float* I_meas;
  double* loss_out;
  float* g_delta;
  float* g_beta;
  float* g_probe;
  float* g_pos;
  float* I_out;
} adorym_request;

/* Serving loop.  adorym_submit queues a request and returns at once with *ticket.  A request
 * is admitted when a slot is free and its device workspace fits the context's footprint
 * budget, in arrival order except that requests which fit may go ahead of an older one that
 * does not (at most 8 admissions past any one waiting request, so none is starved); admitted
 * requests run concurrently on separate streams as captured CUDA graphs (one graph per problem
 * shape and slot), so requests that arrive while others run overlap with them on the device.
 * Half of the slots (rounded down) are reserved for short requests (B M L N^2 pixel-slices of at
 * most 2^26, doubled for N >= 256) and run at the device's highest stream priority, so a short
 * request does not wait behind long ones for a slot (a short request that takes a short-request
 * slot while a long one waits for a normal slot neither waits nor counts as overtaking it) and its
 * thread blocks are scheduled first when SMs free up.
 * Completion is event driven (a blocked waiter per slot, no polling).  Array pointers must be
 * device memory and stay valid until the request completes.  Requests whose footprint can never
 * fit return ENOMEM at submit. */
int adorym_submit(adorym_ctx* ctx, const adorym_request* req, uint64_t* ticket);

/* Wait up to timeout_us microseconds (<0: forever, 0: test) for a ticket.  Returns ADORYM_OK
 * once the request's outputs are complete (the ticket is then retired), ETIMEDOUT if it is still
 * queued or running, ENOENT for an unknown ticket, or the request's own error code. */
int adorym_poll(adorym_ctx* ctx, uint64_t ticket, int64_t timeout_us);

/* adorym_poll that also reports where the request's time went (times_us[3], may be NULL):
 * times_us[0] = time from submission to admission (queueing for a slot and memory),
 * times_us[1] = time from admission to completion (graph capture or update, launch and device
 * execution, including time shared with other admitted requests), times_us[2] = the admission
 * instant since the serving loop was configured (-1 if never admitted).  Host clock,
 * microseconds.  Same return codes. */
int adorym_poll_times(adorym_ctx* ctx, uint64_t ticket, int64_t timeout_us, double* times_us);

/* Serving configuration: number of concurrent slots (streams, 1..16) and the device-memory
 * footprint budget in bytes for admitted requests' workspaces (0 = no limit).  Only allowed
 * while no request is in flight. */
int adorym_serve_config(adorym_ctx* ctx, int slots, uint64_t budget_bytes);

/* Cancel a serving request that is still waiting for admission: it is removed from the queue and
 * its adorym_poll returns ADORYM_ECANCELED.  Returns ADORYM_OK, ADORYM_ENOENT for an unknown
 * ticket, or ADORYM_EINVAL when the request has already been admitted (its GPU work is not
 * interrupted) or has finished.  No counterpart in the paper (serving). */
int adorym_cancel(adorym_ctx* ctx, uint64_t ticket);

/* Failure injection for tests of error handling, host side only: the next `count` workspace
 * allocations of ctx fail with ADORYM_ENOMEM without touching the device (the context's existing
 * workspace is kept, later calls allocate normally).  No counterpart in the paper. */
int adorym_inject_alloc_failures(adorym_ctx* ctx, int count);

/* Serving statistics since the context was created: completed requests and the number of
 * times a request had to wait for admission. */
int adorym_serve_stats(adorym_ctx* ctx, uint64_t* completed, uint64_t* admission_waits);

/* Kernel timing for roofline measurements.  With enable = 1, each later direct call records a
 * CUDA event pair around its fused path kernel on the context's stream (not inside serving
 * graphs).  adorym_kernel_ms returns the path kernel time of the most recent such call in
 * milliseconds (it waits for that call's stop event). */
int adorym_enable_kernel_timing(adorym_ctx* ctx, int enable);
int adorym_kernel_ms(adorym_ctx* ctx, float* path_ms);

/* Device workspace (bytes) that a served request (adorym_submit) needs for this problem, for
 * admission planning by callers.  grads: bitmask 1 = object, 2 = probe, 4 = positions.  A direct
 * adorym_loss_grad call with N <= 128 and a batch below the device's SM count takes more: the
 * SMs the batch leaves idle recompute checkpoint segments into a store of
 * B * M * (ncp - 1) * cp * N^2 * 8 bytes (ncp checkpoints every cp slices). */
int adorym_workspace_bytes(const adorym_problem* p, int grads, uint64_t* bytes);

/* Size of the fixed device scratch array used by adorym_loss_grad_noalloc. */
#define ADORYM_NOALLOC_SCRATCH_BYTES ((uint64_t)64 << 20)

/* adorym_loss_grad for callers that cannot allocate device memory.  The paper has no
 * counterpart: this is a deployment variant of the same computation.
 *
 * Who needs it: code that runs where cudaMalloc is not allowed or not wanted -- a plug-in whose
 * host framework owns all device memory through its own pool, or a latency-critical loop that
 * must not allocate (an allocation can synchronise the device).  This call takes no context and
 * allocates nothing (no cudaMalloc, cudaFree or allocating library routine): its workspace and
 * tables live in one file-scope device array of ADORYM_NOALLOC_SCRATCH_BYTES (64 MiB), reserved
 * on every GPU that loads the library until the process exits.  The twiddle and propagator
 * tables are computed into that array by a kernel on cuda_stream.
 *
 * Arguments are those of adorym_loss_grad (same layouts and accumulate/overwrite rules), except
 * that the object volumes delta, beta ([Lz][Ly][Lx] FP32) are passed directly, every pointer
 * must be device memory, and variable slice spacing is not offered (p->gaps with L > 1 returns
 * ADORYM_EINVAL).  Work is enqueued on cuda_stream (a cudaStream_t) on the current device.
 *   status  optional device int: with it, the kernels OR the call's ADORYM status bits into
 *           *status (the caller zeroes it beforehand; nonzero afterwards means a position was
 *           not finite or beyond +-2^24 px, or a bounded device wait gave up, and the outputs are
 *           then meaningless).  NULL: the status is kept in the scratch array only and not
 *           reported.
 *
 * Returns ADORYM_ETOOBIG when the problem's workspace exceeds the array (e.g. large batches of
 * 128x128 tiles: use adorym_loss_grad there), EINVAL for invalid sizes or non-device pointers.
 * The array's device address is looked up on the first call made on each device.  All calls
 * share the array and it keeps the previous call's contents (each call clears on its stream what
 * must start at zero); calls that overlap on the GPU -- on different streams or from several
 * host threads -- race on it, so the caller must serialise them (e.g. one stream). */
int adorym_loss_grad_noalloc(void* cuda_stream, const adorym_problem* p, const float* delta, const float* beta,
                             const float* probe, const float* pos, const float* I_meas, double* loss_out,
                             float* g_delta, float* g_beta, float* g_probe, float* g_pos, float* I_out,
                             int* status);

#ifdef __cplusplus
}
#endif

#endif /* ADORYM_H */
