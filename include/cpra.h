/*
 * cpra.h - C ABI of the GB300 carousel phase retrieval (CPRA) library.
 *
 * The library reconstructs Np projected objects (POs) from Np measured N x N
 * far-field intensity patterns (Eq. 1-3 of arXiv 2402.05283), couples each PO
 * with its periodic neighbours between episodes (Eq. 4, Step B), and
 * assembles the retrieved spectra into a 3D reciprocal grid followed by an
 * inverse 3D FFT (Step D).  All compute runs in hand-written sm_103a kernels
 * on the caller's CUDA stream; there is no CPU fallback.
 *
 * Conventions shared by every call
 *   - Images are row-major [z][u]: rows run along the rotation axis z,
 *     columns along u.  Stacks are [angle][row][col].
 *   - Intensities arrive centred (q = 0 at pixel (N/2, N/2)).
 *   - Forward FFTs are unnormalised with exp(-2 pi i jk/N); inverse FFTs carry
 *     1/N per axis.
 *   - Pointers may be host or device memory; the library tells them apart
 *     with cudaPointerGetAttributes.  Host memory is read or written with
 *     stream-ordered copies; a call that reads host memory returns after its
 *     data was consumed, a call that writes host memory returns after the
 *     data is there.  Device pointers are used in stream order on the plan's
 *     stream; the caller keeps them alive until the stream has passed them.
 *   - Every call returns a cpra_status and never aborts or throws.  A failing
 *     call records a message readable with cpra_last_error(plan)
 *     (cpra_last_error(NULL) for failures without a plan).
 */
#ifndef CPRA_H
#define CPRA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cpra_plan_s* cpra_plan_t;

typedef enum {
  CPRA_OK = 0,
  CPRA_ERR_INVALID_ARG = 1,   /* bad size, pointer, weight or input value   */
  CPRA_ERR_OUT_OF_MEMORY = 2, /* the allocator returned NULL               */
  CPRA_ERR_CUDA = 3,          /* a CUDA runtime call failed                */
  CPRA_ERR_NOT_READY = 4,     /* inputs missing (e.g. angles not loaded)   */
  CPRA_ERR_TIMEOUT = 5,       /* a bounded device wait gave up             */
  CPRA_ERR_UNSUPPORTED = 6,   /* valid request the library cannot run     */
  CPRA_ERR_NONFINITE = 7      /* a non-finite iterate (diverged, NaN state) */
} cpra_status;

/* Device-side failures.  Each plan has a status word in pinned host memory
 * that its kernels write (cudaHostAlloc, mapped; besides the device buffers
 * the allocator callbacks provide).  The kernel that publishes an angle's
 * FP64 Fourier error flags it when the error sums are not finite: a
 * non-finite iterate (a diverged run, a loaded state holding NaN or Inf) or
 * an invalid pattern (a negative or non-finite intensity, which the
 * preparation turns into a NaN error constant).  Calls read the word without
 * waiting for the stream: cpra_iterate, cpra_assemble_3d, cpra_refine_3d,
 * cpra_result and cpra_batch_iterate report a flag set by work that has
 * completed by the time they are called, and every call that waits for the
 * stream (cpra_sync, results copied to host memory, cpra_iterate with
 * err_out) reports a flag set by any work queued before it.  The status is
 * CPRA_ERR_INVALID_ARG (naming the angle) when a loaded pattern was invalid,
 * CPRA_ERR_NONFINITE otherwise; it stays set until cpra_reset or
 * cpra_load_state clears it. */

enum { CPRA_WRAP_LITERAL = 0, CPRA_WRAP_MIRROR = 1 };
enum { CPRA_BLEND_STATE = 0, CPRA_BLEND_OBJECT = 1 };
enum { CPRA_FP32 = 0, CPRA_BF16_TC = 1, CPRA_FP16_TC = 2 };
enum { CPRA_UPDATE_HIO = 0, CPRA_UPDATE_RAAR = 1 };
enum {
  CPRA_ENGINE_AUTO = 0,
  CPRA_ENGINE_TWO_PASS = 1,
  CPRA_ENGINE_FUSED = 2,
  CPRA_ENGINE_WARP = 3,
  CPRA_ENGINE_TUNED = 4
};
enum {
  CPRA_RESULT_PO = 0,      /* Np*N*N float: P_{S+} g (iterate on its valid set)  */
  CPRA_RESULT_STATE = 1,   /* Np*N*N float: the iterate g itself                 */
  CPRA_RESULT_SUPPORT = 2, /* Np*N*N uint8: support, 1 inside                    */
  CPRA_RESULT_ERRORS = 3,  /* t*Np double: Fourier error of every iteration so far,
                              [iteration][angle]                                 */
  CPRA_RESULT_VOLUME = 4,  /* N*N*N complex64 [z][y][x], centred (after assemble
                              or merge)                                          */
  CPRA_RESULT_MERGED_SPECTRA = 5 /* Np*N*N complex64 [angle][kz][ku], FFT order: the
                              merged spectra E_n of the last cpra_merge into this
                              plan (NOT_READY before)                             */
};

#define CPRA_MAX_TAPS 15

/*
 * Reconstruction parameters.  cpra_default_config fills the paper's example
 * values; fields map to the paper as follows.
 *   N, Np          pattern size and number of angles (Eq. 1-3).  N = 2^a 3^b,
 *                  a multiple of 16, 16 <= N <= 1024; Np >= 1.
 *   n_ei           conventional 2D iterations per episode, N_ei (Step B).
 *   n_taps, alpha  coupling weights alpha_k, k = -(n_taps/2)..n_taps/2 (Eq. 4);
 *                  n_taps odd, <= CPRA_MAX_TAPS, sum 1 within 1e-12.
 *   beta           feedback of the update rule: HIO's beta (Fienup) or RAAR's
 *                  relaxation (Luke); the paper uses 0.9 for both.
 *   wrap_mode      180-degree seam: LITERAL couples angle Np-1 with angle 0 as
 *                  is; MIRROR flips u once per wrap.
 *   blend_target   STATE blends the iterate g, OBJECT blends P_{S+} g.
 *   hio_iters, er_iters  global schedule: iteration t runs the update rule
 *                  (HIO or RAAR, see `update`) while t < hio_iters, ER
 *                  afterwards.
 *   shrinkwrap_every, sw_sigma, sw_tau   support update after iteration t
 *                  when (t+1) % every == 0 (0 = off): blur P_{S+} g with a
 *                  periodic Gaussian of sw_sigma pixels and keep pixels at or
 *                  above sw_tau times the maximum (the paper's 0.1 threshold).
 *   n_pre          Step A: iterations of the update rule run on angle 0
 *                  alone before t = 0.
 *   precision      CPRA_FP32 (default) or tensor-core FFT stages.
 *   com_align      1: move each PO's mass centre to the origin before
 *                  assembly (Step C); 0: use the frame centre.
 *   engine         kernel family.  TWO_PASS: row and column passes with
 *                  block-wide shared-memory FFTs (every supported N).  WARP:
 *                  the same passes with warp-resident two-level FFTs
 *                  (N = 64, 128, 256, 512, 1024).  FUSED: one launch per
 *                  run of iterations between coupling steps, each angle's
 *                  spectrum held in the distributed shared memory of a
 *                  thread-block cluster (N = 64, 128, 256, 512; FP32; needs a
 *                  GPU that can hold an N/32-CTA cluster at N = 512, an
 *                  N/64-CTA cluster below, else UNSUPPORTED at cpra_plan).
 *                  AUTO: FUSED for N <= 256 in FP32 where the device holds
 *                  its clusters, else WARP where available, else TWO_PASS.
 *                  TUNED: the fastest engine for this N on this GPU
 *                  according to cpra_autotune (its default cache).
 *   update         real-space rule of the iterations before hio_iters.
 *                  CPRA_UPDATE_HIO (default): g' on V = {x in S, g'(x) >= 0},
 *                  g - beta g' elsewhere.  CPRA_UPDATE_RAAR (relaxed averaged
 *                  alternating reflections, Luke 2005; the paper's rule for
 *                  its S. aureus data): g' on {x in S, 2 g'(x) - g(x) >= 0},
 *                  beta g + (1 - 2 beta) g' elsewhere, which is
 *                  beta/2 (R_S R_M + I) g + (1 - beta) P_M g with the
 *                  reflections R = 2P - I of the support-positivity and
 *                  modulus projections.
 *   sweep          0 (default): Jacobi episodes, every angle starts an
 *                  episode from Eq. 4 over the previous episode (the
 *                  equation's literal form; all angles run in parallel).
 *                  1: Gauss-Seidel sweep (Step B's "consecutively, from n = 1
 *                  to N_p"): angle n starts from Eq. 4 with this episode's
 *                  images of the angles before it and the previous
 *                  episode's of the others, and runs its n_ei iterations
 *                  before angle n + 1 starts, so one episode carries a
 *                  pre-reconstructed PO around the whole carousel.  Calls
 *                  run whole episodes (t and n_iters multiples of n_ei);
 *                  shrink-wrap runs at episode ends (shrinkwrap_every a
 *                  multiple of n_ei); no present mask (UNSUPPORTED);
 *                  batches run many sweep plans together.
 *   seed           seeds the random initial guess (SplitMix64 per pixel).
 *   alloc, free, alloc_ctx  device allocator; NULL alloc = cudaMalloc.
 */
typedef struct {
  int32_t N, Np;
  int32_t n_ei;
  int32_t n_taps;
  double alpha[CPRA_MAX_TAPS];
  float beta;
  int32_t wrap_mode;
  int32_t blend_target;
  int32_t hio_iters, er_iters;
  int32_t shrinkwrap_every;
  float sw_sigma, sw_tau;
  int32_t n_pre;
  int32_t precision;
  int32_t com_align;
  int32_t engine;
  int32_t update;
  int32_t sweep;
  uint64_t seed;
  void* (*alloc)(size_t bytes, void* ctx);
  void (*free)(void* ptr, void* ctx);
  void* alloc_ctx;
} cpra_config;

/* Fill *cfg with defaults for an N x N, Np-angle problem: n_ei 10, alpha
 * (0.2, 0.6, 0.2) and beta 0.9 (the paper's Eq. 4 example and HIO value),
 * 200 HIO + 20 ER, shrink-wrap off, sigma 2, tau 0.1, LITERAL, STATE, FP32,
 * com_align 1, engine AUTO, update HIO, sweep 0, seed 0, cudaMalloc.  Returns INVALID_ARG for a NULL cfg. */
cpra_status cpra_default_config(int32_t N, int32_t Np, cpra_config* cfg);

/* Device bytes a plan for *cfg holds while iterating (iter_bytes) and the
 * extra bytes cpra_assemble_3d allocates (assemble_bytes); either may be NULL.
 * Used for admission by free HBM.  Validates cfg like cpra_plan. */
cpra_status cpra_plan_bytes(const cpra_config* cfg, size_t* iter_bytes, size_t* assemble_bytes);

/* Create a plan: validate *cfg (copied), allocate the iteration state through
 * cfg->alloc and build FFT twiddle tables (FP64 on the host, stored FP32).
 * stream is a cudaStream_t (NULL = legacy default stream); the plan uses it
 * for all work.  On failure *out is NULL and the status says why
 * (INVALID_ARG, UNSUPPORTED for N outside the supported set,
 * OUT_OF_MEMORY, CUDA). */
cpra_status cpra_plan(const cpra_config* cfg, void* stream, cpra_plan_t* out);

/* Load `count` centred intensity patterns I[count][N][N] (float32) for angles
 * first_angle .. first_angle+count-1 with their angles theta_rad[count]
 * (radians, host memory, may be NULL to keep theta_n = n*pi/Np).  Prepares
 * A = sqrt(I) in FFT order, its Hermitian-symmetrised half plane and the FP64
 * error constants (Eq. 1-3).  The call queues the upload and the preparation
 * and returns without waiting for them.  An upload from host memory runs on
 * a second, plan-owned stream into a plan-owned buffer (Np*N*N floats,
 * allocated on the first host upload through the plan's allocator), so it
 * overlaps work already queued on the plan's stream; the preparation on the
 * plan's stream waits for it, and a later upload waits until the
 * preparation has read the buffer.  Host buffers in pinned memory must stay
 * unchanged until the plan's stream has passed the preparation (cpra_sync);
 * pageable buffers are copied before the call returns.  Non-finite or
 * negative intensities are reported by the first iteration on them, through
 * the plan's status word (see above: INVALID_ARG naming the angle). */
cpra_status cpra_load_intensities(cpra_plan_t plan, const float* I, int32_t first_angle,
                                  int32_t count, const double* theta_rad);

/* Missing data (the beamstop of measured patterns): mask marks the measured
 * pixels (uint8, nonzero = measured), centred like the intensities;
 * per_angle = 1: mask is [Np][N][N], 0: one [N][N] mask for every angle;
 * NULL: every pixel measured (the default).  It applies to the intensities
 * loaded after the call.  A frequency pair {k, -k} is constrained only when
 * both pixels are measured (a real PO has |G(-k)| = |G(k)|, and a centred
 * beamstop is symmetric): the modulus projection leaves the others' G as it
 * is and the Fourier error sums over the constrained pixels only.  Paper:
 * its cell patterns were cropped with a beamstop in the centre (results
 * section).  Host or device memory; the copy is queued on the plan's stream
 * (pinned host buffers must stay unchanged until the stream has passed it). */
cpra_status cpra_load_mask(cpra_plan_t plan, const uint8_t* mask, int32_t per_angle);

/* Set the support from S (uint8, nonzero = inside).  per_angle = 1: S is
 * [Np][N][N]; per_angle = 0: one [N][N] mask for every angle.  S = NULL sets
 * the padded bounding box (central N/2 x N/2 square) for every angle.  Like
 * cpra_load_intensities, the call returns once the copy is queued. */
cpra_status cpra_load_support(cpra_plan_t plan, const uint8_t* S, int32_t per_angle);

/* Checkpoint restore: set the iterate g[Np][N][N] (float32) and the global
 * iteration counter t (>= 0).  Without this call the first cpra_iterate
 * starts from the seeded random guess on the current support (Step A).
 * Waits for the plan's stream and clears its status word. */
cpra_status cpra_load_state(cpra_plan_t plan, const float* g, int64_t t);

/* Run n_iters global iterations (Step B): coupling (Eq. 4) before every
 * iteration t with t % n_ei == 0, then FFT -> modulus projection -> inverse
 * FFT -> HIO/RAAR/ER update for every angle, shrink-wrap on schedule.  If err_out
 * is not NULL it receives the Fourier error of every angle and iteration,
 * err_out[i*Np + n] (double, host or device).  Returns NOT_READY until every
 * iterating angle (every angle unless cpra_set_present restricted them) has
 * intensities. */
cpra_status cpra_iterate(cpra_plan_t plan, int32_t n_iters, double* err_out);

/* Let only the angles with mask[n] != 0 iterate (mask: host memory, Np
 * bytes, read during the call; NULL = every angle), so that a reconstruction
 * can start while its patterns are still arriving.  Reading of the paper's
 * concurrent partial reconstruction: the iterating angles run Step B as
 * usual, and Eq. 4 couples each of them with its present neighbours only,
 * the alpha_k of the present taps divided by their sum; absent angles keep
 * their state (the seeded start until they join) and their error entries
 * stay 0.  INVALID_ARG when no angle is present, UNSUPPORTED with
 * shrink-wrap on; cpra_assemble_3d returns NOT_READY while an angle is
 * absent.  Batches follow a member's mask from their next iterate call. */
cpra_status cpra_set_present(cpra_plan_t plan, const uint8_t* mask);

/* Step D: spectra of P_{S+} g with the centre-of-mass phase ramp, Fourier
 * slice gridding (bilinear in kx, ky; exact kz) into an N^3 grid, inverse 3D
 * FFT.  The centred complex64 volume [z][y][x] stays in the plan (read it
 * with CPRA_RESULT_VOLUME) and is also copied to out_volume when that is not
 * NULL (N^3 * 8 bytes, host or device). */
cpra_status cpra_assemble_3d(cpra_plan_t plan, void* out_volume);

/* cpra_assemble_3d, then a download of the volume to out that the call does
 * not wait for: the volume is copied device-to-device into a plan-owned
 * staging buffer (N^3 * 8 bytes, allocated on first use through the plan's
 * allocator) on the plan's stream, and from there to out on a second,
 * plan-owned stream, so that whatever the caller queues next on the plan
 * (the next reconstruction's upload and iterations) overlaps the download.
 * out: page-locked host memory (cudaHostAlloc or cudaHostRegister), N^3
 * complex floats; INVALID_ARG for any other memory.  The caller must leave
 * out alone until cpra_download_wait returns.  A later call orders its
 * staging copy after the previous download on the device; the host never
 * waits here.  Errors as cpra_assemble_3d. */
cpra_status cpra_assemble_3d_async(cpra_plan_t plan, void* out);

/* Wait until every download cpra_assemble_3d_async queued has landed in host
 * memory, then report the plan's status word as a waiting call does
 * (CPRA_OK when nothing is pending). */
cpra_status cpra_download_wait(cpra_plan_t plan);

/* Step C (repeating and merging): combine n_r finished reconstructions of
 * the same patterns, each from its own random start (its own seed), into one
 * episode and assemble it (Step D) into dst's volume.
 *   1. Keep the n_l guesses of lowest reconstruction error, best first; the
 *      error of a guess is the mean over its POs of the Fourier error of its
 *      last iteration.
 *   2. Move the mass centre of every PO of every kept guess to the origin
 *      (Delta r_n = -int O'_n r dv, as a phase ramp on its spectrum
 *      E_n = FFT2(P_{S+} g_n), as in cpra_assemble_3d).
 *   3. Twin: compare PO twin_ref of each kept guess with PO twin_ref of the
 *      best one, as is and centrally inverted (spectrum conj(E_n)); the
 *      version at the smaller Euclidean distance (computed on the spectra,
 *      Parseval) is used for every PO of that guess.
 *   4. Average the corrected spectra: the final E_n, readable as
 *      CPRA_RESULT_MERGED_SPECTRA; gridding and the inverse 3D FFT put the
 *      volume into dst (CPRA_RESULT_VOLUME).
 *   guesses   n_r plans with dst's N and Np (dst may be one of them), every
 *             angle present and at least one iteration run
 *   twin_ref  the PO compared for the twin choice, 0 <= twin_ref < Np
 *   dst       receives the merged spectra and volume; its angles grid them
 *   selected  NULL or host int32[n_l]: the kept guesses, best first
 *   inverted  NULL or host int32[n_l]: 1 where that guess was inverted
 *   prtf      NULL or float32[Np][N/2] (host or device): per PO, the phase
 *             retrieval transfer function |sum_g E'_g| / sum_g |E'_g| over the
 *             kept, corrected guesses, averaged over rings round(|k|) = s
 *             (signed k), s = 0..N/2-1 (0 where sum |E'| = 0)
 * Paper: Step C (N_r random guesses, the N_l best kept, mass-centre move,
 * twin choice against the best episode, averaging); PRTF as in its results
 * section (its ref. 23).  The call runs on the guesses' and dst's streams and
 * returns when the merge is complete.  Besides the assembly buffers, dst
 * allocates about 8 N^2 Np bytes of scratch on first use (4 N^2 Np more
 * with prtf).  Each guess's
 * state is only read; its row spectra buffer is reused.  INVALID_ARG for bad
 * counts, sizes or pointers, NOT_READY for a guess that has not iterated or
 * has absent angles. */
cpra_status cpra_merge(const cpra_plan_t* guesses, int32_t n_r, int32_t n_l, int32_t twin_ref,
                       cpra_plan_t dst, int32_t* selected, int32_t* inverted, float* prtf);

/* Step D refinement: the paper's tomographic 3D reconstruction "like
 * conventional 3D CXDI but using E(q)" (about 50 iterations, the 3D support
 * from the 2D supports projected back, shrunk every 5 iterations in its cell
 * example).  Alternating projections on the plan's Step D result:
 *   V = the gridded spectrum E(q) (the FFT of the last volume of
 *       cpra_assemble_3d or cpra_merge), M = the (kx, ky) cells the slices
 *       reach (every kz);
 *   S3 = voxels whose projection lands inside the plan's current 2D support
 *       at every angle (nearest pixel in u, exact z), each 2D support first
 *       moved by the whole-pixel part of its PO's mass-centre move (the
 *       plan's own state; no move with com_align 0);
 *   the iteration runs on the centred volume (the frame of the supports);
 *   start: rho = the real part of that volume;
 *   each iteration: X = FFT3(P_{S3+} rho); X <- V on M; rho = Re IFFT3(X);
 *   after iteration t with (t+1) % shrink_every == 0 (0 = never):
 *   S3 <- {blur(P_{S3+} rho) >= tau * max}, blur = periodic Gaussian of
 *   sigma voxels along x, y, z.
 * The refined volume P_{S3+} rho replaces the plan's volume (centred,
 * complex64 with imaginary part 0; CPRA_RESULT_VOLUME).  Successive calls
 * continue the refinement (and its shrink-wrap count); the next assemble or
 * merge restarts it.  err_out (NULL, or n_iters doubles, host or device):
 * sqrt(sum_M |X - V|^2 / sum_M |V|^2) of every iteration (FP64 sums).
 * Allocates about 25 N^3 bytes on first use.  NOT_READY without a Step D
 * volume, INVALID_ARG for negative counts or bad shrink-wrap parameters.
 * Runs on the plan's stream; returns after queuing (after the copy when
 * err_out is given). */
cpra_status cpra_refine_3d(cpra_plan_t plan, int32_t n_iters, int32_t shrink_every, float sigma,
                           float tau, double* err_out);

/* Copy one result (CPRA_RESULT_*) into dst, which holds `bytes` bytes (host
 * or device).  INVALID_ARG if bytes is smaller than the result, NOT_READY for
 * a volume before cpra_assemble_3d. */
cpra_status cpra_result(cpra_plan_t plan, int32_t what, void* dst, size_t bytes);

/* Restart the reconstruction: t = 0, the error history is cleared and the
 * next cpra_iterate starts again from the seeded guess (Step A).
 * Intensities, angles and the current support are kept.  A set status word
 * (device-side failure) is cleared after waiting for the plan's stream; a
 * failure that work queued before the reset flags after it is reported on
 * the new run, so call cpra_sync first to see it on the old one. */
cpra_status cpra_reset(cpra_plan_t plan);

/* Kernel classes for cpra_kernel_stats. */
enum {
  CPRA_KERNEL_COLPASS = 0,   /* two-pass engine: column FFT + modulus projection */
  CPRA_KERNEL_ROWPASS = 1,   /* two-pass engine: C2R + HIO/ER + R2C rows          */
  CPRA_KERNEL_PRIME = 2,     /* coupling (Eq. 4) + R2C rows                        */
  CPRA_KERNEL_SHRINKWRAP = 3,
  CPRA_KERNEL_ASSEMBLE = 4,
  CPRA_KERNEL_FUSED = 5,     /* fused engine: prime + a run of whole iterations    */
  CPRA_KERNEL_PREPARE = 6,
  CPRA_KERNEL_REFINE = 7,    /* Step D refinement (3D line passes, support)       */
  CPRA_KERNEL_KINDS = 8
};

/* Device-time profiling: with on = 1 the plan records CUDA events around each
 * of its kernel launches on its stream (a small overhead per launch).
 * cpra_kernel_stats waits for the stream and returns, for one kernel class,
 * the summed device milliseconds and the launch count since profiling was
 * switched on (or since the last cpra_set_profiling call). */
cpra_status cpra_set_profiling(cpra_plan_t plan, int32_t on);
cpra_status cpra_kernel_stats(cpra_plan_t plan, int32_t kind, double* total_ms, int64_t* launches);

/* Number of kernels this library has launched in this process. */
int64_t cpra_launch_count(void);

/* Shrink-wrap support update without any device allocation.
 *
 * The paper has no counterpart: this is a library service.  It runs the same
 * kernels and the same arithmetic as the shrink-wrap step of cpra_iterate
 * (blur P_{S+} g with the periodic Gaussian of sigma pixels, keep pixels at
 * or above tau times each pattern's maximum; a pattern whose maximum is 0
 * keeps S_in), for callers that cannot call cudaMalloc: cudaMalloc and
 * cudaFree can synchronize the whole device and take driver locks, which a
 * pipeline that must keep up with a detector while other work runs on the
 * same GPU, or a process that has handed its whole memory budget to another
 * allocator, cannot afford.  Plans allocate through cpra_config.alloc; this
 * call allocates nothing.
 *
 *   g      count*N*N float32, device memory: iterates [count][N][N]
 *   S_in   count*N*N uint8, device memory: current supports (nonzero = in)
 *   S_out  count*N*N uint8, device memory: new supports (0/1); may be S_in
 *   stream cudaStream_t the work is queued on (NULL = legacy default stream)
 *
 * Scratch lives in file-scope device arrays of the library (about 8.3 MB on
 * every GPU that loads it, held until the process exits).  The first call on
 * a device looks up their addresses on that device (cudaGetSymbolAddress);
 * make that first call before any stream capture.  Every call shares the
 * arrays, so calls that overlap on the GPU race: queue them on one stream or
 * order them.  count*N*N may be at most CPRA_SHRINKWRAP_STATIC_MAX_PIXELS
 * (2^20, e.g. 4 patterns of 512^2 or 256 of 64^2); larger requests return
 * INVALID_ARG.  Host pointers, and device pointers of a device other than
 * the current one, return INVALID_ARG.  The Gaussian taps are passed to the
 * device as a kernel argument, so no host buffer outlives the call.  The
 * call returns after queuing the work; errors are readable with
 * cpra_last_error(NULL). */
#define CPRA_SHRINKWRAP_STATIC_MAX_PIXELS (1 << 20)
cpra_status cpra_shrinkwrap_static(const float* g, const uint8_t* S_in, uint8_t* S_out, int32_t N,
                                   int32_t count, float sigma, float tau, void* stream);

/* ------------------------------------------------------------------------
 * Batching (many reconstructions per launch) and the engine autotuner.
 *
 * A batch iterates several plans together: for every group of plans with
 * the same N and engine, each kernel of an iteration runs as ONE launch
 * whose tiles are the (plan, angle) pairs of the whole group (for the FUSED
 * engine: one launch per round, round r running every member's r-th run of
 * iterations between its coupling steps); each plan
 * keeps its own schedule (its own t, episode boundaries, HIO/ER switch), so
 * every plan computes exactly what cpra_iterate would (bit-identical).  With
 * use_graph = 1 the launches of one cpra_batch_iterate call are captured
 * once into a CUDA graph and replayed while the call pattern repeats.
 * Paper: the reconstructions are independent (Steps A-B per guess and per
 * object); this is a throughput form, not a step of the method.
 * ------------------------------------------------------------------------ */
typedef struct cpra_batch_s* cpra_batch_t;

/* plans: n plans (n >= 1) on the same device, all using plans[0]'s stream.
 * Jacobi plans must not use shrink-wrap (UNSUPPORTED).  Gauss-Seidel plans
 * (sweep 1) of the same N, engine and n_ei form a group whose sweeps run
 * together: their Step A as rows over every member's angle 0, then one
 * launch per angle of the sweep (fused engine; prime + n_ei column and row
 * launches otherwise) over every member that has that angle, shrink-wrap at
 * episode ends; calls must run whole episodes (INVALID_ARG otherwise) and
 * are not captured in a graph.  Plans must stay alive until
 * cpra_batch_destroy.  The batch holds device tables only. */
cpra_status cpra_batch_create(const cpra_plan_t* plans, int32_t n, int32_t use_graph,
                              cpra_batch_t* out);

/* Advance every plan of the batch by n_iters iterations (NOT_READY if a plan
 * lacks intensities).  Error histories are kept per plan. */
cpra_status cpra_batch_iterate(cpra_batch_t batch, int32_t n_iters);

/* Number of kernel launches one cpra_batch_iterate(n_iters) issues (or the
 * graph holds); -1 for a NULL batch. */
int64_t cpra_batch_launches(cpra_batch_t batch, int32_t n_iters);

/* Persistent work-queue mode (mode 1; 0 returns to one launch per kernel
 * and size group).  Each call then splits at the iterations where a member
 * couples (Eq. 4 at its episode starts); for every such segment the size
 * groups' coupling launches run first, then ONE persistent launch per size
 * group runs all of the segment's column and row passes of every (member,
 * angle) tile: its CTAs take tasks from a device queue and wait on
 * per-tile completion counts instead of launch boundaries, so an angle's
 * row pass starts as soon as its own column pass is done.  The queue runs
 * the tiles in chunks of chunk_tiles: a chunk takes every iteration of the
 * segment (column tasks of its tiles, then their row tasks, block by block)
 * before the next chunk starts, so a chunk's iterates, spectra and
 * amplitudes stay in L2 between passes.  chunk_tiles = 0 takes as many
 * tiles as half the device's L2 holds (about 10 N^2 bytes a tile); a value
 * of at least the group's tile count gives the plain (iteration, pass,
 * tile, block) order.  The groups' launches are forked onto a stream each
 * (in the CUDA graph when the batch uses one), so one size group's tail
 * overlaps the next group's start.  Every tile computes what the warp
 * engine computes for it alone (states bit for bit; FP64 error sums to
 * rounding).  Needs every Jacobi group on the FP32 warp engine with
 * N in {64, 128, 192, 256, 384, 512} (UNSUPPORTED otherwise).
 * wait_budget_s bounds every device-side wait (0 = 2 s): a wait that runs
 * out sets TIMEOUT in the members' status words (reported by their next
 * calls, see cpra_sync) and ends its CTA.  Mode 2 exists to test that path:
 * the first task of every launch waits on a count that no task increments.
 * The paper has no batching: this serves several reconstructions at once
 * for throughput.  Waits for the batch's stream. */
cpra_status cpra_batch_set_persistent(cpra_batch_t batch, int32_t mode, double wait_budget_s,
                                      int32_t chunk_tiles);

cpra_status cpra_batch_destroy(cpra_batch_t batch);

/* Autotuner: time each engine available for N (TWO_PASS, WARP, FUSED) on a sample
 * of 64 random patterns with CUDA events on a private stream, and keep the
 * fastest per (N, precision, SM count, device name) in a JSON cache file.
 * cache_path NULL = $CPRA_TUNE_CACHE or $HOME/.cache/cpra_tune.json.  A
 * cached entry is returned without timing.  *engine_out receives the engine,
 * *ms_out (nullable) the measured or cached milliseconds per iteration of the
 * sample. */
cpra_status cpra_autotune(int32_t N, int32_t precision, const char* cache_path,
                          int32_t* engine_out, double* ms_out);

/* ------------------------------------------------------------------------
 * Serving: continuous batching of reconstructions while patterns stream in.
 *
 * A library-owned host thread admits submitted requests in order while the
 * device's free memory minus the request's footprint (cpra_plan_bytes:
 * iteration state + assembly) stays above hbm_reserve_bytes; prepares the
 * patterns pushed for resident requests as they arrive; and advances every
 * request whose angles have all arrived (with early_start: whose first
 * angles have arrived) in rounds of iters_per_round iterations, all running
 * requests together through one batch (see cpra_batch_create), so requests
 * arriving while others run join at the next round.  After its first
 * episode with every angle present (n_ei iterations) a request gets a
 * first 3D estimate (cpra_assemble_3d), after hio_iters + er_iters
 * iterations its final volume.  Without early_start each request computes
 * exactly what a standalone plan would; with it, what a plan computes whose
 * present mask follows the arrivals round by round.  The paper motivates this by reconstructing while
 * the experiment runs ("concurrent partial reconstructions", concluding
 * section); the serving loop itself has no counterpart in the paper.
 * Times are seconds since cpra_server_start.
 * ------------------------------------------------------------------------ */
typedef struct cpra_server_s* cpra_server_t;

typedef struct {
  size_t hbm_reserve_bytes;  /* device memory left free (default 2 GiB)        */
  int32_t max_active;        /* resident requests at most (0 = no limit)        */
  int32_t iters_per_round;   /* iterations per batched round (default 10)       */
  int32_t use_graph;         /* capture each round's launches in a CUDA graph   */
  void* stream;              /* cudaStream_t of the serving thread (NULL = own) */
  int32_t early_start;       /* 1: a request iterates its arrived angles while the
                                others stream in (cpra_set_present), holding its
                                last early_tail iterations until every angle is
                                there; 0 (default): it starts once every angle
                                arrived                                         */
  int32_t early_tail;        /* iterations kept for after the last pattern with
                                early_start (0 = half the schedule, rounded up
                                to whole episodes; at least one episode)        */
} cpra_server_config;

enum { CPRA_EVENT_FIRST_ESTIMATE = 1, CPRA_EVENT_FINAL = 2, CPRA_EVENT_FAILED = 3 };

typedef struct {
  int64_t id;
  int32_t kind;            /* CPRA_EVENT_*                                 */
  double t_event;          /* when it happened                             */
  double t_submit;         /* when the request was submitted               */
  double t_last_pattern;   /* when its latest pattern push arrived         */
} cpra_server_event;

typedef struct {
  int32_t state;           /* 0 queued, 1 resident, 2 running, 3 done, 4 failed */
  int64_t iterations_done;
  int32_t angles_arrived;
  double t_submit, t_admit, t_last_pattern, t_first_estimate, t_final;  /* -1 = not yet */
} cpra_server_request;

typedef struct {
  int64_t submitted, admitted, completed, rounds, max_batch, angle_iterations;
} cpra_server_stats;

cpra_status cpra_server_default_config(cpra_server_config* cfg);
/* Start the serving thread on the current device. */
cpra_status cpra_server_start(const cpra_server_config* cfg, cpra_server_t* out);
/* Queue a request (cfg is copied; shrink-wrap and the Gauss-Seidel sweep
 * unsupported; the serving thread allocates with cudaMalloc, cfg->alloc is
 * ignored). */
cpra_status cpra_server_submit(cpra_server_t s, const cpra_config* cfg, int64_t* request_id);
/* Stream count patterns [count][N][N] (host or device float32, centred) for
 * angles first..first+count-1, with optional angles theta (host).  The data
 * are copied before the call returns. */
cpra_status cpra_server_push(cpra_server_t s, int64_t request_id, const float* I, int32_t first,
                             int32_t count, const double* theta);
/* Take up to max_events finished events (non-blocking); *got = how many. */
cpra_status cpra_server_poll(cpra_server_t s, cpra_server_event* ev, int32_t max_events,
                             int32_t* got);
/* Block until the request is done (TIMEOUT after timeout_s seconds). */
cpra_status cpra_server_wait(cpra_server_t s, int64_t request_id, double timeout_s);
cpra_status cpra_server_request_info(cpra_server_t s, int64_t request_id, cpra_server_request* info);
/* cpra_result of a finished request (NOT_READY before). */
cpra_status cpra_server_result(cpra_server_t s, int64_t request_id, int32_t what, void* dst,
                               size_t bytes);
/* Free a finished request's device memory. */
cpra_status cpra_server_release(cpra_server_t s, int64_t request_id);
cpra_status cpra_server_get_stats(cpra_server_t s, cpra_server_stats* out);
/* Stop the thread and free every request. */
cpra_status cpra_server_stop(cpra_server_t s);

/* Global iteration counter t of the plan (-1 for a NULL plan). */
int64_t cpra_iteration(cpra_plan_t plan);

/* Wait for the plan's stream; reports device-side failures (CUDA, and the
 * status word: INVALID_ARG for an invalid pattern, NONFINITE). */
cpra_status cpra_sync(cpra_plan_t plan);

/* Free every device buffer through cfg->free and the plan itself. */
cpra_status cpra_destroy(cpra_plan_t plan);

/* Message of the last failure on this plan (NULL plan: last failure of a
 * call that had no plan on this thread).  The string lives until the next
 * call on the same plan. */
const char* cpra_last_error(cpra_plan_t plan);

#ifdef __cplusplus
}
#endif

#endif /* CPRA_H */
