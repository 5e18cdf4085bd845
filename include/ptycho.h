/*
 * ptycho.h -- C ABI of a B300-native (sm_103a) library for the per-iteration
 * hot path of ptychographic reconstruction: ePIE, DM and LSQML.
 *
 * The ptychopy paper (Yue et al., arXiv 2202.03144) exposes its CUDA engine
 * through a "whole" call per algorithm and a "step" API -- init (parameters,
 * data upload, sample/probe initialisation), step (iterations on the GPU),
 * resobj/resprobe (copy results back at any time), post (free) -- Sec. 3.2,
 * Fig. 3 and Listing 1.  This header is that step API with plain pointers:
 *
 *   paper            this ABI
 *   epieinit()       ptycho_create + ptycho_set_data + ptycho_set_init
 *   epiestep()       ptycho_iterate(ctx, alg, 1)
 *   epie(para)       ptycho_iterate(ctx, alg, n)
 *   epieresobj()     ptycho_get_object
 *   epieresprobe()   ptycho_get_probe
 *   epiepost()       ptycho_destroy
 *
 * Conventions used by every entry point
 * -------------------------------------
 *  - Complex arrays are interleaved float32 pairs (re, im), row-major.
 *    object: [obj_ny][obj_nx][2]; probe: [K][M][M][2];
 *    exit waves / residuals: [J][K][M][M][2].
 *  - intensities: [J][M][M] float32, detector-centred (zero spatial
 *    frequency at pixel (M/2, M/2)); a negative value marks a masked pixel
 *    (saturated or bad, Sec. 2.2), which the modulus projection leaves free.
 *  - positions: [J][2] float32 (y, x) of each patch's top-left corner on the
 *    object grid, in pixels; rounded half-to-even to integers, or, with
 *    ptycho_params.subpixel = S, quantised to 1/S pixel with the probe
 *    Fourier-shifted by the fractional part.  Every patch must lie inside
 *    the object.
 *  - on_device != 0: the pointer is CUDA device memory of the current device;
 *    otherwise it is host memory (pageable or pinned).
 *  - Ownership: the library COPIES every input; the caller keeps its
 *    buffers.  get_* calls write into caller memory and may be made at any
 *    time without disturbing the reconstruction (Sec. 3.2, step mode).
 *  - Stream: all GPU work is issued on ptycho_params.stream (a cudaStream_t;
 *    NULL = the legacy default stream).  Only get_*, fourier_error and the
 *    host-pointer variants synchronise that stream.
 *  - Errors: every int-returning call returns PTYCHO_OK (0) or a negative
 *    PTYCHO_ERR_* code; ptycho_last_error() gives a message.  After an error
 *    the context stays valid and can be destroyed (or used again).
 *  - The library allocates its device memory with cudaMalloc at
 *    ptycho_create/ptycho_set_data and frees it in ptycho_destroy.
 */
#ifndef PTYCHO_H
#define PTYCHO_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ptycho_ctx ptycho_ctx;

/* Reconstruction algorithms (Abstract, Sec. 2.3). */
enum { PTYCHO_EPIE = 0, PTYCHO_DM = 1, PTYCHO_LSQML = 2 };

/* Storage precision of the measured data on the device.  F16/BF16 store
 * sqrt(I) divided by its per-frame maximum, plus one float32 scale per frame;
 * all arithmetic stays float32. */
enum { PTYCHO_I_F32 = 0, PTYCHO_I_F16 = 1, PTYCHO_I_BF16 = 2 };

/* Storage of LSQML's residuals between the passes of an iteration
 * (ptycho_params.residual_store). */
enum { PTYCHO_R_F32 = 0, PTYCHO_R_F16 = 1 };

/* Transform engine of the Fourier passes (ptycho_params.fft_engine). */
enum { PTYCHO_FFT_AUTO = -1, PTYCHO_FFT_REGISTER = 0, PTYCHO_DFT_TENSOR_BF16X3 = 1 };

/* LSQML likelihood (ptycho_params.likelihood). */
enum { PTYCHO_LIK_AMPLITUDE = 0, PTYCHO_LIK_POISSON = 1 };

#define PTYCHO_OK 0
#define PTYCHO_ERR_ARG (-1)         /* bad argument or size                     */
#define PTYCHO_ERR_BOUNDS (-2)      /* a patch falls outside the object         */
#define PTYCHO_ERR_NONFINITE (-3)   /* NaN/Inf in an input                      */
#define PTYCHO_ERR_OOM (-4)         /* device allocation failed                 */
#define PTYCHO_ERR_CUDA (-5)        /* a CUDA call failed                       */
#define PTYCHO_ERR_TIMEOUT (-6)     /* a bounded device wait gave up            */
#define PTYCHO_ERR_DIVERGED (-7)    /* non-finite Fourier error                 */
#define PTYCHO_ERR_STATE (-8)       /* call out of order (e.g. iterate first)   */
#define PTYCHO_ERR_UNSUPPORTED (-9) /* (M, K) combination not compiled in       */

typedef struct {
  int M;            /* probe / detector side in pixels (16, 32, 64, 96, 128,
                       192, 256; for 96 and 192 ePIE runs only with
                       subpixel > 0, through the general kernels)            */
  int K;            /* number of incoherent probe modes (1..3), Sec. 2.2       */
  int J;            /* number of scan positions (diffraction frames)          */
  int obj_ny;       /* object rows                                            */
  int obj_nx;       /* object columns                                         */
  int istore;       /* PTYCHO_I_F32 / _F16 / _BF16                            */
  int probe_start;  /* first iteration index that updates the probe, Sec. 2.2 */
  double epie_alpha;  /* ePIE object step (default 1)                         */
  double epie_beta;   /* ePIE probe step (default 1)                          */
  double lsqml_beta;  /* LSQML relaxation of the final update (default 0.9)   */
  double reg;         /* DM/LSQML denominators: delta = reg * max(den), 1e-3  */
  unsigned long long seed; /* ePIE visiting order: 0 = identity, else a
                              SplitMix64-driven Fisher-Yates shuffle per
                              iteration, keyed by seed XOR iteration index   */
  void* stream;     /* cudaStream_t for all GPU work (may be NULL)            */
  int cluster;      /* CTAs per scan position in the Fourier kernel: 0 = the
                       built-in choice, -1 = autotuned (ptycho_autotune),
                       > 0 = that size (must be compiled for (M, K))          */
  int likelihood;   /* LSQML noise model (Odstrcil et al. 2018, cited for
                       LSQML in Sec. 1): PTYCHO_LIK_AMPLITUDE (default,
                       Gaussian noise on sqrt I: chi = F^-1 Pi F(phi) - phi)
                       or PTYCHO_LIK_POISSON (photon counts:
                       chi = F^-1 [(I - A^2)/(I + A^2) F(phi)], A^2 = sum_k
                       |F(phi_k)|^2: one per-pixel Newton step of the Poisson
                       negative log-likelihood along its gradient; masked
                       pixels 0).  DM and ePIE ignore it;
                       ptycho_fourier_residual follows it.                   */
  int probe_ortho;  /* 1: after every iteration that updates the probe,
                       orthogonalise its modes (Thibault & Menzel 2013, cited
                       in Sec. 1): rotate them into the eigenbasis of their
                       Gram matrix <P_l, P_k>, decreasing power, each
                       eigenvector's largest entry real positive; DM's exit
                       waves are mixed with the same unitary.  0 (default):
                       modes are left as the updates make them.              */
  int subpixel;     /* 0 (default): positions rounded half-to-even to whole
                       pixels.  S = 2, 4, 8 or 16: positions quantised to 1/S
                       pixel, q = rint(S y); corner p = floor((q + S/2) / S);
                       the probe seen at the position is the probe translated
                       by delta = q/S - p in [-1/2, 1/2) with the Fourier shift
                       theorem, F(T P)(f) = F(P)(f) exp(-2 pi i f . delta),
                       f = k/M, k >= M/2 taken as k - M.  (The script
                       example of Sec. 3.2 scans in 50 nm steps at a
                       2.8 nm pixel: 17.76 pixels.)  The
                       probe sums take the adjoint shift.  LSQML scales its
                       probe direction by the unshifted den_P = sum |O_j|^2;
                       DM's probe update solves its normal equations
                       sum_j T_j^H |O_j|^2 T_j P + d P = rhs by 4
                       preconditioned conjugate-gradient iterations from the
                       current probe (the diagonal form makes the difference
                       map diverge).  ePIE takes each position's probe step
                       in its shifted frame (the probe is carried from one
                       position's frame to the next by the difference of
                       their shifts), one position at a time through the
                       general kernels (slower than the whole-pixel sweep).
                       All algorithms, the Fourier error, simulation and
                       residual calls.  Device memory: three tables of
                       S^2 K M^2 complex values and S^2 M^2 floats.          */
  int block_positions; /* 0 (default): the residuals of all J positions stay
                       in device memory (J K M^2 complex values).  B > 0 (and
                       < J): LSQML keeps those of B positions at a time, for
                       scans whose residuals exceed device memory (the paper's
                       data larger than one GPU's memory, Sec. 3.3): each
                       iteration computes every block's residual twice, once
                       for the directions and once for the step sizes and the
                       update (two Fourier passes instead of one); same
                       results as B = 0 up to the grouping of the sums.  DM
                       (whose state is every exit wave) and sub-pixel
                       positions return PTYCHO_ERR_UNSUPPORTED.               */
  unsigned long long mem_limit; /* 0 (default): no cap.  > 0: the context
                       allocates at most this many bytes of device memory in
                       total (a share of a GPU shared with other work); an
                       allocation that would pass the cap fails with
                       PTYCHO_ERR_OOM exactly as a failed cudaMalloc does:
                       the call returns the code, nothing of it is applied
                       and the context stays valid and destroyable.         */
  int fft_engine;   /* 2-D transforms of the DM, LSQML, Fourier-error and
                       forward-model passes (the paper's batched transforms of
                       every diffraction pattern, Sec. 2.3):
                       PTYCHO_FFT_REGISTER (default): FP32 radix FFT in
                       registers and shared memory;
                       PTYCHO_DFT_TENSOR_BF16X3: each 1-D transform is one
                       product with the DFT matrix on the tensor cores, in
                       BF16 with a three-term split (hi*hi + lo*hi + hi*lo)
                       and FP32 accumulation -- about 17 significant bits
                       per transform stage instead of 24.  Compiled for M = 64,
                       K = 1 (else PTYCHO_ERR_UNSUPPORTED).  ePIE's sweep
                       keeps its own kernels.
                       PTYCHO_FFT_AUTO: the faster engine for (M, K) as
                       ptycho_autotune_engine measures it (with cluster = -1
                       also its cluster size).                               */
  int residual_store; /* LSQML's residuals chi between the Fourier pass that
                       writes them and the five passes that read them (object
                       and probe directions, step sizes, object and probe
                       updates): PTYCHO_R_F32 (default) or PTYCHO_R_F16
                       (half the bytes of the iteration's dominant traffic;
                       chi rounded to 11 significant bits, every sum and
                       update still FP32 / FP64).  The reduced-precision
                       storage pattern applied to the residual; DM's exit
                       waves, ptycho_fourier_residual's output and the
                       position refinement stay FP32.                      */
} ptycho_params;

/* Fill *p with the defaults above (M, K, J and the object size are zero). */
void ptycho_default_params(ptycho_params* p);

/* Create a context for one reconstruction and allocate its device buffers
 * (object, probe, per-position state).  *out receives the handle, or NULL on
 * error.  Returns PTYCHO_ERR_ARG for out-of-range sizes,
 * PTYCHO_ERR_UNSUPPORTED when no kernel is compiled for (M, K), and
 * PTYCHO_ERR_OOM / PTYCHO_ERR_CUDA on device failure. */
int ptycho_create(ptycho_ctx** out, const ptycho_params* p);

/* Upload the measured data: intensities [J][M][M] (see conventions) and
 * positions [J][2].  Positions are always host memory; intensities are host
 * or device memory as on_device says.  Checks every patch is inside the
 * object (PTYCHO_ERR_BOUNDS) and every intensity is finite
 * (PTYCHO_ERR_NONFINITE), then stores sqrt(I) in FFT order at the context's
 * storage precision.  Resets the DM exit-wave state. */
int ptycho_set_data(ptycho_ctx* ctx, const float* intensities, const float* positions,
                    int on_device);

/* ---- Raw detector frames (Sec. 2.2 preprocessing parameters) ------------
 * ptycho_set_data_raw replaces ptycho_set_data for frames straight from the
 * detector: raw[J][raw_h][raw_w] of dtype, host or device (on_device),
 * copied.  Each frame becomes the detector-centred M x M intensity whose
 * pixel (y, x), at offset d = (y - M/2, x - M/2) from the zero frequency,
 * reads the raw pixel (round(center_y), round(center_x)) + R^-rot90 d, with R
 * a quarter turn counter-clockwise, (a, b) -> (-b, a), and offsets wrapped
 * into [-M/2, M/2) (the DFT grid is periodic).  A raw pixel outside the
 * frame, negative, or at / above 2^saturation_bits - 1 (saturation_bits > 0,
 * at most 24) is masked; values below threshold (> 0) become 0 (noise
 * removal).  Then as ptycho_set_data (same storage, checks and errors;
 * PTYCHO_ERR_ARG for bad parameters). */
enum { PTYCHO_RAW_U16 = 0, PTYCHO_RAW_U32 = 1, PTYCHO_RAW_F32 = 2 };
typedef struct {
  int raw_h, raw_w;        /* raw frame size in pixels                       */
  int dtype;               /* PTYCHO_RAW_U16 / _U32 / _F32                    */
  float center_y;          /* raw pixel of zero frequency (rounded half-even) */
  float center_x;
  int saturation_bits;     /* 0: no saturation test; 1..24: pixel bit depth  */
  float threshold;         /* <= 0: off                                      */
  int rot90;               /* 0..3 quarter turns counter-clockwise            */
} ptycho_preprocess;
int ptycho_set_data_raw(ptycho_ctx* ctx, const void* raw, const ptycho_preprocess* pp, const float* positions,
                        int on_device);

/* Upload the scan positions only ([J][2], host memory), e.g. before
 * ptycho_simulate.  Same checks as ptycho_set_data. */
int ptycho_set_positions(ptycho_ctx* ctx, const float* positions);

/* Upload the object [obj_ny][obj_nx][2] and probe [K][M][M][2] guesses
 * (Sec. 2.2 lets the user supply either or both starting estimates).  Either
 * pointer may be NULL to keep the current value (initially object = 1 and
 * probe = 0).  Resets the DM exit-wave state. */
int ptycho_set_init(ptycho_ctx* ctx, const float* object, const float* probe, int on_device);

/* Orthogonalise the probe modes now (see ptycho_params.probe_ortho; the DM
 * exit-wave state, if any, is mixed too).  Asynchronous on the context's
 * stream; K = 1: no change. */
int ptycho_orthogonalize_probe(ptycho_ctx* ctx);

/* Switch the LSQML likelihood of an existing context (PTYCHO_LIK_*), e.g.
 * Poisson refinement after amplitude-model iterations.  Takes effect at the
 * next LSQML iteration; errors: PTYCHO_ERR_ARG. */
int ptycho_set_likelihood(ptycho_ctx* ctx, int likelihood);

/* Run n_iter iterations of alg (PTYCHO_EPIE / _DM / _LSQML) entirely on the
 * device; the iteration counter t continues across calls, so n calls of 1
 * iteration equal one call of n.  The probe is updated from t >= probe_start.
 * DM keeps its exit waves [J][K][M][M] between calls; they are (re)initialised
 * to P_k O_j on the first DM iteration after set_data / set_init or after
 * another algorithm ran.  Asynchronous on the context stream. */
int ptycho_iterate(ptycho_ctx* ctx, int alg, int n_iter);

/* Bounded waits.  The Fourier kernels exchange data between the CTAs of a
 * cluster and wait for it on shared-memory barriers; each such wait polls at
 * most `polls` times (default 1 << 20, about a millisecond; 0 = give up at
 * once).  A wait that gives up sets the context's device error flag, after
 * which the kernel still waits (with a fixed bound) for the data already in
 * flight into its shared memory and returns; the next call that reads the
 * flag (get_object, get_probe, fourier_error) returns PTYCHO_ERR_TIMEOUT and
 * clears it.  The results of the passes that gave up are meaningless.
 * Errors: PTYCHO_ERR_ARG for polls < 0. */
int ptycho_set_wait_limit(ptycho_ctx* ctx, long long polls);

/* Copy the current object [obj_ny][obj_nx][2] / probe [K][M][M][2] out. */
int ptycho_get_object(ptycho_ctx* ctx, float* out, int on_device);
int ptycho_get_probe(ptycho_ctx* ctx, float* out, int on_device);

/* Fourier error E = sum m (A - sqrt I)^2 / sum m I over all frames and
 * unmasked pixels m, A = sqrt(sum_k |F(P_k O_j)|^2), from a fresh forward
 * pass at the current (O, P); sums in FP64 in a fixed order.  Synchronises.
 * Returns PTYCHO_ERR_DIVERGED if E is not finite. */
int ptycho_fourier_error(ptycho_ctx* ctx, double* out);

/* Forward model (Sec. 2.3): far-field intensities of the current (O, P) at
 * the current positions, I_j = fftshift(sum_k |F(P_k O_j)|^2), written as
 * [J][M][M] float32 (detector-centred) to out. */
int ptycho_simulate(ptycho_ctx* ctx, float* out, int on_device);

/* Fourier residual of the current (O, P): chi_jk = F^-1 Pi(F(P_k O_j)) - P_k O_j,
 * written as [J][K][M][M][2] to out.  Pi replaces the mode-summed modulus by
 * sqrt(I) (masked pixels unchanged).  Does not change the reconstruction. */
int ptycho_fourier_residual(ptycho_ctx* ctx, float* out, int on_device);

/* DM exit-wave state psi [J][K][M][M][2] (PTYCHO_ERR_STATE if none). */
int ptycho_get_exit_waves(ptycho_ctx* ctx, float* out, int on_device);

/* Iterations run so far (the counter t). */
long long ptycho_iteration(const ptycho_ctx* ctx);

/* Checkpoint / resume (for runs longer than one session; the DM state
 * included): a run is
 * resumed bit for bit from (object, probe, iteration index) -- plus, for DM,
 * the exit waves of ptycho_get_exit_waves.
 * ptycho_set_iteration: the index t of the next iteration (>= 0; sets the
 *   probe_start test and the ePIE visiting order).
 * ptycho_set_exit_waves: the DM state psi [J][K][M][M][2] (host or device,
 *   copied; NaN/Inf rejected with the state unchanged); later DM iterations
 *   continue from it instead of P_k O_j.  Errors: PTYCHO_ERR_* codes. */
int ptycho_set_iteration(ptycho_ctx* ctx, long long t);
int ptycho_set_exit_waves(ptycho_ctx* ctx, const float* psi, int on_device);

/* Position refinement (sub-pixel contexts; the position-correction step of
 * the LSQML method of Odstrcil et al. 2018, cited in Sec. 1).  One call takes
 * a fresh Fourier residual chi at the current (O, P) and positions (under the
 * context's likelihood), and for every position the shift s = (s_y, s_x)
 * minimising ||chi_j - s_y a_y - s_x a_x||^2 + lam |s|^2 over modes and
 * pixels, a_y = P_jk dO_j/dy, a_x = P_jk dO_j/dx (P_j the shifted probe the
 * position sees, dO central differences of the object with indices past the
 * edge clamped; lam = 1e-6 (A11 + A22) / 2, FP64 solve).  Each position moves
 * by step * clamp(s, -max_shift, max_shift) pixels (float32) and is
 * re-quantised.  The residual pass overwrites the DM exit-wave state: a DM
 * iteration after this call restarts from psi = P_j O_j.
 * Errors: PTYCHO_ERR_UNSUPPORTED (subpixel = 0), PTYCHO_ERR_STATE (no data),
 * PTYCHO_ERR_ARG (non-finite step, negative max_shift), PTYCHO_ERR_BOUNDS (a
 * moved patch would leave the object: no position changes). */
int ptycho_refine_positions(ptycho_ctx* ctx, double step, double max_shift);

/* The current positions [J][2] (y, x) in float32 pixels: as last set, or as
 * moved by ptycho_refine_positions.  Host memory. */
int ptycho_get_positions(ptycho_ctx* ctx, float* out);

/* Number of this library's kernel launches issued so far on the context. */
long long ptycho_launch_count(const ptycho_ctx* ctx);

/* Bytes of device memory the context holds now (all its buffers; the figure
 * ptycho_params.mem_limit caps); -1 for ctx = NULL. */
long long ptycho_memory_used(const ptycho_ctx* ctx);

/* Logging and feedback (Sec. 3.4: progress and error reports while a
 * reconstruction runs).  The sink is called synchronously, on the calling
 * thread, from inside the library call that produces the message:
 *   PTYCHO_LOG_ERROR  a call on this context failed; msg is the text that
 *                     ptycho_last_error() returns for it;
 *   PTYCHO_LOG_INFO   a progress report of ptycho_iterate:
 *                     "<alg> iteration <t>: E = <Fourier error>", t counting
 *                     completed iterations of the context.
 * error_every > 0: ptycho_iterate reports after every error_every-th
 * iteration (and after its last one), each report one extra Fourier-error
 * pass and a host synchronisation -- the iterates are unchanged, bit for bit;
 * 0: errors only.  fn = NULL removes the sink.  The message is valid during
 * the call only.  The sink runs inside a library call on this context: it
 * may call ptycho_last_error(ctx) but no other function on the same
 * context.  Errors: PTYCHO_ERR_ARG (ctx NULL, error_every < 0). */
typedef void (*ptycho_log_fn)(void* user, int level, const char* msg);
enum { PTYCHO_LOG_ERROR = 0, PTYCHO_LOG_INFO = 1 };
int ptycho_set_log(ptycho_ctx* ctx, ptycho_log_fn fn, void* user, int error_every);

/* Per-kernel timing.  When enabled, every launch is bracketed by CUDA events
 * on the context stream and its duration is accumulated per kernel family. */
typedef struct {
  const char* name;     /* kernel family                                    */
  long long launches;   /* launches since profiling was enabled             */
  double ms;            /* summed device time (ms)                          */
  double bytes;         /* summed algorithmic DRAM bytes of those launches  */
} ptycho_kernel_stat;

int ptycho_set_profiling(ptycho_ctx* ctx, int enabled);
/* Writes up to max entries; *n receives the number of kernel families. */
int ptycho_get_profile(ptycho_ctx* ctx, ptycho_kernel_stat* out, int max, int* n);

/* CTAs per scan position of the Fourier kernels of this context (1, 2, 4, 8
 * or 16). */
int ptycho_cluster_size(const ptycho_ctx* ctx);

/* CTAs of the persistent ePIE sweep (the widest compiled cluster for (M, K)
 * unless ptycho_params.cluster fixed it); 0 if no ePIE kernel fits.  With
 * sub-pixel positions (ptycho_params.subpixel > 0) the sweep visits one
 * position at a time through the general kernels, and this is the cluster
 * of that per-position Fourier pass (chosen the same way). */
int ptycho_epie_cluster_size(const ptycho_ctx* ctx);

/* ---- Many reconstructions per launch --------------------------------------
 * The paper's batch GPU mode queues many small scans, one job per GPU
 * (Sec. 3.3).  On one B300 a batch groups N reconstructions of unequal size:
 * one iteration of every member is captured into a single CUDA graph (each
 * member's kernels on its own stream branch) and replayed once per iteration.
 * Members run in groups, one group after another, so that large members do
 * not contend with each other for L2 and SMs while small ones still share
 * the GPU: a member whose per-iteration working set (J*K*M^2*8 bytes of
 * residuals, the stored amplitudes, 24 bytes per object pixel) reaches the
 * group budget runs alone; the others are packed, largest first, into
 * groups whose working sets sum to at most the budget (default 512 MiB).
 *
 * ptycho_batch_create: params[n] describes each member (its stream field is
 *   ignored: the batch creates one stream per member); stream is the batch
 *   stream the graph runs on (NULL: the batch creates its own).
 * ptycho_batch_member: the member's context, for ptycho_set_data,
 *   ptycho_set_init, ptycho_get_*, ptycho_fourier_error (owned by the batch;
 *   do not destroy it).
 * ptycho_batch_iterate: n_iter iterations of DM or LSQML (ePIE:
 *   PTYCHO_ERR_UNSUPPORTED) on every member; every member must have data.
 *   The graph is captured again when the algorithm or a member's
 *   probe-update state changes.  Asynchronous on the batch stream; member
 *   streams are ordered after it.
 * ptycho_batch_kernels_per_iteration: kernel nodes in the captured graph.
 * ptycho_batch_set_group_bytes: the group budget in bytes (<= 0: all members
 *   in one group); the graph is captured again at the next iterate.
 * ptycho_batch_groups: number of groups (lanes in lanes mode) of the current
 *   plan; if group_of is not NULL it receives each member's group (lane)
 *   index (n ints).  The schedule
 *   changes only the order of independent work: results are bit-identical
 *   for every budget.
 * ptycho_batch_set_lanes: lanes > 0 replaces the groups by that many
 *   chains: members sorted by work (J K M^2 (log2 M + 6)), largest first,
 *   each to the chain with the least work so far; a chain runs its members
 *   one after another and the chains run side by side, with no barrier
 *   between chains until the end of the iteration.  0 returns to groups
 *   (as does ptycho_batch_set_group_bytes).  Errors: PTYCHO_ERR_ARG
 *   (lanes < 0).
 * ptycho_batch_lanes: the current number of lanes (0: groups mode; -1 for
 *   b = NULL).
 * ptycho_batch_autotune: time n_iter iterations of alg under each candidate
 *   schedule -- group budgets (all members at once, then 64 MiB .. 4 GiB)
 *   and lanes (2 .. 32 chains, fewer than the members); candidates giving
 *   the same schedule are timed once -- keep the fastest and write its group
 *   budget to *best_bytes, its lanes (0 for a group schedule) to
 *   *best_lanes and its time per iteration (ms) to *best_ms (any may be
 *   NULL).  The timed iterations are real iterations of every member (one
 *   untimed iteration per candidate captures its graph): the iteration
 *   counters advance by (n_iter + 1) per distinct schedule.
 * Errors: PTYCHO_ERR_* codes; ptycho_batch_last_error(b) (b = NULL: last
 * failed create). */
typedef struct ptycho_batch ptycho_batch;
int ptycho_batch_create(ptycho_batch** out, int n, const ptycho_params* params, void* stream);
ptycho_ctx* ptycho_batch_member(ptycho_batch* b, int i);
int ptycho_batch_size(const ptycho_batch* b);
int ptycho_batch_iterate(ptycho_batch* b, int alg, int n_iter);
long long ptycho_batch_kernels_per_iteration(const ptycho_batch* b);
int ptycho_batch_set_group_bytes(ptycho_batch* b, long long bytes);
int ptycho_batch_set_lanes(ptycho_batch* b, int lanes);
int ptycho_batch_lanes(const ptycho_batch* b);
int ptycho_batch_autotune(ptycho_batch* b, int alg, int n_iter, long long* best_bytes, int* best_lanes,
                          double* best_ms);
int ptycho_batch_groups(ptycho_batch* b, int* group_of);
int ptycho_batch_synchronize(ptycho_batch* b);
const char* ptycho_batch_last_error(const ptycho_batch* b);
void ptycho_batch_destroy(ptycho_batch* b);

/* FFT shape autotuner: times the Fourier kernel (residual pass) of every
 * compiled cluster size for (M, K) on synthetic data of about 512 MB, keeps
 * the fastest in a process-wide table (later calls return it at once) and
 * writes it to *best_cluster and its time per scan position to
 * *ms_per_position (either may be NULL).  Allocates and frees temporary
 * contexts; synchronises the device work it issues. */
int ptycho_autotune(int M, int K, int* best_cluster, double* ms_per_position);

/* FFT-variant autotuner: ptycho_autotune over the transform engines too --
 * the register FFT at its best cluster size and, where it is compiled
 * (M = 64, K = 1), the tensor-core DFT, timed the same way -- writing the
 * faster engine (PTYCHO_FFT_REGISTER or PTYCHO_DFT_TENSOR_BF16X3), the
 * register FFT's best cluster size and the winner's time per scan position
 * (any output may be NULL).  Cached per (M, K) like ptycho_autotune.
 * Errors: PTYCHO_ERR_ARG (M < 2, K < 1), PTYCHO_ERR_UNSUPPORTED (nothing
 * compiled for (M, K)). */
int ptycho_autotune_engine(int M, int K, int* best_engine, int* best_cluster, double* ms_per_position);

/* ---- Learned warm start ----------------------------------------------------
 * A convolutional encoder-decoder (6 levels, 128^2 -> 4^2 -> 64^2, ~1.96M
 * parameters, BF16 weights and activations, FP32 sums) maps one diffraction
 * frame, x = log(1 + I) / 10 of a 128 x 128 detector-centred pattern, to the
 * amplitude and phase of the central 64 x 64 object patch under the probe.
 * Its predictions, stitched together, replace the flat initial object of a
 * DM or LSQML reconstruction, which has the last word.  Not in the paper; it
 * uses the paper's option of a user-supplied initial probe or object
 * (Sec. 2.2).  Training, inference and every gradient run in this library's CUDA
 * kernels.
 *
 * Parameter vector (FP32, host order used by get/set): for each of the 12
 * layers, weights [co][ci][3][3] then biases [co].
 * ptycho_net_create: He-normal weights from SplitMix64(seed), zero biases;
 *   max_batch bounds B in the calls below; flags = 0 (BF16 activations, the
 *   method; forward convolutions as implicit GEMMs on the tcgen05 tensor
 *   cores, backward on CUDA cores), PTYCHO_NET_F32_ACTIVATIONS (CUDA-core
 *   kernels with FP32 activation storage, for checking the kernels against an
 *   unrounded reference) or PTYCHO_NET_CUDA_CORES (BF16, CUDA-core forward);
 *   stream as for contexts.
 * ptycho_net_predict: intensities device [B][128][128] (detector-centred);
 *   out device [B][2][64][64] (amplitude, phase).
 * ptycho_net_gradients: loss L = sum (out - target)^2 / (B * 2 * 64 * 64)
 *   against targets device [B][2][64][64]; grads (host, may be NULL)
 *   receives dL/dparams; *loss (may be NULL) receives L.  Synchronises.
 * ptycho_net_train_step: one AdamW step (beta 0.9 / 0.999, eps 1e-8, weight
 *   decay 1e-4 on weights) at learning rate lr; *loss as above (NULL: no sync).
 * ptycho_object_patches: amplitude and phase of the central 64 x 64 patch of
 *   the context's current object at every position, device [J][2][64][64]
 *   (training targets from a known object).
 * ptycho_warm_start: predicts the patch of every position of ctx (M must be
 *   128) from its stored data and writes their per-pixel mean into ctx's
 *   object where at least one patch covers it.  Synchronises. */
typedef struct ptycho_net ptycho_net;
#define PTYCHO_NET_F32_ACTIVATIONS 1 /* FP32 activation storage (verification)      */
#define PTYCHO_NET_CUDA_CORES 2      /* forward convolutions on CUDA cores instead of
                                        the tensor cores (comparison)               */
int ptycho_net_create(ptycho_net** out, unsigned long long seed, int max_batch, int flags, void* stream);
long long ptycho_net_num_params(const ptycho_net* n);
int ptycho_net_get_params(ptycho_net* n, float* out);
int ptycho_net_set_params(ptycho_net* n, const float* in);
int ptycho_net_predict(ptycho_net* n, const float* intensities, int B, float* out);
int ptycho_net_gradients(ptycho_net* n, const float* intensities, const float* targets, int B, float* grads,
                         double* loss);
int ptycho_net_train_step(ptycho_net* n, const float* intensities, const float* targets, int B, float lr,
                          double* loss);
const char* ptycho_net_last_error(const ptycho_net* n);
void ptycho_net_destroy(ptycho_net* n);
int ptycho_object_patches(ptycho_ctx* ctx, float* out);
int ptycho_warm_start(ptycho_ctx* ctx, ptycho_net* n);

/* Fourier error without any device allocation.
 *
 * The paper has no counterpart to this call.  It exists for callers that
 * cannot call cudaMalloc: code embedded in a host application that owns all
 * device memory through its own pool and forbids other allocations, or a
 * live-feedback loop that cannot afford the implicit device-wide
 * synchronisation an allocation may bring.  Such a caller keeps its data in
 * its own device buffers and gets E without creating a context.
 *
 * E is computed exactly as ptycho_fourier_error computes it (same kernel,
 * same cluster split, same fixed-order FP64 sums).  Inputs:
 *   object      device, [obj_ny][obj_nx][2] float32 (re, im)
 *   probe       device, [K][M][M][2] float32
 *   positions   HOST, [J][2] float32 (y, x) top-left, rounded half-to-even;
 *               every patch must lie inside the object (PTYCHO_ERR_BOUNDS)
 *   amplitudes  device, [J][M][M] float32 = sqrt(I) in FFT order (zero
 *               frequency at pixel (0, 0), i.e. NOT detector-centred);
 *               a negative value marks a masked pixel
 *   out         HOST, receives E
 *   stream      cudaStream_t for the work (NULL = legacy default stream);
 *               the call synchronises it before returning.
 * Limits: J <= 16384 and M <= 256, beyond which the call fails with
 * PTYCHO_ERR_ARG; (M, K) must be a compiled combination (else
 * PTYCHO_ERR_UNSUPPORTED).  Errors are reported by ptycho_last_error(NULL) on the calling thread.
 * Pointer checks before any device work: object and probe must be 8-byte
 * aligned and amplitudes 16-byte aligned, and all three must be device (or
 * managed) memory of the current device; otherwise PTYCHO_ERR_ARG.
 *
 * Scratch: one fixed array of about 4.3 MB in device memory, defined at file
 * scope in the library, which every GPU that loads the library keeps until
 * the process exits.  Every call looks up that array's device address on
 * the current device (a lookup, not an allocation).  All calls share the
 * array: two calls whose GPU work overlaps (different streams or threads)
 * race on it and must be serialised by the caller.  The call copies the
 * positions from host memory and reads E back, synchronising its stream, so
 * it cannot be recorded into a CUDA graph by stream capture.  The call itself
 * allocates no device memory (no cudaMalloc, no cudaFree, no allocating
 * library routine); it stages the positions in an ordinary host buffer. */
int ptycho_fourier_error_noalloc(const float* object, int obj_ny, int obj_nx, const float* probe, int M, int K,
                                 const float* positions, int J, const float* amplitudes, double* out,
                                 void* stream);

/* FP32 fused multiply-add throughput of the current device, measured (a
 * measurement utility with no counterpart in the paper: the denominator of
 * the FP32 roofline of the instruction-bound Fourier passes).  A kernel of
 * independent FMA chains filling every SM (8 CTAs of 256 threads per SM,
 * 2 flops per FMA) is timed with CUDA events on `stream` (NULL = legacy
 * default stream), best of three runs after one warm-up run.
 * Out (host): *tflops (TFLOP/s), *ms (time of the best run, may be NULL),
 * *sm_count (the device's multiprocessor count, may be NULL).  The rate
 * follows the SM clock of the run: record the clock beside it.  Synchronises
 * the stream; errors: PTYCHO_ERR_ARG (tflops NULL), PTYCHO_ERR_CUDA. */
int ptycho_fp32_fma_peak(double* tflops, double* ms, int* sm_count, void* stream);

/* Message of the last error on ctx (or, for ctx = NULL, of the last failed
 * create or context-free call made on the calling thread: that message is
 * kept per thread).  Valid until the next call on the same context (thread). */
const char* ptycho_last_error(const ptycho_ctx* ctx);

/* Free all device memory of ctx ("post", Sec. 3.2).  NULL is ignored. */
void ptycho_destroy(ptycho_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* PTYCHO_H */
