/*
 * nlinv.h -- C ABI of the GB300 (sm_103a) NLINV hot path.
 *
 * NLINV (Schaetz, Voit, Frahm, Uecker 2017, Sec. 2.2) reconstructs an image
 * rho and J coil sensitivities c_j from multi-channel k-space by minimising
 *     || F x - y ||^2 + alpha || W (x - x_prev) ||^2                  (Eq. 1)
 * with the iteratively regularised Gauss-Newton method (IRGNM, Eqs. 2-3)
 * after the change of variables x^ = W x, F^ = F o W^-1, each Newton step
 * solved by conjugate gradients on (DF^H DF + alpha_n I) (Eqs. 4-5).  The
 * non-uniform transform pair is a truncated convolution with the
 * point-spread function (PSF) on the twofold-oversampled grid (Sec. 2.2
 * footnote, Fig. 4); W is a Fourier-domain Sobolev weight on the coils only
 * (Fig. 4, Fig. 7); coil coefficients are stored on a G_c = floor(G/4) grid
 * (Sec. 3.2).
 *
 * Conventions (all entry points):
 *   - complex data are complex64, interleaved (re, im) float pairs, row-major;
 *   - N = image side, G grid side (2N, or 2 gamma N of Eq. 8), J channels,
 *     Gc coil grid side (odd or even);
 *   - unitary 2-D DFT U, unshifted frequency order; the field of view is
 *     rows/cols [0, N) of the G grid;
 *   - the unknown x^ is ONE contiguous vector of n_x = N*N + J*Gc*Gc complex
 *     values: rho [N][N] followed by c^ [J][Gc][Gc], the c^ grid holding
 *     frequency f at index f mod Gc (f in [-floor(Gc/2), (Gc-1)/2]);
 *   - D_W^-1(f) = (1 + w_a |2f/G|^2)^(-w_l/2) (Fig. 7's (1+880|k|^2)^16 with
 *     k = f/G for w_a = 220, w_l = 32);
 *   - the PSF P [U][G][G] is real, unshifted; sampling enters only through
 *     P (P = 0/1 mask for Cartesian sampling);
 *   - data Y [J][G][G] are gridded so that crop_N U^H Y_j = A^H y_j.
 *
 * Memory and streams: every pointer argument marked "device" is
 * caller-owned device memory (8-byte aligned for complex data) that must
 * stay valid until the stream has passed the call.  The plan owns its
 * workspace, its PSFs and its weight tables.  All compute calls are
 * asynchronous on `stream` (a cudaStream_t; NULL = legacy default stream).
 *
 * Errors: every call returns NLINV_OK (0) or a negative code.  Host-side
 * validation failures return before anything is enqueued.  Errors detected
 * on the device (an expired bounded wait, a CG breakdown) are latched in the
 * plan and returned by nlinv_sync().  No C++ exception crosses this ABI.
 */
#ifndef NLINV_H
#define NLINV_H

#ifdef __cplusplus
extern "C" {
#endif

#define NLINV_OK 0
#define NLINV_EINVAL (-1)      /* bad size, null/unaligned pointer, bad turn */
#define NLINV_ECUDA (-2)       /* a CUDA runtime call failed */
#define NLINV_ENOMEM (-3)      /* device allocation failed */
#define NLINV_ETIMEOUT (-4)    /* a bounded device-side wait expired */
#define NLINV_ENUMERIC (-5)    /* CG breakdown: Re<p, A p> <= 0 or not finite */
#define NLINV_EUNSUPPORTED (-6)/* grid size without a compiled FFT schedule */

typedef struct nlinv_plan_s* nlinv_plan_t;
typedef void* nlinv_stream_t; /* cudaStream_t */

typedef struct {
  int N;              /* image side (the field of view is N x N) */
  int J;              /* receive channels */
  int Gc;             /* coil grid side, <= G; 0 -> floor(G/4) (Sec. 3.2) */
  int newton_steps;   /* M, 1..32 (Sec. 2.2: 6 to 10) */
  int cg_iters;       /* fixed CG iterations per Newton step, 0..4096 */
  int n_turns;        /* U: PSFs held by the plan (Sec. 2.1, Fig. 3) */
  double alpha0, q;   /* alpha_n = alpha0 * q^n, alpha0 > 0, 0 < q <= 1 */
  double damping;     /* x_ref = damping * x_prev (1.0 = Eq. 1 literally) */
  double w_a, w_l;    /* Sobolev weight constants (220, 32) */
  long long spin_limit; /* polls before a device-side wait gives up; 0 -> default */
  int exec_mode;      /* how nlinv_frame runs a frame:
                         0: default -- the CUDA graph of 4, which measured
                            fastest on the configurations' sizes (the tuner,
                            tune.py, records the fastest per size);
                         1: one launch per phase (unfused comparator);
                            each launch covers every frame of the call
                            (nlinv_batch: CTA b works on frame b / n_b);
                            the frames' pointers are read from a plan-owned
                            device table written at the start of the call;
                         2: one persistent cooperative launch, CTAs
                            synchronised by grid barriers between phases;
                         3: one persistent cooperative launch with one
                            thread-block cluster per channel (per-channel
                            passes exchange data in distributed shared
                            memory; grid barriers only for the channel sum
                            and the CG inner products); nlinv_plan returns
                            NLINV_EUNSUPPORTED when the J clusters cannot be
                            co-resident;
                         4: the launches of 1 captured into a CUDA graph
                            with programmatic dependent launches between the
                            phases, one graph per frame count, replayed per
                            call (captured on first use and again after
                            nlinv_set_alpha0; the capture is on a plan-owned
                            stream, so such a call must not be issued while
                            the calling thread captures) */
  int max_batch;      /* frames of this plan one nlinv_batch call may hold, 1..64;
                         0 -> 1 (the plan allocates one workspace per frame) */
  int G;              /* grid side: 0 -> 2N (gamma = 1); else a grid G = 2 gamma N
                         of Eq. 8 (G >= 2N) among the compiled (G, N) pairs
                         (nlinv_grid_list; NLINV_EUNSUPPORTED otherwise) */
  int cluster_cs;     /* CTAs per channel cluster of the cluster kernel
                         (exec_mode 3): 0 -> the largest size whose J
                         clusters are co-resident; else exactly this size
                         (NLINV_EUNSUPPORTED when it does not fit) */
} nlinv_params_t;

/* The compiled grids: (G_out[i], N_out[i]) for i < the returned count (at
 * most cap entries are written; either array may be NULL to count only).
 * Host-only. */
int nlinv_grid_list(int* G_out, int* N_out, int cap);

/* Fill `p` with the defaults for an N x N image and J channels:
 * G = 2N, Gc = G/4, 7 Newton steps x 10 CG, alpha0 = 1, q = 1/2, damping 1,
 * w_a = 220, w_l = 32, one turn, the default execution (exec_mode 0). */
int nlinv_default_params(nlinv_params_t* p, int N, int J);

/* Create a plan (Sec. 2.2, Fig. 4 set-up: twiddles, D_W^-1 table, PSFs,
 * workspace).  psf: device float [U][G][G] copied into the plan, or NULL
 * (PSFs then start at zero; set them with nlinv_set_psf / nlinv_psf).
 * Allocates device memory; synchronises `stream` before returning. */
int nlinv_plan(nlinv_plan_t* out, const nlinv_params_t* p, const float* psf,
               nlinv_stream_t stream);
int nlinv_plan_destroy(nlinv_plan_t plan);

/* n_x, G and Gc of a plan (host values). */
int nlinv_plan_sizes(nlinv_plan_t plan, long long* nx, int* G, int* Gc);

/* How nlinv_frame runs this plan's frames: *exec_path = 1 (per-phase
 * launches), 2 (grid kernel), 3 (cluster kernel) or 4 (per-phase launches in
 * a CUDA graph), see exec_mode, and
 * *cluster_size = CTAs per channel cluster (0 unless exec_path is 3).
 * Either pointer may be NULL. */
int nlinv_plan_path(nlinv_plan_t plan, int* exec_path, int* cluster_size);

/* Copy one turn's PSF (device float [G][G]) into the plan. */
int nlinv_set_psf(nlinv_plan_t plan, int turn, const float* psf, nlinv_stream_t stream);

/* PSF of a trajectory (Sec. 2.2 footnote): P(f) = sum_d p(d) e^{-2 pi i f.d/G},
 * p(d) = (2N)^-2 sum_s e^{2 pi i k_s.d} for d in [-(N-1), N-1]^2, evaluated as
 * (2N)^-2 sum_s Dir(kx_s - fx/G) Dir(ky_s - fy/G) with the Dirichlet kernel
 * Dir(t) = sin((2N-1) pi t) / sin(pi t).  (A sample is (2N)^-1 sum_r x_r
 * e^{-2 pi i k.r}: its scale is fixed by the image size N.)
 * kxy: device double [S][2] (kx, ky) in cycles/pixel.  The result goes into
 * the plan's slot `turn` and, if P_out != NULL, to device float [G][G]. */
int nlinv_psf(nlinv_plan_t plan, int turn, int S, const double* kxy, float* P_out,
              nlinv_stream_t stream);

/* Gridding by the exact adjoint NDFT (the preprocessing stage of Sec. 3.1
 * in its brute-force form): Y_j = U pad(A^H y_j) with
 * (A^H y)(r) = (2N)^-1 sum_s y_s e^{+2 pi i k_s.r}.
 * kxy: device double [S][2]; y: device complex64 [J][S];
 * Y_out: device complex64 [J][G][G].  Uses the plan's workspace. */
int nlinv_grid(nlinv_plan_t plan, int S, const double* kxy, const void* y, void* Y_out,
               nlinv_stream_t stream);

/* Gridding by convolution (the preprocessing stage of Sec. 3.1 as a
 * non-uniform FFT): the same Y_j = U pad(A^H y_j) as nlinv_grid, with A^H y
 * evaluated by spreading each sample onto the W x W grid points nearest to
 * G k_s with a Kaiser-Bessel kernel phi(u) = I0(beta sqrt(1 - (2u/W)^2)),
 * beta = pi sqrt((W/sigma)^2 (sigma - 1/2)^2 - 0.8), sigma = G/N, modulated by
 * the centre N/2 of the field of view; an inverse FFT of the grid; division by
 * the kernel's continuous transform (deapodisation) on the field of view.
 * The relative error against nlinv_grid falls geometrically with W (about
 * 7e-6 at W = 6 and 6e-8 at W = 8 for sigma = 2, in exact arithmetic).
 * kxy: device double [S][2]; y: device complex64 [J][S]; W: 2..16;
 * Y_out: device complex64 [J][G][G].  Uses the plan's workspace (J G^2
 * complex values for the spread grid); float atomics make the summation
 * order, and so the last bits, vary between runs. */
int nlinv_grid_nufft(nlinv_plan_t plan, int S, const double* kxy, const void* y, int W, void* Y_out,
                     nlinv_stream_t stream);

/* Temporal median filter of the post-processing stage (Sec. 3.1): for a
 * window of T consecutive images (T odd, 1..15; imgs: host array of T
 * device pointers to complex64 [n], e.g. the img_out of T frames),
 * out[i] = the median of |img_t[i]| over t (device float [n]).  One launch,
 * asynchronous on `stream`; needs no plan. */
int nlinv_median(const void* const* imgs, int T, long long n, float* out, nlinv_stream_t stream);

/* DF at x^_n applied to dx (Eq. 5 before the PSF):
 *   z_j = U pad_N(c_j drho + rho W^-1 dc^_j),  c_j = W^-1 c^_j of x^_n.
 * xhat, dx: device complex64 [n_x]; z: device complex64 [J][G][G]. */
int nlinv_apply_DF(nlinv_plan_t plan, const void* xhat, const void* dx, void* z,
                   nlinv_stream_t stream);

/* The exact adjoint of nlinv_apply_DF (Eq. 4 without the PSF):
 *   t_j = crop_N U^H z_j;  dx = (sum_j conj(c_j) t_j, W^-H(conj(rho) t_j)).
 * xhat: device [n_x]; z: device [J][G][G]; dx_out: device [n_x]. */
int nlinv_apply_DFH(nlinv_plan_t plan, const void* xhat, const void* z, void* dx_out,
                    nlinv_stream_t stream);

/* The CG operator of one Newton step (Eqs. 2, 4, 5):
 *   out = (DF^H P_turn DF + alpha I) dx   at x^_n = xhat.
 * xhat, dx, out: device [n_x]; out must not alias xhat or dx. */
int nlinv_apply_normal(nlinv_plan_t plan, const void* xhat, const void* dx, int turn,
                       double alpha, void* out, nlinv_stream_t stream);

/* Allocation-free variant of nlinv_apply_normal (the paper has no
 * counterpart: this is a deployment convenience).  It is for callers that
 * cannot call cudaMalloc -- a running real-time reconstruction loop that
 * must not allocate or implicitly synchronise the device, or a host
 * framework that owns all device memory through its own pools.  It needs
 * no plan:
 *   out = (DF^H P DF + alpha I) dx  at x^_n = xhat,
 * with G = 2N, Gc (0 -> G/4, even), D_W^-1 constants w_a, w_l, and
 * psf: device float [G][G].  xhat, dx, out: device complex64 [n_x],
 * n_x = N*N + J*Gc*Gc; out must not alias xhat or dx.
 * Every intermediate lives in one 16 MiB __device__ array inside
 * libnlinv.so, which every GPU that loads the library holds until the
 * process exits; a problem needing more than that (about 40 J N^2 bytes,
 * e.g. N = 160 with J <= 16, N = 256 with J <= 6) returns NLINV_EINVAL
 * before anything is enqueued.  The call allocates nothing: no cudaMalloc,
 * no cudaFree, no allocating library routine.  The first call on a device
 * does a one-time set-up (looks up the array's device address and uploads
 * a small constant table); make that first call before any stream capture.
 * All calls share the one array, so calls that overlap on the GPU (other
 * streams, other threads) race and must be serialised by the caller; each
 * call writes every intermediate before reading it, so nothing has to be
 * cleared between calls.  The twiddle and D_W^-1 tables in the array are
 * kept from the previous call on the device when G, Gc, w_a and w_l are
 * unchanged (only a change of them rewrites the tables). */
int nlinv_apply_normal_static(int N, int J, int Gc, double w_a, double w_l,
                              const void* xhat, const void* dx, const float* psf,
                              double alpha, void* out, nlinv_stream_t stream);

/* One NLINV frame (Eqs. 2-3): M Newton steps from x^_0 = x_prev, each
 *   (DF^H P DF + alpha_n I) delta = DF^H (Y - P F^(x^_n)) - alpha_n (x^_n - x_ref)
 * solved by cg_iters CG iterations from zero, x^_{n+1} = x^_n + delta,
 * alpha_n = alpha0 q^n, x_ref = damping * x_prev.  The per-phase paths
 * (exec_mode 0, 1, 4) run the CG with the operator applied to the residual
 * (one reduction point per iteration; the same iterates as the textbook CG
 * in exact arithmetic) and stop a Newton step's CG once |r_k|^2 falls to
 * 1e-8 |r_0|^2 and its step length is no longer positive (rounding floor);
 * the persistent kernels (exec_mode 2, 3) run the textbook CG.  A step
 * length that is not positive above that floor is a breakdown:
 * NLINV_ENUMERIC from nlinv_sync.
 * Y: device complex64 [J][G][G]; turn selects the PSF; x_prev: device [n_x]
 * or NULL (rho = 1, c^ = 0: the first frame of Sec. 3.3); x_out: device
 * [n_x] (may alias x_prev); rho_out: device [N][N] or NULL; img_out: device
 * [N][N] rho * sqrt(sum_j |c_j|^2) or NULL. */
int nlinv_frame(nlinv_plan_t plan, const void* Y, int turn, const void* x_prev,
                void* x_out, void* rho_out, void* img_out, nlinv_stream_t stream);

/* One frame of an nlinv_batch call. */
typedef struct {
  nlinv_plan_t plan;    /* size class (N, J, Gc, M, K, alpha schedule) of the frame */
  const void* Y;        /* device complex64 [J][G][G] gridded data */
  int turn;             /* PSF slot of the plan */
  const void* x_prev;   /* device [n_x] initial value and regulariser, or NULL
                           (rho = 1, c^ = 0) */
  void* x_out;          /* device [n_x]; may alias this frame's x_prev, not another's */
  void* rho_out;        /* device [N][N] or NULL */
  void* img_out;        /* device [N][N] rho * sqrt(sum_j |c_j|^2) or NULL */
  const void* x_last;   /* device [n_x] or NULL: regulariser of the LAST Newton step
                           (x_ref = damping * x_last there; Eq. 10's exception:
                           frame n's last step uses x^_{n-1}).  It may be the x_out
                           of an EARLIER frame of the same plan in this call: that
                           step then waits (bounded, NLINV_ETIMEOUT) until the
                           earlier frame is written.  Any other frame's x_out of
                           this call is rejected (NLINV_EINVAL). */
} nlinv_frame_desc_t;

/* Frames in flight together (the temporal decomposition of Sec. 3.3,
 * Eq. 10: frames whose initial/regularisation values are already available
 * are reconstructed at the same time).  Each frame is nlinv_frame with its
 * own inputs (and, with x_last, another regulariser in its last Newton
 * step); frames may belong to different plans (grid sizes, channel counts).
 * Frames of one plan (at most its max_batch) run together: on the
 * per-phase path (exec_mode 0, 1, 4) every phase is one launch over all of
 * them, each frame on its own workspace with the same CTA count; with
 * exec_mode 2 or 3, or when a frame's last step waits for another frame of
 * the call, in one persistent cooperative launch whose CTAs are split into
 * one group per frame, each group with its own barrier.  Different plans run
 * concurrently on the plans' own streams (the persistent launches each on a
 * share of the SMs proportional to its work), and the call is ordered on
 * `stream` before and after.  Which frame serves as whose
 * x_prev (the schedule) is the caller's choice: no frame's x_prev may be
 * another frame's x_out of the same call (x_last may, see above). */
int nlinv_batch(const nlinv_frame_desc_t* frames, int nframes, nlinv_stream_t stream);

/* Temporal decomposition of Sec. 3.3 (Eq. 10): *src_out = the frame whose
 * x^ starts (and regularises) frame n of a stream reconstructed with `delay`
 * frames in flight after `warmup` frames in order.  Frames n <= warmup use
 * n - 1; later frames go in groups of `delay` and each uses the last frame of
 * the previous group (frame `warmup` for the first group), which lies in
 * [n - delay, n - 1]; -1 stands for the initial value (rho = 1, c^ = 0).
 * Returns NLINV_OK, or NLINV_EINVAL for n < 0, delay < 1, warmup < 0 or a
 * NULL src_out.  Host-only: launches nothing. */
int nlinv_stream_source(int n, int delay, int warmup, int* src_out);

/* The whole schedule of one stream of nframes frames (host arrays of
 * nframes ints, each may be NULL): group_out[n] = the launch group of frame
 * n (0..warmup in order, then groups of `delay`), source_out[n] =
 * the source of nlinv_stream_source, last_out[n] = the frame whose x^ regularises the
 * last Newton step of frame n when last_from_prev is set and differs from
 * the source (n - 1), else -1.  Returns the number of groups, or
 * NLINV_EINVAL.  Host-only: launches nothing. */
int nlinv_stream_schedule(int nframes, int delay, int warmup, int last_from_prev, int* group_out,
                          int* source_out, int* last_out);

/* One stream of frames for nlinv_run_streams (host arrays of device
 * pointers, each of length nframes). */
typedef struct {
  nlinv_plan_t plan;        /* size class of every frame of the stream; its
                               max_batch must be >= delay, and no other
                               stream of the call may use the same plan */
  int nframes;
  const void* const* Y;     /* device complex64 [J][G][G] per frame */
  const int* turns;         /* PSF slot per frame (host ints) */
  void* const* x_out;       /* device [n_x] per frame: frame n's x^ */
  void* const* img_out;     /* device [N][N] per frame, or NULL (none) */
  const void* x_init;       /* device [n_x]: x^ of the frame before frame 0,
                               or NULL (rho = 1, c^ = 0) */
  int delay;                /* frames in flight after the warm-up (>= 1; 1 = in order) */
  int warmup;               /* frames 0..warmup are reconstructed in order (>= 0) */
  int last_from_prev;       /* nonzero: Eq. 10's exception, the last Newton
                               step of frame n regularised towards x^_{n-1}
                               (waiting for it when it is in the same group) */
} nlinv_stream_desc_t;

/* Reconstruct several independent streams with the temporal decomposition
 * of Sec. 3.3 (Eq. 10): the library forms each stream's launch groups
 * (nlinv_stream_source) and issues group g of every stream together as one
 * nlinv_batch call, g = 0, 1, ...; frame n starts from and is regularised
 * towards damping * x^ of its source frame.  Everything is asynchronous on
 * `stream`; device errors are latched in the plans (nlinv_sync). */
int nlinv_run_streams(const nlinv_stream_desc_t* streams, int nstreams, nlinv_stream_t stream);

/* Change alpha_0 of the plan's schedule alpha_n = alpha0 q^n (alpha0 > 0);
 * applies to calls issued afterwards. */
int nlinv_set_alpha0(nlinv_plan_t plan, double alpha0);

/* Reverse-mode derivative of nlinv_frame through the unrolled IRGNM / CG
 * (Sec. 2.2, Eqs. 2-5: every Newton step and CG iteration exactly as
 * computed, with the data-dependent step lengths).  A forward sweep records
 * every Newton step (checkpoint x^_n, residual, the CG vectors p_k, q_k, r_k)
 * in the workspace and the reverse sweep reads that record: per frame
 * (M + 1 + M (3 K + 1) + 13) n_x + (M + 2) J G^2 + J N^2 complex64 values, ~0.24 GB
 * at N = 160, J = 10, G = 320, M = 7, K = 10.  With gbar = dL/dx^_M (device [n_x]; for
 * complex vectors the gradient of a real L is dL/dRe + i dL/dIm):
 *   Ybar_out       device [J][G][G] complex64: dL/dY
 *   alpha0_bar_out host double: dL/dalpha_0 (alpha_n = alpha0 q^n), or NULL
 *   xprev_bar_out  device [n_x]: dL/dx_prev through the initial value and
 *                  the regulariser x_ref = damping x_prev, or NULL (zero
 *                  when x_prev is NULL).
 * Y, turn and x_prev as in nlinv_frame.  The scalars of the recorded CG
 * and of its reverse stay on the device (FP64); the call reads alpha0-bar
 * back once at the end, so it returns after the work on `stream` is
 * complete.  Uses a plan-owned workspace that is allocated on first use.
 * Returns NLINV_ENUMERIC if the recorded CG breaks down. */
int nlinv_frame_vjp(nlinv_plan_t plan, const void* Y, int turn, const void* x_prev,
                    const void* gbar, void* Ybar_out, double* alpha0_bar_out,
                    void* xprev_bar_out, nlinv_stream_t stream);

/* nlinv_frame_vjp of nframes independent frames of one plan (nframes <= its
 * max_batch): host arrays of device pointers Y[f], x_prev[f] (the array or
 * an entry may be NULL), gbar[f], Ybar_out[f], xprev_bar_out[f] (array or
 * entry NULL: not wanted), host ints turns[f]; alpha0_bar_out: host double
 * [nframes] (or NULL).  Each frame's reverse pass runs on its own stream and
 * frame workspace of the plan, forked from and joined back into `stream`;
 * the call returns once all are complete.  A slot's reverse pass is captured
 * into a CUDA graph on its first use (and again when alpha_0, the turn or the
 * presence of x_prev / xprev_bar_out change) and replayed through the slot's
 * staging buffers; do not call while the calling thread captures a stream. */
int nlinv_batch_vjp(nlinv_plan_t plan, int nframes, const void* const* Y, const int* turns,
                    const void* const* x_prev, const void* const* gbar, void* const* Ybar_out,
                    double* alpha0_bar_out, void* const* xprev_bar_out, nlinv_stream_t stream);

/* Bounded device-side wait until *flag == expected (flag: device int),
 * polling at most spin_limit times; on expiry the plan latches
 * NLINV_ETIMEOUT, which nlinv_sync() returns.  This is the wait primitive of
 * the frame dependencies; it also lets a caller check the timeout path. */
int nlinv_wait_flag(nlinv_plan_t plan, const int* flag, int expected, long long spin_limit,
                    nlinv_stream_t stream);

/* Wait for `stream`, then return and clear the plan's latched device error
 * (NLINV_OK, NLINV_ETIMEOUT or NLINV_ENUMERIC) or NLINV_ECUDA. */
int nlinv_sync(nlinv_plan_t plan, nlinv_stream_t stream);

/* Static description of an error code. */
const char* nlinv_strerror(int code);

/* Last CUDA error string seen by the library on this thread (or ""). */
const char* nlinv_last_cuda_error(void);

#ifdef __cplusplus
}
#endif
#endif /* NLINV_H */
