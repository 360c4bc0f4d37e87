/*
 * mes.h -- C ABI of the GB300 (sm_103a) library for the Tucker-ALS stage of
 * multi-exposure stereo coding (Sharma & Grover, arXiv 2104.04726).
 *
 * The library covers the data-parallel path of the coding scheme:
 *   colour pre-pass (Section III-A)  ->  Tucker-ALS / HOOI decomposition of
 *   the stacked tensor (Section III-B, Eq. 1 to Eq. 8)  ->  core quantiser
 *   and reconstruction.
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Every call returns mes_status.  No C++ exception crosses the ABI.  On an
 *    error, mes_last_error() returns a thread-local message.
 *  - Array arguments are DEVICE pointers owned by the caller unless a
 *    parameter says otherwise.  The library never frees them.
 *  - Work is enqueued on the caller's CUDA stream (`stream`, a cudaStream_t
 *    passed as void*; NULL is the legacy default stream) and the call returns
 *    without synchronising, except where a parameter says so.  Scalar results
 *    (fit, iteration count, norms) are written to device memory so calls stay
 *    asynchronous.
 *  - Tensors are dense with the FIRST mode fastest: element (i_1, ..., i_N)
 *    of a tensor of dims (s_1, ..., s_N) is at
 *    i_1 + s_1 * (i_2 + s_2 * (i_3 + ...)).
 *    Factor matrices are column-major s_n x r_n (element (i, q) at i + s_n*q).
 *  - Internal scratch memory is taken from the stream-ordered allocator
 *    (cudaMallocAsync on `stream`) and released on the same stream before
 *    the call returns.  MES_ERR_OOM reports a failed allocation.
 *  - Invalid arguments are rejected before anything is enqueued.
 *
 * Environment variables read by the library
 * -----------------------------------------
 *  - MES_TRACE=<file>: mes_tucker_als, mes_reconstruct, mes_colour_convert
 *    and mes_quantize_core time their phases (setup, layout, init, sweep k,
 *    core, orthonormalise, canonical, fit for the decomposition) with CUDA
 *    events on their stream and append one JSON line per call to <file>:
 *    {"call": name, "phases": [[phase, ms], ...], "total_ms": ms}.  A traced
 *    call synchronises its stream before it returns; a call made while its
 *    stream is being captured is not timed.  Every phase is also an NVTX
 *    range (named like the phase, nested in a range named like the call)
 *    whether MES_TRACE is set or not; NVTX costs nothing without a tool.
 *  - MES_FAULT: host-side fault injection for tests of the failure paths (a
 *    comma-separated list): "alloc:<k>" makes internal allocation k of each
 *    call fail with MES_ERR_OOM; "admit" makes the serving loop refuse every
 *    admission (the ticket's status is MES_ERR_OOM).  Nothing touches the GPU.
 *  - MES_TUNE=1: the first use of a tensor-core product shape times every
 *    tile width (128, 256) and split-K factor (1..16) on the caller's stream
 *    and keeps the fastest for the process (never under stream capture);
 *    MES_TUNE_CACHE=<file> loads and appends the choices.  Off by default.
 *  - MES_TC_VARIANT=p1|p2: the TF32 and BF16 products run on the persistent
 *    tensor-core kernel (p1: one CTA per SM; p2: 128-wide tiles, two CTAs per
 *    SM) instead of one tile per CTA.  Same results up to split-K rounding
 *    order; a measurement switch, off by default.
 *  - MES_DEBUG: diagnostic messages on stderr.
 */
#ifndef MES_H
#define MES_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum mes_status {
  MES_OK = 0,
  MES_ERR_INVALID_ARG = 1,   /* null pointer, bad size, bad enum            */
  MES_ERR_RANK = 2,          /* r_n < 1, r_n > s_n, or r_n > prod_{m!=n} r_m */
  MES_ERR_OOM = 3,           /* device allocation failed                    */
  MES_ERR_CUDA = 4,          /* a CUDA runtime call or launch failed        */
  MES_ERR_TIMEOUT = 5,       /* a bounded device-side wait gave up          */
  MES_ERR_NONFINITE = 6,     /* NaN or Inf met where the method forbids it  */
  MES_ERR_NOT_IMPLEMENTED = 7
} mes_status;

typedef enum mes_colour {
  MES_YCBCR601 = 0,   /* ITU-R BT.601 Y'CbCr, full range, no offsets        */
  MES_IPT = 1,        /* Ebner-Fairchild IPT from gamma-linearised sRGB    */
  MES_YCBCR2020CL = 2 /* ITU-R BT.2020 constant-luminance Y'CbCr from
                         gamma-linearised sRGB: BT.709 -> BT.2020 primaries
                         (BT.2087), Yc = 0.2627R + 0.6780G + 0.0593B,
                         BT.2020 transfer function (alpha 1.0993, beta
                         0.0181) on Yc, B, R; Cb, Cr divided by 1.9404 /
                         1.5816 and 1.7184 / 0.9936 by the sign of the
                         difference                                         */
} mes_colour;

typedef enum mes_precision {
  MES_PREC_FP32 = 0,  /* every contraction in FP32 (CUDA cores)            */
  MES_PREC_BF16 = 1,  /* products with T as an operand (the mode products
                         of Eq. 8 and of the T-HOSVD) on BF16 copies of T
                         and the factors, FP32 accumulation; the factored
                         Gram products as in MES_PREC_TF32; the returned
                         core from T itself.  Needs s_1, s_2 multiples of
                         8 (16-byte BF16 rows), else runs as MES_PREC_TF32 */
  MES_PREC_TF32 = 2   /* tensor-core TF32 inputs (FP32 data), FP32 accum.  */
} mes_precision;

typedef enum mes_init {
  MES_INIT_THOSVD = 0,      /* truncated HOSVD (Eq. 6, Eq. 7): every factor
                               from the unfolding Gram of T itself          */
  MES_INIT_INTERLACED = 1   /* interlaced HOSVD (end of the initialisation
                               subsection): modes in order 1..N, mode n's
                               factor from the Gram of T already truncated
                               in modes 1..n-1 (T x_1 S^(1)T ...), so the
                               later modes work on a smaller tensor         */
} mes_init;

/* Thread-local text of the last error on this thread ("" if none). */
const char* mes_last_error(void);

/* Library version string, e.g. "mes 0.1.0 sm_103a". */
const char* mes_version(void);

/*
 * mes_colour_convert -- colour pre-pass of Section III-A and the stacking of
 * Section III-B ("T_MES^c", the tensor of multi-exposure stereo images).
 *
 *  rgb8   [in]  K images, each row-major with s1 pixels per row and s2 rows,
 *               interleaved R,G,B bytes: byte (k, y, x, c) at
 *               ((k*s2 + y)*s1 + x)*3 + c.  Image k = view*E + exposure.
 *  s1, s2, K    image width, height and count (each >= 1).
 *  space        MES_YCBCR601, MES_IPT or MES_YCBCR2020CL.
 *  gamma        IPT and BT.2020 CL: linearisation exponent R = (R')^gamma (> 0).
 *  out    [out] FP32 tensor of dims (s1, s2, 3, K), first mode fastest, i.e.
 *               channel plane (c, k) is the contiguous s1*s2 block number
 *               c + 3k.
 *  norm2  [out] nullable; one double receiving ||out||_F^2 (accumulated in
 *               FP64 with a fixed reduction order: bitwise reproducible).
 * Errors: MES_ERR_INVALID_ARG for null rgb8/out, non-positive sizes, an
 *         unknown space or gamma <= 0; MES_ERR_CUDA on a launch failure.
 */
mes_status mes_colour_convert(const uint8_t* rgb8, int64_t s1, int64_t s2, int64_t K,
                              int space, float gamma, float* out, double* norm2,
                              void* stream);

/*
 * mes_colour_invert -- inverse of the colour pre-pass: a tensor in the colour
 * space of Section III-A (typically the low-rank approximation from
 * mes_reconstruct) back to 8-bit R'G'B' images, the form in which the
 * approximated views go on to the 3D-HEVC encoder (Section III-C).  Each
 * space is solved back to R'G'B' from its definition (mes_colour_convert);
 * linear values below zero keep their sign through the power functions.
 *
 *  X      [in]  FP32 tensor of dims (s1, s2, 3, K), first mode fastest (the
 *               layout mes_colour_convert writes).
 *  s1, s2, K, space, gamma   as for mes_colour_convert.
 *  rgb8   [out] nullable; K images in the layout mes_colour_convert reads,
 *               each channel clamp(rint(255 R'), 0, 255), ties to even.
 *  rgbp   [out] nullable; the same images as FP32 R'G'B' before rounding and
 *               clamping (interleaved like rgb8).
 *  ref8   [in]  nullable; 8-bit images in the layout of rgb8 (e.g. the
 *               input of mes_colour_convert).  Given together with sse8.
 *  sse8   [out] nullable device double: sum over all bytes of (out - ref8)^2,
 *               exact (integer sums), for the PSNR of the decoded views
 *               (Figs. 3 and 4 report it per view after coding).
 * Errors: MES_ERR_INVALID_ARG for a null X, no output at all (rgb8, rgbp,
 *         sse8 all null), only one of ref8 / sse8, non-positive sizes, an
 *         unknown space or gamma <= 0; MES_ERR_OOM; MES_ERR_CUDA on a launch
 *         failure.  A NaN gives byte 0, not an error.
 */
mes_status mes_colour_invert(const float* X, int64_t s1, int64_t s2, int64_t K, int space,
                             float gamma, uint8_t* rgb8, float* rgbp, const uint8_t* ref8,
                             double* sse8, void* stream);

/*
 * Options of mes_tucker_als.  Zero-initialise and set what you need; a NULL
 * options pointer means all defaults.  Fields equal to 0 take the default.
 */
typedef struct mes_als_opts {
  int precision;        /* mes_precision of the large contractions (FP32).
                           The Gram and orthonormalisation products of the
                           factor update stay FP32 in every form.           */
  int init_iters;       /* subspace steps of the T-HOSVD initialisation
                           (default 2; 24 when max_iters <= 2)                */
  int inner_iters;      /* subspace steps per factor update in a sweep
                           (default 1; 12 when max_iters <= 2: a run of one
                           or two sweeps needs each update close to the exact
                           eigenvectors, later sweeps refine them anyway)     */
  uint64_t seed;        /* seed of the random start block of the init (1)     */
  const float* const* init_factors; /* nullable: device factors to start from
                                       instead of T-HOSVD (warm start / resume) */
  int* iters_done;      /* nullable device int: sweeps actually run           */
  double* fit_history;  /* nullable device array of max_iters doubles: fit
                           after each sweep from ||T||^2 - ||Q||^2            */
  int canonical;        /* 0 = default (1): rotate each factor to the
                           eigenvectors of the core's mode-n Gram, sorted by
                           decreasing eigenvalue, sign-fixed; -1 = off        */
  int init;             /* mes_init of the start when init_factors is null
                           (MES_INIT_THOSVD)                                  */
  float* reconstruction; /* nullable device FP32 tensor of dims `dims`: receives
                           T_hat = Q x_1 S^(1) ... x_N S^(N) (Eq. 1) of the
                           returned decomposition, from the same pass that
                           measures the fit (as mes_reconstruct gives with
                           precision FP32 for the FP32 form, TF32 otherwise) */
  int* status;          /* nullable device int, written at the end of the call
                           (stream-ordered): MES_OK, or a failure found on the
                           device -- MES_ERR_TIMEOUT when a bounded tensor-core
                           pipeline wait gave up, MES_ERR_NONFINITE when
                           ||T||^2 or the fit is not finite (NaN or Inf in T).
                           On either failure *fit is NaN, status or not.  The
                           host call itself cannot see these (it returns
                           before the device runs).                           */
  int64_t wait_ns;      /* bound of every tensor-core pipeline wait, in ns (0:
                           2 s).  A wait that runs out sets the timeout status
                           and the kernel finishes without hanging; a bound of
                           a few ns forces that path (tests of error handling) */
  int concurrency;      /* how many decompositions the caller keeps running
                           side by side on this GPU (0 or 1: this one alone).
                           Products whose tile grid does not fill the GPU
                           split their reduction dimension over at most
                           SMs / concurrency CTA slots instead of all SMs:
                           less SM time (fewer partial sums to write and
                           reduce), a longer single call.  Results do not
                           depend on it beyond rounding order (bitwise
                           reproducible for a given value).  The batched and
                           served forms set it from their stream / slot count
                           when a problem leaves it 0.                        */
} mes_als_opts;

/*
 * mes_tucker_als -- Tucker-ALS / HOOI of Section III-B.
 *
 * Computes T ~= Q x_1 S^(1) x_2 ... x_N S^(N) (Eq. 1) with orthonormal
 * factors S^(n) (s_n x r_n), initialised by the truncated HOSVD (Eq. 6,
 * Eq. 7) or the interlaced HOSVD (opts->init) and refined by sweeps n = 1..N in which S^(n) becomes the r_n
 * leading left singular vectors of Y^(n) = T x_{i!=n} S^(i)T (Eq. 8), i.e.
 * the leading eigenvectors of the Gram Y^(n)_(n) Y^(n)_(n)^T.
 *
 *  X        [in]  FP32 tensor of dims `dims`, first mode fastest.
 *  N              order, 2..8.  Modes 1 and 2 may have any size; modes 3..N
 *                 must have s_n <= 32 and prod_{n>=3} s_n <= 1024.
 *  dims, ranks    HOST arrays of N int64.
 *  max_iters      maximum number of sweeps (>= 1).
 *  tol            stop after sweep t > 1 when |fit_t - fit_{t-1}| < tol.
 *  core     [out] FP32 tensor of dims `ranks`, first mode fastest.
 *  factors  [in]  HOST array of N DEVICE pointers; factors[n] [out] receives
 *                 S^(n), column-major s_n x r_n.
 *  fit      [out] nullable device double: 1 - ||T - T_hat||_F / ||T||_F of the
 *                 returned decomposition, from the explicit residual; NaN
 *                 when the device met a failure (see opts->status).
 *  opts           nullable, see mes_als_opts.
 * Errors (returned): MES_ERR_INVALID_ARG (null pointers, N out of range, bad
 *         sizes or options), MES_ERR_RANK (rank constraints), MES_ERR_OOM,
 *         MES_ERR_CUDA.  Failures the device meets while the enqueued work
 *         runs (a pipeline wait that ran out, NaN or Inf in T) arrive in
 *         opts->status and as a NaN fit.
 */
mes_status mes_tucker_als(const float* X, int N, const int64_t* dims, const int64_t* ranks,
                          int max_iters, double tol, float* core, float* const* factors,
                          double* fit, const mes_als_opts* opts, void* stream);

/*
 * mes_tucker_als_workspace_size -- device workspace that mes_tucker_als takes
 * from the stream-ordered allocator for this shape and these options (each
 * request rounded up to 256 bytes), without touching the device.  A caller
 * that budgets device memory (the serving loop) admits a decomposition by
 * this figure plus its own input and output buffers.  The paper has no
 * counterpart; it is bookkeeping for the Section III-B decomposition.
 *
 *  N, dims, ranks, opts   as for mes_tucker_als.
 *  bytes    [out] HOST size_t.
 * Errors: as mes_tucker_als for the shape and options; MES_ERR_INVALID_ARG
 *         for a null `bytes`.
 */
mes_status mes_tucker_als_workspace_size(int N, const int64_t* dims, const int64_t* ranks,
                                         const mes_als_opts* opts, size_t* bytes);

/*
 * mes_reconstruct -- T_hat = Q x_1 S^(1) x_2 ... x_N S^(N) (Eq. 1, Eq. 2).
 *
 *  core     [in]  FP32 tensor of dims `ranks`.
 *  factors  [in]  HOST array of N device pointers, column-major s_n x r_n.
 *  out      [out] FP32 tensor of dims `dims`.
 *  ref      [in]  nullable FP32 tensor of dims `dims`; when given, sse
 *                 receives sum((ref - out)^2) in FP64 (fused into the last
 *                 contraction; bitwise reproducible), or NaN if a tensor-core
 *                 pipeline wait gave up.
 *  sse      [out] nullable device double.
 *  precision      MES_PREC_FP32: every product on CUDA cores in FP32;
 *                 MES_PREC_TF32 or MES_PREC_BF16: the two large products on
 *                 tensor cores with each operand split into two TF32 terms
 *                 (hi*hi + hi*lo + lo*hi, FP32-level accuracy: about 3 * 2^-22
 *                 relative per product); falls back to CUDA cores when r_1
 *                 or r_2 is not a multiple of 4 (16-byte rows for TMA).
 * Same shape limits and errors as mes_tucker_als; MES_ERR_INVALID_ARG for an
 * unknown precision.
 */
mes_status mes_reconstruct(const float* core, const float* const* factors, int N,
                           const int64_t* dims, const int64_t* ranks, float* out,
                           const float* ref, double* sse, int precision, void* stream);

/*
 * mes_quantize_core -- core quantiser, the rate knob of the scheme (the
 * abstract and Section I set the bit rate through the core's ranks and its
 * quantisation; the paper does not define the quantiser).
 *
 * The core (r_1 x r_2 x r_3 x ... x r_N) is cut into P = prod_{n>=3} r_n
 * planes of r_1 x r_2 (plane p is the contiguous block p of the first-mode-
 * fastest core).  Per plane: m = max|x|, qmax = 2^(bits-1) - 1,
 * scale = m / qmax (one FP32 division), q = clamp(rint(x / scale), -qmax,
 * qmax) with FP32 division and round-half-to-even; m == 0 gives scale 0 and
 * q 0.  Results are bit-exact against any IEEE FP32 implementation of the
 * same steps.
 *
 *  core    [in]  FP32, N >= 1 modes (N = 1: one plane of r_1 x 1).
 *  ranks   HOST array of N int64 (each >= 1).
 *  bits    2..16.
 *  q       [out] int16, same element order as the core.
 *  scales  [out] FP32, P entries.
 * Errors: MES_ERR_INVALID_ARG (also for more than 65535 planes or a plane of
 *         more than 2^40 elements); MES_ERR_NONFINITE if a plane holds NaN or
 *         Inf (reported only when `status_host_sync` != 0, since it needs a
 *         device-to-host read; otherwise such planes get scale NaN).
 */
mes_status mes_quantize_core(const float* core, int N, const int64_t* ranks, int bits,
                             int16_t* q, float* scales, int status_host_sync, void* stream);

/*
 * mes_quantize_core_noalloc -- the quantiser of mes_quantize_core for callers
 * that cannot allocate device memory.  The paper has no counterpart; this is
 * an engineering variant.  Same arguments, layouts, arithmetic and results as
 * mes_quantize_core (bit-identical codes and scales), without the NaN/Inf
 * report (a non-finite plane gets scale NaN).
 *
 * Who needs it: code that must not call the device allocator once it is
 * running -- a serving or streaming loop with a fixed memory budget, or a host
 * program that gives the library only buffers it owns -- cannot use
 * mes_quantize_core, whose per-plane scratch comes from cudaMallocAsync.
 * Here that scratch is a fixed array of 4096 words (16 KiB) in device global
 * memory, part of the library image: every GPU that loads the library holds
 * it until the process exits.  The call allocates nothing and calls no
 * allocating routine.
 *
 * Limits and behaviour:
 *  - at most 4096 planes (prod_{n>=3} r_n); more gives MES_ERR_INVALID_ARG
 *    (ranks are checked one by one, so a product that would overflow int64
 *    is rejected too);
 *  - the first call on a device looks up the array's device address (once
 *    per device, with that device current) and keeps it -- make that first
 *    call before any stream capture, and do not call this entry point on a
 *    device after cudaDeviceReset there (the kept address is then stale);
 *  - every call shares the one array: calls whose work overlaps on the GPU
 *    (different streams without ordering) race and give wrong results; calls
 *    ordered on one stream are safe;
 *  - the array keeps the previous call's contents; each call clears the
 *    words it uses before using them.
 */
mes_status mes_quantize_core_noalloc(const float* core, int N, const int64_t* ranks, int bits,
                                     int16_t* q, float* scales, void* stream);

/*
 * mes_problem -- one stack of the batched and served forms: the colour
 * pre-pass (when rgb8 is given), the decomposition and the quantiser (when
 * quant_bits > 0), exactly as mes_colour_convert, mes_tucker_als and
 * mes_quantize_core would run them one after another on one stream, so each
 * result is the same as that of the single calls.  Pointers are caller-owned
 * DEVICE memory; dims, ranks and the factor pointers are held by value, so a
 * problem may be a temporary.
 */
typedef struct mes_problem {
  const uint8_t* rgb8;   /* nullable: K images laid out as for mes_colour_convert;
                            then N = 4 and dims = (s1, s2, 3, K)            */
  int space;             /* mes_colour of rgb8                              */
  float gamma;           /* IPT linearisation exponent (0 means 2.2)        */
  float* X;              /* FP32 tensor of dims: written when rgb8 is given,
                            otherwise the input                             */
  int N;                 /* order, 2..8                                     */
  int64_t dims[8];
  int64_t ranks[8];
  int max_iters;
  double tol;
  mes_als_opts opts;     /* as for mes_tucker_als; all zero = defaults      */
  float* core;
  float* factors[8];
  double* fit;           /* nullable device double                          */
  int quant_bits;        /* 0 = no quantiser, else 2..16                    */
  int16_t* q;            /* quantised core when quant_bits > 0              */
  float* scales;         /* per-plane scales when quant_bits > 0            */
} mes_problem;

/*
 * Batched form: many stacks of uneven size, rank and colour space in one
 * submission.  The paper decomposes one stack at a time; this is the
 * engineering form of Section III-B for many stacks.
 *
 * mes_batch_create(max_streams, out): a batch context on the current device
 *   with max_streams (1..64) internal streams.  *out is a HOST handle.
 * mes_batch_run(b, probs, n, statuses, stream): validates every problem
 *   (statuses: nullable HOST array of n entries receiving each problem's
 *   validation status; nothing is enqueued if any fails), orders them by
 *   estimated work, longest first, and deals them to the internal streams so
 *   each stream's total work is balanced; the streams are forked from and
 *   joined back into `stream`, so all work is ordered after what `stream`
 *   already holds and before what it gets next.
 * mes_batch_capture(b, probs, n, stream): the same enqueue captured into one
 *   CUDA graph held by the context (replacing any previous one); nothing
 *   runs.  Call mes_batch_run once first on the same shapes so one-time setup
 *   happens outside the capture.  The graph holds the problems' pointers.
 * mes_batch_launch(b, stream): replays the captured graph on `stream`.
 * mes_batch_destroy(b): frees the context (after its work completes).
 * Failures the device meets while a problem runs (a tensor-core wait that ran
 * out, NaN or Inf in its tensor) arrive in that problem's opts.status (when
 * set) and as a NaN fit; `statuses` only reports validation and enqueue.
 * Errors: MES_ERR_INVALID_ARG (null handle or arrays, n < 1, a problem that
 *   fails validation, launch without capture, capture while the kernel
 *   profiler is on), errors of the single calls, MES_ERR_CUDA.
 */
typedef struct mes_batch mes_batch;
mes_status mes_batch_create(int max_streams, mes_batch** out);
mes_status mes_batch_run(mes_batch* b, const mes_problem* probs, int n, mes_status* statuses, void* stream);
mes_status mes_batch_capture(mes_batch* b, const mes_problem* probs, int n, void* stream);
mes_status mes_batch_launch(mes_batch* b, void* stream);
mes_status mes_batch_destroy(mes_batch* b);

/*
 * Serving form: a request loop with continuous batching.  Requests are
 * admitted in arrival order as soon as one of `max_slots` slots (each an
 * internal stream) is free and the device memory they need fits in
 * `hbm_budget_bytes` next to the requests already running; a request that
 * does not fit lets later ones that do fit pass it (never more than
 * max_slots of them).  A request's device memory is its workspace
 * (mes_tucker_als_workspace_size plus the quantiser's planes) and its input
 * and output buffers.  State stays on the device; the caller reads results
 * from its own buffers after completion.  The paper has no counterpart; this
 * serves Section III-B decompositions.
 *
 * mes_serve_create(hbm_budget_bytes, max_slots, out): starts the loop (one
 *   host thread) on the current device.
 * mes_serve_submit(s, p, ticket): validates and queues a copy of *p; HOST
 *   *ticket receives its id.  MES_ERR_OOM if it can never fit the budget.
 * mes_serve_poll(s, ticket, done, result, latency_ms): HOST outputs; *done 1
 *   once the request's device work has completed, with its status and its
 *   latency from submission to observed completion (nullable outputs).  The
 *   status includes failures met on the device (MES_ERR_TIMEOUT,
 *   MES_ERR_NONFINITE; the server reads the request's opts.status word, or a
 *   word of its own when the request gives none, after completion).
 * mes_serve_wait(s, ticket, timeout_ms, result, latency_ms): blocks until
 *   done or timeout_ms (< 0: no limit); MES_ERR_TIMEOUT on timeout.
 * mes_serve_get_stats(s, out): counts, latency percentiles of completed
 *   requests and memory in use (HOST struct).
 * mes_serve_destroy(s): waits for queued and running requests, stops the
 *   loop and frees the server.
 * Errors: MES_ERR_INVALID_ARG (null handle or pointer, unknown ticket,
 *   budget 0, max_slots outside 1..64), MES_ERR_OOM, MES_ERR_TIMEOUT,
 *   MES_ERR_CUDA.
 */
typedef struct mes_server mes_server;
typedef struct mes_serve_stats {
  uint64_t submitted, completed, failed, queued, running;
  double p50_ms, p99_ms, max_ms, mean_ms;  /* submit-to-completion latency */
  double first_admit_s, last_done_s;       /* host clock, seconds since creation */
  size_t hbm_in_use, hbm_peak;
} mes_serve_stats;
mes_status mes_serve_create(size_t hbm_budget_bytes, int max_slots, mes_server** out);
mes_status mes_serve_submit(mes_server* s, const mes_problem* p, uint64_t* ticket);
mes_status mes_serve_poll(mes_server* s, uint64_t ticket, int* done, mes_status* result, double* latency_ms);
mes_status mes_serve_wait(mes_server* s, uint64_t ticket, double timeout_ms, mes_status* result,
                          double* latency_ms);
mes_status mes_serve_get_stats(mes_server* s, mes_serve_stats* out);
mes_status mes_serve_destroy(mes_server* s);

/* Inverse of mes_quantize_core: x = q * scale (FP32), same layouts. */
mes_status mes_dequantize_core(const int16_t* q, const float* scales, int N,
                               const int64_t* ranks, float* core, void* stream);

/*
 * Measurement helpers (the paper has no counterpart: they exist to report
 * per-kernel time against the roofline).  When enabled, every kernel launch
 * of the library is bracketed by CUDA events recorded on the launch stream
 * and its algorithmic flops and bytes are accumulated per kernel family.
 * Not for use while a stream is being captured into a CUDA graph.
 *
 * mes_profile_enable(1) clears the records and starts recording; 0 stops.
 * mes_profile_count() is the number of kernel families recorded.
 * mes_profile_get(i, ...) synchronises on family i's events and returns its
 *   name (NUL-terminated, at most name_len bytes, host buffer), launch count,
 *   total device milliseconds, flops and bytes (host pointers, nullable).
 *   MES_ERR_INVALID_ARG for a bad index or buffer, MES_ERR_CUDA if an event
 *   query fails.
 */
void mes_profile_enable(int on);
int mes_profile_count(void);
mes_status mes_profile_get(int i, char* name, int name_len, int64_t* launches, double* ms,
                           double* flops, double* bytes);

/*
 * Test hook for the library's matrix-product kernels (no counterpart in the
 * paper; used by the test suite to check each kernel in isolation).
 * C[b][m][n] = sum_k A[b][m][k] * B[b][n][k], all row-major FP32 device
 * arrays, batch >= 1.  impl 0: CUDA-core FP32 kernel; 1: tcgen05 kind::tf32;
 * 2: tcgen05 kind::f16 on BF16-rounded copies of A and B; 3: tcgen05
 * kind::tf32 on the three-term split (hi + lo of A and B); 4: tcgen05
 * kind::f16 on the six-term split (three BF16 parts of A and B, the six
 * part products down to 2^-16 of the leading one).  Synchronises the
 * stream.  MES_ERR_INVALID_ARG for bad sizes or operands the tensor-core
 * kernel cannot address (row strides must be multiples of 16 bytes);
 * MES_ERR_TIMEOUT if a bounded pipeline wait gave up.
 */
mes_status mes_gemm_selftest(int impl, const float* A, const float* B, float* C, int64_t M, int64_t N,
                             int64_t K, int batch, void* stream);

/*
 * Test hook for the factorization and solve of one CholeskyQR pass (the
 * factor update after Eq. 8 runs them on every r x r Gram; used by the test
 * suite to check the kernels in isolation).  H: r x r symmetric positive
 * definite, column-major (only the lower part is read); W, V: s x r
 * column-major; all FP32 device arrays, 1 <= r <= 1024.  Computes
 * dinv = diag(H)^-1/2, L lower triangular with L L^T = D^-1 H D^-1
 * (D = diag(dinv)^-1; only the lower part of L is written), and
 * V = W D^-1 L^-T, i.e. V R = W for the upper triangular R = (D L)^T with
 * R^T R = H.  The factorization raises a diagonal shift and restarts when a
 * pivot falls below its floor; *restarts (nullable host int) receives the
 * number of restarts.  Synchronises the stream.  MES_ERR_INVALID_ARG for bad
 * sizes or W == V; MES_ERR_NONFINITE when diag(H) has a non-positive or
 * non-finite entry.
 */
mes_status mes_solve_selftest(const float* H, int r, const float* W, int64_t s, float* L, float* dinv,
                              float* V, int* restarts, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* MES_H */
