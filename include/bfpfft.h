/*
 * bfpfft -- block-floating-point FP16 FFT and SAR range-Doppler compression
 * for NVIDIA GB300 (sm_103a).  C ABI.
 *
 * Paper: "Range, Not Precision: Block-Floating-Point Half-Precision FFT and
 * SAR Imaging" (arXiv 2605.28451).  Section references below are to it.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Every call returns an int status (enum bfpfft_status); no exception or
 *   longjmp crosses this boundary.  bfpfft_error_string() names a status.
 * - Complex data is interleaved (re, im), row-major: a batch of lines of n
 *   points each, consecutive lines n points apart unless a call says otherwise.
 *   Element types by dtype: BFPFFT_F32 -> float2 (8 B / point);
 *   BFPFFT_F16_BFP and BFPFFT_F16_NAIVE -> __half2 (4 B / point);
 *   BFPFFT_E4M3_BFP and BFPFFT_E5M2_BFP -> two FP8 bytes (2 B / point).
 * - Device pointers are owned by the caller (e.g. torch tensors) and must be
 *   16-byte aligned; a misaligned pointer returns BFPFFT_ERR_MISALIGNED.
 *   In-place execution (in == out) is allowed wherever input and output have
 *   the same element type and layout.
 * - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *   Exec calls only enqueue work; they return after the launch, and a launch
 *   failure is reported as BFPFFT_ERR_CUDA.
 * - Arithmetic is FP32 in registers and shared memory for every dtype; the
 *   dtype fixes only the storage format in HBM (Section VI's "FP16 storage /
 *   FP32 compute" mode).  Twiddle tables are generated on the GPU in FP64.
 * - Supported lengths: powers of two with 16 <= n <= 65536 for the row
 *   transforms; anything else returns BFPFFT_ERR_UNSUPPORTED.
 */
#ifndef BFPFFT_H_
#define BFPFFT_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum bfpfft_status {
  BFPFFT_OK = 0,
  BFPFFT_ERR_INVALID_ARG = 1,   /* null pointer, negative size, bad enum value */
  BFPFFT_ERR_UNSUPPORTED = 2,   /* length / dtype / direction combination not provided */
  BFPFFT_ERR_CUDA = 3,          /* a CUDA runtime call or kernel launch failed */
  BFPFFT_ERR_OOM = 4,           /* device allocation for a plan failed */
  BFPFFT_ERR_TIMEOUT = 5,       /* a bounded device-side wait expired */
  BFPFFT_ERR_NONFINITE = 6,     /* informational: output holds Inf or NaN */
  BFPFFT_ERR_MISALIGNED = 7     /* a buffer is not 16-byte aligned */
};

enum bfpfft_dtype {
  BFPFFT_F32 = 0,        /* FP32 storage: the comparison path (Section V, Table II) */
  BFPFFT_F16_BFP = 1,    /* FP16 storage with the fixed 1/N block shift (Eq. 1) */
  BFPFFT_F16_NAIVE = 2,  /* FP16 storage without the shift (Section III-B's failing path) */
  BFPFFT_E4M3_BFP = 3,   /* FP8 E4M3 storage, static block exponents (Section VII) */
  BFPFFT_E5M2_BFP = 4,   /* FP8 E5M2 storage, static block exponents (Section VII) */
  BFPFFT_F16_ADAPTIVE = 5,  /* FP16 mantissas (half2) plus one int32 exponent per line, chosen from
                               the line's block maximum (Section VIII): bfpfft_exec_adaptive */
  BFPFFT_BF16 = 6           /* bfloat16 storage (re, im pairs, 4 B / point) and bfloat16 arithmetic,
                               with the 1/N shift (Section IV-C); n <= 16384, uniform plans */
};

/*
 * Arithmetic of a plan's transforms (bfpfft_plan_set_arith), the precision
 * modes of Section VI (and Table I's pure FP16, Section IV-C's bfloat16).
 * The storage dtype is unchanged by the mode.
 */
enum bfpfft_arith {
  BFPFFT_ARITH_F32 = 0,             /* FP32 registers and shared memory (default; FP16 storage + FP32
                                       compute for the FP16 dtypes) */
  BFPFFT_ARITH_F16 = 1,             /* pure FP16: every add and multiply in half2, FP16 twiddles, FP16
                                       shared-memory exchange (F16_BFP / F16_NAIVE, n <= 16384) */
  BFPFFT_ARITH_F16_MUL_F32_ACC = 2, /* FP16 operands, FP32 accumulation: each radix-16 DFT block on the
                                       tensor cores (tcgen05.mma kind::f16), twiddles FP32 (F16_BFP,
                                       E4M3_BFP or E5M2_BFP, n = 4096; FP8 values convert exactly to
                                       FP16 operands and the block exponent scales the first pass's FP32
                                       results, so the stored scale is the FP8 plan's own) */
  BFPFFT_ARITH_BF16 = 3             /* bfloat16 arithmetic; the one mode of BFPFFT_BF16 plans */
};

/* Plan flags (bfpfft_plan_set_flags). */
enum bfpfft_flags {
  BFPFFT_CHECK_FINITE = 1  /* every output store checks its value; a non-finite one sets the
                              plan's status to BFPFFT_ERR_NONFINITE (read by bfpfft_plan_status) */
};

enum bfpfft_direction {
  BFPFFT_FORWARD = -1,   /* X[k] = sum_n x[n] exp(-2 pi i n k / N), unnormalised */
  BFPFFT_INVERSE = +1    /* x[n] = (1/N) sum_k X[k] exp(+2 pi i n k / N) */
};

typedef struct bfpfft_plan_s* bfpfft_plan;

/* Library version as major * 10000 + minor * 100 + patch. */
int bfpfft_version(void);

/* Static text for a status code; never NULL. */
const char* bfpfft_error_string(int status);

/*
 * Create a plan for `batch` transforms of length `n` (Section V: batched
 * radix-16 Stockham transforms, one line per thread group, all passes on
 * chip).  direction = BFPFFT_INVERSE computes the normalised inverse DFT as
 * conj(FFT(conj(z) * 1/N)): the 1/N is the fixed block shift folded into the
 * pre-inverse conjugate (Section IV-A, Eq. 1).  With BFPFFT_F16_NAIVE the
 * inverse instead stores the unnormalised result to FP16 and then scales by
 * 1/N, which overflows to Inf once |N y| > 65504 (Section III-B).
 * FP8 plans carry static block exponents, see bfpfft_plan_scale_exp().
 * batch may be 0 (exec is then a no-op).  The plan allocates its twiddle
 * table on the current device; it must be executed on that device.
 * Errors: INVALID_ARG (out NULL, batch < 0, unknown dtype or direction),
 * UNSUPPORTED (n not a power of two in [16, 65536]), OOM, CUDA.
 * On error *out is set to NULL.
 */
int bfpfft_plan_create(bfpfft_plan* out, int64_t n, int64_t batch, int dtype, int direction);

/*
 * Enqueue the planned transforms on `stream`: in and out are buffers of
 * batch * n points in the plan's dtype, 16-byte aligned.  in == out is allowed.
 * Either may also be pinned host memory (cudaHostAlloc / cudaMallocHost),
 * which the kernels then read or write in place over the CPU-GPU link; the
 * caller keeps it alive and unmodified until the stream has passed the call.
 * Errors: INVALID_ARG (NULL plan or buffer), MISALIGNED, CUDA.
 */
int bfpfft_exec(bfpfft_plan plan, const void* in, void* out, void* stream);

/* Free a plan's device resources (synchronous).  NULL is accepted. */
int bfpfft_plan_destroy(bfpfft_plan plan);

/*
 * Uneven batch: `count` transforms of lengths n[i] (powers of two in
 * [16, 65536], mixed freely) at point offsets offset_pts[i] of the in / out
 * buffers, by default all computed by ONE persistent launch.  The plan sorts
 * the lines into tasks of 65,536 points of one length, largest length first;
 * thread-block clusters of 16 CTAs take every clusters-th task in turn (a
 * line of 65536 spans the whole cluster, shorter lines one CTA or part of
 * one) and never wait on each other.  bfpfft_plan_tune or
 * bfpfft_plan_set_many_schedule may choose another schedule (two-pass long
 * lines, FP16 row exchanges, one launch per length).  Offsets must be
 * multiples of 16 points.  dtype: BFPFFT_F32, BFPFFT_F16_BFP, BFPFFT_E4M3_BFP or
 * BFPFFT_E5M2_BFP (FP8 transforms of length n use the block exponents of a
 * uniform plan of that length); direction as for bfpfft_plan_create.
 * Transforms must not overlap each other in `out`; in == out is allowed.
 * The arrays n and offset_pts are host memory, read during the call only.
 * Errors: INVALID_ARG (also an offset that is not a multiple of 16), UNSUPPORTED
 * (a length, BFPFFT_F16_NAIVE, or no room for a 16-CTA cluster on this device),
 * OOM, CUDA.  Execute with bfpfft_exec or bfpfft_exec_graph.
 */
int bfpfft_plan_create_many(bfpfft_plan* out, int64_t count, const int64_t* n, const int64_t* offset_pts,
                            int dtype, int direction);

/* Schedule flags of an uneven plan (bfpfft_plan_set_many_schedule; the tuner's
 * code carries them as clusters + 65536 * flags). */
enum bfpfft_many_schedule {
  BFPFFT_MANY_TWO_PASS = 1,    /* lines of 32768 / 65536 points by the two-pass kernels, before the
                                  persistent launch */
  BFPFFT_MANY_FP16_ROWS = 2,   /* FP16 storage: four-step lines exchange their rows as FP16 words (one more
                                  FP16 rounding inside the transform, within the FP16 error budget) */
  BFPFFT_MANY_PER_LENGTH = 4   /* one launch per length over its listed lines, each with the dense-row kernel
                                  of a uniform plan of that length, instead of the persistent kernel (the
                                  four-step lines still follow BFPFFT_MANY_FP16_ROWS; TWO_PASS does not apply) */
};

/*
 * Set an uneven plan's schedule by hand (what bfpfft_plan_tune chooses):
 * clusters = persistent clusters (0: all resident ones), flags = OR of enum
 * bfpfft_many_schedule.  The arithmetic of every transform stays FP32; only
 * BFPFFT_MANY_FP16_ROWS changes results (one more FP16 storage point).  A graph
 * captured by bfpfft_exec_graph is captured again.
 * Errors: INVALID_ARG (NULL or uniform plan, clusters < 0, unknown flag bits,
 * BFPFFT_MANY_FP16_ROWS without FP16 storage).
 */
int bfpfft_plan_set_many_schedule(bfpfft_plan plan, int clusters, int flags);

/*
 * Autotuner (not in the paper).  Times the candidate kernels of this plan on
 * its own shape -- a uniform plan: the row-kernel variants (plain, with or
 * without an L2 prefetch one wave ahead, at 3 or 4 CTAs per SM, or bulk-copy
 * pipelined; one or two FP32 exchange buffers; with allow_fp16_exchange != 0
 * and FP16 storage also the FP16 shared-memory exchanges, which round at
 * every pass and so change the results within the FP16 error budget; lines
 * of 32768 and 65536 points: the four-step kernel or the two-pass kernels,
 * and with allow_fp16_exchange the four-step kernel with its row exchange in
 * FP16 words); an uneven plan: the number of persistent clusters, whether
 * lines of 32768 / 65536 points run inside the persistent kernel or in the
 * two-pass kernels before it, and with allow_fp16_exchange and FP16 storage
 * whether lines of 8192 points or more exchange their rows in FP16 words --
 * on scratch buffers it allocates and frees (synchronous), keeps the fastest
 * in the plan, and writes it to the tuning cache (file named by
 * BFPFFT_TUNE_CACHE, default $HOME/.cache/bfpfft/tune.txt, keyed by GPU name
 * and shape).  chosen: a uniform plan's variant code, or an uneven plan's
 * clusters + 65536 * (two-pass long lines) + 131072 * (FP16 row exchange);
 * best_ms (may be NULL): its median time.  An FP16 row exchange is one more
 * FP16 storage point: every output stays within the FP16 error budget, not
 * within one rounding of the FP32 result.
 * Plans created while BFPFFT_TUNE=cached apply a cached choice;
 * BFPFFT_TUNE=full also tunes shapes missing from the cache.  The variable
 * BFPFFT_ROWS, when set, overrides any tuned row variant.
 * Errors: INVALID_ARG, OOM, CUDA.
 */
int bfpfft_plan_tune(bfpfft_plan plan, int allow_fp16_exchange, int* chosen, float* best_ms);

/* Tasks and persistent clusters of an uneven plan (both 0 for a uniform plan). */
int bfpfft_plan_info(bfpfft_plan plan, int64_t* tasks, int64_t* clusters);

/*
 * bfpfft_exec through a CUDA graph: the first call for a given (in, out) pair
 * captures the plan's launches (for an uneven plan: the task-counter reset
 * and the persistent kernel) into a graph and instantiates it; every call
 * then launches that graph on `stream`.  A new (in, out) pair re-captures.
 * The graph belongs to the plan and is freed by bfpfft_plan_destroy.
 * Errors: as bfpfft_exec.
 */
int bfpfft_exec_graph(bfpfft_plan plan, const void* in, void* out, void* stream);

/*
 * Static block exponents of a plan: the true value of a stored input point is
 * stored * 2^in_exp and that of a stored output point is stored * 2^out_exp.
 * FP8 forward plans store the spectrum with out_exp = ceil(log2(n) / 2) (the
 * unitary sqrt(N) growth of noise-like data); FP8 inverse plans expect that
 * exponent on input and produce out_exp = 0.  Both are 0 for FP32 and FP16.
 */
int bfpfft_plan_scale_exp(bfpfft_plan plan, int* in_exp, int* out_exp);

/*
 * Read and clear the current device's status word after a device-wide
 * synchronisation.  The calls that take no plan (the SAR compressions,
 * sar_make_filter and autofocus) record errors of their device-side bounded
 * waits there: BFPFFT_ERR_TIMEOUT where a wait expired instead of spinning
 * forever; BFPFFT_OK means no wait expired since the last call.  Plans have
 * a word of their own (bfpfft_plan_status).  Errors: INVALID_ARG (status
 * NULL), CUDA.
 */
int bfpfft_device_status(int* status);

/*
 * Read and clear the plan's own status word after a device-wide
 * synchronisation (call it on the plan's device).  Its kernels record there:
 *   BFPFFT_ERR_TIMEOUT   a bounded device-side wait expired (bulk-copy
 *                        pipelines, four-step exchanges, tensor-core commits);
 *                        the kernel stopped working and returned, and its
 *                        output is not valid;
 *   BFPFFT_ERR_NONFINITE with BFPFFT_CHECK_FINITE set: an output value was Inf
 *                        or NaN (the naive FP16 schedule of Section III-B
 *                        overflows; the shifted schedule of Eq. 1 does not).
 * The first error recorded since the last read is kept (a timeout may replace
 * a non-finite report, not the reverse).  BFPFFT_OK: neither happened.
 * Errors: INVALID_ARG (NULL plan or status), CUDA.
 */
int bfpfft_plan_status(bfpfft_plan plan, int* status);

/*
 * Set the plan's flags: 0 or BFPFFT_CHECK_FINITE (the output stores of every
 * later exec check their values; the check costs no extra memory traffic).
 * A graph captured by bfpfft_exec_graph is dropped and captured again.
 * Errors: INVALID_ARG (NULL plan or an unknown flag bit).
 */
int bfpfft_plan_set_flags(bfpfft_plan plan, int flags);

/*
 * Select the arithmetic of a uniform plan's transforms (enum bfpfft_arith).
 * The 16-bit twiddle table a mode needs is built here, so call it before any
 * stream capture.  A graph captured by bfpfft_exec_graph is captured again.
 * Results change with the mode within its error budget: pure FP16 rounds every
 * operation (about 60 dB SQNR at N = 4096 on N(0,1) lines against the ~74 dB
 * of FP16 storage with FP32 compute); bfloat16 about 18 dB lower than FP16.
 * Errors: INVALID_ARG (NULL plan, unknown mode), UNSUPPORTED (a mode the
 * plan's dtype, length or kind does not offer), OOM, CUDA.
 */
int bfpfft_plan_set_arith(bfpfft_plan plan, int arith);

/*
 * Failure-detection self-test (not in the paper): enqueue on `stream` one
 * small kernel that arms a device-side barrier for a copy that is never
 * issued and waits for it with the same bounded wait the transform kernels
 * use.  The bound (one second of GPU wall time) expires, the kernel records
 * BFPFFT_ERR_TIMEOUT in the plan's status word and returns; the context stays
 * usable.  bfpfft_plan_status then reads BFPFFT_ERR_TIMEOUT.  The plan's
 * buffers and tables are not touched.  Errors: INVALID_ARG, CUDA.
 */
int bfpfft_plan_selftest_wait(bfpfft_plan plan, void* stream);

/*
 * sar_range_compress / sar_azimuth_compress in a chosen arithmetic (Section
 * VI's precision modes of the range-Doppler chain, Table IV): arith
 * BFPFFT_ARITH_F32 is the calls above (FP32 registers; FP16, FP32 or naive
 * storage); BFPFFT_ARITH_F16 runs every transform, the filter product and the
 * 1/N shift in FP16 arithmetic (the "pure FP16" mode; the filter spectrum is
 * rounded to FP16 once; a complex64 raw echo is rounded to FP16 as it is
 * loaded) and needs FP16 output (F16_BFP, or F16_NAIVE for the unshifted
 * schedule) and, for the azimuth call, FP16 input.
 * BFPFFT_ARITH_F16_MUL_F32_ACC (the "FP16 multiply, FP32 accumulate" mode) runs
 * both transforms of a line on the tensor cores (the tensor-core rows of
 * bfpfft_plan_set_arith: FP16 operands at every pass, FP32 accumulation) and
 * the filter product and 1/N shift in FP32 between them; lines of 4096 points
 * only, FP16-BFP output, FP32 or FP16 input (rounded to FP16 operands as it is
 * loaded).  Both 16-bit modes turn corners with the tiled transpose whatever
 * BFPFFT_SAR_TURN says.
 * Errors: as the calls above; INVALID_ARG for an unknown arith; UNSUPPORTED for
 * a length or storage combination the mode does not offer.
 */
int sar_range_compress_arith(const void* raw, int raw_dtype, void* out, int out_dtype, const void* hr,
                             int64_t n_az, int64_t n_rg, int transpose_out, int arith, void* stream);
int sar_azimuth_compress_arith(const void* rc, int rc_dtype, int rc_layout, void* img, int img_dtype,
                               const void* ha, int64_t n_az, int64_t n_rg, int arith, void* stream);

/* ---------------------------------------------------------------------------
 * Adaptive per-line block exponents (Section VIII, Limitations).
 *
 * The fixed 1/N shift of Eq. 1 suits inputs of known scale.  For inputs of any
 * amplitude the paper names the alternative: one exponent per block, picked
 * by a block-max reduction.  Here a block is one line.  After the line's
 * transform(s) in FP32, m = max over the line of |Re| and |Im|; the exponent
 * e is the smallest integer with m * 2^-e <= 2^14, read from the bits of the
 * FP32 maximum; the line is stored as FP16 mantissas RN(v * 2^-e) (largest
 * component in (2^13, 2^14]) plus e.  Its value is mantissa * 2^e.  A zero
 * line gets e = 0; a line holding Inf or NaN is stored unscaled with e = 0.
 * Mantissas: half2 [lines][n]; exponents: int32 [lines] device arrays.
 * Lengths: powers of two in [16, 16384].
 * ------------------------------------------------------------------------- */

/*
 * Execute a plan of dtype BFPFFT_F16_ADAPTIVE (created by bfpfft_plan_create;
 * n <= 16384; bfpfft_exec rejects such a plan with INVALID_ARG).  in: FP16
 * mantissas [batch][n]; in_exp: int32 [batch] input exponents, or NULL for all
 * zero (values = the FP16 numbers themselves; exponents are clamped to
 * [-252, 252]); out: FP16 mantissas [batch][n]; out_exp: int32 [batch],
 * written.  Forward: X = DFT(x); inverse: the normalised inverse DFT with its
 * 1/N folded into the pre-inverse conjugate (Eq. 1).  Arithmetic FP32.
 * in == out is allowed (and in_exp == out_exp).  Asynchronous on `stream`.
 * Errors: INVALID_ARG (NULL plan / buffer / out_exp, or a plan of another
 * dtype), MISALIGNED, CUDA.
 */
int bfpfft_exec_adaptive(bfpfft_plan plan, const void* in, const int32_t* in_exp, void* out, int32_t* out_exp,
                         void* stream);

/*
 * Forward-multiply-inverse with an adaptive output exponent per line (the
 * general pipeline of Section VIII's Generality paragraph, stored as above):
 * out, out_exp = IDFT(DFT(x) . H) per line of n points, `lines` lines.
 *   x      x_dtype BFPFFT_F32 (complex64 values; x_exp must be NULL) or
 *          BFPFFT_F16_ADAPTIVE (FP16 mantissas with x_exp, or NULL for zeros)
 *   h      float2[n] filter spectrum (conj(DFT(ref)) for a matched filter)
 *   out    FP16 mantissas [lines][n]; out_exp int32 [lines]
 * A SAR range line of any amplitude compresses without overflow: the fixed
 * shift keeps an unnormalised matched filter's output in FP16 range only for
 * unit-scale echoes.  lines = 0 is a no-op.  Asynchronous on `stream`.
 * Errors: INVALID_ARG, UNSUPPORTED (n or x_dtype), MISALIGNED, CUDA.
 */
int bfp_spectral_adaptive(const void* x, int x_dtype, const int32_t* x_exp, const void* h, void* out,
                          int32_t* out_exp, int64_t n, int64_t lines, void* stream);

/*
 * Batched forward-multiply-inverse, y = IDFT(DFT(x) . H) per line, with the
 * fixed 1/N shift of Eq. 1 (Section VIII, Generality: FFT convolution and
 * correlation, and the spectral layers of Fourier neural operators, reuse the
 * schedule).  The kernels are those of the SAR compression calls below; the
 * line is held on chip from load to store.
 *   x         [lines][n], x_dtype BFPFFT_F32 or BFPFFT_F16_BFP (16-byte aligned)
 *   h         float2 filter spectra: h_stride = 0 applies h[n] to every line
 *             (convolution with DFT(g), correlation with conj(DFT(g)));
 *             h_stride = n gives line l its own h[l n .. l n + n) (a spectral
 *             layer's per-channel weights; zeros above a cut-off truncate the
 *             modes).  Other strides: INVALID_ARG.
 *   out       [lines][n], out_dtype BFPFFT_F32, BFPFFT_F16_BFP or BFPFFT_F16_NAIVE
 *             (no shift: overflows as Section III-B predicts)
 *   n         a power of two in [256, 16384]
 *   arith     BFPFFT_ARITH_F32, BFPFFT_ARITH_F16 or BFPFFT_ARITH_F16_MUL_F32_ACC,
 *             with the storage combinations and lengths of
 *             sar_range_compress_arith
 * lines = 0 is a no-op.  Asynchronous on `stream`.
 * Errors: INVALID_ARG, UNSUPPORTED (n, dtype or arith combination), MISALIGNED,
 * CUDA.
 */
int bfp_spectral_filter(const void* x, int x_dtype, const void* h, int64_t h_stride, void* out, int out_dtype,
                        int64_t n, int64_t lines, int arith, void* stream);

/* ---------------------------------------------------------------------------
 * SAR range-Doppler compression (Section VI, Fig. 1).
 *
 * Matched-filter compression y = IDFT(DFT(x) . H) of every line, computed as
 * conj(DFT(conj(DFT(x) . H) * 1/N)): forward transform, filter multiply and
 * the 1/N block shift folded into the conjugate (Eq. 1), then the inverse,
 * all in one kernel with the line held on chip.  FP32 arithmetic; the dtype
 * arguments fix only the storage formats.  With an F16_NAIVE output the shift
 * is dropped: the unnormalised inverse (O(N^2) for an unnormalised filter,
 * Section III-B) is stored to FP16 before the 1/N, and overflows to Inf.
 * Supported line lengths: powers of two in [256, 16384].
 * ------------------------------------------------------------------------- */

/*
 * Filter spectrum from a time-domain reference line: h_out = conj(DFT(ref)),
 * divided by max_k |DFT(ref)[k]| when peak_normalise != 0 (|H| <= 1, the
 * filter of Section III-B's magnitude argument).  ref and h_out are float2[n]
 * device buffers; ref is the transmitted pulse placed circularly centred at
 * index 0.  Errors: INVALID_ARG, MISALIGNED, UNSUPPORTED (n), CUDA.
 * The first call for a given device and length allocates that length's
 * twiddle table; make it before any stream capture.
 */
int sar_make_filter(const void* ref, int64_t n, int peak_normalise, void* h_out, void* stream);

/*
 * Range compression: for each of the n_az azimuth lines raw[eta][0..n_rg),
 * out = IDFT(DFT(raw[eta]) . Hr).
 *   raw        [n_az][n_rg], raw_dtype BFPFFT_F32 (complex64) or BFPFFT_F16_BFP (half2)
 *   out        out_dtype BFPFFT_F32, BFPFFT_F16_BFP or BFPFFT_F16_NAIVE;
 *              transpose_out = 0: [n_az][n_rg];  transpose_out = 1: [n_rg][n_az]
 *   hr         float2[n_rg], the range filter spectrum
 * The corner turn of transpose_out = 1 is by default a tiled transpose of the
 * compressed rows through stream-ordered scratch (n_az * n_rg points of the
 * output type) from a library-owned CUDA memory pool that keeps its memory
 * between calls; with the environment variable BFPFFT_SAR_TURN=fused it is
 * done on chip by a thread-block cluster instead (no scratch).
 * n_az = 0 is a no-op.  out must not overlap raw when transpose_out = 1.
 * With transpose_out = 0 this is the general batched forward-multiply-inverse
 * pipeline of Section VIII (Generality) on dense lines: hr = DFT(g) gives the
 * circular convolution of each line with g, hr = conj(DFT(g)) the circular
 * correlation (the range matched filter is the correlation with the pulse).
 * Errors: INVALID_ARG, MISALIGNED, UNSUPPORTED (n_rg or dtypes), OOM (scratch),
 * CUDA.
 */
int sar_range_compress(const void* raw, int raw_dtype, void* out, int out_dtype, const void* hr,
                       int64_t n_az, int64_t n_rg, int transpose_out, void* stream);

/*
 * Azimuth compression: for each of the n_rg range columns,
 * img[:, r] = IDFT(DFT(rc[:, r]) . Ha), lines of length n_az.
 *   rc         rc_dtype BFPFFT_F32 or BFPFFT_F16_BFP;
 *              rc_layout = 0: [n_az][n_rg];
 *              rc_layout = 1: [n_rg][n_az] (as written by sar_range_compress
 *              with transpose_out = 1)
 *   img        [n_az][n_rg], img_dtype BFPFFT_F32, BFPFFT_F16_BFP or BFPFFT_F16_NAIVE
 *   ha         float2[n_az], the azimuth filter spectrum
 * By default the azimuth lines are compressed as dense rows into
 * stream-ordered scratch and turned into img by a tiled transpose (layout 0
 * is first turned into scratch as well); BFPFFT_SAR_TURN=fused gathers and
 * scatters the columns on chip through thread-block clusters instead.
 * n_rg = 0 is a no-op.  img must not overlap rc.
 * Errors: INVALID_ARG, MISALIGNED, UNSUPPORTED (n_az or dtypes), OOM (scratch),
 * CUDA.
 */
int sar_azimuth_compress(const void* rc, int rc_dtype, int rc_layout, void* img, int img_dtype,
                         const void* ha, int64_t n_az, int64_t n_rg, void* stream);

/*
 * Range-Doppler image with range-cell-migration correction and a
 * range-dependent azimuth filter (Section VI: the RCMC stage of the
 * range-Doppler chain).  For the hyperbolic range history sqrt(R^2 + v^2 t^2)
 * a target at Doppler frequency f sits dR(f) = R (1/D(f) - 1) further out,
 * D(f) = sqrt(1 - (lambda f / (2 v))^2), and its azimuth chirp has the FM
 * rate k_a(R) = 2 v^2 / (lambda R PRF^2) cycles per pulse^2.  Steps:
 *   1. range compression of every azimuth line (as sar_range_compress);
 *   2. azimuth DFT of every range line: the range-Doppler domain;
 *   3. SAR_RDA_RCMC: every Doppler row f (signed bin k, f = k PRF / n_az) moved
 *      back by dR(f, R0) / range_cell cells by an exact band-limited shift
 *      (DFT along range, linear phase, 1/N shift, inverse);
 *   4. every range bin r: the filter conj(DFT(ref_r)) of its own reference
 *      chirp exp(-i pi k_a(R_r) n^2), n in [-L/2, L/2), circularly centred at
 *      index 0, with R_r = R0 + (r - n_rg/2) range_cell (SAR_RDA_RANGE_DEPENDENT;
 *      else R_r = R0), divided by its largest magnitude with
 *      SAR_RDA_PEAK_NORMALISE; times the line; the 1/N-shifted inverse DFT.
 *   raw       [n_az][n_rg], raw_dtype BFPFFT_F32 or BFPFFT_F16_BFP
 *   img       [n_az][n_rg], img_dtype BFPFFT_F32 or BFPFFT_F16_BFP (FP16
 *             requires SAR_RDA_PEAK_NORMALISE: an unnormalised filter lifts a
 *             unit target's image peak past 65504)
 *   hr        float2[n_rg], the range filter spectrum
 *   geometry  host double[5]: range cell (m), PRF (Hz), wavelength (m), speed
 *             (m/s), slant range of cell n_rg/2 (m)
 *   aperture  azimuth chirp length L (even, 2 <= L <= n_az)
 * n_az, n_rg: powers of two in [256, 8192].  Intermediates are stored in the
 * image's format; scratch (2 n_az n_rg points) comes from the library's
 * stream-ordered pool, as for the corner turns of the SAR calls.
 * Asynchronous on `stream`.  Errors: INVALID_ARG (NULL, flags, geometry with
 * lambda PRF / (4 v) >= 1, aperture), UNSUPPORTED (sizes, dtypes), MISALIGNED,
 * OOM, CUDA.
 */
enum sar_rda_flags { SAR_RDA_RCMC = 1, SAR_RDA_RANGE_DEPENDENT = 2, SAR_RDA_PEAK_NORMALISE = 4 };
int sar_rda_image(const void* raw, int raw_dtype, void* img, int img_dtype, const void* hr, int64_t n_az,
                  int64_t n_rg, const double* geometry, int64_t aperture, int flags, void* stream);

/* ---------------------------------------------------------------------------
 * Entropy phase autofocus with a hand-written adjoint.
 *
 * The paper has no autofocus section; this builds standard SAR entropy
 * autofocus on its azimuth compression (Fig. 1).  For range-compressed data
 * rc[r][n] (range bin r, pulse n) and a per-pulse phase correction phi[n]:
 *   v = rc . exp(-j phi[n]),  I[r] = IDFT(DFT(v[r]) . Ha),  q = |I|^2,
 *   S = sum q,  E = -sum (q/S) ln(q/S) = ln S - (1/S) sum q ln q,
 *   dE/dphi[n] = 2 sum_r Im( conj((A^H G)[r][n]) v[r][n] ),
 *   G = -(ln(q/S) + E) / S . I,  A^H = IDFT(DFT(.) . conj(Ha)).
 * The image is never stored: the gradient pass recomputes the forward
 * transforms.  FP32 arithmetic; FP64 sums across CTAs.
 * Layout: rc is [n_rg][n_az] (each row one range bin's azimuth line, as written
 * by sar_range_compress with transpose_out = 1), dtype BFPFFT_F32 or
 * BFPFFT_F16_BFP; phi float[n_az], Ha float2[n_az] (device).
 * stats_out: device double[4] = {S, sum q ln q, E, ln S}.
 * workspace: caller-owned device scratch of at least
 * sar_autofocus_workspace_bytes(n_az) bytes (overwritten).
 * Supported n_az: powers of two in [256, 8192].  Asynchronous on `stream`.
 * Errors: INVALID_ARG (NULL, n_rg < 0, workspace too small), UNSUPPORTED,
 * MISALIGNED, CUDA.
 * ------------------------------------------------------------------------- */

/* Workspace bytes for the autofocus calls at azimuth length n_az (0 if unsupported). */
size_t sar_autofocus_workspace_bytes(int64_t n_az);

/* Entropy only (forward pass): writes stats_out. */
int sar_autofocus_entropy(const void* rc, int rc_dtype, const float* phi, const void* ha, int64_t n_az,
                          int64_t n_rg, void* stats_out, void* workspace, size_t ws_bytes, void* stream);

/* Entropy (stats_out) and its gradient grad_out = dE/dphi (device float[n_az]). */
int sar_autofocus_grad(const void* rc, int rc_dtype, const float* phi, const void* ha, int64_t n_az,
                       int64_t n_rg, float* grad_out, void* stats_out, void* workspace, size_t ws_bytes,
                       void* stream);

/*
 * The same two calls in a chosen arithmetic: BFPFFT_ARITH_F32 is the calls
 * above; BFPFFT_ARITH_F16_MUL_F32_ACC runs every transform on the tensor cores
 * (FP16 operands at each radix-16 pass, FP32 accumulation; the filter product,
 * |I|^2, the logarithms and all sums in FP32 / FP64 as above), n_az = 4096
 * only.  The gradient pass scales G by a power of two taken from the largest
 * |I|^2 of the entropy pass, so its FP16 operands stay in range; like the
 * FP16 transforms, the mode expects unit-scale rc (|rc| well below 256) and a
 * peak-normalised Ha.  Same workspace as above.
 * Errors: as above; INVALID_ARG for another arith, UNSUPPORTED for another n_az.
 */
int sar_autofocus_entropy_arith(const void* rc, int rc_dtype, const float* phi, const void* ha, int64_t n_az,
                                int64_t n_rg, void* stats_out, void* workspace, size_t ws_bytes, int arith,
                                void* stream);
int sar_autofocus_grad_arith(const void* rc, int rc_dtype, const float* phi, const void* ha, int64_t n_az,
                             int64_t n_rg, float* grad_out, void* stats_out, void* workspace, size_t ws_bytes,
                             int arith, void* stream);

/* ---------------------------------------------------------------------------
 * FP64 metric reductions on the GPU (Section IV-B, Section VI).
 * ------------------------------------------------------------------------- */

/*
 * Point-target metrics of a SAR image, FP64 on the GPU (Section VI, Table
 * III).  The paper names PSLR, ISLR, target SNR and 3 dB resolution without
 * defining windows; per target (eta, r) this computes:
 *   peak cell = argmax |I| within +-4 cells of (eta, r); a 64 x 64 window
 *   around it interpolated x16 by zero-padding its 2-D DFT; the interpolated
 *   maximum within +-1 cell; the range and azimuth cuts through it (1024 fine
 *   samples); per cut the mainlobe (peak to the first minimum on each side),
 *   PSLR = 20 log10(max sidelobe / peak), ISLR = 10 log10(sidelobe / mainlobe
 *   energy), 3 dB width in cells (linear interpolation of the half-power
 *   crossings); SNR = 10 log10(peak^2 / mean |I|^2 over every cell at least
 *   `guard` cells from every target in both axes; each |I|^2 is formed in
 *   FP32 -- exact products of FP16 pixels -- and summed in FP64).  Targets
 *   go through in chunks of 16, with their FP64 intermediates in `workspace`.
 *   img       [n_az][n_rg], dtype BFPFFT_F32 or BFPFFT_F16_*, n_az, n_rg >= 64
 *   targets   device int32 [k][2] = (eta, r)
 *   out       device double [k][12] = PSLR range, PSLR azimuth, ISLR range,
 *             ISLR azimuth, width range, width azimuth (cells), peak |I|, SNR
 *             (dB), noise power, peak cell eta, peak cell r, (reserved)
 *   workspace caller-owned device scratch of sar_point_target_workspace_bytes().
 * Errors: INVALID_ARG, UNSUPPORTED (dtype), MISALIGNED, CUDA.
 */
size_t sar_point_target_workspace_bytes(int64_t n_az, int64_t n_rg);
int sar_point_target_metrics(const void* img, int img_dtype, int64_t n_az, int64_t n_rg, const int32_t* targets,
                             int64_t k, int guard, void* out, void* workspace, size_t ws_bytes, void* stream);

/* Device workspace bytes bfp_sqnr_sums() needs, for any count. */
size_t bfp_sqnr_workspace_bytes(void);

/*
 * The five FP64 sums of the scale-aligned SQNR between a reference `ref` and
 * a test array `test`, `count` complex points each (dtypes BFPFFT_F32 or
 * BFPFFT_F16_*; the two may differ), written to the device buffer
 * sums_out = double[5]:
 *   [0] sum |ref|^2   [1] sum |test|^2   [2] Re sum conj(test) ref
 *   [3] sum |ref - test|^2   [4] number of test points with a non-finite part
 * Non-finite test points are counted and left out of [0..3].  The aligned SQNR
 * (optimal real scale, Section IV-B) is 10 log10([0] / ([0] - [2]^2 / [1])),
 * the unaligned one 10 log10([0] / [3]).  The reduction is two-stage with a
 * fixed summation order (bitwise reproducible).  workspace: caller-owned
 * device scratch of ws_bytes >= bfp_sqnr_workspace_bytes(); its contents are
 * overwritten.  count = 0 writes zeros.  Asynchronous on `stream`.
 * Errors: INVALID_ARG (NULL pointer, count < 0, workspace too small),
 * UNSUPPORTED (dtype), MISALIGNED, CUDA.
 */
int bfp_sqnr_sums(const void* ref, int ref_dtype, const void* test, int test_dtype, int64_t count,
                  void* sums_out, void* workspace, size_t ws_bytes, void* stream);

/*
 * bfp_sqnr_sums_noalloc -- the sums of bfp_sqnr_sums without any workspace.
 * The paper has no counterpart; this entry point exists for callers that
 * cannot allocate device memory: for example a radar processing chain that
 * fixes its whole device-memory budget at start-up and forbids allocation
 * afterwards for predictable latency, or a host application whose own memory
 * pool owns every device byte and has no way to lend the library a
 * workspace.  The caller passes only inputs and the output.
 *
 * Arguments and results are those of bfp_sqnr_sums (ref, test: `count`
 * complex points, dtypes BFPFFT_F32 or BFPFFT_F16_*; sums_out: device
 * double[5]).  The partial sums live in a fixed 160 KB array inside the
 * library that every GPU loading the library keeps until the process exits;
 * this call allocates nothing (no cudaMalloc, no cudaFree).
 * Limit: count <= bfp_sqnr_sums_noalloc_max_count() = 16,777,216 points;
 * larger counts return BFPFFT_ERR_UNSUPPORTED without launching anything.
 * The first call on each device looks up the array's device address (with
 * that device current); make that first call before any stream capture.
 * All calls share the one array: calls that overlap on the GPU (different
 * streams, no ordering between them) race and may return wrong sums; calls
 * ordered on one stream are safe.  Stage 1 rewrites every partial the call
 * reads, so leftovers from an earlier call never leak into a result.
 * Errors: INVALID_ARG, UNSUPPORTED (count or dtype), MISALIGNED, CUDA.
 */
long long bfp_sqnr_sums_noalloc_max_count(void);
int bfp_sqnr_sums_noalloc(const void* ref, int ref_dtype, const void* test, int test_dtype, int64_t count,
                          void* sums_out, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* BFPFFT_H_ */
