/*
 * s2w.h - C ABI of libs2w, the GB300 (sm_103a) source-to-waveform library.
 *
 * The library evaluates the two-stage linear time-invariant map of the paper
 * (arXiv 2608.21763, Sec. II):
 *
 *     m_n = sum_{k=0}^{n} F_{G,k} s_{n-k}       Eq. (elastic-response)
 *     v   = D_t m                               Sec. II-B.2
 *     q_n = sum_{k=0}^{n} F_{q,k} v_{n-k}       Eq. (waveform-response)
 *
 * i.e. q = F_q D_t F_G s (Alg. 1 steps 2-4, on one GPU, with the sum over
 * grid partitions of Eq. (distributed-composition) done inside the device),
 * with each block-Toeplitz matvec evaluated by FFT along time (Alg. 2):
 * zero-pad to L = 2 Nt, real FFT, per-bin complex contraction over bins
 * l = 0..Nt, inverse FFT, keep the first Nt samples.
 *
 * Notation: Ns = subfaults (N_f), Ng = seafloor grid points (N_m), No =
 * observations (N_q), Nt = time steps, Nb = Nt + 1 bins, B = ruptures per call.
 *
 * Conventions shared by every entry point:
 *  - Arrays are row-major float32 with the time index fastest.
 *  - Pointer arguments may be host or device memory; the library tells them
 *    apart with cudaPointerGetAttributes.  Device pointers must belong to the
 *    context's device.  The caller owns every array it passes; the library
 *    never keeps a pointer past the call.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  Work is
 *    enqueued on it.  When an output is host memory, the call copies the
 *    result back and synchronises `stream` before returning; when all outputs
 *    are device memory, the call returns once the work is enqueued and the
 *    caller must keep inputs alive until the stream has passed the work.
 *  - Every call returns an s2w_status.  A message for the last failure is
 *    available from s2w_last_error.  Nothing aborts or prints.
 *  - Kernel-side failures (a bounded wait that expired) are latched in a
 *    device status word and reported by the next s2w_sync as S2W_ERR_TIMEOUT.
 */
#ifndef S2W_H
#define S2W_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct s2w_ctx s2w_ctx;

typedef enum {
  S2W_OK = 0,
  S2W_ERR_ARG = -1,         /* invalid argument (size, pointer, alignment) */
  S2W_ERR_OOM = -2,         /* device allocation failed */
  S2W_ERR_STATE = -3,       /* call out of order (e.g. operators not loaded) */
  S2W_ERR_CUDA = -4,        /* a CUDA runtime call failed */
  S2W_ERR_TIMEOUT = -5,     /* a kernel-side bounded wait expired */
  S2W_ERR_UNSUPPORTED = -6  /* valid request outside what this build supports */
} s2w_status;

/* Storage of a resident operator spectrum.  Products accumulate in FP32
 * (FP32 pairs for FP32_HILO).  BF16: round-to-nearest-even bf16 complex.
 * BF16_HILO: two bf16 arrays hi = bf16(x), lo = bf16(x - hi), used as
 * hi + lo.  FP8_E4M3: e4m3 complex with one FP32 scale per (bin, 256
 * consecutive grid rows), scale = amax / 448 computed in FP64 (stage-1
 * operator only).
 * FP32_HILO: two FP32 arrays hi + lo holding each spectrum to about 48
 * significant bits (twice the FP32 bytes), and every step of the stream
 * engine (the slip FFT, both contractions, the retransform, the reduction
 * and the final IFFT) carried in FP32 pairs with error-free sums and
 * products; only the waveforms are rounded to FP32 at the end.  An FFT
 * evaluation errs relative to its whole 2 Nt-sample window, so when a
 * waveform's energy lies mostly past the kept Nt samples (late arrivals)
 * the kept head's relative error grows with that energy ratio; FP32 pairs
 * keep the head at FP32 accuracy for ratios up to ~10^8.  For both
 * operators or neither; stream engine only; no adjoint.  Spectra loaded as
 * complex64 (s2w_load_*_spectra) carry no low-order part (lo = 0): load
 * time-domain responses, whose spectra the library computes in pairs. */
typedef enum {
  S2W_PREC_FP32 = 0,
  S2W_PREC_BF16 = 1,
  S2W_PREC_BF16_HILO = 2,
  S2W_PREC_FP8_E4M3 = 3,
  S2W_PREC_FP32_HILO = 4
} s2w_prec;

/* D_t between the stages.  The paper (Sec. II-B.2) names "a discrete
 * temporal-difference stencil" without printing it; BACKWARD is the
 * first-order backward difference v[n] = (m[n] - m[n-1]) / dt, m[-1] = 0.
 * NONE gives v = m (two plain consecutive convolutions). */
typedef enum { S2W_DT_BACKWARD = 0, S2W_DT_NONE = 1 } s2w_dt_mode;

/* Contraction engine for s2w_waveforms.  STREAM: CUDA-core kernels that
 * stream the resident spectra once per rupture (any storage precision).
 * TENSOR: tcgen05 tensor-core GEMMs over the whole rupture batch (one pass
 * over the spectra per sub-batch); needs prec_g = BF16, BF16_HILO or
 * FP8_E4M3, Nt <= 256, No <= 128.  With BF16 the activations (slip and
 * velocity spectra) and the stage-2 operator are rounded to BF16 and the
 * retransform runs as a GEMM (sub-batches of up to 256 ruptures).  FP8 works
 * the same way except in stage 1: its tiles are widened exactly to FP16 in
 * shared memory and multiplied by the slip spectra packed as FP16 (scaled by a
 * power of two from their largest magnitude), with the per-(bin, 256 rows)
 * scales and that power of two undone in the epilogue.  With BF16_HILO every
 * operand (both operators, both activations and the retransform matrix) is
 * split into hi + lo BF16 parts and each K step issues three MMAs (hi hi,
 * hi lo, lo hi) into FP32 accumulators (sub-batches of up to 128).  A call
 * that asks for the seafloor field runs on the stream kernels.  AUTO: TENSOR
 * for calls with B >= the batch threshold (2, or what s2w_autotune measured,
 * which may be 1) when prec_g allows it, STREAM otherwise.  The stream engine
 * handles the ruptures of a call in groups of up to 64. */
typedef enum { S2W_ENGINE_AUTO = 0, S2W_ENGINE_STREAM = 1, S2W_ENGINE_TENSOR = 2 } s2w_engine;

typedef struct {
  int prec_g;     /* s2w_prec of the stage-1 spectrum Ghat (default FP32) */
  int prec_p;     /* s2w_prec of the stage-2 spectrum Phat: FP32, BF16 or FP32_HILO */
  int dt_mode;    /* s2w_dt_mode (default BACKWARD) */
  double dt;      /* time step of D_t in seconds (default 1.0, Sec. II-A) */
  int max_batch;  /* largest B accepted by s2w_waveforms (sizes workspaces) */
  int device;     /* CUDA device ordinal (default 0) */
  int engine;     /* s2w_engine (default AUTO) */
  int tc_adjoint; /* 1: also keep transposed copies of both operator spectra
                     (K-major along the grid) so that s2w_adjoint and
                     s2w_misfit_gradient run on the tensor engine for
                     batches (same rules as s2w_waveforms); doubles the
                     stage-1 operator memory.  0 (default): the adjoint
                     streams the spectra once per rupture. */
  int single_pass; /* 1: the single-pass variant (an ablation of the
                      truncate-and-retransform step): both operators are kept
                      at FFT length L = 4 Nt (2 Nt + 1 bins, twice the bytes),
                      D_t is folded into the stage-2 spectra as the factor
                      (1 - exp(-2 pi i l / L)) / dt, and the seafloor spectra
                      go straight into stage 2 with no IFFT / Truncate / FFT
                      between the stages.  L >= 3 Nt - 1 keeps the circular
                      convolution of the three factors free of wrap onto the
                      kept samples.  Stream engine only; Nt <= 256; no
                      seafloor output, adjoint or no-alloc path.  The
                      spectral loaders then take 2 Nt + 1 bins of length-4 Nt
                      DFTs.  0 (default): L = 2 Nt with the retransform. */
  int tc_pair;     /* tensor engine: S2W_PAIR_ON runs each GEMM whose shape
                      allows it (BF16 or hi/lo operands, N a
                      multiple of 32, at least two 128-row M tiles) as
                      two-SM MMAs: a pair of CTAs computes one 256-row tile
                      with each CTA staging half of the B tile.  S2W_PAIR_OFF
                      keeps one CTA per 128-row tile; S2W_PAIR_AUTO (0,
                      default) takes the two-SM form for the 512-column
                      GEMMs of BF16 operators (256-rupture sub-batches).
                      The BF16 stage-2 GEMM, whose adjoint operand is stored
                      once (the embedding's second rows are built in shared
                      memory), runs on one CTA per tile in every mode; the
                      FP8-activation stage-1 GEMM is always two-SM. */
  int tc_fp8_act;  /* prec_g = FP8_E4M3 only.  1: the tensor engine also
                      rounds the slip spectra, stage 1's B operand, to e4m3
                      with one power-of-two scale per (bin, rupture) (amax to
                      <= 448), and runs stage 1 as FP8 x FP8 MMAs (tcgen05
                      kind::f8f6f4, two-SM tiles): twice the BF16 MMA rate
                      and no widening of the operator, at the cost of the
                      activation rounding (<= 2^-4 relative per entry) on
                      top of the operator's.  2 (default): the same with the
                      slip spectra as hi + lo e4m3 parts in that frame (lo =
                      the rounded remainder), two FP8 x FP8 MMAs per K step:
                      activations kept to ~2^-8, the FP16 path's accuracy
                      for these contractions, with both operands read as
                      bytes straight from TMA.  0: the operator tiles
                      widened exactly to FP16 in shared memory, FP16
                      activations.  1 and 2 are used for sub-batches whose
                      grid spans at least two 128-row tiles; others take the
                      FP16-activation path.  With another prec_g the default
                      2 is ignored and 1 is an argument error. */
  int tc_bsub;     /* tensor engine: ruptures per GEMM pass (the sub-batch),
                      128 or 256 (BF16_HILO: 128); 0 (default) = 256, or 128
                      for BF16_HILO, capped by max_batch.  The workspaces are
                      sized for it; s2w_autotune may lower it to 128. */
  int tc_s2_chunks; /* tensor engine: chunks of the grid (the K extent) that
                      split the stage-2 GEMM, 1..16; 0 (default) = the count
                      that balances bins x row tiles x chunks over the SMs,
                      and for BF16_HILO at least the count that keeps each
                      chunk within 2,048 K elements (one FP32 accumulation
                      each; longer ones cost that precision accuracy).
                      Results depend on it (the partial sums are added in
                      chunk order). */
  const char *tune_cache; /* path of the autotuner's cache file, or NULL
                      (default).  s2w_autotune reads its choices from it
                      when the file holds an entry for this problem (Ns,
                      Ng, No, Nt, the batch, both precisions, the FP8
                      activation and adjoint options and the GPU model) and
                      otherwise measures and writes one.  The string is read
                      during s2w_create and s2w_autotune only. */
  int fault;        /* test hook, an s2w_fault (default S2W_FAULT_NONE).  When
                      it is NONE, s2w_create reads the environment variable
                      S2W_FAULT ("wait", "oom_load" or "launch") instead. */
  int fault_wait_us; /* with fault = S2W_FAULT_WAIT: the bound of every wait
                      in the streaming kernels, in microseconds (default
                      5000; otherwise those waits are bounded by 2 s). */
} s2w_opts;

enum { S2W_PAIR_AUTO = 0, S2W_PAIR_ON = 1, S2W_PAIR_OFF = 2 };

/* Injected failures for testing the error paths (the paper has no
 * counterpart).  None of them faults, traps or hangs the GPU.
 *   WAIT      the streaming stage-1 kernel's copy producer skips its first
 *             copy, so the consumers' bounded wait on that stage runs out
 *             after fault_wait_us: the kernel latches the timeout in the
 *             device status word, drains its own copies and returns; the
 *             next s2w_sync returns S2W_ERR_TIMEOUT (the waveforms of that
 *             call are undefined).  Stream engine only.
 *   OOM_LOAD  every operator load fails as if its staging allocation had
 *             failed (S2W_ERR_OOM); no row is marked loaded.
 *   LAUNCH    s2w_waveforms fails before its first launch as if the launch
 *             had failed (S2W_ERR_CUDA); nothing is enqueued. */
typedef enum { S2W_FAULT_NONE = 0, S2W_FAULT_WAIT = 1, S2W_FAULT_OOM_LOAD = 2, S2W_FAULT_LAUNCH = 3 } s2w_fault;

/* Fill *o with the defaults listed above (max_batch = 1). */
void s2w_default_opts(s2w_opts *o);

/* Create a context for Ns x Ng x No operators over Nt steps.  Allocates the
 * resident spectra (sizes: s2w_operator_bytes) and workspaces on
 * opts->device.  Supported: Nt in {32, 64, 128, 256, 512}; 1 <= Ns <= 1024;
 * Ng >= 1; 1 <= No.  *out is NULL on failure.  opts may be NULL (defaults). */
int s2w_create(int Ns, int Ng, int No, int Nt, const s2w_opts *opts, s2w_ctx **out);

/* Release every device allocation of the context.  NULL is accepted. */
int s2w_destroy(s2w_ctx *ctx);

/* Bytes of the resident stage-1 and stage-2 spectra of a context. */
int s2w_operator_bytes(const s2w_ctx *ctx, size_t *g_bytes, size_t *p_bytes);

/* Load grid rows g0 .. g0+ng-1 of the stage-1 operator from its time-domain
 * impulse responses G[r][j][k] = [F_{G,k}]_{g0+r, j} (Sec. II-B.1), layout
 * [ng][Ns][Nt].  The library zero-pads each response to L = 2 Nt, takes its
 * real FFT with FP64-generated twiddles (Sec. II-C.1: spectra computed once
 * at setup and kept resident), and stores bins 0..Nt in the context's
 * precision.  Rows may be loaded in any order and in any number of calls;
 * s2w_waveforms requires every row to have been loaded once.  FP8 storage
 * requires g0 to be a multiple of 256 and ng a multiple of 256 unless the
 * chunk ends at Ng.  Synchronises `stream` before returning. */
int s2w_load_greens(s2w_ctx *ctx, int g0, int ng, const float *G, void *stream);

/* Load grid columns g0 .. g0+ng-1 of the stage-2 operator from its
 * time-domain responses P[o][r][k] = [F_{q,k}]_{o, g0+r} (Sec. II-B.2,
 * adjoint acoustic-gravity responses), layout [No][ng][Nt].  Same transform
 * and rules as s2w_load_greens (no alignment rule). */
int s2w_load_adjoint(s2w_ctx *ctx, int g0, int ng, const float *P, void *stream);

/* Load operator spectra directly (the form the paper keeps resident, Sec.
 * II-C.1: the blocks' zero-padded DFTs, bins l = 0..Nt of length 2 Nt):
 *   Ghat[l][r][j] = sum_{k<Nt} G[g0+r][j][k] exp(-2 pi i k l / (2 Nt)),
 * complex64 (re, im interleaved), layout [Nt+1][ng][Ns].  Same storage
 * conversion (precision, FP8 scales, 256-row chunk rule), transposed copies
 * and pointer rules as s2w_load_greens; rows of both loaders may be mixed. */
int s2w_load_greens_spectra(s2w_ctx *ctx, int g0, int ng, const float *Ghat, void *stream);

/* Phat[l][o][r] = sum_{k<Nt} P[o][g0+r][k] exp(-2 pi i k l / (2 Nt)),
 * complex64, layout [Nt+1][No][ng].  Rules as s2w_load_adjoint. */
int s2w_load_adjoint_spectra(s2w_ctx *ctx, int g0, int ng, const float *Phat, void *stream);

/* Waveforms for B ruptures: q[b] = F_q D_t F_G slip[b].
 *   slip      [B][Ns][Nt]  slip-rate histories s_j[n]          (input)
 *   q         [B][No][Nt]  observation waveforms q_o[n]        (output)
 *   seafloor  [B][Ng][Nt]  seafloor motion m_i[n], or NULL     (output)
 * 0 <= B <= max_batch (B = 0 does nothing).  Requires both operators fully
 * loaded (else S2W_ERR_STATE). */
int s2w_waveforms(s2w_ctx *ctx, const float *slip, int B, float *q, float *seafloor, void *stream);

/* s2w_waveforms for ruptures with uneven active durations: rupture b's
 * slip-rate histories are taken as zero from sample active_len[b] on (those
 * samples are never read, so they may hold anything).  active_len: host
 * array of B ints in [0, Nt] (S2W_ERR_ARG otherwise); NULL = all Nt.  The
 * frequency-domain contractions stay dense in the bins, so the cost is that
 * of s2w_waveforms; results equal s2w_waveforms on zero-filled tails, bit for
 * bit. */
int s2w_waveforms_active(s2w_ctx *ctx, const float *slip, const int *active_len, int B, float *q,
                         float *seafloor, void *stream);

/* Adjoint of s2w_waveforms (the paper has no adjoint of the pipeline; this is
 * the transpose of the same map): for B residual sets r[b] ([No][Nt]),
 *   grad_s[b] = F_G^T D_t^T F_q^T r[b]     ([Ns][Nt]),
 * i.e. the gradient of 0.5 ||q(s) - d||^2 with respect to the slip-rate
 * histories when r = q(s) - d.  Each transpose is a correlation with the
 * conjugate spectra, (F^T y)_j[n] = sum_i sum_{k <= Nt-1-n} f_ij[k] y_i[n+k],
 * evaluated as conj(Fhat_l) yhat_l per bin with zero padding to 2 Nt (no
 * wrap reaches the kept samples), and D_t^T w[n] = (w[n] - w[n+1]) / dt with
 * w[Nt] = 0.  Without opts.tc_adjoint: the streaming kernels, one rupture at
 * a time, for every storage precision.  With opts.tc_adjoint (BF16 or
 * BF16_HILO storage) and B >= the AUTO batch threshold (or ENGINE_TENSOR):
 * both correlations run as tcgen05 GEMMs over the sub-batch against the
 * transposed spectra, with the same hi/lo splitting as the forward tensor
 * path and the FP32 FFT retransform with D_t^T between them.  Pointer and
 * stream rules as s2w_waveforms. */
int s2w_adjoint(s2w_ctx *ctx, const float *r, int B, float *grad_s, void *stream);

/* Gradient of the waveform misfit L_b = 0.5 ||q(slip[b]) - d[b]||^2 for B
 * ruptures: forward waveforms, residual r = q - d, then s2w_adjoint(r).
 *   slip [B][Ns][Nt], d [B][No][Nt] (inputs); grad_s [B][Ns][Nt] (output);
 *   loss [B] (output, may be NULL; same memory kind as grad_s).
 * Pointer and stream rules as s2w_waveforms. */
int s2w_misfit_gradient(s2w_ctx *ctx, const float *slip, const float *d, int B, float *grad_s, float *loss,
                        void *stream);

/* Waveforms for ONE rupture without allocating any memory (the paper has no
 * counterpart; this serves callers that cannot let a library allocate device
 * memory: applications whose device memory all comes from their own pool,
 * code inside a CUDA stream capture, latency-bound loops that must not wait on
 * the allocator).  Same result as s2w_waveforms with B = 1 and no seafloor
 * output; the intermediates live in a static 32 MiB device array that every
 * GPU which loads libs2w holds until the process exits.
 *   slip [Ns][Nt], q [No][Nt]: device pointers of the context's device.
 * Limits: the problem's scratch (slip, seafloor and velocity spectra, stage-2
 * partials: about 16 (Nt + 1) Ng bytes plus small terms) must fit in 32 MiB,
 * e.g. Ng <= ~7,700 at Ns = 963, Nt = 256; larger problems get
 * S2W_ERR_UNSUPPORTED with the required size in s2w_last_error.
 * The first call on a device looks up the array's device address (one
 * cudaGetSymbolAddress per device); make that first call before any stream
 * capture.  All calls in the process share the array, which keeps the last
 * call's contents (the call clears what must start at zero): calls that can
 * overlap on the GPU (different streams, contexts or threads without
 * ordering) race on it and must be serialised by the caller.  Returns once
 * the work is enqueued on `stream`. */
int s2w_waveforms_noalloc(s2w_ctx *ctx, const float *slip, float *q, void *stream);

/* s2w_waveforms for device pointers, run as a CUDA graph: the first call
 * with a given (slip, q, B) captures the whole launch sequence once (on an
 * internal stream, after synchronising `stream`) and instantiates it; later
 * calls with the same arguments replay it on `stream` with one graph launch
 * and no per-kernel host work.  Up to 8 graphs are kept per context (least
 * recently replayed evicted).  No seafloor output.  Results equal those of
 * s2w_waveforms bit for bit.  The graphs use the context's workspaces:
 * replays on different streams must not overlap, as for s2w_waveforms.
 * S2W_ERR_ARG for host pointers or pointers of another device. */
int s2w_waveforms_graph(s2w_ctx *ctx, const float *slip, int B, float *q, void *stream);

/* Measured choices of the tensor engine, from s2w_autotune. */
typedef struct {
  int from_cache;               /* 1: the choices below came from opts.tune_cache; nothing was timed */
  int tc_min_batch;             /* smallest B that ENGINE_AUTO sends to the tensor engine */
  int tc_bsub;                  /* chosen ruptures per GEMM pass (<= 256) */
  int tc_pair;                  /* chosen GEMM form (S2W_PAIR_AUTO, _ON or _OFF) */
  int tc_s2_chunks;             /* chosen stage-2 K chunk count */
  int probe_batch;              /* batch size of the form and chunk probes */
  float ms_stream_per_rupture;  /* stream engine, one rupture (0 = not run) */
  int form_bsub[6];             /* GEMM forms probed: ruptures per pass (0 = no entry) ... */
  int form_pair[6];             /* ... and S2W_PAIR_* mode */
  float ms_form[6];             /* tensor engine at probe_batch in each form */
  int s2_chunk_cand[4];         /* stage-2 chunk counts probed in the chosen form (0 = none) */
  float ms_s2_chunks[4];        /* tensor engine at probe_batch with each of them */
  float ms_tensor_batch[7];     /* tensor engine at B = 1, 2, 4, 8, 16, 32, 64 (0 = not run) */
} s2w_tuning;

/* Choose the tensor engine's schedule for this problem by timing it on the
 * loaded operators (dummy inputs: the timings do not depend on the data):
 * the GEMM form (ruptures per pass and two-SM or single-CTA tiles), the
 * stage-2 K chunk count (how the grid is split between the persistent
 * CTAs; with the BF16 hi/lo split, only counts at or above the default,
 * since each chunk is one FP32 accumulation and a longer one costs that
 * precision accuracy), and the batch size from which AUTO uses the tensor engine instead
 * of streaming the spectra once per rupture.  The choices are kept in the
 * context (and written to opts.tune_cache when one is set); an entry already
 * in that cache is applied without timing.  Options the caller fixed
 * (tc_bsub, tc_pair other than AUTO, tc_s2_chunks) are not searched.
 * Uses up to B ruptures (<= max_batch).  Without the tensor engine only
 * ms_stream_per_rupture is measured.  Captured graphs (s2w_waveforms_graph)
 * are dropped: they hold the old schedule.  `out` may be NULL. */
int s2w_autotune(s2w_ctx *ctx, int B, s2w_tuning *out, void *stream);

/* Zero-padded real FFT of `rows` signals of Nt samples (the transform of
 * Alg. 2 steps 1-2): X[r][l] = sum_{n<Nt} x[r][n] exp(-2 pi i n l / (2 Nt)),
 * l = 0..Nt, X as interleaved (re, im) float pairs [rows][Nt+1][2].
 * x and X must be device pointers. */
int s2w_rfft(s2w_ctx *ctx, const float *x, long long rows, float *X, void *stream);

/* Inverse of the above with truncation (Alg. 2 steps 4-5): from bins
 * X[r][0..Nt] of a real length-2Nt signal, x[r][n] for n < Nt.  Device
 * pointers only. */
int s2w_irfft(s2w_ctx *ctx, const float *X, long long rows, float *x, void *stream);

/* The retransform between the two stages (Alg. 2: IFFT, Truncate to Nt
 * samples, D_t, ZeroPad to 2 Nt, FFT) of one real signal's Nt + 1 bins,
 * written as the real 2 Nt x 2 Nt matrix that the tensor engine applies
 * (rounded to BF16 there): T[n][k] row-major, over the degrees of freedom
 * k = 0: Re bin 0, k = 1: Re bin Nt, k = 2l / 2l + 1: Re / Im bin l
 * (0 < l < Nt), the same ordering for the outputs n.  transpose = 1 gives
 * the adjoint's map (D_t^T in place of D_t).  dt_mode / dt as in s2w_opts.
 * Evaluated in FP64 on the host; T (caller-owned) receives 4 Nt^2 doubles.
 * Touches no device.  S2W_ERR_ARG for a NULL T, a bad dt_mode, dt <= 0 or
 * transpose not 0 / 1; S2W_ERR_UNSUPPORTED for Nt outside 32, 64, 128,
 * 256. */
int s2w_retransform_matrix(int Nt, int dt_mode, double dt, int transpose, double *T);

/* Per-stage CUDA-event timers (the per-stage timing of Sec. III-B).
 * Stages: 0 rfft of slip, 1 stage-1 contraction, 2 retransform (IFFT,
 * Truncate, D_t, ZeroPad, FFT), 3 stage-2 contraction, 4 partial reduction +
 * IFFT + Truncate, 5 host<->device copies made by s2w_waveforms, 6 packing
 * of tensor-engine operands (slip spectra into the stage-1 B operand), 7 a
 * whole replayed graph (s2w_waveforms_graph). */
#define S2W_NUM_STAGES 8
typedef struct {
  double ms[S2W_NUM_STAGES];           /* summed event-timed durations */
  long long count[S2W_NUM_STAGES];     /* timed launches per stage */
  long long launches;                  /* kernel launches by the library (always counted) */
} s2w_profile;

/* on != 0: clear the totals and start recording a CUDA event before and after
 * every stage launch, on the stream the stage runs on.  on == 0: stop. */
int s2w_profile_enable(s2w_ctx *ctx, int on);

/* Synchronise the recorded events and return the totals since enable.
 * `launches` counts every kernel the library launched since the context was
 * created (recording on or off). */
int s2w_profile_read(s2w_ctx *ctx, s2w_profile *out);

/* Wait for all work of the context's device, then report and clear the
 * device status word (S2W_ERR_TIMEOUT if a kernel-side wait expired). */
int s2w_sync(s2w_ctx *ctx);

/* Message of the last failing call on ctx (or of the last failing
 * s2w_create when ctx is NULL).  Valid until the next call on ctx. */
const char *s2w_last_error(const s2w_ctx *ctx);

/* Static name of a status code. */
const char *s2w_status_string(int status);

#ifdef __cplusplus
}
#endif

#endif /* S2W_H */
