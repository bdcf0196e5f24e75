/*
 * pfb.h -- C ABI of the GB300 polyphase filter bank (PFB) channeliser.
 *
 * The operation (TINA, arXiv 2408.16551, Sec. 5.2 with Sec. 4.3 and 4.1):
 *   an input stream x[n] is cut into frames of P samples, branch p of frame f
 *   being x_p(f) = x[f*P + p]; each branch runs a T-tap FIR (the paper's
 *   FIR-as-convolution, Sec. 4.3, in its cross-correlation form
 *   O(w) = sum_n I(w+n) K(n)), and every spectrum of P branch sums goes
 *   through a P-point DFT (the Fourier-matrix product Z = X F of Sec. 4.1):
 *
 *     y[s,p] = sum_{m<T} h[m*P + p] * x[(s+m)*P + p]            (Sec. 5.2)
 *     X[s,k] = sum_{p<P} y[s,p] * exp(-2*pi*i*p*k/P)             (Sec. 4.1)
 *
 *   for s < S = max(0, floor(N/P) - T + 1) ("valid" spectra, hop P).
 *   h[0..P*T) is the prototype filter: a symmetric window (Hann, Hamming,
 *   Blackman) times sinc((n - (L-1)/2) / P), normalised to sum(h) = 1, or
 *   caller-supplied taps.
 *
 * Conventions for every entry point:
 *   - Device pointers are plain CUDA device addresses on the plan's device,
 *     16-byte aligned.  The caller owns all input/output buffers; they must
 *     stay alive until the work that uses them completes (stream order for
 *     pfb_execute*, pfb_poll()==PFB_OK for pfb_submit).  The library owns plan
 *     tables, batch tables and per-stream filter state.
 *   - Errors are reported by status code only; nothing aborts or throws across
 *     this ABI.  Arguments are validated before any launch, so an invalid call
 *     has no effect on the device.  pfb_last_error() gives a message for the
 *     calling thread's last failed call.
 *   - pfb_execute* are asynchronous on the given CUDA stream (a cudaStream_t
 *     passed as void*; NULL = legacy default stream) and never synchronise.
 *   - Output layout: complex64 (interleaved fp32 re, im) X[s][k], spectrum-
 *     major, bin k contiguous (the paper's Z(m,n): m = spectrum, n = bin).
 *   - Input layouts: PFB_IN_R32 = float32[N]; PFB_IN_C64 = complex64[N]
 *     (interleaved re, im); PFB_IN_CI8 = int8[2N] (interleaved re, im),
 *     dequantised in-kernel as value * in_scale.
 */
#ifndef PFB_H_
#define PFB_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PFB_API_VERSION 4

#if defined(__GNUC__)
#define PFB_API __attribute__((visibility("default")))
#else
#define PFB_API
#endif

typedef enum pfb_status {
    PFB_OK = 0,
    PFB_PENDING = 1,          /* pfb_poll: submitted work not finished yet */
    PFB_ERR_INVALID = -1,     /* bad argument; nothing was launched */
    PFB_ERR_OOM = -2,         /* device or host allocation failed */
    PFB_ERR_CUDA = -3,        /* a CUDA runtime call failed */
    PFB_ERR_BUSY = -4,        /* server: over budget/slots and not queuing */
    PFB_ERR_TIMEOUT = -5,     /* a bounded wait ran out (host or device side) */
    PFB_ERR_INTERNAL = -6,    /* a kernel reported an internal consistency error */
    PFB_ERR_UNSUPPORTED = -7  /* valid request this build has no kernel for */
} pfb_status;

typedef enum pfb_in_dtype { PFB_IN_R32 = 0, PFB_IN_C64 = 1, PFB_IN_CI8 = 2 } pfb_in_dtype;

typedef enum pfb_window {
    PFB_WIN_HANN = 0, PFB_WIN_HAMMING = 1, PFB_WIN_BLACKMAN = 2, PFB_WIN_USER = 3
} pfb_window;

/* How the P-point DFT of Sec. 4.1 is computed. */
typedef enum pfb_dft_path {
    PFB_DFT_FFT_F32 = 0,      /* radix shared-memory FFT, FP32 (the fast path) */
    PFB_DFT_GEMM_F32 = 1,     /* product with the DFT matrix, FP32 on the SIMT cores */
    PFB_DFT_GEMM_BF16X3 = 2   /* product with the DFT matrix on the tensor cores:
                                 y and W split into bf16 hi+lo, three products
                                 (hi*hi + hi*lo + lo*hi), FP32 accumulation */
} pfb_dft_path;

typedef struct pfb_plan_s *pfb_plan_t;
typedef struct pfb_batch_s *pfb_batch_t;
typedef struct pfb_server_s *pfb_server_t;

/* Order of the T taps within a branch. */
typedef enum pfb_tap_order {
    PFB_TAPS_CORRELATION = 0, /* y[s,p] = sum_m h[m*P+p] x[(s+m)*P+p]: the FIR-as-
                                 convolution mapping of Sec. 4.3, O(w) = sum_n I(w+n) K(n) */
    PFB_TAPS_CONVOLUTION = 1  /* y[s,p] = sum_m h[(T-1-m)*P+p] x[(s+m)*P+p]: the
                                 convolution y_p(n') = sum_m h_p(m) x_p(n'-m) of the
                                 Sec. 5.2 equation, taps reversed within each branch */
} pfb_tap_order;

/* Plan descriptor.  P: branches = channels, a power of two in [4, 4096].
 * T: taps per branch, 1..64.  in_scale: dequantisation factor for
 * PFB_IN_CI8 (must be finite; ignored for other dtypes).  user_taps_host:
 * P*T doubles (host memory, read during pfb_plan_create only) when
 * window == PFB_WIN_USER, else NULL; user taps are used as given.
 * device: CUDA ordinal, or -1 for the calling thread's current device.
 * hop: samples between consecutive spectra; 0 (or P) = critically sampled.
 * A hop D < P gives an oversampled channeliser (R = P/D spectra per frame):
 *     X[s,k] = sum_{n<P*T} h'[n] x[s*D + n] exp(-2 pi i n k / P)
 * (the windowed-overlap-add form of the P-hop PFB, evaluated every D
 * samples, no phase correction), with h' the taps in tap_order.  D must
 * divide P, R <= 32, and D * (bytes per input sample) must be a multiple of
 * 16.  tap_order: pfb_tap_order.  reserved: must be 0. */
typedef struct pfb_plan_desc {
    int32_t P;
    int32_t T;
    int32_t in_dtype;        /* pfb_in_dtype */
    float in_scale;
    int32_t window;          /* pfb_window */
    int32_t path;            /* pfb_dft_path */
    const double *user_taps_host;
    int32_t device;
    int32_t hop;             /* 0 = P */
    int32_t tap_order;       /* pfb_tap_order */
    int32_t reserved;        /* must be 0 */
} pfb_plan_desc;

/* Build a plan: validates the descriptor, then generates on the GPU, in FP64,
 * the prototype filter (Sec. 5.2 taps), the FFT twiddles and, for the GEMM
 * paths, the DFT matrix of Sec. 4.1 (bf16 hi/lo splits or fp32), and stores
 * them in device memory owned by the plan.  Synchronises the device once.
 * Errors: PFB_ERR_INVALID (descriptor), PFB_ERR_OOM, PFB_ERR_CUDA. */
PFB_API pfb_status pfb_plan_create(const pfb_plan_desc *desc, pfb_plan_t *out_plan);

/* Free the plan's device tables.  The caller must ensure no launched work
 * still uses the plan.  NULL is accepted. */
PFB_API pfb_status pfb_plan_destroy(pfb_plan_t plan);

/* Kernel-side status of the plan's launches.  Every kernel bounds its
 * device-side waits (1 s of %globaltimer by default); a wait that runs out
 * makes the kernel wind down and write an error code into the plan's error
 * word, which lives in mapped, pinned host memory.  This call reads and
 * clears that word without blocking or synchronising: PFB_OK if no launch of
 * the plan has failed since the last read, PFB_ERR_TIMEOUT if a device-side
 * wait ran out, PFB_ERR_INTERNAL for any other kernel error code.  Call it
 * after the work of interest has completed (e.g. after a stream or event
 * synchronisation); the word is shared by all launches of the plan, so a
 * failure cannot be attributed to one of several overlapping launches.
 * pfb_execute_host and pfb_execute_host_noalloc read and clear the word
 * themselves before returning; the server gives every batch its own word. */
PFB_API pfb_status pfb_plan_status(pfb_plan_t plan);

/* Test hook for the error reporting above (no paper counterpart; the
 * failure-detection path of the channeliser).  mode 1 makes the producer
 * role of the single-CTA warp-specialised FFT kernel (FFT path, P = 1024,
 * variant 5) issue no input copies, so every consumer's bounded wait runs
 * out after wait_ns nanoseconds and the launch reports PFB_ERR_TIMEOUT; no
 * memory is touched and no GPU fault is provoked.  mode 0 restores normal
 * operation.  wait_ns (0 = the default of 1 s, at most 4 s) bounds the
 * device-side waits of the plan's launches in either mode; kernels other
 * than that one ignore the mode and keep the default bound.
 * Errors: PFB_ERR_INVALID for an unknown mode or wait_ns out of range. */
PFB_API pfb_status pfb_plan_set_fault(pfb_plan_t plan, int32_t mode, int64_t wait_ns);

/* Spectra produced for n_samples input samples: max(0, floor(n/P) - T + 1)
 * (Sec. 5.2 valid outputs, hop P); with a hop D < P, floor((n - P*T)/D) + 1
 * for n >= P*T, else 0.  Returns -1 for a NULL plan or n < 0. */
PFB_API int64_t pfb_out_spectra(pfb_plan_t plan, int64_t n_samples);

/* Copy the plan's FP64 prototype filter h[0..P*T) (as generated on the GPU)
 * to host memory.  cap = number of doubles available at host_out. */
PFB_API pfb_status pfb_plan_get_taps(pfb_plan_t plan, double *host_out, int64_t cap);

/* Channelise one stream: X = DFT(FIR(x)) for all S valid spectra.
 * d_in: n_samples samples in the plan's in_dtype (device memory).
 * d_out: complex64 [out_cap_spectra][P] (device memory); S rows are written.
 * Errors: PFB_ERR_INVALID if out_cap_spectra < S, pointers misaligned or NULL
 * while S > 0; PFB_ERR_CUDA if the launch fails.  S == 0 is valid (no-op).
 * A failure inside the kernel (a bounded device-side wait that ran out) is
 * reported afterwards, once the work has completed, by pfb_plan_status. */
PFB_API pfb_status pfb_execute(pfb_plan_t plan, const void *d_in, int64_t n_samples,
                       void *d_out, int64_t out_cap_spectra, void *cuda_stream);

/* Same as pfb_execute, from and to HOST memory; returns after the output is
 * in host_out and starts after the work already queued on cuda_stream.  Two
 * routes, chosen as in pfb_execute_batch_host (pfb_set_host_route):
 *  - mapped: both buffers page-locked and mapped into the device's address
 *    space (both ends of each range), 16-byte aligned, and the plan on the
 *    four-step cluster kernel (FFT path, P = 4096, variant 3): the kernel
 *    reads the input and writes the spectra in host memory over the CPU-GPU
 *    link;
 *  - staged: the library stages the input through device buffers it owns,
 *    pipelined over chunks of about 16 MB of input: host->device copies on an
 *    internal stream, kernels on cuda_stream, device->host copies on a second
 *    internal stream, so both copy directions and the kernels overlap.
 *    Pinned host memory gives the fastest copies.
 * Results equal those of pfb_execute on both routes.  Returns
 * PFB_ERR_TIMEOUT (output not valid) if a device-side wait of a kernel ran
 * out; the plan's error word is cleared by the call. */
PFB_API pfb_status pfb_execute_host(pfb_plan_t plan, const void *host_in, int64_t n_samples,
                            void *host_out, int64_t out_cap_spectra, void *cuda_stream);

/* Size of the static device staging area of pfb_execute_host_noalloc. */
#define PFB_NOALLOC_SCRATCH_BYTES (32ll << 20)

/* pfb_execute_host that allocates nothing.  The paper has no counterpart: it
 * exists for callers that must not allocate device memory -- a process whose
 * device memory is owned by another allocator (a framework's caching pool, a
 * fixed reservation), or a latency-critical thread that cannot take the
 * device-wide synchronisation cudaMalloc/cudaFree may imply -- while
 * pfb_execute_host grows plan-owned staging buffers with cudaMalloc and
 * creates copy streams and events.
 * Same arguments and results as pfb_execute_host (host_in, host_out in host
 * memory; pinned memory copies fastest).  The whole frames of the input and
 * the S output spectra are staged through one fixed area of static device
 * memory, PFB_NOALLOC_SCRATCH_BYTES (32 MiB) per device, held by every device
 * that loads the library until the process exits: input at offset 0, output
 * at the next multiple of 256 bytes.  Copy in, kernel and copy out run in
 * order on cuda_stream (after the work already queued there); the call
 * returns once host_out is written.  No cudaMalloc, cudaFree, stream or event
 * creation happens in the call.
 *  - The area's device address is looked up (cudaGetSymbolAddress, with
 *    the device current) and cached by pfb_plan_create on the plan's device.
 *    That lookup loads the module holding the area: under CUDA's lazy module
 *    loading this is when the device reserves the 32 MiB, so it happens at
 *    the first plan creation on a device, never inside this entry point.
 *  - Every call on a device shares the one area, which keeps the last call's
 *    contents.  Calls whose work overlaps on the GPU (several host threads,
 *    or several streams) race on it: serialise them.
 * Errors: as pfb_execute_host (PFB_ERR_TIMEOUT from the kernel's error
 * word included); PFB_ERR_INVALID also when the staged input (rounded up to
 * 256 bytes) plus the output exceed PFB_NOALLOC_SCRATCH_BYTES, with nothing
 * launched. */
PFB_API pfb_status pfb_execute_host_noalloc(pfb_plan_t plan, const void *host_in, int64_t n_samples,
                                            void *host_out, int64_t out_cap_spectra, void *cuda_stream);

/* Synthesis (inverse) filter bank, the adjoint of pfb_execute up to the
 * IDFT's 1/P: every spectrum X[s] goes back through the inverse DFT
 * (Sec. 4.2, y~[s,p] = (1/P) sum_k X[s,k] exp(+2 pi i p k / P)) and each
 * branch value is spread over the T frames it was analysed from:
 *     xh[f*P + p] = sum_{m<T} h'[m*P + p] y~[f - m, p],  f < n_spectra + T - 1
 * (y~ = 0 outside the given spectra; h' = the plan's taps in its tap_order).
 * d_spectra: complex64 [n_spectra][P]; d_out: complex64 samples, at least
 * pfb_synth_out_samples() of them.  Needs an FFT-path plan with P in {512,
 * 1024}, T <= 16 and hop P (else PFB_ERR_UNSUPPORTED).  Asynchronous on
 * cuda_stream.  Errors as pfb_execute. */
PFB_API int64_t pfb_synth_out_samples(pfb_plan_t plan, int64_t n_spectra);
PFB_API pfb_status pfb_synthesize(pfb_plan_t plan, const void *d_spectra, int64_t n_spectra, void *d_out,
                                  int64_t out_cap_samples, void *cuda_stream);

/* One stream of a batch. */
typedef struct pfb_batch_item {
    pfb_plan_t plan;
    const void *d_in;
    int64_t n_samples;
    void *d_out;
    int64_t out_cap_spectra;
} pfb_batch_item;

/* Channelise many independent streams of uneven P, T and length in one call:
 * streams are grouped by kernel variant and each group runs as one persistent
 * launch over the flattened list of (stream, spectrum-batch) work units.
 * Streams producing 0 spectra are skipped.  All plans must be on one device.
 * Results equal per-stream pfb_execute bit for bit. */
PFB_API pfb_status pfb_execute_batch(const pfb_batch_item *items, int32_t n_items, void *cuda_stream);

/* pfb_execute_batch from and to HOST memory: items[i].d_in and d_out are
 * host pointers here.  Two routes:
 *  - mapped (taken under PFB_HOST_ROUTE_AUTO when every buffer of the batch
 *    is page-locked host memory mapped into the device's address space --
 *    cudaHostAlloc, cudaMallocHost or cudaHostRegister under unified
 *    addressing -- with both ends of each range mapped and 16-byte aligned,
 *    and every plan's kernel reads and writes the caller's buffers per thread;
 *    in this build that is the four-step cluster kernel, variant 3 of the
 *    FFT path at P = 4096): the kernels read the input and write the spectra
 *    in host memory over the CPU-GPU link, one launch per variant group on
 *    cuda_stream, no staging copies;
 *  - staged (every other case): the streams are staged through device
 *    buffers the library owns (per device, grown with cudaMalloc and kept),
 *    in chunks of consecutive items of about 32 MB of input: chunk c's
 *    copy-in, kernels and copy-out run on a copy-in stream, cuda_stream and a
 *    copy-out stream, three chunks in flight, so copies in both directions
 *    overlap the kernels; calls on one device are serialised.
 * Either route starts after the work already queued on cuda_stream and
 * returns once every output is in host memory (cuda_stream drained).
 * Results equal those of pfb_execute_batch (and of pfb_execute per stream)
 * bit for bit on both routes.  Oversampled plans return
 * PFB_ERR_UNSUPPORTED.  Errors: as pfb_execute_batch; PFB_ERR_OOM for the
 * staging buffers; PFB_ERR_TIMEOUT if a device-side wait of a kernel ran out
 * (every plan's error word is read and cleared). */
PFB_API pfb_status pfb_execute_batch_host(const pfb_batch_item *items, int32_t n_items, void *cuda_stream);

/* Route selection of pfb_execute_batch_host, process-wide (default AUTO). */
#define PFB_HOST_ROUTE_AUTO 0   /* mapped when the batch allows it, else staged */
#define PFB_HOST_ROUTE_STAGED 1 /* always staged */
/* Errors: PFB_ERR_INVALID for another value (the route is unchanged). */
PFB_API pfb_status pfb_set_host_route(int32_t route);

/* The route the calling thread's last pfb_execute_batch_host or
 * pfb_execute_host took: 1 staged, 2 mapped, 0 if it launched nothing (an
 * invalid call, or no spectra). */
PFB_API int32_t pfb_last_host_route(void);

/* A reusable batch: the launches of pfb_execute_batch captured once into a
 * CUDA graph (tile shapes from the autotuner cache), replayed by
 * pfb_batch_launch.  The plans' workspaces (the two-pass DFT-matrix
 * products) are grown before the capture.  The items' buffers and plans must
 * stay valid while the batch object is used. */
PFB_API pfb_status pfb_batch_create(const pfb_batch_item *items, int32_t n_items, pfb_batch_t *out_batch);
PFB_API pfb_status pfb_batch_launch(pfb_batch_t batch, void *cuda_stream);
PFB_API pfb_status pfb_batch_destroy(pfb_batch_t batch);

/* ---------------------------------------------------------------------- */
/* Autotuning: kernel variants (tile shapes) of a plan's kernel family     */
/* ---------------------------------------------------------------------- */

/* Number of kernel variants the plan's family offers (>= 1), and the one in
 * use.  A new plan starts from the variant cached for its shape (see
 * pfb_plan_autotune) or from a built-in default. */
PFB_API int32_t pfb_plan_num_variants(pfb_plan_t plan);
PFB_API int32_t pfb_plan_variant(pfb_plan_t plan);
/* Select a variant explicitly (0 <= variant < pfb_plan_num_variants);
 * PFB_ERR_UNSUPPORTED if the variant has no kernel for the plan's P and T.
 * Variants: FP32 FFT path, P <= 1024: 0-4 tile shapes of the fused kernel,
 * 5 warp-specialised; P = 2048, 4096: 0 synchronous cluster kernel, 1 and 2
 * warp-specialised cluster kernels, 3 (P = 4096) the four-step 64 x 64
 * cluster kernel.  Split-bf16 path: 0 the fused dense DFT-matrix product,
 * 1 the factored (four-step) tensor-core DFT, 2 (P = 1024, 2048, 4096,
 * T <= 16) the dense product in two passes -- the FIR into a plan-owned
 * workspace of 4 * P bytes per spectrum (rounded up to 128-spectrum tiles per
 * stream), then a pipelined tcgen05 GEMM.  The workspace grows on demand
 * inside pfb_execute / pfb_execute_batch (PFB_ERR_OOM if it cannot), so
 * launches of one plan in that variant must not overlap on different
 * streams; pfb_batch_create grows it before capturing, and a graph the caller
 * captures itself needs an earlier launch of the same size (else
 * PFB_ERR_UNSUPPORTED).  A buffer the workspace outgrows is kept until the
 * plan is destroyed, so graphs captured earlier stay valid.  The FP32
 * DFT-matrix path keeps a workspace by the same rules for P a multiple of
 * 128 (8 * P bytes per spectrum, rounded up to 128-spectrum blocks per
 * stream): the FIR pass writes the branch sums there and the GEMM reads
 * them. */
PFB_API pfb_status pfb_plan_set_variant(pfb_plan_t plan, int32_t variant);
/* Time every variant on an input of n_samples (device scratch buffers the
 * call allocates, fills and frees; it synchronises cuda_stream), keep the
 * fastest in the plan and cache it per (GPU, P, T, dtype, family) -- in the
 * process, and in the JSON file named by the environment variable
 * PFB_AUTOTUNE_CACHE if set.  out_best_ms (may be NULL) receives the winner's
 * time per pfb_execute. */
PFB_API pfb_status pfb_plan_autotune(pfb_plan_t plan, int64_t n_samples, void *cuda_stream, double *out_best_ms);

/* ---------------------------------------------------------------------- */
/* Serving: continuous batching of channelisation requests                */
/* ---------------------------------------------------------------------- */

/* hbm_budget_bytes: device bytes the server may hold for in-flight work and
 * resident filter state (admission control).  max_slots: requests allowed
 * on the device at once (1..64).  timeout_ms: a request not finished this
 * long after launch reports PFB_ERR_TIMEOUT.  queue_when_busy: 1 = pfb_submit
 * queues a request that does not fit yet; 0 = it returns PFB_ERR_BUSY. */
typedef struct pfb_server_desc {
    int64_t hbm_budget_bytes;
    int32_t max_slots;
    int32_t timeout_ms;
    int32_t queue_when_busy;
    int32_t device;
} pfb_server_desc;

typedef struct pfb_server_stats {
    int64_t submitted, completed, failed, rejected;
    int64_t queued_now, in_flight_now;
    int64_t reserved_bytes_now, peak_reserved_bytes;
    int64_t samples_completed;
    int64_t batches, batched_requests;  /* launches formed so far and requests they held */
    double p50_latency_us, p99_latency_us, mean_latency_us; /* submit -> completion */
} pfb_server_stats;

PFB_API pfb_status pfb_server_create(const pfb_server_desc *desc, pfb_server_t *out_server);
/* Waits (bounded by timeout_ms per request) for in-flight work, then frees. */
PFB_API pfb_status pfb_server_destroy(pfb_server_t server);

/* Open a stream: allocates its resident filter state (the last T-1 frames of
 * input, device memory, counted against the budget).  The stream starts
 * empty: its first chunk emits floor(n/P) - T + 1 spectra, later chunks
 * floor(n/P) each, so the concatenated outputs equal pfb_execute on the
 * concatenated input. */
PFB_API pfb_status pfb_stream_open(pfb_server_t server, pfb_plan_t plan, int64_t *out_stream_id);
PFB_API pfb_status pfb_stream_close(pfb_server_t server, int64_t stream_id);

/* Spectra the next chunk of n_samples on this stream will emit, counting the
 * chunks already submitted. */
PFB_API int64_t pfb_stream_next_spectra(pfb_server_t server, int64_t stream_id, int64_t n_samples);

/* Submit one chunk (n_samples a multiple of P, device memory) of a stream.
 * Non-blocking: the request is admitted as soon as a slot and budget are
 * free, runs with the stream's resident state, and chunks of one stream
 * complete in submission order.  d_out must hold pfb_stream_next_spectra()
 * rows.  Returns a ticket for pfb_poll/pfb_wait. */
PFB_API pfb_status pfb_submit(pfb_server_t server, int64_t stream_id, const void *d_chunk,
                      int64_t n_samples, void *d_out, int64_t out_cap_spectra,
                      int64_t *out_ticket);

/* n_chunks consecutive chunks of one stream in one call, the same as
 * n_chunks pfb_submit calls in order: chunk i is samples_per_chunk samples
 * (a multiple of P) at d_chunks + i * samples_per_chunk samples; its spectra
 * go to d_out right after those of chunks 0..i-1 (out_cap_spectra rows in
 * all).  out_tickets receives n_chunks tickets.  On an error the chunks
 * before the failing one stay submitted (their tickets are set, the rest are
 * 0) and the error is returned. */
PFB_API pfb_status pfb_submit_chunks(pfb_server_t server, int64_t stream_id, const void *d_chunks, int32_t n_chunks,
                                     int64_t samples_per_chunk, void *d_out, int64_t out_cap_spectra,
                                     int64_t *out_tickets);

/* The server's timestamps of a ticket, in seconds of the library's steady
 * clock (CLOCK_MONOTONIC on Linux): when pfb_submit accepted it and when the
 * server saw it finish (its batch's completion event, polled every few
 * microseconds by the server thread); *t_done_s = 0 while it is pending. */
PFB_API pfb_status pfb_ticket_times(pfb_server_t server, int64_t ticket, double *t_submit_s, double *t_done_s);

/* PFB_PENDING while queued or running, PFB_OK once the output is complete,
 * or the request's error.  Never blocks.  A finished ticket can be polled
 * until pfb_server_destroy. */
PFB_API pfb_status pfb_poll(pfb_server_t server, int64_t ticket);

/* Block until the ticket finishes or timeout_ms passes (PFB_ERR_TIMEOUT). */
PFB_API pfb_status pfb_wait(pfb_server_t server, int64_t ticket, int32_t timeout_ms);

PFB_API pfb_status pfb_server_get_stats(pfb_server_t server, pfb_server_stats *out_stats);

/* Checkpoint of a stream's filter state (the last T-1 frames of raw input
 * that the per-branch FIR of Sec. 5.2 carries from one chunk to the next).
 * The blob is a 48-byte header (magic "PFBSTATE", version 1, P, T, dtype,
 * frames taken so far, frames stored) followed by min(T-1, frames taken)
 * frames of raw input in the plan's dtype.
 * pfb_stream_state_size: bytes of the blob once the chunks submitted so far
 * have run (-1 for an unknown stream).
 * pfb_stream_state_export: waits (bounded by the server's timeout_ms) until
 * the stream has no chunk queued or in flight, then copies the blob to
 * host_buf (cap bytes available).  Errors: PFB_ERR_INVALID (unknown stream,
 * cap too small, an earlier chunk failed), PFB_ERR_TIMEOUT, PFB_ERR_CUDA.
 * pfb_stream_state_import: loads a blob into an open, idle stream of a plan
 * with the same P, T and dtype; its next chunk then continues the exporting
 * stream: the spectra equal those of an uninterrupted stream bit for bit.
 * Errors: PFB_ERR_INVALID (not a blob, other P/T/dtype, truncated), as above
 * otherwise. */
PFB_API int64_t pfb_stream_state_size(pfb_server_t server, int64_t stream_id);
PFB_API pfb_status pfb_stream_state_export(pfb_server_t server, int64_t stream_id, void *host_buf, int64_t cap);
PFB_API pfb_status pfb_stream_state_import(pfb_server_t server, int64_t stream_id, const void *host_buf,
                                           int64_t size);

/* ---------------------------------------------------------------------- */
/* Diagnostics                                                            */
/* ---------------------------------------------------------------------- */

PFB_API const char *pfb_status_string(pfb_status status);
/* Message for the calling thread's most recent failed call ("" if none). */
PFB_API const char *pfb_last_error(void);
/* Number of kernel launches this library has issued so far (all threads). */
PFB_API int64_t pfb_launch_count(void);
/* Name of the kernel variant pfb_execute uses for a plan ("" for NULL). */
PFB_API const char *pfb_plan_kernel_name(pfb_plan_t plan);

#ifdef __cplusplus
}
#endif

#endif /* PFB_H_ */
