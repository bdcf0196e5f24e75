// Internal declarations shared by the translation units of libpfb.
// Not part of the public ABI (include/pfb.h is).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/pfb.h"

namespace pfb {

// ---------------------------------------------------------------------------
// error reporting
// ---------------------------------------------------------------------------
void set_error(const std::string &msg);
void clear_error();
pfb_status fail(pfb_status st, const std::string &msg);
pfb_status cuda_fail(cudaError_t e, const char *what);
extern std::atomic<int64_t> g_launches;

#define PFB_CUDA_TRY(expr)                                           \
    do {                                                             \
        cudaError_t _e = (expr);                                     \
        if (_e != cudaSuccess) return ::pfb::cuda_fail(_e, #expr);   \
    } while (0)

// Device-side error word values (written by kernels, read by the host).
enum : int {
    KERR_NONE = 0,
    KERR_BOUNDS = 1,     // a work index fell outside its descriptor table
    KERR_TIMEOUT = 2,    // a bounded device-side wait ran out
    KERR_CONFIG = 3,     // kernel launched with a configuration it does not support
};

// ---------------------------------------------------------------------------
// per-stream work descriptor (one stream = one contiguous run of frames)
//
// The frames of a stream are the n_state frames of `state` followed by the
// frames of `in`; spectra s = 0 .. S-1 use frames s .. s+T-1 of that sequence.
// ---------------------------------------------------------------------------
struct StreamDesc {
    const void *in;        // input samples (raw dtype)
    const void *state;     // resident state frames (raw dtype) or nullptr
    float2 *out;           // output spectra [S][P] complex64
    int64_t n_state;       // frames taken from `state` (precede `in`)
    int64_t n_frames;      // total frames available (state + in)
    int64_t S;             // spectra to produce
    int64_t unit0;         // index of this stream's first work unit in the launch
    int64_t ldo;           // output row stride in complex64 elements (P; R*P for hop P/R)
    const float *taps;     // fp32 taps, layout depends on the kernel family
    float scale;           // dequantisation factor (CI8)
    int32_t T;             // taps per branch
};

constexpr int kMaxStreamsPerLaunch = 64;
constexpr int kMaxOversampling = 32;          // most spectra per frame (P / hop)
constexpr uint64_t kDefaultWaitNs = 1000000000ull;  // bound of every device-side wait

// Fault modes of the error-reporting test hook (pfb_plan_set_fault).
enum : int32_t {
    FAULT_NONE = 0,
    FAULT_NO_COPIES = 1,  // the producer issues no input copies: every consumer wait runs out
};

struct LaunchArgs {
    StreamDesc s[kMaxStreamsPerLaunch];
    int32_t nstreams;
    int32_t units_per_cta;  // contiguous work units per CTA (persistent ranges)
    int64_t nunits;         // total work units in this launch
    const float2 *tw;       // FFT twiddle table for the family's P
    const void *aux;        // family-specific table (DFT matrix for GEMM paths)
    int *err;               // error word (host-mapped memory): KERR_* of a failed launch
    uint64_t wait_ns;       // bound of the kernel's device-side waits (%globaltimer ns)
    int32_t fault;          // FAULT_* test hook (0 in normal use)
    int32_t pad_;
};

// ---------------------------------------------------------------------------
// plan
// ---------------------------------------------------------------------------
enum KernelFamily : int {
    FAM_FFT_FAST = 0,     // fused FIR + radix-16 Stockham FFT, P in [64,1024], T <= 16
    FAM_FFT_GENERIC = 1,  // fused FIR + radix-2 Stockham FFT, any supported P, T
    FAM_GEMM_F32 = 2,     // fused FIR + DFT-matrix product, FP32 SIMT
    FAM_GEMM_BF16X3 = 3,  // fused FIR + DFT-matrix product, tcgen05 split-bf16
    FAM_FFT_CLUSTER = 4,  // fused FIR + four-step FFT across a CTA cluster, P in {2048, 4096}
};

constexpr int kPipeChunks = 32;  // most chunks of one pfb_execute_host pipeline

struct Plan {
    pfb_plan_desc desc;
    int device = 0;
    int P = 0, T = 0, TT = 0;       // TT: tap count the kernel is compiled for (>= T)
    int in_dtype = 0;
    int path = 0;
    int family = 0;
    int esize = 0;                  // bytes per input sample
    int variant = 0;                // kernel variant (tile shape) within the family
    int hop = 0;                    // samples between spectra (P = critically sampled)
    int R = 1;                      // P / hop: spectra per frame (oversampling factor)
    // device tables (owned)
    double *d_h64 = nullptr;        // FP64 prototype [P*T]
    float *d_taps = nullptr;        // fp32 taps [T][P]
    float *d_taps_pad = nullptr;    // fp32 taps zero-extended to [TT][P] (rows T..TT-1 zero)
    float2 *d_tw = nullptr;         // FFT twiddles (layout per family; radix-16 pass list)
    float2 *d_tw32 = nullptr;       // radix-32 pass list twiddles (fast FFT family)
    float2 *d_tw_r2 = nullptr;      // radix-2 table w^r, r < P/2 (generic family)
    void *d_dft = nullptr;          // DFT matrix (GEMM families)
    void *d_tcf = nullptr;          // factored split-bf16 DFT: 32-point matrix hi/lo + twiddles
    size_t dft_bytes = 0;
    int *h_err = nullptr;           // error word in mapped, pinned host memory (written by kernels)
    int *d_err = nullptr;           // its device address
    uint64_t wait_ns = kDefaultWaitNs;  // device-side wait bound of the plan's launches
    int32_t fault = 0;              // FAULT_* test hook
    // synthesis routes other than the fused kernel: the inverse-DFT buffer
    // y~ [S][P] and (split-bf16 plans) the internal one-tap inverse plan
    void *d_synth_y = nullptr;
    size_t synth_y_bytes = 0;
    // the two-pass DFT-matrix products (split-bf16 variant 2, FP32 GEMM for P a
    // multiple of 128): the branch sums between the passes, grown on demand;
    // a buffer it outgrows is kept until the plan is destroyed, because a CUDA
    // graph captured earlier may still use it
    mutable void *d_ws2 = nullptr;
    mutable size_t ws2_bytes = 0;
    mutable std::vector<void *> ws2_retired;
    // guards the workspace alone: pfb_execute_host launches while it holds
    // stage_mu, and a launch may grow the workspace
    mutable std::mutex ws2_mu;
    Plan *inv = nullptr;
    // host staging for pfb_execute_host
    std::mutex stage_mu;
    void *d_stage_in = nullptr, *d_stage_out = nullptr;
    size_t stage_in_bytes = 0, stage_out_bytes = 0;
    // host-buffer pipeline: copy-in and copy-out streams, per-chunk events
    cudaStream_t s_copy_in = nullptr, s_copy_out = nullptr;
    cudaEvent_t ev_pipe[2 * kPipeChunks + 2] = {};
    std::string kernel_name;
};

int64_t out_spectra(const Plan &p, int64_t n_samples);
// Descriptors of one stream of the plan: one, or R = P/hop interleaved
// critically sampled ones for an oversampled plan (input shifted by j*hop,
// output rows j, j+R, ...).  Validates the buffers; returns the count in *n.
pfb_status make_stream_descs(const Plan &plan, const void *d_in, int64_t n_samples, void *d_out, int64_t out_cap,
                             StreamDesc *descs, int *n);
bool is_pow2(int64_t v);
int ilog2(int64_t v);

// Launch one kernel of the plan's family over the given streams (all with
// the plan's P, T, dtype).  `descs` unit0 fields are filled in here.  The
// kernels report failures into `err` (device address of a host-mapped word;
// nullptr = the plan's own word).
pfb_status launch_family(const Plan &plan, StreamDesc *descs, int n, cudaStream_t stream, int *err = nullptr);

// Read and clear a host-mapped error word: PFB_OK, or the status a kernel's
// KERR_* code maps to (KERR_TIMEOUT -> PFB_ERR_TIMEOUT, others ->
// PFB_ERR_INTERNAL), with the message set.
pfb_status take_kernel_error(int *h_err, const char *what);

// Resolve (and cache) the device address of the static staging area of
// pfb_execute_host_noalloc on `device` (current); loads its module there.
pfb_status noalloc_prepare(int device);

// Mapped, pinned host words the kernels write their error codes to.
pfb_status alloc_error_words(int n, int **h_err, int **d_err);
void free_error_words(int *h_err);

// Family-specific launchers (defined in their .cu files).
pfb_status launch_fft_fast(const Plan &plan, LaunchArgs &args, cudaStream_t stream);
pfb_status launch_fft_generic(const Plan &plan, LaunchArgs &args, cudaStream_t stream);
pfb_status launch_gemm_f32(const Plan &plan, LaunchArgs &args, cudaStream_t stream);
size_t gemm_f32_workspace_bytes(const Plan &plan, int64_t nunits);   // 0: no workspace
size_t gemm2p_workspace_bytes(const Plan &plan, int64_t nunits);
// bytes of the plan-owned workspace (d_ws2) one launch of nunits work units needs (0: none)
size_t family_workspace_bytes(const Plan &plan, int64_t nunits);
// grow the plan's workspace to at least `bytes` (kept; PFB_ERR_OOM if it cannot;
// PFB_ERR_UNSUPPORTED if it would have to grow while `stream` is capturing)
pfb_status grow_plan_workspace(const Plan &plan, size_t bytes, cudaStream_t stream);
void free_plan_workspaces(Plan &plan);
pfb_status launch_gemm_bf16x3(const Plan &plan, LaunchArgs &args, cudaStream_t stream);
pfb_status launch_gemm_bf16x3_2p(const Plan &plan, LaunchArgs &args, cudaStream_t stream);  // variant 2
int64_t gemm2p_units(const Plan &plan, int64_t S);
bool gemm2p_supported(const Plan &plan);
pfb_status launch_gemm_bf16x3_tcf(const Plan &plan, LaunchArgs &args, cudaStream_t stream);
bool tcf_supported(const Plan &plan);
pfb_status build_tcf_table(Plan &plan);
pfb_status launch_fft_cluster(const Plan &plan, LaunchArgs &args, cudaStream_t stream);
bool fft_cluster_supported(int P, int T);
bool ws_cluster_supported(const Plan &plan);   // variant 1 of the cluster family
bool wcf_supported(const Plan &plan);          // variant 3 of the cluster family (P = 4096)
pfb_status prepare_family(const Plan &plan);
pfb_status ensure_variant_tables(Plan &plan);
const float *family_taps(const Plan &plan);   // tap layout the family's kernels read
// work units a stream of S spectra contributes to a launch of the plan's family
int64_t family_units(const Plan &plan, int64_t S);
bool fft_fast_supported(int P, int T);
int fft_fast_tt(int T);
int family_variants(const Plan &plan);        // number of variants the autotuner may pick from
int default_variant(const Plan &plan);

// Synthesis routes (synth_generic.cu): any P, T, path at hop P
bool synth_generic_supported(const Plan &p);
pfb_status launch_synth_generic(Plan &p, const float2 *X, int64_t S, float2 *xh, cudaStream_t stream);
void free_inverse_plan(Plan &p);

// Table generators (plan.cu)
pfb_status build_fft_fast_twiddles(Plan &plan);
pfb_status build_gemm_tables(Plan &plan);

// stream-state update for serving: new_state = last n_keep frames of (state ++ chunk)
pfb_status launch_state_update(const void *old_state, int64_t old_frames, const void *chunk,
                               int64_t chunk_frames, void *new_state, int64_t n_keep,
                               int64_t frame_bytes, cudaStream_t stream);

}  // namespace pfb
