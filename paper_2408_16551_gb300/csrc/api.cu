// Host side of the C ABI: status strings, error messages, pfb_execute,
// pfb_execute_host and the batched entry points (work grouping, CUDA graphs).
#include <algorithm>
#include <atomic>
#include <mutex>
#include <vector>
#include <cstring>
#include <map>
#include <new>
#include <tuple>

#include "internal.h"

namespace pfb {

std::atomic<int64_t> g_launches{0};
static thread_local std::string t_err;

void set_error(const std::string &msg) { t_err = msg; }
void clear_error() { t_err.clear(); }
pfb_status fail(pfb_status st, const std::string &msg) {
    t_err = msg;
    return st;
}
pfb_status cuda_fail(cudaError_t e, const char *what) {
    t_err = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    return PFB_ERR_CUDA;
}

int64_t generic_units(int P, int64_t S);
int64_t fast_units(const Plan &plan, int64_t S);
int64_t gemm_f32_units(const Plan &plan, int64_t S);
int64_t gemm_bf16x3_units(const Plan &plan, int64_t S);
int64_t fft_cluster_units(const Plan &plan, int64_t S);

int64_t family_units(const Plan &plan, int64_t S) {
    switch (plan.family) {
    case FAM_FFT_FAST: return fast_units(plan, S);
    case FAM_FFT_GENERIC: return generic_units(plan.P, S);
    case FAM_GEMM_F32: return gemm_f32_units(plan, S);
    case FAM_GEMM_BF16X3: return gemm_bf16x3_units(plan, S);
    case FAM_FFT_CLUSTER: return fft_cluster_units(plan, S);
    default: return 0;
    }
}

size_t family_workspace_bytes(const Plan &plan, int64_t nunits) {
    if (plan.family == FAM_GEMM_F32) return gemm_f32_workspace_bytes(plan, nunits);
    if (plan.family == FAM_GEMM_BF16X3 && plan.variant == 2) return gemm2p_workspace_bytes(plan, nunits);
    return 0;
}

const float *family_taps(const Plan &plan) { return plan.d_taps_pad ? plan.d_taps_pad : plan.d_taps; }

pfb_status alloc_error_words(int n, int **h_err, int **d_err) {
    *h_err = nullptr;
    *d_err = nullptr;
    void *h = nullptr;
    cudaError_t e = cudaHostAlloc(&h, sizeof(int) * (size_t)n, cudaHostAllocMapped | cudaHostAllocPortable);
    if (e != cudaSuccess) return cuda_fail(e, "cudaHostAlloc (error words)");
    std::memset(h, 0, sizeof(int) * (size_t)n);
    void *d = nullptr;
    e = cudaHostGetDevicePointer(&d, h, 0);
    if (e != cudaSuccess) {
        cudaFreeHost(h);
        return cuda_fail(e, "cudaHostGetDevicePointer (error words)");
    }
    *h_err = static_cast<int *>(h);
    *d_err = static_cast<int *>(d);
    return PFB_OK;
}

void free_error_words(int *h_err) {
    if (h_err) cudaFreeHost(h_err);
}

pfb_status take_kernel_error(int *h_err, const char *what) {
    if (!h_err) return PFB_OK;
    volatile int *w = h_err;
    const int v = *w;
    if (v == KERR_NONE) return PFB_OK;
    *w = KERR_NONE;
    if (v == KERR_TIMEOUT)
        return fail(PFB_ERR_TIMEOUT, std::string(what) + ": a device-side wait of the kernel ran out (error word)");
    return fail(PFB_ERR_INTERNAL, std::string(what) + ": the kernel reported error code " + std::to_string(v));
}

// Launch the plan's family kernel over n stream descriptors (all of this
// family/P/T/dtype), in groups of kMaxStreamsPerLaunch.
pfb_status launch_family(const Plan &plan, StreamDesc *descs, int n, cudaStream_t stream, int *err) {
    for (int g0 = 0; g0 < n; g0 += kMaxStreamsPerLaunch) {
        const int g1 = std::min(n, g0 + kMaxStreamsPerLaunch);
        LaunchArgs a;
        std::memset(&a, 0, sizeof(a));
        int64_t units = 0;
        int k = 0;
        for (int i = g0; i < g1; ++i) {
            if (descs[i].S <= 0) continue;
            a.s[k] = descs[i];
            a.s[k].unit0 = units;
            units += family_units(plan, descs[i].S);
            ++k;
        }
        if (k == 0) continue;
        a.nstreams = k;
        a.nunits = units;
        a.tw = plan.d_tw;
        a.aux = plan.d_dft;
        a.err = err ? err : plan.d_err;
        a.wait_ns = plan.wait_ns;
        a.fault = plan.fault;
        pfb_status st;
        switch (plan.family) {
        case FAM_FFT_FAST: st = launch_fft_fast(plan, a, stream); break;
        case FAM_FFT_GENERIC: st = launch_fft_generic(plan, a, stream); break;
        case FAM_GEMM_F32: st = launch_gemm_f32(plan, a, stream); break;
        case FAM_GEMM_BF16X3: st = launch_gemm_bf16x3(plan, a, stream); break;
        case FAM_FFT_CLUSTER: st = launch_fft_cluster(plan, a, stream); break;
        default: st = fail(PFB_ERR_INTERNAL, "unknown kernel family");
        }
        if (st != PFB_OK) return st;
    }
    return PFB_OK;
}

// Set kernel attributes and occupancy caches for the plan's variant outside
// any stream capture (the launchers do it on first use).
pfb_status prepare_family(const Plan &plan) {
    LaunchArgs a;
    std::memset(&a, 0, sizeof(a));
    a.wait_ns = kDefaultWaitNs;
    switch (plan.family) {
    case FAM_FFT_FAST: return launch_fft_fast(plan, a, nullptr);
    case FAM_FFT_GENERIC: return launch_fft_generic(plan, a, nullptr);
    case FAM_GEMM_F32: return launch_gemm_f32(plan, a, nullptr);
    case FAM_GEMM_BF16X3: return launch_gemm_bf16x3(plan, a, nullptr);
    case FAM_FFT_CLUSTER: return launch_fft_cluster(plan, a, nullptr);
    default: return PFB_OK;
    }
}

static bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// Fill a descriptor for a plain (stateless) stream; validates the arguments.
static pfb_status make_desc(const Plan &plan, const void *d_in, int64_t n_samples, void *d_out,
                            int64_t out_cap, StreamDesc &d) {
    if (n_samples < 0) return fail(PFB_ERR_INVALID, "n_samples < 0");
    const int64_t S = out_spectra(plan, n_samples);
    std::memset(&d, 0, sizeof(d));
    d.S = S;
    if (S == 0) return PFB_OK;
    if (!d_in || !d_out) return fail(PFB_ERR_INVALID, "NULL buffer with S > 0");
    if (!aligned16(d_in) || !aligned16(d_out)) return fail(PFB_ERR_INVALID, "buffers must be 16-byte aligned");
    if (out_cap < S) return fail(PFB_ERR_INVALID, "out_cap_spectra smaller than the spectra produced");
    d.in = d_in;
    d.state = nullptr;
    d.out = static_cast<float2 *>(d_out);
    d.n_state = 0;
    d.n_frames = n_samples / plan.P;
    d.ldo = plan.P;
    d.taps = family_taps(plan);
    d.scale = plan.desc.in_scale;
    d.T = plan.T;
    return PFB_OK;
}

}  // namespace pfb

pfb_status pfb::make_stream_descs(const Plan &plan, const void *d_in, int64_t n_samples, void *d_out, int64_t out_cap,
                                  StreamDesc *descs, int *n) {
    *n = 0;
    if (plan.R <= 1) {
        pfb_status st = make_desc(plan, d_in, n_samples, d_out, out_cap, descs[0]);
        if (st == PFB_OK && descs[0].S > 0) *n = 1;
        return st;
    }
    // oversampled: spectrum s = R s' + j is spectrum s' of the critically
    // sampled PFB of the input shifted by j*hop samples (the window of spectrum
    // s starts at s*hop = s'*P + j*hop), written to output row s
    if (n_samples < 0) return fail(PFB_ERR_INVALID, "n_samples < 0");
    const int64_t S = out_spectra(plan, n_samples);
    if (S == 0) return PFB_OK;
    if (!d_in || !d_out) return fail(PFB_ERR_INVALID, "NULL buffer with S > 0");
    if (!aligned16(d_in) || !aligned16(d_out)) return fail(PFB_ERR_INVALID, "buffers must be 16-byte aligned");
    if (out_cap < S) return fail(PFB_ERR_INVALID, "out_cap_spectra smaller than the spectra produced");
    int64_t total = 0;
    for (int j = 0; j < plan.R; ++j) {
        const int64_t nj = n_samples - (int64_t)j * plan.hop;
        StreamDesc &d = descs[*n];
        std::memset(&d, 0, sizeof(d));
        d.S = nj > 0 ? std::max<int64_t>(0, nj / plan.P - plan.T + 1) : 0;
        if (d.S == 0) continue;
        d.in = static_cast<const char *>(d_in) + (int64_t)j * plan.hop * plan.esize;
        d.out = static_cast<float2 *>(d_out) + (int64_t)j * plan.P;
        d.ldo = (int64_t)plan.R * plan.P;
        d.n_frames = nj / plan.P;
        d.taps = family_taps(plan);
        d.scale = plan.desc.in_scale;
        d.T = plan.T;
        total += d.S;
        ++*n;
    }
    if (total != S) return fail(PFB_ERR_INTERNAL, "oversampled spectra count mismatch");
    return PFB_OK;
}

namespace pfb {

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
        else prev = -1;
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

}  // namespace pfb

using namespace pfb;

extern "C" const char *pfb_status_string(pfb_status s) {
    switch (s) {
    case PFB_OK: return "PFB_OK";
    case PFB_PENDING: return "PFB_PENDING";
    case PFB_ERR_INVALID: return "PFB_ERR_INVALID";
    case PFB_ERR_OOM: return "PFB_ERR_OOM";
    case PFB_ERR_CUDA: return "PFB_ERR_CUDA";
    case PFB_ERR_BUSY: return "PFB_ERR_BUSY";
    case PFB_ERR_TIMEOUT: return "PFB_ERR_TIMEOUT";
    case PFB_ERR_INTERNAL: return "PFB_ERR_INTERNAL";
    case PFB_ERR_UNSUPPORTED: return "PFB_ERR_UNSUPPORTED";
    default: return "PFB_UNKNOWN_STATUS";
    }
}

extern "C" const char *pfb_last_error(void) { return t_err.c_str(); }

extern "C" pfb_status pfb_plan_status(pfb_plan_t plan) {
    clear_error();
    if (!plan) return fail(PFB_ERR_INVALID, "plan is NULL");
    return take_kernel_error(reinterpret_cast<Plan *>(plan)->h_err, "pfb_plan_status");
}

extern "C" pfb_status pfb_plan_set_fault(pfb_plan_t plan, int32_t mode, int64_t wait_ns) {
    clear_error();
    if (!plan) return fail(PFB_ERR_INVALID, "plan is NULL");
    if (mode != FAULT_NONE && mode != FAULT_NO_COPIES) return fail(PFB_ERR_INVALID, "unknown fault mode");
    if (wait_ns < 0 || wait_ns > 4ll * (int64_t)kDefaultWaitNs) return fail(PFB_ERR_INVALID, "wait_ns outside [0, 4 s]");
    Plan &p = *reinterpret_cast<Plan *>(plan);
    p.fault = mode;
    p.wait_ns = wait_ns == 0 ? kDefaultWaitNs : (uint64_t)wait_ns;
    return PFB_OK;
}
extern "C" int64_t pfb_launch_count(void) { return g_launches.load(); }

extern "C" pfb_status pfb_execute(pfb_plan_t plan, const void *d_in, int64_t n_samples, void *d_out,
                                  int64_t out_cap_spectra, void *cuda_stream) {
    clear_error();
    if (!plan) return fail(PFB_ERR_INVALID, "plan is NULL");
    const Plan &p = *reinterpret_cast<Plan *>(plan);
    StreamDesc d[kMaxStreamsPerLaunch];
    int nd = 0;
    pfb_status st = make_stream_descs(p, d_in, n_samples, d_out, out_cap_spectra, d, &nd);
    if (st != PFB_OK || nd == 0) return st;
    DeviceGuard g(p.device);
    return launch_family(p, d, nd, static_cast<cudaStream_t>(cuda_stream));
}

namespace pfb {

// Route of the host-buffer calls (PFB_HOST_ROUTE_*), and the route the
// calling thread's last one took (0 none, 1 staged, 2 mapped).
static std::atomic<int> g_host_route{PFB_HOST_ROUTE_AUTO};
static thread_local int t_last_host_route = 0;

// True when the kernel the plan launches touches the caller's input and
// spectra only with per-thread accesses (16-byte cp.async reads, plain
// stores): the four-step cluster kernel.  Kernels that move the caller's
// buffers with bulk copies, or read each input frame more than once from
// memory, stay on the staged route.  (A per-thread copy producer for the
// warp-specialised single-CTA kernel measured 3 % slower than staging on a
// 2^24-sample stream at P = 1024, so it has none.)
static bool takes_mapped_buffers(const Plan &p) { return p.family == FAM_FFT_CLUSTER && p.variant == 3 && p.R == 1; }

// The device address of the host range [ptr, ptr + bytes) when both its ends
// are page-locked host memory mapped into the current device's address
// space (cudaHostAlloc, cudaMallocHost, cudaHostRegister under unified
// addressing), else nullptr.  Pageable memory gives nullptr.
static const char *mapped_host_range(const void *ptr, size_t bytes) {
    cudaPointerAttributes a{}, b{};
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (a.type != cudaMemoryTypeHost || !a.devicePointer) return nullptr;
    const char *dev = static_cast<const char *>(a.devicePointer);
    if (bytes > 1) {
        if (cudaPointerGetAttributes(&b, static_cast<const char *>(ptr) + bytes - 1) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        if (b.type != cudaMemoryTypeHost || static_cast<const char *>(b.devicePointer) != dev + bytes - 1) return nullptr;
    }
    return dev;
}

}  // namespace pfb

extern "C" pfb_status pfb_execute_host(pfb_plan_t plan, const void *host_in, int64_t n_samples, void *host_out,
                                       int64_t out_cap_spectra, void *cuda_stream) {
    clear_error();
    if (!plan) return fail(PFB_ERR_INVALID, "plan is NULL");
    Plan &p = *reinterpret_cast<Plan *>(plan);
    if (p.R > 1) return fail(PFB_ERR_UNSUPPORTED, "pfb_execute_host: oversampled plans (hop < P) run through pfb_execute");
    if (n_samples < 0) return fail(PFB_ERR_INVALID, "n_samples < 0");
    const int64_t S = out_spectra(p, n_samples);
    if (S == 0) return PFB_OK;
    if (!host_in || !host_out) return fail(PFB_ERR_INVALID, "NULL buffer with S > 0");
    if (out_cap_spectra < S) return fail(PFB_ERR_INVALID, "out_cap_spectra smaller than the spectra produced");
    const size_t in_bytes = (size_t)n_samples * p.esize;
    const size_t out_bytes = (size_t)S * p.P * sizeof(float2);
    t_last_host_route = 0;
    // Mapped route (as in pfb_execute_batch_host): page-locked, mapped,
    // 16-byte aligned buffers and a kernel that takes them; it reads the
    // input and writes the spectra in host memory, then the stream drains.
    if (g_host_route.load() == PFB_HOST_ROUTE_AUTO && takes_mapped_buffers(p)) {
        DeviceGuard g(p.device);
        const int64_t fr = (n_samples / p.P) * p.P;  // whole frames only
        const char *di = mapped_host_range(host_in, (size_t)fr * p.esize);
        const char *dq = di ? mapped_host_range(host_out, out_bytes) : nullptr;
        if (di && dq && aligned16(di) && aligned16(dq)) {
            t_last_host_route = 2;
            cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
            StreamDesc d[kMaxStreamsPerLaunch];
            int nd = 0;
            pfb_status st = make_stream_descs(p, di, fr, const_cast<char *>(dq), S, d, &nd);
            if (st == PFB_OK && nd > 0) st = launch_family(p, d, nd, s);
            cudaError_t e = cudaStreamSynchronize(s);
            if (st != PFB_OK) return st;
            if (e != cudaSuccess) return cuda_fail(e, "pfb_execute_host kernels (mapped)");
            return take_kernel_error(p.h_err, "pfb_execute_host");
        }
    }
    t_last_host_route = 1;
    std::lock_guard<std::mutex> lk(p.stage_mu);
    DeviceGuard g(p.device);
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    if (p.stage_in_bytes < in_bytes) {
        cudaFree(p.d_stage_in);
        p.d_stage_in = nullptr;
        p.stage_in_bytes = 0;
        if (cudaMalloc(&p.d_stage_in, in_bytes) != cudaSuccess) return fail(PFB_ERR_OOM, "staging input");
        p.stage_in_bytes = in_bytes;
    }
    if (p.stage_out_bytes < out_bytes) {
        cudaFree(p.d_stage_out);
        p.d_stage_out = nullptr;
        p.stage_out_bytes = 0;
        if (cudaMalloc(&p.d_stage_out, out_bytes) != cudaSuccess) return fail(PFB_ERR_OOM, "staging output");
        p.stage_out_bytes = out_bytes;
    }
    // Pipeline over spectrum chunks: chunk c's new input frames go up on the
    // copy-in stream, its kernel runs on the caller's stream, its spectra come
    // back on the copy-out stream, so both copy directions and the kernels
    // overlap.  Chunk c reads frames [s_a, s_b + T - 1); the T - 1 frames it
    // shares with chunk c + 1 are copied once.
    // 16 MB chunks measured best on c2 (4 and 8 MB: more per-chunk overhead)
    constexpr int64_t kChunkBytes = 16ll << 20;
    constexpr int kMaxChunks = kPipeChunks;
    const int64_t fbytes = (int64_t)p.P * p.esize;
    int nch = (int)std::min<int64_t>(kMaxChunks, std::max<int64_t>(1, (int64_t)in_bytes / kChunkBytes));
    nch = (int)std::min<int64_t>(nch, S);
    if (!p.s_copy_in) {
        PFB_CUDA_TRY(cudaStreamCreateWithFlags(&p.s_copy_in, cudaStreamNonBlocking));
        PFB_CUDA_TRY(cudaStreamCreateWithFlags(&p.s_copy_out, cudaStreamNonBlocking));
        for (cudaEvent_t &e : p.ev_pipe) PFB_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    }
    cudaEvent_t *ev_in = p.ev_pipe, *ev_k = p.ev_pipe + kMaxChunks;
    cudaEvent_t ev_start = p.ev_pipe[2 * kMaxChunks], ev_done = p.ev_pipe[2 * kMaxChunks + 1];
    // copies start after the caller's earlier work on s
    PFB_CUDA_TRY(cudaEventRecord(ev_start, s));
    PFB_CUDA_TRY(cudaStreamWaitEvent(p.s_copy_in, ev_start, 0));
    PFB_CUDA_TRY(cudaStreamWaitEvent(p.s_copy_out, ev_start, 0));
    const char *hin = static_cast<const char *>(host_in);
    char *hout = static_cast<char *>(host_out);
    char *din = static_cast<char *>(p.d_stage_in);
    float2 *dout = static_cast<float2 *>(p.d_stage_out);
    int64_t copied = 0;  // input bytes already on the device
    for (int c = 0; c < nch; ++c) {
        const int64_t sa = S * c / nch, sb = S * (c + 1) / nch;
        const int64_t need = (c == nch - 1) ? (int64_t)in_bytes : (sb + p.T - 1) * fbytes;
        if (need > copied)
            PFB_CUDA_TRY(cudaMemcpyAsync(din + copied, hin + copied, need - copied, cudaMemcpyHostToDevice,
                                         p.s_copy_in));
        copied = std::max(copied, need);
        PFB_CUDA_TRY(cudaEventRecord(ev_in[c], p.s_copy_in));
        PFB_CUDA_TRY(cudaStreamWaitEvent(s, ev_in[c], 0));
        StreamDesc d;
        pfb_status st = make_desc(p, din + sa * fbytes, need / p.esize - sa * p.P, dout + sa * p.P, sb - sa, d);
        if (st == PFB_OK) st = launch_family(p, &d, 1, s);
        if (st != PFB_OK) {  // nothing may still be writing host_out when the call returns
            cudaStreamSynchronize(p.s_copy_in);
            cudaStreamSynchronize(s);
            cudaStreamSynchronize(p.s_copy_out);
            return st;
        }
        PFB_CUDA_TRY(cudaEventRecord(ev_k[c], s));
        PFB_CUDA_TRY(cudaStreamWaitEvent(p.s_copy_out, ev_k[c], 0));
        PFB_CUDA_TRY(cudaMemcpyAsync(hout + sa * p.P * sizeof(float2), dout + sa * p.P,
                                     (size_t)(sb - sa) * p.P * sizeof(float2), cudaMemcpyDeviceToHost,
                                     p.s_copy_out));
    }
    PFB_CUDA_TRY(cudaEventRecord(ev_done, p.s_copy_out));
    PFB_CUDA_TRY(cudaStreamWaitEvent(s, ev_done, 0));
    PFB_CUDA_TRY(cudaStreamSynchronize(s));
    return take_kernel_error(p.h_err, "pfb_execute_host");
}

// ---------------------------------------------------------------------------
// batches: group streams by kernel variant, one persistent launch per group
// ---------------------------------------------------------------------------
namespace pfb {

struct Group {
    const Plan *plan;  // representative (P, T, dtype, family, tables of this shape)
    std::vector<StreamDesc> descs;
};

static pfb_status build_groups(const pfb_batch_item *items, int32_t n, std::vector<Group> &groups, int &device) {
    if (n < 0 || (n > 0 && !items)) return fail(PFB_ERR_INVALID, "bad item list");
    std::map<std::tuple<int, int, int, int, int, int>, size_t> index;
    device = -1;
    for (int i = 0; i < n; ++i) {
        const pfb_batch_item &it = items[i];
        if (!it.plan) return fail(PFB_ERR_INVALID, "item with NULL plan");
        const Plan &p = *reinterpret_cast<Plan *>(it.plan);
        if (device < 0) device = p.device;
        if (p.device != device) return fail(PFB_ERR_INVALID, "batch items span devices");
        StreamDesc d[kMaxStreamsPerLaunch];
        int nd = 0;
        pfb_status st = make_stream_descs(p, it.d_in, it.n_samples, it.d_out, it.out_cap_spectra, d, &nd);
        if (st != PFB_OK) return fail(st, "item " + std::to_string(i) + ": " + pfb_last_error());
        if (nd == 0) continue;
        // streams share a launch when the kernel variant is the same; taps are
        // per stream (descriptor), twiddles/DFT tables depend only on P
        auto key = std::make_tuple(p.family, p.P, p.TT, p.in_dtype, p.variant, p.R);
        auto f = index.find(key);
        if (f == index.end()) {
            index[key] = groups.size();
            groups.push_back(Group{&p, {}});
            f = index.find(key);
        }
        for (int k = 0; k < nd; ++k) groups[f->second].descs.push_back(d[k]);
    }
    return PFB_OK;
}

struct Batch {
    int device = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

}  // namespace pfb

extern "C" pfb_status pfb_execute_batch(const pfb_batch_item *items, int32_t n_items, void *cuda_stream) {
    clear_error();
    std::vector<Group> groups;
    int device = -1;
    pfb_status st = build_groups(items, n_items, groups, device);
    if (st != PFB_OK || groups.empty()) return st;
    DeviceGuard g(device);
    for (auto &gr : groups) {
        st = launch_family(*gr.plan, gr.descs.data(), (int)gr.descs.size(), static_cast<cudaStream_t>(cuda_stream));
        if (st != PFB_OK) return st;
    }
    return PFB_OK;
}

// ---------------------------------------------------------------------------
// pfb_execute_batch_host: a batch from and to host memory, pipelined
// ---------------------------------------------------------------------------
namespace pfb {

// Per-device staging for host batches: kHostSlots chunk slots (input and
// output areas), a copy-in and a copy-out stream, per-slot events.
struct HostBatchCtx {
    static constexpr int kHostSlots = 3;
    std::mutex mu;
    bool ready = false;
    void *d_in[kHostSlots] = {}, *d_out[kHostSlots] = {};
    size_t in_cap[kHostSlots] = {}, out_cap[kHostSlots] = {};
    cudaStream_t s_in = nullptr, s_out = nullptr;
    cudaEvent_t ev_in[kHostSlots] = {}, ev_k[kHostSlots] = {}, ev_free[kHostSlots] = {};
    cudaEvent_t ev_start = nullptr, ev_done = nullptr;
};
constexpr int kHostCtxDevices = 64;
static HostBatchCtx g_host_ctx[kHostCtxDevices];

static size_t round256(size_t v) { return (v + 255) / 256 * 256; }

static pfb_status grow(void **p, size_t *cap, size_t need) {
    if (*cap >= need) return PFB_OK;
    cudaFree(*p);
    *p = nullptr;
    *cap = 0;
    if (cudaMalloc(p, need) != cudaSuccess) {
        cudaGetLastError();
        return fail(PFB_ERR_OOM, "host-batch staging buffer");
    }
    *cap = need;
    return PFB_OK;
}

}  // namespace pfb

extern "C" pfb_status pfb_set_host_route(int32_t route) {
    clear_error();
    if (route != PFB_HOST_ROUTE_AUTO && route != PFB_HOST_ROUTE_STAGED) return fail(PFB_ERR_INVALID, "unknown host route");
    g_host_route.store(route);
    return PFB_OK;
}

extern "C" int32_t pfb_last_host_route(void) { return t_last_host_route; }

extern "C" pfb_status pfb_execute_batch_host(const pfb_batch_item *items, int32_t n_items, void *cuda_stream) {
    clear_error();
    if (n_items < 0 || (n_items > 0 && !items)) return fail(PFB_ERR_INVALID, "bad item list");
    // validate every item before anything is copied or launched
    int device = -1;
    std::vector<int64_t> S(n_items), fr_bytes(n_items);
    for (int i = 0; i < n_items; ++i) {
        const pfb_batch_item &it = items[i];
        if (!it.plan) return fail(PFB_ERR_INVALID, "item with NULL plan");
        const Plan &p = *reinterpret_cast<Plan *>(it.plan);
        if (device < 0) device = p.device;
        if (p.device != device) return fail(PFB_ERR_INVALID, "batch items span devices");
        if (p.R > 1) return fail(PFB_ERR_UNSUPPORTED, "oversampled plans (hop < P) run through pfb_execute_batch");
        if (it.n_samples < 0) return fail(PFB_ERR_INVALID, "item " + std::to_string(i) + ": n_samples < 0");
        S[i] = out_spectra(p, it.n_samples);
        fr_bytes[i] = (it.n_samples / p.P) * p.P * (int64_t)p.esize;  // whole frames only
        if (S[i] == 0) continue;
        if (!it.d_in || !it.d_out) return fail(PFB_ERR_INVALID, "item " + std::to_string(i) + ": NULL buffer with S > 0");
        if (it.out_cap_spectra < S[i])
            return fail(PFB_ERR_INVALID, "item " + std::to_string(i) + ": out_cap_spectra smaller than the spectra produced");
    }
    t_last_host_route = 0;
    if (device < 0) return PFB_OK;
    if (device >= kHostCtxDevices) return fail(PFB_ERR_INVALID, "device ordinal out of range");
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    // Mapped route: every buffer page-locked and mapped, every plan's kernel
    // reading and writing them per thread.  The kernels then read the input
    // and write the spectra in host memory directly (one launch per variant
    // group, no staging copies), and the call returns after the stream has
    // drained.
    if (g_host_route.load() == PFB_HOST_ROUTE_AUTO) {
        DeviceGuard g(device);
        std::vector<pfb_batch_item> mapped;
        bool ok = true;
        for (int i = 0; i < n_items && ok; ++i) {
            if (S[i] == 0) continue;
            const Plan &p = *reinterpret_cast<Plan *>(items[i].plan);
            const char *di = takes_mapped_buffers(p) ? mapped_host_range(items[i].d_in, (size_t)fr_bytes[i]) : nullptr;
            const char *dq = di ? mapped_host_range(items[i].d_out, (size_t)S[i] * p.P * sizeof(float2)) : nullptr;
            ok = di && dq && aligned16(di) && aligned16(dq);
            if (!ok) break;
            pfb_batch_item d = items[i];
            d.d_in = di;
            d.n_samples = fr_bytes[i] / p.esize;
            d.d_out = const_cast<char *>(dq);
            d.out_cap_spectra = S[i];
            mapped.push_back(d);
        }
        if (ok && !mapped.empty()) {
            t_last_host_route = 2;
            std::vector<Group> groups;
            int dev2 = -1;
            pfb_status st = build_groups(mapped.data(), (int32_t)mapped.size(), groups, dev2);
            for (auto &gr : groups) {
                if (st != PFB_OK) break;
                st = launch_family(*gr.plan, gr.descs.data(), (int)gr.descs.size(), s);
            }
            // nothing may still be writing host memory when the call returns
            cudaError_t e = cudaStreamSynchronize(s);
            if (st != PFB_OK) return st;
            if (e != cudaSuccess) return cuda_fail(e, "host batch kernels (mapped)");
            pfb_status kst = PFB_OK;
            for (int i = 0; i < n_items; ++i) {
                pfb_status k = take_kernel_error(reinterpret_cast<Plan *>(items[i].plan)->h_err, "pfb_execute_batch_host");
                if (kst == PFB_OK) kst = k;
            }
            return kst;
        }
    }
    t_last_host_route = 1;
    // chunks: runs of consecutive items of about kChunkBytes of input
    constexpr int64_t kChunkBytes = 32ll << 20;
    struct Chunk { int i0, i1; size_t in_bytes, out_bytes; };
    std::vector<Chunk> chunks;
    for (int i = 0; i < n_items;) {
        if (S[i] == 0) { ++i; continue; }
        Chunk c{i, i, 0, 0};
        while (c.i1 < n_items) {
            const int j = c.i1;
            if (S[j] > 0) {
                const Plan &p = *reinterpret_cast<Plan *>(items[j].plan);
                const size_t ib = round256((size_t)fr_bytes[j]);
                if (c.i1 > c.i0 && (int64_t)(c.in_bytes + ib) > kChunkBytes) break;
                c.in_bytes += ib;
                c.out_bytes += round256((size_t)S[j] * p.P * sizeof(float2));
            }
            ++c.i1;
        }
        chunks.push_back(c);
        i = c.i1;
    }
    if (chunks.empty()) return PFB_OK;
    HostBatchCtx &x = g_host_ctx[device];
    std::lock_guard<std::mutex> lk(x.mu);
    DeviceGuard g(device);
    if (!x.ready) {
        PFB_CUDA_TRY(cudaStreamCreateWithFlags(&x.s_in, cudaStreamNonBlocking));
        PFB_CUDA_TRY(cudaStreamCreateWithFlags(&x.s_out, cudaStreamNonBlocking));
        for (int b = 0; b < HostBatchCtx::kHostSlots; ++b) {
            PFB_CUDA_TRY(cudaEventCreateWithFlags(&x.ev_in[b], cudaEventDisableTiming));
            PFB_CUDA_TRY(cudaEventCreateWithFlags(&x.ev_k[b], cudaEventDisableTiming));
            PFB_CUDA_TRY(cudaEventCreateWithFlags(&x.ev_free[b], cudaEventDisableTiming));
        }
        PFB_CUDA_TRY(cudaEventCreateWithFlags(&x.ev_start, cudaEventDisableTiming));
        PFB_CUDA_TRY(cudaEventCreateWithFlags(&x.ev_done, cudaEventDisableTiming));
        x.ready = true;
    }
    size_t need_in = 0, need_out = 0;
    for (const Chunk &c : chunks) {
        need_in = std::max(need_in, c.in_bytes);
        need_out = std::max(need_out, c.out_bytes);
    }
    // slots in use by an earlier call have finished (the call returns after
    // its last copy), so growing them here is safe
    for (int b = 0; b < HostBatchCtx::kHostSlots && b < (int)chunks.size(); ++b) {
        pfb_status st = grow(&x.d_in[b], &x.in_cap[b], need_in);
        if (st == PFB_OK) st = grow(&x.d_out[b], &x.out_cap[b], need_out);
        if (st != PFB_OK) return st;
    }
    // Chunk c uses slot c mod kHostSlots: its copy-in waits until the slot's
    // previous chunk has been copied out; its kernels run on the caller's
    // stream after its copy-in; its copy-out follows its kernels.
    PFB_CUDA_TRY(cudaEventRecord(x.ev_start, s));
    PFB_CUDA_TRY(cudaStreamWaitEvent(x.s_in, x.ev_start, 0));
    PFB_CUDA_TRY(cudaStreamWaitEvent(x.s_out, x.ev_start, 0));
    std::vector<pfb_batch_item> dev_items;
    pfb_status st = PFB_OK;
    for (size_t c = 0; c < chunks.size() && st == PFB_OK; ++c) {
        const Chunk &ch = chunks[c];
        const int b = (int)(c % HostBatchCtx::kHostSlots);
        if (c >= (size_t)HostBatchCtx::kHostSlots) {
            cudaError_t e = cudaStreamWaitEvent(x.s_in, x.ev_free[b], 0);
            if (e != cudaSuccess) { st = cuda_fail(e, "cudaStreamWaitEvent"); break; }
        }
        char *din = static_cast<char *>(x.d_in[b]);
        char *dout = static_cast<char *>(x.d_out[b]);
        dev_items.clear();
        size_t oi = 0, oo = 0;
        for (int i = ch.i0; i < ch.i1 && st == PFB_OK; ++i) {
            if (S[i] == 0) continue;
            const Plan &p = *reinterpret_cast<Plan *>(items[i].plan);
            cudaError_t e = cudaMemcpyAsync(din + oi, items[i].d_in, (size_t)fr_bytes[i], cudaMemcpyHostToDevice, x.s_in);
            if (e != cudaSuccess) { st = cuda_fail(e, "cudaMemcpyAsync (host batch input)"); break; }
            pfb_batch_item d = items[i];
            d.d_in = din + oi;
            d.n_samples = fr_bytes[i] / p.esize;
            d.d_out = dout + oo;
            d.out_cap_spectra = S[i];
            dev_items.push_back(d);
            oi += round256((size_t)fr_bytes[i]);
            oo += round256((size_t)S[i] * p.P * sizeof(float2));
        }
        if (st != PFB_OK) break;
        cudaError_t e = cudaEventRecord(x.ev_in[b], x.s_in);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, x.ev_in[b], 0);
        if (e != cudaSuccess) { st = cuda_fail(e, "host batch copy-in event"); break; }
        std::vector<Group> groups;
        int dev2 = -1;
        st = build_groups(dev_items.data(), (int32_t)dev_items.size(), groups, dev2);
        for (auto &gr : groups) {
            if (st != PFB_OK) break;
            st = launch_family(*gr.plan, gr.descs.data(), (int)gr.descs.size(), s);
        }
        if (st != PFB_OK) break;
        e = cudaEventRecord(x.ev_k[b], s);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(x.s_out, x.ev_k[b], 0);
        if (e != cudaSuccess) { st = cuda_fail(e, "host batch kernel event"); break; }
        for (size_t k = 0, i = ch.i0; i < (size_t)ch.i1 && st == PFB_OK; ++i) {
            if (S[i] == 0) continue;
            const Plan &p = *reinterpret_cast<Plan *>(items[i].plan);
            e = cudaMemcpyAsync(items[i].d_out, dev_items[k].d_out, (size_t)S[i] * p.P * sizeof(float2),
                                cudaMemcpyDeviceToHost, x.s_out);
            if (e != cudaSuccess) st = cuda_fail(e, "cudaMemcpyAsync (host batch output)");
            ++k;
        }
        if (st == PFB_OK) {
            e = cudaEventRecord(x.ev_free[b], x.s_out);
            if (e != cudaSuccess) st = cuda_fail(e, "host batch slot event");
        }
    }
    // nothing may still be writing host memory (or reading the slots) when
    // the call returns, whatever happened above
    cudaError_t e1 = cudaEventRecord(x.ev_done, x.s_out);
    if (e1 == cudaSuccess) e1 = cudaStreamWaitEvent(s, x.ev_done, 0);
    cudaError_t e2 = cudaStreamSynchronize(x.s_in);
    cudaError_t e3 = cudaStreamSynchronize(s);
    cudaError_t e4 = cudaStreamSynchronize(x.s_out);
    if (st != PFB_OK) return st;
    if (e1 != cudaSuccess) return cuda_fail(e1, "host batch completion event");
    if (e2 != cudaSuccess) return cuda_fail(e2, "host batch copy-in");
    if (e3 != cudaSuccess) return cuda_fail(e3, "host batch kernels");
    if (e4 != cudaSuccess) return cuda_fail(e4, "host batch copy-out");
    // kernel error words of every plan of the batch
    pfb_status kst = PFB_OK;
    for (int i = 0; i < n_items; ++i) {
        pfb_status k = take_kernel_error(reinterpret_cast<Plan *>(items[i].plan)->h_err, "pfb_execute_batch_host");
        if (kst == PFB_OK) kst = k;
    }
    return kst;
}

extern "C" pfb_status pfb_batch_create(const pfb_batch_item *items, int32_t n_items, pfb_batch_t *out_batch) {
    clear_error();
    if (!out_batch) return fail(PFB_ERR_INVALID, "out_batch is NULL");
    *out_batch = nullptr;
    std::vector<Group> groups;
    int device = -1;
    pfb_status st = build_groups(items, n_items, groups, device);
    if (st != PFB_OK) return st;
    if (device < 0) {
        cudaGetDevice(&device);
    }
    DeviceGuard g(device);
    // workspaces of the plans that need one (the two-pass DFT-matrix products)
    // are grown here, outside the capture, to what each launch will use
    for (auto &gr : groups) {
        size_t need = 0;
        const int nd = (int)gr.descs.size();
        for (int g0 = 0; g0 < nd; g0 += kMaxStreamsPerLaunch) {
            int64_t units = 0;
            for (int i = g0; i < std::min(nd, g0 + kMaxStreamsPerLaunch); ++i) units += family_units(*gr.plan, gr.descs[i].S);
            need = std::max(need, family_workspace_bytes(*gr.plan, units));
        }
        if (need > 0 && (st = grow_plan_workspace(*gr.plan, need, nullptr)) != PFB_OK) return st;
    }
    Batch *b = new (std::nothrow) Batch();
    if (!b) return fail(PFB_ERR_OOM, "host allocation");
    b->device = device;
    // Capture every group's launch on its own forked stream so independent
    // groups may overlap on the device; one graph, one replay.
    cudaStream_t main = nullptr;
    std::vector<cudaStream_t> side(groups.size(), nullptr);
    std::vector<cudaEvent_t> done(groups.size(), nullptr);
    cudaEvent_t fork = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&main, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
    for (size_t i = 0; e == cudaSuccess && i < groups.size(); ++i) {
        e = cudaStreamCreateWithFlags(&side[i], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&done[i], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaStreamBeginCapture(main, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) e = cudaEventRecord(fork, main);
    for (size_t i = 0; e == cudaSuccess && st == PFB_OK && i < groups.size(); ++i) {
        e = cudaStreamWaitEvent(side[i], fork, 0);
        if (e != cudaSuccess) break;
        st = launch_family(*groups[i].plan, groups[i].descs.data(), (int)groups[i].descs.size(), side[i]);
        if (st == PFB_OK) e = cudaEventRecord(done[i], side[i]);
        if (e == cudaSuccess && st == PFB_OK) e = cudaStreamWaitEvent(main, done[i], 0);
    }
    cudaGraph_t graph = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(main, &graph);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess && st == PFB_OK) e = cudaGraphInstantiate(&b->exec, graph, 0);
    b->graph = graph;
    for (size_t i = 0; i < groups.size(); ++i) {
        if (side[i]) cudaStreamDestroy(side[i]);
        if (done[i]) cudaEventDestroy(done[i]);
    }
    if (fork) cudaEventDestroy(fork);
    if (main) cudaStreamDestroy(main);
    if (st != PFB_OK || e != cudaSuccess) {
        if (b->exec) cudaGraphExecDestroy(b->exec);
        if (b->graph) cudaGraphDestroy(b->graph);
        delete b;
        return st != PFB_OK ? st : cuda_fail(e, "batch graph capture");
    }
    *out_batch = reinterpret_cast<pfb_batch_t>(b);
    return PFB_OK;
}

extern "C" pfb_status pfb_batch_launch(pfb_batch_t batch, void *cuda_stream) {
    clear_error();
    if (!batch) return fail(PFB_ERR_INVALID, "batch is NULL");
    Batch *b = reinterpret_cast<Batch *>(batch);
    DeviceGuard g(b->device);
    PFB_CUDA_TRY(cudaGraphLaunch(b->exec, static_cast<cudaStream_t>(cuda_stream)));
    g_launches++;
    return PFB_OK;
}

extern "C" pfb_status pfb_batch_destroy(pfb_batch_t batch) {
    clear_error();
    if (!batch) return PFB_OK;
    Batch *b = reinterpret_cast<Batch *>(batch);
    DeviceGuard g(b->device);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    delete b;
    return PFB_OK;
}
