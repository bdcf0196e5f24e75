// pfb_execute_host_noalloc: pfb_execute_host without any device allocation.
//
// pfb_execute_host stages the caller's host buffers through device buffers
// that the plan grows with cudaMalloc (and frees with cudaFree) and pipelines
// the copies over streams and events it creates.  Some callers cannot let a
// library do that: a process whose device memory is handed out by another
// allocator that already holds it (a framework's caching pool, a fixed
// real-time reservation), or a latency-critical thread that cannot take the
// device-wide synchronisation cudaMalloc/cudaFree may imply.  This variant
// stages through a fixed area in static device memory instead, on the
// caller's stream only, and creates nothing.
#include <cstring>

#include "internal.h"

namespace pfb {

// The staging area: input samples at offset 0, output spectra after them
// (offset rounded up to 256 bytes).  Every device that loads the library
// holds it until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[PFB_NOALLOC_SCRATCH_BYTES];

static_assert(PFB_NOALLOC_SCRATCH_BYTES % 256 == 0, "staging area must be a multiple of 256 bytes");

// Device address of g_noalloc_scratch per device.  In host code the array's
// name is only a host-side handle, so the address is looked up once per
// device (with that device current) and cached.
constexpr int kMaxDevices = 64;
static pfb_status scratch_address(int device, void **out);
static std::mutex g_scratch_mu;
static void *g_scratch_ptr[kMaxDevices] = {};

}  // namespace pfb

// Called by pfb_plan_create with the plan's device current: resolving the
// address loads this translation unit's module on that device (under lazy
// module loading that is when the static area is reserved), so the first
// pfb_execute_host_noalloc call neither loads a module nor reserves memory.
pfb_status pfb::noalloc_prepare(int device) {
    void *p = nullptr;
    return scratch_address(device, &p);
}

namespace pfb {

static pfb_status scratch_address(int device, void **out) {
    if (device < 0 || device >= kMaxDevices) return fail(PFB_ERR_INVALID, "device ordinal out of range");
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (!g_scratch_ptr[device]) {
        void *ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
        if (!ptr) return fail(PFB_ERR_CUDA, "cudaGetSymbolAddress(g_noalloc_scratch) returned NULL");
        g_scratch_ptr[device] = ptr;
    }
    *out = g_scratch_ptr[device];
    return PFB_OK;
}

}  // namespace pfb

using namespace pfb;

extern "C" pfb_status pfb_execute_host_noalloc(pfb_plan_t plan, const void *host_in, int64_t n_samples,
                                               void *host_out, int64_t out_cap_spectra, void *cuda_stream) {
    clear_error();
    if (!plan) return fail(PFB_ERR_INVALID, "plan is NULL");
    const Plan &p = *reinterpret_cast<Plan *>(plan);
    if (p.R > 1) return fail(PFB_ERR_UNSUPPORTED, "oversampled plans (hop < P) run through pfb_execute");
    if (n_samples < 0) return fail(PFB_ERR_INVALID, "n_samples < 0");
    const int64_t S = out_spectra(p, n_samples);
    if (S == 0) return PFB_OK;
    if (!host_in || !host_out) return fail(PFB_ERR_INVALID, "NULL buffer with S > 0");
    if (out_cap_spectra < S) return fail(PFB_ERR_INVALID, "out_cap_spectra smaller than the spectra produced");
    // Only whole frames are staged: the kernel never reads the N mod P tail.
    const int64_t frames = n_samples / p.P;
    const int64_t in_bytes = frames * p.P * p.esize;
    const int64_t out_off = (in_bytes + 255) / 256 * 256;
    const int64_t out_bytes = S * p.P * (int64_t)sizeof(float2);
    if (out_off + out_bytes > PFB_NOALLOC_SCRATCH_BYTES)
        return fail(PFB_ERR_INVALID, "input (" + std::to_string(in_bytes) + " B) plus output (" +
                                         std::to_string(out_bytes) + " B) exceed the " +
                                         std::to_string((long long)PFB_NOALLOC_SCRATCH_BYTES) +
                                         "-byte static staging area of pfb_execute_host_noalloc");

    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != p.device) {
        cudaError_t e = cudaSetDevice(p.device);
        if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    }
    pfb_status st = PFB_OK;
    do {
        void *base = nullptr;
        st = scratch_address(p.device, &base);
        if (st != PFB_OK) break;
        char *din = static_cast<char *>(base);
        float2 *dout = reinterpret_cast<float2 *>(din + out_off);
        cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
        // Nothing in the area needs clearing: the kernel reads only the input
        // bytes copied here by this call and writes every output row it copies
        // back, so whatever an earlier call left behind is never read.
        cudaError_t e = cudaMemcpyAsync(din, host_in, (size_t)in_bytes, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) { st = cuda_fail(e, "cudaMemcpyAsync (host to staging area)"); break; }
        StreamDesc d;
        std::memset(&d, 0, sizeof(d));
        d.in = din;
        d.state = nullptr;
        d.out = dout;
        d.n_state = 0;
        d.n_frames = frames;
        d.S = S;
        d.ldo = p.P;
        d.taps = family_taps(p);
        d.scale = p.desc.in_scale;
        d.T = p.T;
        st = launch_family(p, &d, 1, s);
        if (st != PFB_OK) {
            cudaStreamSynchronize(s);  // the input copy must not outlive the call
            break;
        }
        e = cudaMemcpyAsync(host_out, dout, (size_t)out_bytes, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) st = cuda_fail(e, "staging area to host copy");
        // the kernel's error word (host-mapped, allocated with the plan)
        if (st == PFB_OK) st = take_kernel_error(p.h_err, "pfb_execute_host_noalloc");
    } while (0);
    if (prev >= 0 && prev != p.device) cudaSetDevice(prev);
    return st;
}
