// Synthesis (inverse) filter bank: launcher and C ABI (kernel in fft_synth.cuh).
#include <cstring>

#include "fft_synth.cuh"

namespace pfb {

static bool synth_supported(const Plan &p) {
    return p.family == FAM_FFT_FAST && (p.P == 512 || p.P == 1024) && p.R == 1 &&
           (p.TT == 4 || p.TT == 8 || p.TT == 16) && p.T <= p.TT;
}

template <int P, int TT>
static pfb_status launch_synth_k(LaunchArgs &a, cudaStream_t stream) {
    using C = SyCfg<P, TT>;
    auto k = k_synth_ws<P, TT>;
    static int grid_cap = 0;
    if (grid_cap == 0) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
        if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(k_synth_ws)");
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        grid_cap = sms;
    }
    int64_t grid = a.nunits < grid_cap ? a.nunits : grid_cap;
    if (grid < 1) return PFB_OK;
    if ((a.nunits + grid - 1) / grid > INT32_MAX - 64)  // 32-bit segment counters in the kernel
        return fail(PFB_ERR_INVALID, "too many output frames for one launch of k_synth_ws");
    a.units_per_cta = (int32_t)((a.nunits + grid - 1) / grid);
    grid = (a.nunits + a.units_per_cta - 1) / a.units_per_cta;
    k<<<(unsigned)grid, C::NTHREADS, C::SMEM, stream>>>(a);
    g_launches++;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "launch k_synth_ws");
    return PFB_OK;
}

static pfb_status launch_synth(const Plan &p, LaunchArgs &a, cudaStream_t stream) {
    switch (p.P * 100 + p.TT) {
    case 512 * 100 + 4: return launch_synth_k<512, 4>(a, stream);
    case 512 * 100 + 8: return launch_synth_k<512, 8>(a, stream);
    case 512 * 100 + 16: return launch_synth_k<512, 16>(a, stream);
    case 1024 * 100 + 4: return launch_synth_k<1024, 4>(a, stream);
    case 1024 * 100 + 8: return launch_synth_k<1024, 8>(a, stream);
    case 1024 * 100 + 16: return launch_synth_k<1024, 16>(a, stream);
    default: return fail(PFB_ERR_UNSUPPORTED, "synthesis: no kernel for this P/T");
    }
}

}  // namespace pfb

using namespace pfb;

extern "C" int64_t pfb_synth_out_samples(pfb_plan_t plan, int64_t n_spectra) {
    if (!plan || n_spectra < 0) return -1;
    const Plan &p = *reinterpret_cast<Plan *>(plan);
    return n_spectra > 0 ? (n_spectra + p.T - 1) * (int64_t)p.P : 0;
}

extern "C" pfb_status pfb_synthesize(pfb_plan_t plan, const void *d_spectra, int64_t n_spectra, void *d_out,
                                     int64_t out_cap_samples, void *cuda_stream) {
    clear_error();
    if (!plan) return fail(PFB_ERR_INVALID, "plan is NULL");
    Plan &p = *reinterpret_cast<Plan *>(plan);
    if (n_spectra < 0) return fail(PFB_ERR_INVALID, "n_spectra < 0");
    if (n_spectra == 0) return PFB_OK;
    if (!synth_supported(p) && !synth_generic_supported(p))
        return fail(PFB_ERR_UNSUPPORTED, p.R != 1 ? "synthesis needs a critically sampled plan (hop P)"
                                                  : "split-bf16 synthesis needs P >= 128");
    if (!d_spectra || !d_out) return fail(PFB_ERR_INVALID, "NULL buffer with spectra to synthesise");
    if ((reinterpret_cast<uintptr_t>(d_spectra) & 15u) || (reinterpret_cast<uintptr_t>(d_out) & 15u))
        return fail(PFB_ERR_INVALID, "buffers must be 16-byte aligned");
    const int64_t frames = n_spectra + p.T - 1;
    if (out_cap_samples < frames * p.P) return fail(PFB_ERR_INVALID, "out_cap_samples smaller than the output");
    if (!synth_supported(p)) {
        int prev = -1;
        cudaGetDevice(&prev);
        if (prev != p.device) cudaSetDevice(p.device);
        pfb_status st = launch_synth_generic(p, static_cast<const float2 *>(d_spectra), n_spectra,
                                             static_cast<float2 *>(d_out), static_cast<cudaStream_t>(cuda_stream));
        if (prev >= 0 && prev != p.device) cudaSetDevice(prev);
        return st;
    }
    LaunchArgs a;
    std::memset(&a, 0, sizeof(a));
    StreamDesc &d = a.s[0];
    d.in = d_spectra;
    d.out = static_cast<float2 *>(d_out);
    d.n_frames = n_spectra;  // spectrum rows
    d.S = frames;            // work units: output frames
    d.ldo = p.P;
    d.taps = family_taps(p);
    d.T = p.T;
    d.unit0 = 0;
    a.nstreams = 1;
    a.nunits = frames;
    a.aux = p.d_tw_r2;
    a.err = p.d_err;
    a.wait_ns = p.wait_ns;
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != p.device) cudaSetDevice(p.device);
    pfb_status st = launch_synth(p, a, static_cast<cudaStream_t>(cuda_stream));
    if (prev >= 0 && prev != p.device) cudaSetDevice(prev);
    return st;
}
