// Launcher of the cluster FFT family (P = 2048, 4096): variant 0 is the
// synchronous kernel of fft_cluster.cuh (units of 8 spectra), variant 1 the
// warp-specialised TMA-fed kernel of fft_ws_cluster.cuh (cross-CTA step in
// the FFT warps), variant 2 the warp-specialised kernel of fft_wc2.cuh (one
// exchange between the FIR warps' radix-4 step and the receiving FFT warps'
// radix-CS step, the default); 1 and 2 take one unit per spectrum and T
// equal to their compiled tap count 4, 8 or 16.
#include "fft_cluster.cuh"
#include "fft_wc2.cuh"
#include "fft_wcf.cuh"
#include "fft_ws_cluster.cuh"

namespace pfb {

int64_t cluster_units(int64_t S) { return (S + 7) / 8; }
int64_t fft_cluster_units(const Plan &plan, int64_t S) { return plan.variant >= 1 ? S : cluster_units(S); }

bool wcf_supported(const Plan &plan) { return plan.P == 4096 && plan.T == plan.TT && (plan.TT == 4 || plan.TT == 8 || plan.TT == 16); }

bool ws_cluster_supported(const Plan &plan) {
    return (plan.P == 2048 || plan.P == 4096) && plan.T == plan.TT && (plan.TT == 4 || plan.TT == 8 || plan.TT == 16);
}

template <int CS, int TT, int IN, bool TC>
static pfb_status launch_ws_cluster_k(LaunchArgs &a, cudaStream_t stream) {
    using C = WcCfg<CS, TT, IN, TC>;
    auto k = k_fft_ws_cluster<CS, TT, IN, TC>;
    static int cap_clusters = 0;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CS;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.blockDim = dim3(C::NTHREADS, 1, 1);
    cfg.dynamicSmemBytes = C::SMEM;
    cfg.stream = stream;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (cap_clusters == 0) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
        if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(k_fft_ws_cluster)");
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cfg.gridDim = dim3((unsigned)(sms / CS * CS), 1, 1);
        int n = 0;
        e = cudaOccupancyMaxActiveClusters(&n, k, &cfg);
        if (e != cudaSuccess || n < 1) return cuda_fail(e == cudaSuccess ? cudaErrorInvalidConfiguration : e,
                                                        "cudaOccupancyMaxActiveClusters(k_fft_ws_cluster)");
        cap_clusters = n;
    }
    int64_t clusters = a.nunits < cap_clusters ? a.nunits : cap_clusters;
    if (clusters < 1) return PFB_OK;
    if ((a.nunits + clusters - 1) / clusters > INT32_MAX - 64)  // 32-bit segment counters in the kernels
        return fail(PFB_ERR_INVALID, "too many spectra for one cluster launch");
    a.units_per_cta = (int32_t)((a.nunits + clusters - 1) / clusters);
    clusters = (a.nunits + a.units_per_cta - 1) / a.units_per_cta;
    cfg.gridDim = dim3((unsigned)(clusters * CS), 1, 1);
    cudaError_t e = cudaLaunchKernelEx(&cfg, k, a);
    g_launches++;
    if (e != cudaSuccess) return cuda_fail(e, "launch k_fft_ws_cluster");
    return PFB_OK;
}

template <int CS, int TT, int IN>
static pfb_status launch_wc2_k(LaunchArgs &a, cudaStream_t stream) {
    using C = Wc2Cfg<CS, TT, IN>;
    auto k = k_fft_wc2<CS, TT, IN>;
    static int cap_clusters = 0;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CS;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.blockDim = dim3(C::NTHREADS, 1, 1);
    cfg.dynamicSmemBytes = C::SMEM;
    cfg.stream = stream;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (cap_clusters == 0) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
        if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(k_fft_wc2)");
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cfg.gridDim = dim3((unsigned)(sms / CS * CS), 1, 1);
        int n = 0;
        e = cudaOccupancyMaxActiveClusters(&n, k, &cfg);
        if (e != cudaSuccess || n < 1) return cuda_fail(e == cudaSuccess ? cudaErrorInvalidConfiguration : e,
                                                        "cudaOccupancyMaxActiveClusters(k_fft_wc2)");
        cap_clusters = n;
    }
    int64_t clusters = a.nunits < cap_clusters ? a.nunits : cap_clusters;
    if (clusters < 1) return PFB_OK;
    if ((a.nunits + clusters - 1) / clusters > INT32_MAX - 64)  // 32-bit segment counters in the kernel
        return fail(PFB_ERR_INVALID, "too many spectra for one cluster launch");
    a.units_per_cta = (int32_t)((a.nunits + clusters - 1) / clusters);
    clusters = (a.nunits + a.units_per_cta - 1) / a.units_per_cta;
    cfg.gridDim = dim3((unsigned)(clusters * CS), 1, 1);
    cudaError_t e = cudaLaunchKernelEx(&cfg, k, a);
    g_launches++;
    if (e != cudaSuccess) return cuda_fail(e, "launch k_fft_wc2");
    return PFB_OK;
}

template <int TT, int IN>
static pfb_status launch_wcf_k(LaunchArgs &a, cudaStream_t stream) {
    using C = WcfCfg<TT, IN>;
    auto k = k_fft_wcf<TT, IN>;
    static int cap_clusters = 0;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C::CS;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.blockDim = dim3(C::NTHREADS, 1, 1);
    cfg.dynamicSmemBytes = C::SMEM;
    cfg.stream = stream;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (cap_clusters == 0) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
        if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(k_fft_wcf)");
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cfg.gridDim = dim3((unsigned)(sms / C::CS * C::CS), 1, 1);
        int n = 0;
        e = cudaOccupancyMaxActiveClusters(&n, k, &cfg);
        if (e != cudaSuccess || n < 1) return cuda_fail(e == cudaSuccess ? cudaErrorInvalidConfiguration : e,
                                                        "cudaOccupancyMaxActiveClusters(k_fft_wcf)");
        cap_clusters = n;
    }
    int64_t clusters = a.nunits < cap_clusters ? a.nunits : cap_clusters;
    if (clusters < 1) return PFB_OK;
    if ((a.nunits + clusters - 1) / clusters > INT32_MAX - 64)  // 32-bit segment counters in the kernel
        return fail(PFB_ERR_INVALID, "too many spectra for one cluster launch");
    a.units_per_cta = (int32_t)((a.nunits + clusters - 1) / clusters);
    clusters = (a.nunits + a.units_per_cta - 1) / a.units_per_cta;
    cfg.gridDim = dim3((unsigned)(clusters * C::CS), 1, 1);
    cudaError_t e = cudaLaunchKernelEx(&cfg, k, a);
    g_launches++;
    if (e != cudaSuccess) return cuda_fail(e, "launch k_fft_wcf");
    return PFB_OK;
}

static pfb_status launch_wcf(const Plan &plan, LaunchArgs &a, cudaStream_t stream) {
    if (plan.P != 4096) return fail(PFB_ERR_UNSUPPORTED, "cluster variant 3: P must be 4096");
    for (int i = 0; i < a.nstreams; ++i)
        if (a.s[i].T != plan.TT) return fail(PFB_ERR_UNSUPPORTED, "cluster variant 3 needs T in {4, 8, 16}");
    switch (plan.in_dtype * 100 + plan.TT) {
    case PFB_IN_C64 * 100 + 4: return launch_wcf_k<4, PFB_IN_C64>(a, stream);
    case PFB_IN_C64 * 100 + 8: return launch_wcf_k<8, PFB_IN_C64>(a, stream);
    case PFB_IN_C64 * 100 + 16: return launch_wcf_k<16, PFB_IN_C64>(a, stream);
    case PFB_IN_R32 * 100 + 4: return launch_wcf_k<4, PFB_IN_R32>(a, stream);
    case PFB_IN_R32 * 100 + 8: return launch_wcf_k<8, PFB_IN_R32>(a, stream);
    case PFB_IN_R32 * 100 + 16: return launch_wcf_k<16, PFB_IN_R32>(a, stream);
    case PFB_IN_CI8 * 100 + 4: return launch_wcf_k<4, PFB_IN_CI8>(a, stream);
    case PFB_IN_CI8 * 100 + 8: return launch_wcf_k<8, PFB_IN_CI8>(a, stream);
    case PFB_IN_CI8 * 100 + 16: return launch_wcf_k<16, PFB_IN_CI8>(a, stream);
    default: return fail(PFB_ERR_UNSUPPORTED, "cluster variant 3: no kernel for this T/dtype");
    }
}

template <int CS>
static pfb_status launch_wc2_cs(const Plan &plan, LaunchArgs &a, cudaStream_t stream) {
    for (int i = 0; i < a.nstreams; ++i)
        if (a.s[i].T != plan.TT) return fail(PFB_ERR_UNSUPPORTED, "cluster variant 2 needs T in {4, 8, 16}");
    switch (plan.in_dtype * 100 + plan.TT) {
    case PFB_IN_C64 * 100 + 4: return launch_wc2_k<CS, 4, PFB_IN_C64>(a, stream);
    case PFB_IN_C64 * 100 + 8: return launch_wc2_k<CS, 8, PFB_IN_C64>(a, stream);
    case PFB_IN_C64 * 100 + 16: return launch_wc2_k<CS, 16, PFB_IN_C64>(a, stream);
    case PFB_IN_R32 * 100 + 4: return launch_wc2_k<CS, 4, PFB_IN_R32>(a, stream);
    case PFB_IN_R32 * 100 + 8: return launch_wc2_k<CS, 8, PFB_IN_R32>(a, stream);
    case PFB_IN_R32 * 100 + 16: return launch_wc2_k<CS, 16, PFB_IN_R32>(a, stream);
    case PFB_IN_CI8 * 100 + 4: return launch_wc2_k<CS, 4, PFB_IN_CI8>(a, stream);
    case PFB_IN_CI8 * 100 + 8: return launch_wc2_k<CS, 8, PFB_IN_CI8>(a, stream);
    case PFB_IN_CI8 * 100 + 16: return launch_wc2_k<CS, 16, PFB_IN_CI8>(a, stream);
    default: return fail(PFB_ERR_UNSUPPORTED, "cluster variant 2: no kernel for this T/dtype");
    }
}

template <int CS, bool TC>
static pfb_status launch_ws_cluster_cs(const Plan &plan, LaunchArgs &a, cudaStream_t stream) {
    for (int i = 0; i < a.nstreams; ++i)
        if (a.s[i].T != plan.TT) return fail(PFB_ERR_UNSUPPORTED, "cluster variant 1 needs T in {4, 8, 16}");
    switch (plan.in_dtype * 100 + plan.TT) {
    case PFB_IN_C64 * 100 + 4: return launch_ws_cluster_k<CS, 4, PFB_IN_C64, TC>(a, stream);
    case PFB_IN_C64 * 100 + 8: return launch_ws_cluster_k<CS, 8, PFB_IN_C64, TC>(a, stream);
    case PFB_IN_C64 * 100 + 16: return launch_ws_cluster_k<CS, 16, PFB_IN_C64, TC>(a, stream);
    case PFB_IN_R32 * 100 + 4: return launch_ws_cluster_k<CS, 4, PFB_IN_R32, TC>(a, stream);
    case PFB_IN_R32 * 100 + 8: return launch_ws_cluster_k<CS, 8, PFB_IN_R32, TC>(a, stream);
    case PFB_IN_R32 * 100 + 16: return launch_ws_cluster_k<CS, 16, PFB_IN_R32, TC>(a, stream);
    case PFB_IN_CI8 * 100 + 4: return launch_ws_cluster_k<CS, 4, PFB_IN_CI8, TC>(a, stream);
    case PFB_IN_CI8 * 100 + 8: return launch_ws_cluster_k<CS, 8, PFB_IN_CI8, TC>(a, stream);
    case PFB_IN_CI8 * 100 + 16: return launch_ws_cluster_k<CS, 16, PFB_IN_CI8, TC>(a, stream);
    default: return fail(PFB_ERR_UNSUPPORTED, "cluster variant 1: no kernel for this T/dtype");
    }
}

template <int CS, int TT, int IN, bool TC>
static pfb_status launch_cluster_k(LaunchArgs &a, cudaStream_t stream) {
    using C = ClusterCfg<CS, TC>;
    auto k = k_fft_cluster<CS, TT, IN, TC>;
    static int cap_clusters = 0;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CS;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.blockDim = dim3(C::NT, 1, 1);
    cfg.dynamicSmemBytes = C::SMEM;
    cfg.stream = stream;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (cap_clusters == 0) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
        if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(k_fft_cluster)");
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cfg.gridDim = dim3((unsigned)(sms / CS * CS), 1, 1);
        int n = 0;
        e = cudaOccupancyMaxActiveClusters(&n, k, &cfg);
        if (e != cudaSuccess || n < 1) return cuda_fail(e == cudaSuccess ? cudaErrorInvalidConfiguration : e,
                                                        "cudaOccupancyMaxActiveClusters(k_fft_cluster)");
        cap_clusters = n;
    }
    int64_t clusters = a.nunits < cap_clusters ? a.nunits : cap_clusters;
    if (clusters < 1) return PFB_OK;
    if ((a.nunits + clusters - 1) / clusters > INT32_MAX - 64)  // 32-bit segment counters in the kernels
        return fail(PFB_ERR_INVALID, "too many spectra for one cluster launch");
    a.units_per_cta = (int32_t)((a.nunits + clusters - 1) / clusters);
    clusters = (a.nunits + a.units_per_cta - 1) / a.units_per_cta;
    cfg.gridDim = dim3((unsigned)(clusters * CS), 1, 1);
    cudaError_t e = cudaLaunchKernelEx(&cfg, k, a);
    g_launches++;
    if (e != cudaSuccess) return cuda_fail(e, "launch k_fft_cluster");
    return PFB_OK;
}

template <int CS, bool TC>
static pfb_status launch_cluster_cs(const Plan &plan, LaunchArgs &a, cudaStream_t stream) {
    switch (plan.in_dtype * 100 + plan.TT) {
    case PFB_IN_C64 * 100 + 4: return launch_cluster_k<CS, 4, PFB_IN_C64, TC>(a, stream);
    case PFB_IN_C64 * 100 + 8: return launch_cluster_k<CS, 8, PFB_IN_C64, TC>(a, stream);
    case PFB_IN_C64 * 100 + 16: return launch_cluster_k<CS, 16, PFB_IN_C64, TC>(a, stream);
    case PFB_IN_R32 * 100 + 4: return launch_cluster_k<CS, 4, PFB_IN_R32, TC>(a, stream);
    case PFB_IN_R32 * 100 + 8: return launch_cluster_k<CS, 8, PFB_IN_R32, TC>(a, stream);
    case PFB_IN_R32 * 100 + 16: return launch_cluster_k<CS, 16, PFB_IN_R32, TC>(a, stream);
    case PFB_IN_CI8 * 100 + 4: return launch_cluster_k<CS, 4, PFB_IN_CI8, TC>(a, stream);
    case PFB_IN_CI8 * 100 + 8: return launch_cluster_k<CS, 8, PFB_IN_CI8, TC>(a, stream);
    case PFB_IN_CI8 * 100 + 16: return launch_cluster_k<CS, 16, PFB_IN_CI8, TC>(a, stream);
    default: return fail(PFB_ERR_UNSUPPORTED, "cluster FFT family: no kernel for this T/dtype");
    }
}

bool fft_cluster_supported(int P, int T) { return (P == 2048 || P == 4096) && T >= 1 && T <= 16; }

pfb_status launch_fft_cluster(const Plan &plan, LaunchArgs &a, cudaStream_t stream) {
    a.aux = plan.d_tw_r2;
    if (plan.variant == 3) return launch_wcf(plan, a, stream);
    if (plan.variant == 2) {
        switch (plan.P) {
        case 2048: return launch_wc2_cs<2>(plan, a, stream);
        case 4096: return launch_wc2_cs<4>(plan, a, stream);
        default: return fail(PFB_ERR_UNSUPPORTED, "cluster variant 2: P must be 2048 or 4096");
        }
    }
    if (plan.variant == 1) {
        switch (plan.P) {
        case 2048: return launch_ws_cluster_cs<2, false>(plan, a, stream);
        case 4096: return launch_ws_cluster_cs<4, false>(plan, a, stream);
        default: return fail(PFB_ERR_UNSUPPORTED, "cluster variant 1: P must be 2048 or 4096");
        }
    }
    switch (plan.P) {
    case 2048: return launch_cluster_cs<2, false>(plan, a, stream);
    case 4096: return launch_cluster_cs<4, false>(plan, a, stream);
    default: return fail(PFB_ERR_UNSUPPORTED, "cluster FFT family: P must be 2048 or 4096");
    }
}

// the same cluster kernel with its local 1024-point DFT on the tensor cores
// (factored split-bf16 route for P = 2048, 4096)
pfb_status launch_fft_cluster_tc(const Plan &plan, LaunchArgs &a, cudaStream_t stream) {
    a.aux = plan.d_tw_r2;
    a.tw = static_cast<const float2 *>(plan.d_tcf);
    if (ws_cluster_supported(plan)) {  // warp-specialised cluster kernel, local DFT on the tensor cores
        switch (plan.P) {
        case 2048: return launch_ws_cluster_cs<2, true>(plan, a, stream);
        case 4096: return launch_ws_cluster_cs<4, true>(plan, a, stream);
        default: break;
        }
    }
    switch (plan.P) {
    case 2048: return launch_cluster_cs<2, true>(plan, a, stream);
    case 4096: return launch_cluster_cs<4, true>(plan, a, stream);
    default: return fail(PFB_ERR_UNSUPPORTED, "factored split-bf16 DFT on a cluster: P must be 2048 or 4096");
    }
}

}  // namespace pfb
