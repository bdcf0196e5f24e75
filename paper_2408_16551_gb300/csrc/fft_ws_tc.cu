// Split-bf16 DFT on the tensor cores in factored (four-step) form (variant 1
// of the split-bf16 family).  P = 1024 = 32 x 32: the warp-specialised FIR
// front end of fft_ws.cuh feeding two 32-point DFT-matrix products (Sec. 4.1
// DFT as a matrix product, split into bf16 hi/lo terms).  P = 2048, 4096: the
// cluster kernel (fft_cluster.cuh) with its local 1024-point DFT done the same
// way after the cross-CTA radix-CS step.  Executed tensor work is
// 2 x 3 x 8 x 32 = 1536 bf16 flop per sample instead of 24 P for the dense
// DFT-matrix product, and the FIR runs once per spectrum.
#include "fft_fast.cuh"  // ypad and the warp-specialised kernel (fft_ws.cuh)

namespace pfb {

// P = 1024: the warp-specialised streaming kernel (T must equal a compiled tap
// count); P = 2048, 4096: the cluster kernel (any T <= 16, taps zero-padded)
bool tcf_supported(const Plan &plan) {
    if (plan.P == 1024) return plan.T == plan.TT && plan.TT <= 16;
    return (plan.P == 2048 || plan.P == 4096) && plan.T <= 16;
}

pfb_status launch_fft_cluster_tc(const Plan &plan, LaunchArgs &a, cudaStream_t stream);

// tables: B_hi, B_lo (64 x 64 bf16 each, K-major core-matrix tiles, K = 2 n1 + c_in,
// N = 2 k1 + c_out, real block form of w_32^(n1 k1)), then w_1024^(k1 n2) as [k1][n2]
__global__ void gen_tcf_kernel(__nv_bfloat16 *Bhi, __nv_bfloat16 *Blo, float2 *tw) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < 64 * 64) {
        const int cm = i / 64, within = i % 64;
        const int n = (cm / 8) * 8 + within / 8, k = (cm % 8) * 8 + within % 8;
        const int k1 = n >> 1, c = n & 1, n1 = k >> 1, cin = k & 1;
        double sv, cv;
        sincospi(2.0 * (double)((n1 * k1) % 32) / 32.0, &sv, &cv);
        const double fr = cv, fi = -sv;  // w_32^(n1 k1) = fr + i fi
        const double v = cin == 0 ? (c == 0 ? fr : fi) : (c == 0 ? -fi : fr);
        const __nv_bfloat16 hi = __double2bfloat16(v);
        Bhi[i] = hi;
        Blo[i] = __double2bfloat16(v - (double)__bfloat162float(hi));
    } else if (i < 64 * 64 + 32 * 32) {
        const int t = i - 64 * 64, k1 = t / 32, n2 = t % 32;
        double sv, cv;
        sincospi(2.0 * (double)((k1 * n2) % 1024) / 1024.0, &sv, &cv);
        tw[t] = make_float2((float)cv, (float)-sv);
    }
}

pfb_status build_tcf_table(Plan &plan) {
    constexpr size_t bytes = 2 * 64 * 64 * 2 + 32 * 32 * 8;
    PFB_CUDA_TRY(cudaMalloc(&plan.d_tcf, bytes));
    uint8_t *base = static_cast<uint8_t *>(plan.d_tcf);
    __nv_bfloat16 *bhi = reinterpret_cast<__nv_bfloat16 *>(base);
    gen_tcf_kernel<<<(64 * 64 + 32 * 32 + 255) / 256, 256>>>(bhi, bhi + 64 * 64,
                                                              reinterpret_cast<float2 *>(base + 2 * 64 * 64 * 2));
    g_launches++;
    PFB_CUDA_TRY(cudaGetLastError());
    return PFB_OK;
}

pfb_status launch_gemm_bf16x3_tcf(const Plan &plan, LaunchArgs &a, cudaStream_t stream) {
    if (!tcf_supported(plan))
        return fail(PFB_ERR_UNSUPPORTED, "factored split-bf16 DFT needs P = 1024 with T in {4, 8, 16}, or P = 2048, 4096");
    if (plan.P != 1024) return launch_fft_cluster_tc(plan, a, stream);
    for (int i = 0; i < a.nstreams; ++i)
        if (a.s[i].T != plan.TT) return fail(PFB_ERR_UNSUPPORTED, "factored split-bf16 DFT: T mismatch");
    a.aux = plan.d_tcf;
    switch (plan.in_dtype * 100 + plan.TT) {
    case PFB_IN_C64 * 100 + 4: return launch_fft_ws_k<1024, 4, PFB_IN_C64, true>(a, stream);
    case PFB_IN_C64 * 100 + 8: return launch_fft_ws_k<1024, 8, PFB_IN_C64, true>(a, stream);
    case PFB_IN_C64 * 100 + 16: return launch_fft_ws_k<1024, 16, PFB_IN_C64, true>(a, stream);
    case PFB_IN_R32 * 100 + 4: return launch_fft_ws_k<1024, 4, PFB_IN_R32, true>(a, stream);
    case PFB_IN_R32 * 100 + 8: return launch_fft_ws_k<1024, 8, PFB_IN_R32, true>(a, stream);
    case PFB_IN_R32 * 100 + 16: return launch_fft_ws_k<1024, 16, PFB_IN_R32, true>(a, stream);
    case PFB_IN_CI8 * 100 + 4: return launch_fft_ws_k<1024, 4, PFB_IN_CI8, true>(a, stream);
    case PFB_IN_CI8 * 100 + 8: return launch_fft_ws_k<1024, 8, PFB_IN_CI8, true>(a, stream);
    case PFB_IN_CI8 * 100 + 16: return launch_fft_ws_k<1024, 16, PFB_IN_CI8, true>(a, stream);
    default: return fail(PFB_ERR_UNSUPPORTED, "factored split-bf16 DFT: no kernel for this T/dtype");
    }
}

}  // namespace pfb
