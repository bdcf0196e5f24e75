// Fused polyphase FIR + radix-2 Stockham FFT, FP32, for every supported
// (P, T, dtype) -- the general kernel of the FFT path.  It is the route for
// the shapes the fast family does not cover (P < 64, P > 1024, T > 16).
//
//   y[s,p] = sum_{m<T} h[m*P+p] * x[(s+m)*P+p]     (Sec. 5.2 / Sec. 4.3)
//   X[s,k] = sum_p y[s,p] exp(-2 pi i p k / P)       (Sec. 4.1)
//
// A work unit is RB = max(1, 2048/P) consecutive spectra of one stream.
// The FIR writes the unit's branch sums to shared memory; log2(P) radix-2
// Stockham passes ping-pong between two shared buffers with twiddles
// w^r = exp(-2 pi i r/P) from an FP64-built table; the last pass writes HBM.
#include "devutil.cuh"
#include "internal.h"

namespace pfb {

constexpr int kGenThreads = 256;

static inline int gen_rows(int P) { return P >= 2048 ? 1 : 2048 / P; }

template <int IN>
__global__ void __launch_bounds__(kGenThreads) k_fft_generic(const __grid_constant__ LaunchArgs a, int P, int RB) {
    using L = Loader<IN>;
    extern __shared__ __align__(16) float2 sm[];
    float2 *buf0 = sm;
    float2 *buf1 = sm + (size_t)RB * P;
    const int t = threadIdx.x;
    const int lgP = __ffs(P) - 1;
    const int64_t u0 = (int64_t)blockIdx.x * a.units_per_cta;
    const int64_t u1 = min(u0 + (int64_t)a.units_per_cta, a.nunits);
    for (int64_t u = u0; u < u1; ++u) {
        const int si = find_stream(a, u);
        const StreamDesc &d = a.s[si];
        const int64_t s0 = (u - d.unit0) * RB;
        const int nrows = (int)min((int64_t)RB, d.S - s0);
        __syncthreads();  // buffers free
        for (int idx = t; idx < nrows * P; idx += kGenThreads) {
            const int row = idx >> lgP, p = idx & (P - 1);
            float2 acc = make_float2(0.f, 0.f);
            for (int m = 0; m < d.T; ++m) {
                int64_t smp;
                const void *src = frame_source(d, s0 + row + m, P, smp);
                const float2 v = L::load1(src, smp + p, d.scale);
                const float h = __ldg(d.taps + m * P + p);
                acc.x = fmaf(h, v.x, acc.x);
                acc.y = fmaf(h, v.y, acc.y);
            }
            buf0[idx] = acc;
        }
        __syncthreads();
        float2 *in = buf0, *out = buf1;
        const int half = P >> 1;
        for (int Ns = 1; Ns < P; Ns <<= 1) {
            const bool last = (Ns << 1) == P;
            for (int idx = t; idx < nrows * half; idx += kGenThreads) {
                const int row = idx / half, j = idx - row * half;
                const int jj = j & (Ns - 1);
                const float2 x0 = in[row * P + j];
                const float2 x1 = cmul(in[row * P + j + half], a.tw[jj * (P / (2 * Ns))]);
                const int base = ((j - jj) << 1) + jj;
                if (last) {
                    float2 *o = d.out + (s0 + row) * d.ldo;
                    store_cs(o + base, cadd(x0, x1));
                    store_cs(o + base + Ns, csub(x0, x1));
                } else {
                    out[row * P + base] = cadd(x0, x1);
                    out[row * P + base + Ns] = csub(x0, x1);
                }
            }
            __syncthreads();
            float2 *tmp = in;
            in = out;
            out = tmp;
        }
    }
}

int64_t generic_units(int P, int64_t S) {
    const int RB = gen_rows(P);
    return (S + RB - 1) / RB;
}

template <int IN>
static pfb_status launch_gen_k(const Plan &plan, LaunchArgs &a, cudaStream_t stream) {
    const int P = plan.P, RB = gen_rows(P);
    const size_t smem = 2 * (size_t)RB * P * sizeof(float2);
    auto k = k_fft_generic<IN>;
    static int grid_cap = 0;
    if (grid_cap == 0) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024);
        if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(k_fft_generic)");
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        grid_cap = sms * 4;
    }
    int64_t grid = a.nunits < grid_cap ? a.nunits : grid_cap;
    if (grid < 1) return PFB_OK;
    a.units_per_cta = (int32_t)((a.nunits + grid - 1) / grid);
    grid = (a.nunits + a.units_per_cta - 1) / a.units_per_cta;
    a.tw = plan.d_tw_r2;
    k<<<(unsigned)grid, kGenThreads, smem, stream>>>(a, P, RB);
    g_launches++;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "launch k_fft_generic");
    return PFB_OK;
}

pfb_status launch_fft_generic(const Plan &plan, LaunchArgs &a, cudaStream_t stream) {
    switch (plan.in_dtype) {
    case PFB_IN_C64: return launch_gen_k<PFB_IN_C64>(plan, a, stream);
    case PFB_IN_R32: return launch_gen_k<PFB_IN_R32>(plan, a, stream);
    case PFB_IN_CI8: return launch_gen_k<PFB_IN_CI8>(plan, a, stream);
    default: return fail(PFB_ERR_INVALID, "bad dtype");
    }
}

}  // namespace pfb
