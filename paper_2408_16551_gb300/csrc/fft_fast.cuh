// Fused polyphase FIR + radix-16 Stockham FFT, FP32 (fast FFT family).
//
// Computes, for each work unit of kSB consecutive spectra of one stream,
//   y[s,p] = sum_{m<T} h[m*P+p] * x[(s+m)*P+p]        (Sec. 5.2, FIR per branch,
//                                                       Sec. 4.3 correlation form)
//   X[s,k] = sum_p y[s,p] exp(-2 pi i p k / P)          (Sec. 4.1, the DFT)
// with the branch sums y kept in shared memory (they never go back to HBM).
//
// Mapping (P in [64, 1024], T <= 16 padded with zero taps to TT in {4,8,16}):
//   - one CTA of P/2 threads; thread t owns the branch pair (2t, 2t+1) and
//     keeps its 2*TT fp32 taps in registers for as long as it stays on a stream;
//   - the FIR of a unit reads kSB+TT-1 frames, one 16-byte (C64) load per
//     frame per thread: coalesced, read-only path, each load reused by up to
//     kSB spectra in registers (the TT-1 frame halo is re-read from L1/L2);
//   - the kSB rows of branch sums go to shared memory (rows padded by one
//     slot every 16 entries: all passes are bank-conflict free), then an
//     in-place Stockham autosort FFT runs pass by pass: radix 16 first, one
//     final radix in {2,4,8,16}; each thread carries 16 complex values per
//     pass, twiddles come from a table built in FP64 at plan time;
//   - the last pass stores natural-order bins straight from registers with
//     streaming 8-byte stores, coalesced across the warp.
// A CTA walks a contiguous range of work units (persistent grid sized to the
// resident capacity), so consecutive units reuse their frames from L1.
#pragma once

#include "devutil.cuh"
#include "fftplan.h"
#include "internal.h"

namespace pfb {

constexpr int kSB = 8;  // spectra per work unit (FFT batch)

template <int P>
struct FastCfg {
    static constexpr int NT = P / 2;
    static constexpr int YROW = P + P / 16;
    static constexpr int NTW = fft_tw_entries(P);
    static constexpr size_t SMEM = (size_t)(kSB * YROW + (NTW > 0 ? NTW : 1)) * sizeof(float2);
};

__device__ __forceinline__ int ypad(int i) { return i + (i >> 4); }

template <int P, int PASS>
__device__ __forceinline__ void fft_fast_pass(float2 *Y, const float2 *tw, float2 *out_row0, int nrows) {
    constexpr int R = fft_radix(P, PASS);
    constexpr int NS = fft_ns(P, PASS);
    constexpr int NT = FastCfg<P>::NT;
    constexpr int YROW = FastCfg<P>::YROW;
    constexpr bool LAST = (PASS == fft_npasses(P) - 1);
    constexpr int PER = (kSB * P / R) / NT;  // butterflies per thread (16 / R)
    constexpr int STRIDE = P / R;
    static_assert(PER * R == 16, "each thread carries 16 values per pass");
    const float2 *twp = tw + fft_tw_offset(P, PASS);

    float2 v[PER][R];
#pragma unroll
    for (int q = 0; q < PER; ++q) {
        const int b = threadIdx.x + q * NT;
        const int row = b / STRIDE, j = b % STRIDE;
#pragma unroll
        for (int r = 0; r < R; ++r) v[q][r] = Y[row * YROW + ypad(j + r * STRIDE)];
        if (NS > 1) {
            const int jj = j % NS;
#pragma unroll
            for (int r = 1; r < R; ++r) v[q][r] = cmul(v[q][r], twp[jj * (R - 1) + r - 1]);
        }
        dft_reg<R>(v[q]);
    }
    if (!LAST) {
        __syncthreads();
#pragma unroll
        for (int q = 0; q < PER; ++q) {
            const int b = threadIdx.x + q * NT;
            const int row = b / STRIDE, j = b % STRIDE;
            const int base = (j / NS) * NS * R + (j % NS);
#pragma unroll
            for (int r = 0; r < R; ++r) Y[row * YROW + ypad(base + r * NS)] = v[q][r];
        }
        __syncthreads();
    } else {
        // NS * R == P: bin index j + r*NS, natural order
#pragma unroll
        for (int q = 0; q < PER; ++q) {
            const int b = threadIdx.x + q * NT;
            const int row = b / STRIDE, j = b % STRIDE;
            if (row < nrows) {
                float2 *o = out_row0 + (int64_t)row * P + j;
#pragma unroll
                for (int r = 0; r < R; ++r) store_cs(o + r * NS, v[q][r]);
            }
        }
    }
}

template <int P, int PASS>
__device__ __forceinline__ void fft_fast_passes(float2 *Y, const float2 *tw, float2 *out_row0, int nrows) {
    fft_fast_pass<P, PASS>(Y, tw, out_row0, nrows);
    if constexpr (PASS + 1 < fft_npasses(P)) fft_fast_passes<P, PASS + 1>(Y, tw, out_row0, nrows);
}

template <int P, int TT, int IN>
__global__ void __launch_bounds__(P / 2) k_fft_fast(const __grid_constant__ LaunchArgs a) {
    using L = Loader<IN>;
    constexpr int NT = FastCfg<P>::NT;
    constexpr int YROW = FastCfg<P>::YROW;
    extern __shared__ __align__(16) float2 sm[];
    float2 *Y = sm;
    float2 *tw = sm + kSB * YROW;
    const int t = threadIdx.x;
    for (int i = t; i < FastCfg<P>::NTW; i += NT) tw[i] = a.tw[i];

    const int64_t u0 = (int64_t)blockIdx.x * a.units_per_cta;
    const int64_t u1 = min(u0 + (int64_t)a.units_per_cta, a.nunits);
    int cur = -1;
    float h0[TT], h1[TT];
    for (int64_t u = u0; u < u1; ++u) {
        const int si = find_stream(a, u);
        const StreamDesc &d = a.s[si];
        if (si != cur) {
            cur = si;
#pragma unroll
            for (int m = 0; m < TT; ++m) {
                float2 hv = __ldg(reinterpret_cast<const float2 *>(d.taps + m * P + 2 * t));
                h0[m] = hv.x;
                h1[m] = hv.y;
            }
        }
        const int64_t s0 = (u - d.unit0) * kSB;
        const int nrows = (int)min((int64_t)kSB, d.S - s0);

        // ---- polyphase FIR: kSB spectra x 2 branches, taps in registers ----
        float2 acc0[kSB], acc1[kSB];
#pragma unroll
        for (int j = 0; j < kSB; ++j) acc0[j] = acc1[j] = make_float2(0.f, 0.f);
#pragma unroll
        for (int i = 0; i < kSB + TT - 1; ++i) {
            const int64_t f = s0 + i;
            float2 v0 = make_float2(0.f, 0.f), v1 = v0;
            if (f < d.n_frames) {
                int64_t smp;
                const void *src = frame_source(d, f, P, smp);
                L::load2(src, smp + 2 * t, d.scale, v0, v1);
            }
#pragma unroll
            for (int j = 0; j < kSB; ++j) {
                const int m = i - j;
                if (m >= 0 && m < TT) {
                    acc0[j].x = fmaf(h0[m], v0.x, acc0[j].x);
                    acc1[j].x = fmaf(h1[m], v1.x, acc1[j].x);
                    if (!L::kReal) {
                        acc0[j].y = fmaf(h0[m], v0.y, acc0[j].y);
                        acc1[j].y = fmaf(h1[m], v1.y, acc1[j].y);
                    }
                }
            }
        }
        __syncthreads();  // previous unit's last pass has finished reading Y
        const int c = ypad(2 * t);
#pragma unroll
        for (int j = 0; j < kSB; ++j) {
            Y[j * YROW + c] = acc0[j];
            Y[j * YROW + c + 1] = acc1[j];
        }
        __syncthreads();
        // ---- P-point FFT of the kSB rows, last pass stores to HBM ----
        fft_fast_passes<P, 0>(Y, tw, d.out + s0 * P, nrows);
    }
}

template <int P>
pfb_status launch_fft_fast_p(const Plan &plan, LaunchArgs &a, cudaStream_t stream);

// Dispatch on (TT, dtype) for one P; instantiated once per P in its own
// translation unit (fft_fast_p*.cu) so the build compiles them in parallel.
template <int P, int TT, int IN>
static pfb_status launch_fft_fast_k(LaunchArgs &a, cudaStream_t stream) {
    auto k = k_fft_fast<P, TT, IN>;
    constexpr size_t smem = FastCfg<P>::SMEM;
    static int grid_cap = 0;  // resident CTAs (computed once per instantiation)
    if (grid_cap == 0) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(k_fft_fast)");
        int per_sm = 0, dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, P / 2, smem);
        if (e != cudaSuccess || per_sm < 1) return cuda_fail(e, "occupancy(k_fft_fast)");
        grid_cap = per_sm * sms;
    }
    int64_t grid = a.nunits < grid_cap ? a.nunits : grid_cap;
    if (grid < 1) return PFB_OK;
    a.units_per_cta = (int32_t)((a.nunits + grid - 1) / grid);
    grid = (a.nunits + a.units_per_cta - 1) / a.units_per_cta;
    k<<<(unsigned)grid, P / 2, smem, stream>>>(a);
    g_launches++;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "launch k_fft_fast");
    return PFB_OK;
}

#define PFB_DEFINE_FFT_FAST_P(PV)                                                              \
    template <>                                                                                \
    pfb_status launch_fft_fast_p<PV>(const Plan &plan, LaunchArgs &a, cudaStream_t stream) {   \
        switch (plan.in_dtype * 100 + plan.TT) {                                               \
        case PFB_IN_C64 * 100 + 4: return launch_fft_fast_k<PV, 4, PFB_IN_C64>(a, stream);     \
        case PFB_IN_C64 * 100 + 8: return launch_fft_fast_k<PV, 8, PFB_IN_C64>(a, stream);     \
        case PFB_IN_C64 * 100 + 16: return launch_fft_fast_k<PV, 16, PFB_IN_C64>(a, stream);   \
        case PFB_IN_R32 * 100 + 4: return launch_fft_fast_k<PV, 4, PFB_IN_R32>(a, stream);     \
        case PFB_IN_R32 * 100 + 8: return launch_fft_fast_k<PV, 8, PFB_IN_R32>(a, stream);     \
        case PFB_IN_R32 * 100 + 16: return launch_fft_fast_k<PV, 16, PFB_IN_R32>(a, stream);   \
        case PFB_IN_CI8 * 100 + 4: return launch_fft_fast_k<PV, 4, PFB_IN_CI8>(a, stream);     \
        case PFB_IN_CI8 * 100 + 8: return launch_fft_fast_k<PV, 8, PFB_IN_CI8>(a, stream);     \
        case PFB_IN_CI8 * 100 + 16: return launch_fft_fast_k<PV, 16, PFB_IN_CI8>(a, stream);   \
        default: return fail(PFB_ERR_UNSUPPORTED, "fast FFT family: no kernel for this T/dtype"); \
        }                                                                                      \
    }

}  // namespace pfb
