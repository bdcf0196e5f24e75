// Fused polyphase FIR + radix-16 Stockham FFT, FP32 (fast FFT family).
//
// Computes, for each work unit of SB consecutive spectra of one stream,
//   y[s,p] = sum_{m<T} h[m*P+p] * x[(s+m)*P+p]        (Sec. 5.2, FIR per branch,
//                                                       Sec. 4.3 correlation form)
//   X[s,k] = sum_p y[s,p] exp(-2 pi i p k / P)          (Sec. 4.1, the DFT)
// with the branch sums y kept in shared memory (they never go back to HBM).
//
// Mapping (P in [64, 1024], T <= 16 zero-extended to TT in {4,8,16}):
//   - one CTA of NT = P/NB threads, NB in {2, 4} consecutive branches per
//     thread, SB = 16/NB spectra per unit; the thread's NB*TT fp32 taps stay
//     in registers while it works on a stream;
//   - the FIR of a unit reads SB+TT-1 frames, one 16/32-byte vector load per
//     frame per thread (coalesced, read-only path), each load reused by up to
//     SB spectra in registers; interior units take an unguarded path whose
//     addresses are one base pointer plus compile-time offsets;
//   - the SB rows of branch sums go to shared memory (one pad slot every 16
//     entries: every pass is bank-conflict free), then an in-place Stockham
//     autosort FFT runs pass by pass: radix 16 first, one final radix in
//     {2,4,8,16}; each thread carries 16 complex values per pass; shared and
//     twiddle addresses are a per-thread base plus compile-time offsets;
//     twiddles come from a table built in FP64 at plan time;
//   - the last pass stores natural-order bins straight from registers with
//     streaming 8-byte stores, coalesced across the warp;
//   - a CTA walks a contiguous range of units (persistent grid sized to the
//     resident capacity); one thread issues an L2 bulk prefetch of the
//     frames the unit after next will need.
#pragma once

#include "devutil.cuh"
#include "fftplan.h"
#include "internal.h"

namespace pfb {

template <int G>
__device__ __forceinline__ int ypad(int i) { return i + i / G; }

}  // namespace pfb

#include "fft_ws.cuh"

namespace pfb {

template <int P, int NB, int SB, int MR>
struct FastCfg {
    static constexpr int NT = P / NB;         // threads
    static constexpr int V = SB * NB;         // complex values per thread per FFT pass
    static constexpr int G = MR;              // shared-memory padding: one slot every G entries
    static constexpr int YROW = P + P / G;
    static constexpr int NTW = fft_tw_entries(P, MR);
    static constexpr size_t SMEM = (size_t)(SB * YROW + (NTW > 0 ? NTW : 1)) * sizeof(float2);
    static constexpr int MINB = NT >= 512 ? 1 : 512 / NT;
    static_assert(V % MR == 0 && V >= MR, "a thread carries whole butterflies");
};

// ---------------------------------------------------------------------------
// loads of NB consecutive branches of one frame
// ---------------------------------------------------------------------------
template <int IN, int NB>
__device__ __forceinline__ void load_nb(const void *base, int64_t idx, float s, float2 (&v)[NB]) {
    if constexpr (IN == PFB_IN_C64) {
        const float4 *p = reinterpret_cast<const float4 *>(static_cast<const float2 *>(base) + idx);
#pragma unroll
        for (int k = 0; k < NB / 2; ++k) {
            float4 w = __ldg(p + k);
            v[2 * k] = make_float2(w.x, w.y);
            v[2 * k + 1] = make_float2(w.z, w.w);
        }
    } else if constexpr (IN == PFB_IN_R32) {
        if constexpr (NB == 4) {
            float4 w = __ldg(reinterpret_cast<const float4 *>(static_cast<const float *>(base) + idx));
            v[0] = make_float2(w.x, 0.f); v[1] = make_float2(w.y, 0.f);
            v[2] = make_float2(w.z, 0.f); v[3] = make_float2(w.w, 0.f);
        } else {
            float2 w = __ldg(reinterpret_cast<const float2 *>(static_cast<const float *>(base) + idx));
            v[0] = make_float2(w.x, 0.f); v[1] = make_float2(w.y, 0.f);
        }
    } else {
        const int8_t *b8 = static_cast<const int8_t *>(base) + 2 * idx;
        if constexpr (NB == 4) {
            int2 w = __ldg(reinterpret_cast<const int2 *>(b8));
            char4 a = *reinterpret_cast<char4 *>(&w.x), c = *reinterpret_cast<char4 *>(&w.y);
            v[0] = make_float2((float)a.x * s, (float)a.y * s); v[1] = make_float2((float)a.z * s, (float)a.w * s);
            v[2] = make_float2((float)c.x * s, (float)c.y * s); v[3] = make_float2((float)c.z * s, (float)c.w * s);
        } else {
            char4 a = __ldg(reinterpret_cast<const char4 *>(b8));
            v[0] = make_float2((float)a.x * s, (float)a.y * s); v[1] = make_float2((float)a.z * s, (float)a.w * s);
        }
    }
}

// ---------------------------------------------------------------------------
// one Stockham pass
// ---------------------------------------------------------------------------
template <int P, int NB, int SB, int MR, bool PK, int PASS>
__device__ __forceinline__ void fft_fast_pass(float2 *Y, const float2 *tw, float2 *out_row0, int nrows,
                                              int64_t ldo = P) {
    using C = FastCfg<P, NB, SB, MR>;
    constexpr int R = fft_radix(P, PASS, MR);
    constexpr int NS = fft_ns(P, PASS, MR);
    constexpr int NT = C::NT;
    constexpr int YROW = C::YROW;
    constexpr int G = C::G;
    constexpr bool LAST = (PASS == fft_npasses(P, MR) - 1);
    constexpr int PER = (SB * P / R) / NT;  // butterflies per thread
    constexpr int STRIDE = P / R;
    static_assert(PER * R == C::V, "each thread carries V values per pass");
    const float2 *twp = tw + fft_tw_offset(P, PASS, MR);
    const int t = threadIdx.x;

    // butterfly q of this thread: b = t + q*NT -> (row, j); both are a
    // per-thread base plus a compile-time offset
    auto rowj = [&](int q, int &row, int &j) {
        if constexpr (NT >= STRIDE) {
            row = t / STRIDE + q * (NT / STRIDE);
            j = t % STRIDE;
        } else {
            row = q / (STRIDE / NT);
            j = t + (q % (STRIDE / NT)) * NT;
        }
    };

    float2 v[PER][R];
#pragma unroll
    for (int q = 0; q < PER; ++q) {
        int row, j;
        rowj(q, row, j);
        const float2 *src = Y + row * YROW;
        if constexpr (STRIDE % G == 0) {
            src += ypad<G>(j);
#pragma unroll
            for (int r = 0; r < R; ++r) v[q][r] = src[r * (STRIDE + STRIDE / G)];
        } else {
#pragma unroll
            for (int r = 0; r < R; ++r) v[q][r] = src[ypad<G>(j + r * STRIDE)];
        }
        if constexpr (NS > 1) {
            const float2 *w = twp + (j % NS) * (R - 1);
#pragma unroll
            for (int r = 1; r < R; ++r) v[q][r] = cmul(v[q][r], w[r - 1]);
        }
        dft_reg<R, PK>(v[q]);
    }
    if constexpr (!LAST) {
        __syncthreads();
#pragma unroll
        for (int q = 0; q < PER; ++q) {
            int row, j;
            rowj(q, row, j);
            float2 *dst = Y + row * YROW;
            if constexpr (NS == 1) {
                static_assert(R == G, "the first pass has the padding radix");
                dst += (G + 1) * j;  // ypad(G j + r) = (G+1) j + r
#pragma unroll
                for (int r = 0; r < R; ++r) dst[r] = v[q][r];
            } else {
                static_assert(NS % G == 0, "Ns is a multiple of the padding after the first pass");
                dst += ypad<G>((j / NS) * NS * R + (j % NS));
#pragma unroll
                for (int r = 0; r < R; ++r) dst[r * (NS + NS / G)] = v[q][r];
            }
        }
        __syncthreads();
    } else {
        // NS * R == P: bin index j + r*NS, natural order
        const bool full = (nrows == SB);
#pragma unroll
        for (int q = 0; q < PER; ++q) {
            int row, j;
            rowj(q, row, j);
            if (full || row < nrows) {
                float2 *o = out_row0 + row * ldo + j;
#pragma unroll
                for (int r = 0; r < R; ++r) store_cs(o + r * NS, v[q][r]);
            }
        }
    }
}

template <int P, int NB, int SB, int MR, bool PK, int PASS>
__device__ __forceinline__ void fft_fast_passes(float2 *Y, const float2 *tw, float2 *out_row0, int nrows, int64_t ldo) {
    fft_fast_pass<P, NB, SB, MR, PK, PASS>(Y, tw, out_row0, nrows, ldo);
    if constexpr (PASS + 1 < fft_npasses(P, MR))
        fft_fast_passes<P, NB, SB, MR, PK, PASS + 1>(Y, tw, out_row0, nrows, ldo);
}

// acc[j][b] += h[m][b] * v[b] for the spectra j that frame i feeds
template <int TT, int SB, int NB, bool REAL, bool PK>
__device__ __forceinline__ void fir_frame(int i, const float (&h)[TT][NB], const float2 (&v)[NB],
                                          float2 (&acc)[SB][NB]) {
#pragma unroll
    for (int j = 0; j < SB; ++j) {
        const int m = i - j;
        if (m >= 0 && m < TT) {
#pragma unroll
            for (int b = 0; b < NB; ++b) {
                if constexpr (REAL) {
                    acc[j][b].x = fmaf(h[m][b], v[b].x, acc[j][b].x);
                } else if constexpr (PK) {
                    acc[j][b] = fma2(make_float2(h[m][b], h[m][b]), v[b], acc[j][b]);
                } else {
                    acc[j][b].x = fmaf(h[m][b], v[b].x, acc[j][b].x);
                    acc[j][b].y = fmaf(h[m][b], v[b].y, acc[j][b].y);
                }
            }
        }
    }
}

template <int P, int TT, int IN, int NB, int SB, int MR, bool PK>
__global__ void __launch_bounds__(P / NB, (FastCfg<P, NB, SB, MR>::MINB)) k_fft_fast(const __grid_constant__ LaunchArgs a) {
    using C = FastCfg<P, NB, SB, MR>;
    constexpr int NT = C::NT, YROW = C::YROW;
    constexpr int ESZ = IN == PFB_IN_C64 ? 8 : (IN == PFB_IN_R32 ? 4 : 2);
    constexpr bool REAL = (IN == PFB_IN_R32);
    extern __shared__ __align__(16) float2 sm[];
    float2 *Y = sm;
    float2 *tw = sm + SB * YROW;
    const int t = threadIdx.x;
    const int q0 = NB * t;  // first branch of this thread
    for (int i = t; i < C::NTW; i += NT) tw[i] = a.tw[i];

    const int64_t u0 = (int64_t)blockIdx.x * a.units_per_cta;
    const int64_t u1 = min(u0 + (int64_t)a.units_per_cta, a.nunits);
    int cur = -1;
    float h[TT][NB];
    for (int64_t u = u0; u < u1; ++u) {
        const int si = find_stream(a, u);
        const StreamDesc &d = a.s[si];
        if (si != cur) {
            cur = si;
#pragma unroll
            for (int m = 0; m < TT; ++m)
#pragma unroll
                for (int b = 0; b < NB; ++b) h[m][b] = __ldg(d.taps + m * P + q0 + b);
        }
        const int64_t s0 = (u - d.unit0) * SB;
        const int nrows = (int)min((int64_t)SB, d.S - s0);

        // L2 prefetch of the frames first needed by the unit after next
        if (t == 0) {
            const int64_t f0 = s0 + 2 * SB + TT - 1;
            const int64_t f1 = min(f0 + SB, d.n_frames);
            if (f0 >= d.n_state && f1 > f0) {
                const char *p = static_cast<const char *>(d.in) + (f0 - d.n_state) * (int64_t)P * ESZ;
                asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"((int)((f1 - f0) * P * ESZ))
                             : "memory");
            }
        }

        // ---- polyphase FIR: SB spectra x NB branches, taps in registers ----
        float2 acc[SB][NB];
#pragma unroll
        for (int j = 0; j < SB; ++j)
#pragma unroll
            for (int b = 0; b < NB; ++b) acc[j][b] = make_float2(0.f, 0.f);
        const bool interior = (s0 >= d.n_state) && (s0 + SB + TT - 1 <= d.n_frames);
        if (interior) {
            const char *base = static_cast<const char *>(d.in) + ((s0 - d.n_state) * P + q0) * ESZ;
#pragma unroll
            for (int i = 0; i < SB + TT - 1; ++i) {
                float2 v[NB];
                load_nb<IN, NB>(base + (int64_t)i * P * ESZ, 0, d.scale, v);
                fir_frame<TT, SB, NB, REAL, PK>(i, h, v, acc);
            }
        } else {
#pragma unroll
            for (int i = 0; i < SB + TT - 1; ++i) {
                const int64_t f = s0 + i;
                float2 v[NB];
#pragma unroll
                for (int b = 0; b < NB; ++b) v[b] = make_float2(0.f, 0.f);
                if (f < d.n_frames) {
                    int64_t smp;
                    const void *src = frame_source(d, f, P, smp);
                    load_nb<IN, NB>(src, smp + q0, d.scale, v);
                }
                fir_frame<TT, SB, NB, REAL, PK>(i, h, v, acc);
            }
        }
        __syncthreads();  // previous unit's last pass has finished reading Y
        const int c = ypad<C::G>(q0);
#pragma unroll
        for (int j = 0; j < SB; ++j)
#pragma unroll
            for (int b = 0; b < NB; ++b) Y[j * YROW + c + b] = acc[j][b];
        __syncthreads();
        // ---- P-point FFT of the SB rows, last pass stores to HBM ----
        fft_fast_passes<P, NB, SB, MR, PK, 0>(Y, tw, d.out + s0 * d.ldo, nrows, d.ldo);
    }
}

template <int P>
pfb_status launch_fft_fast_p(const Plan &plan, LaunchArgs &a, cudaStream_t stream);

// Launch one instantiation.  Each P is compiled in its own translation unit
// (fft_fast_p*.cu) so the build runs them in parallel.
template <int P, int TT, int IN, int NB, int SB, int MR, bool PK>
static pfb_status launch_fft_fast_k(LaunchArgs &a, cudaStream_t stream) {
    using C = FastCfg<P, NB, SB, MR>;
    auto k = k_fft_fast<P, TT, IN, NB, SB, MR, PK>;
    constexpr size_t smem = C::SMEM;
    static int grid_cap = 0;  // resident CTAs (computed once per instantiation)
    if (grid_cap == 0) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(k_fft_fast)");
        int per_sm = 0, dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, C::NT, smem);
        if (e != cudaSuccess || per_sm < 1) return cuda_fail(e, "occupancy(k_fft_fast)");
        grid_cap = per_sm * sms;
    }
    int64_t grid = a.nunits < grid_cap ? a.nunits : grid_cap;
    if (grid < 1) return PFB_OK;
    a.units_per_cta = (int32_t)((a.nunits + grid - 1) / grid);
    grid = (a.nunits + a.units_per_cta - 1) / a.units_per_cta;
    k<<<(unsigned)grid, C::NT, smem, stream>>>(a);
    g_launches++;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "launch k_fft_fast");
    return PFB_OK;
}

// variants (tile shapes the autotuner chooses from):
//   0: 2 branches/thread,  8 spectra/unit, radix 16, scalar fp32
//   1: 2 branches/thread,  8 spectra/unit, radix 16, packed fp32x2
//   2: 4 branches/thread,  4 spectra/unit, radix 16, scalar fp32
//   3: 4 branches/thread,  4 spectra/unit, radix 16, packed fp32x2
//   4: 2 branches/thread, 16 spectra/unit, radix 32, packed fp32x2
//   5: warp-specialised, TMA-fed ring, streaming FIR state (fft_ws.cuh);
//      P >= 128 and T equal to the compiled tap count
template <int P, int TT, int IN>
static pfb_status launch_fft_fast_v(int variant, LaunchArgs &a, cudaStream_t stream) {
    switch (variant) {
    case 0: return launch_fft_fast_k<P, TT, IN, 2, 8, 16, false>(a, stream);
    case 1: return launch_fft_fast_k<P, TT, IN, 2, 8, 16, true>(a, stream);
    case 2: return launch_fft_fast_k<P, TT, IN, 4, 4, 16, false>(a, stream);
    case 3: return launch_fft_fast_k<P, TT, IN, 4, 4, 16, true>(a, stream);
    case 4: return launch_fft_fast_k<P, TT, IN, 2, 16, 32, true>(a, stream);
    default:
        if constexpr (P >= 128) {
            for (int i = 0; i < a.nstreams; ++i)
                if (a.s[i].T != TT) return fail(PFB_ERR_UNSUPPORTED, "variant 5 needs T in {4, 8, 16}");
            return launch_fft_ws_k<P, TT, IN>(a, stream);
        } else {
            return fail(PFB_ERR_UNSUPPORTED, "variant 5 needs P >= 128");
        }
    }
}

#define PFB_DEFINE_FFT_FAST_P(PV)                                                                          \
    template <>                                                                                            \
    pfb_status launch_fft_fast_p<PV>(const Plan &plan, LaunchArgs &a, cudaStream_t stream) {               \
        const int v = plan.variant;                                                                        \
        a.tw = (v == 4) ? plan.d_tw32 : plan.d_tw;                                                         \
        a.aux = plan.d_tw_r2;                                                                              \
        switch (plan.in_dtype * 100 + plan.TT) {                                                           \
        case PFB_IN_C64 * 100 + 4: return launch_fft_fast_v<PV, 4, PFB_IN_C64>(v, a, stream);              \
        case PFB_IN_C64 * 100 + 8: return launch_fft_fast_v<PV, 8, PFB_IN_C64>(v, a, stream);              \
        case PFB_IN_C64 * 100 + 16: return launch_fft_fast_v<PV, 16, PFB_IN_C64>(v, a, stream);            \
        case PFB_IN_R32 * 100 + 4: return launch_fft_fast_v<PV, 4, PFB_IN_R32>(v, a, stream);              \
        case PFB_IN_R32 * 100 + 8: return launch_fft_fast_v<PV, 8, PFB_IN_R32>(v, a, stream);              \
        case PFB_IN_R32 * 100 + 16: return launch_fft_fast_v<PV, 16, PFB_IN_R32>(v, a, stream);            \
        case PFB_IN_CI8 * 100 + 4: return launch_fft_fast_v<PV, 4, PFB_IN_CI8>(v, a, stream);              \
        case PFB_IN_CI8 * 100 + 8: return launch_fft_fast_v<PV, 8, PFB_IN_CI8>(v, a, stream);              \
        case PFB_IN_CI8 * 100 + 16: return launch_fft_fast_v<PV, 16, PFB_IN_CI8>(v, a, stream);            \
        default: return fail(PFB_ERR_UNSUPPORTED, "fast FFT family: no kernel for this T/dtype");          \
        }                                                                                                  \
    }

}  // namespace pfb
