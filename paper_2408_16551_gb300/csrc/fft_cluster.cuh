// Fused polyphase FIR + FFT for P = CS * 1024 (P = 2048, 4096) on a cluster
// of CS CTAs that exchange data through distributed shared memory.
//
//   y[s,p] = sum_{m<T} h[m*P+p] * x[(s+m)*P+p]     (Sec. 5.2 / Sec. 4.3)
//   X[s,k] = sum_p y[s,p] exp(-2 pi i p k / P)       (Sec. 4.1)
//
// The branch sums of one spectrum do not fit one SM's registers and shared
// memory together with an FIR window, so CTA c of the cluster owns branches
// p = c*PL + n2 (PL = 1024) and the DFT is factored (four-step form):
//   Z_k1[n2]      = w_P^{n2 k1} * sum_{n1<CS} y[n1*PL + n2] w_CS^{n1 k1}
//   X[k1 + CS k2] = sum_{n2<PL} Z_k1[n2] w_PL^{n2 k2}
// Per work unit (SB = 8 consecutive spectra of one stream):
//   1. FIR of the CTA's branch slice into Y (shared memory), exactly as the
//      single-CTA fast kernel (2 branches per thread, taps in registers);
//   2. cluster barrier; CTA c takes n2 in its quarter, reads y[n1*PL + n2]
//      from every CTA n1 (DSMEM), does the CS-point DFT and the twiddle, and
//      writes Z_k1[n2] into CTA k1's Z buffer (DSMEM);
//   3. cluster barrier; each CTA runs the PL-point Stockham FFT of its Z rows;
//      the last pass sends bin k = k1 + CS*k2 to the CTA that owns bins
//      [o*PL, (o+1)*PL) (o = k / PL), into its staging buffer;
//   4. cluster barrier; each CTA stores its PL contiguous bins per spectrum.
// The branch sums never leave the chip.  The staging buffer aliases Y: no
// CTA writes another's staging before that CTA has passed the next unit's
// barriers, which it reaches only after its own store.
#pragma once

#include <cooperative_groups.h>

#include "fft_fast.cuh"

namespace pfb {

namespace cg = cooperative_groups;

template <int CS>
struct ClusterCfg {
    static constexpr int PL = 1024;          // branches per CTA
    static constexpr int P = CS * PL;
    static constexpr int NB = 2, SB = 8, MR = 16, G = 16;
    static constexpr int NT = PL / NB;        // 512 threads
    static constexpr int YROW = PL + PL / G;
    static constexpr int NTW = fft_tw_entries(PL, MR);
    static constexpr size_t SMEM = (size_t)(2 * SB * YROW + NTW) * sizeof(float2);
};

// w_P^r for 0 <= r < P from the radix-2 table w_P^r, r < P/2
__device__ __forceinline__ float2 tw_full(const float2 *tw_half, int r, int P) {
    if (r < P / 2) return __ldg(tw_half + r);
    const float2 w = __ldg(tw_half + (r - P / 2));
    return make_float2(-w.x, -w.y);
}

// PL-point Stockham FFT of the SB rows of Z: passes 0..n-2 in place (the
// single-CTA pass code, ending in __syncthreads), the last pass sends bin
// k = c + CS*kk (kk = natural local index) to CTA k / PL, row-major [SB][PL].
template <int CS, int PASS>
__device__ __forceinline__ void fft_cluster_passes(float2 *Z, const float2 *tw, float2 *stage, cg::cluster_group &cl,
                                                   int c) {
    using C = ClusterCfg<CS>;
    constexpr int PL = C::PL;
    constexpr int NP = fft_npasses(PL, C::MR);
    if constexpr (PASS < NP - 1) {
        fft_fast_pass<PL, C::NB, C::SB, C::MR, false, PASS>(Z, tw, nullptr, 0);
        fft_cluster_passes<CS, PASS + 1>(Z, tw, stage, cl, c);
    } else {
        constexpr int R = fft_radix(PL, PASS, C::MR);
        constexpr int NS = fft_ns(PL, PASS, C::MR);
        constexpr int STRIDE = PL / R;
        constexpr int NT = C::NT;
        constexpr int PER = (C::SB * PL / R) / NT;
        static_assert(NT >= STRIDE, "row/j split");
        const float2 *twp = tw + fft_tw_offset(PL, PASS, C::MR);
        const int t = threadIdx.x;
#pragma unroll
        for (int q = 0; q < PER; ++q) {
            const int row = t / STRIDE + q * (NT / STRIDE);
            const int j = t % STRIDE;
            float2 v[R];
            const float2 *src = Z + row * C::YROW + ypad<C::G>(j);
#pragma unroll
            for (int r = 0; r < R; ++r) v[r] = src[r * (STRIDE + STRIDE / C::G)];
            const float2 *w = twp + (j % NS) * (R - 1);
#pragma unroll
            for (int r = 1; r < R; ++r) v[r] = cmul(v[r], w[r - 1]);
            dft_reg<R, false>(v);
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int k = c + CS * (j + r * NS);
                cl.map_shared_rank(stage, k / PL)[row * PL + (k % PL)] = v[r];
            }
        }
    }
}

template <int CS, int TT, int IN>
__global__ void __launch_bounds__(ClusterCfg<CS>::NT, 1) k_fft_cluster(const __grid_constant__ LaunchArgs a) {
    using C = ClusterCfg<CS>;
    constexpr int PL = C::PL, P = C::P, NB = C::NB, SB = C::SB, NT = C::NT, YROW = C::YROW, G = C::G;
    constexpr int ESZ = IN == PFB_IN_C64 ? 8 : (IN == PFB_IN_R32 ? 4 : 2);
    constexpr bool REAL = (IN == PFB_IN_R32);
    extern __shared__ __align__(16) float2 csm[];
    float2 *Y = csm;                  // branch sums, later the staging buffer
    float2 *Z = csm + SB * YROW;      // four-step intermediate
    float2 *tw = csm + 2 * SB * YROW; // PL-point pass twiddles
    cg::cluster_group cl = cg::this_cluster();
    const int c = (int)cl.block_rank();
    const int t = threadIdx.x;
    const int q0 = NB * t;            // local branch
    for (int i = t; i < C::NTW; i += NT) tw[i] = a.tw[i];
    const float2 *tw_half = static_cast<const float2 *>(a.aux);  // w_P^r, r < P/2

    const int64_t cid = blockIdx.x / CS;
    const int64_t u0 = cid * a.units_per_cta;
    const int64_t u1 = min(u0 + (int64_t)a.units_per_cta, a.nunits);
    int cur = -1;
    float h[TT][NB];
    __syncthreads();
    for (int64_t u = u0; u < u1; ++u) {
        const int si = find_stream(a, u);
        const StreamDesc &d = a.s[si];
        if (si != cur) {
            cur = si;
#pragma unroll
            for (int m = 0; m < TT; ++m)
#pragma unroll
                for (int b = 0; b < NB; ++b) h[m][b] = __ldg(d.taps + m * P + c * PL + q0 + b);
        }
        const int64_t s0 = (u - d.unit0) * SB;
        const int nrows = (int)min((int64_t)SB, d.S - s0);

        // ---- 1. FIR of this CTA's branch slice ----
        float2 acc[SB][NB];
#pragma unroll
        for (int j = 0; j < SB; ++j)
#pragma unroll
            for (int b = 0; b < NB; ++b) acc[j][b] = make_float2(0.f, 0.f);
        const int qg = c * PL + q0;   // global branch
        const bool interior = (s0 >= d.n_state) && (s0 + SB + TT - 1 <= d.n_frames);
        if (interior) {
            const char *base = static_cast<const char *>(d.in) + ((s0 - d.n_state) * P + qg) * ESZ;
#pragma unroll
            for (int i = 0; i < SB + TT - 1; ++i) {
                float2 v[NB];
                load_nb<IN, NB>(base + (int64_t)i * P * ESZ, 0, d.scale, v);
                fir_frame<TT, SB, NB, REAL, false>(i, h, v, acc);
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
                    load_nb<IN, NB>(src, smp + qg, d.scale, v);
                }
                fir_frame<TT, SB, NB, REAL, false>(i, h, v, acc);
            }
        }
        const int yc = ypad<G>(q0);
#pragma unroll
        for (int j = 0; j < SB; ++j)
#pragma unroll
            for (int b = 0; b < NB; ++b) Y[j * YROW + yc + b] = acc[j][b];

        // ---- 2. cross-CTA CS-point DFTs and twiddles -> Z of the owner ----
        cl.sync();
        {
            constexpr int Q = PL / CS;        // n2 values per CTA
            constexpr int PER = SB * Q / NT;  // per thread
#pragma unroll 1
            for (int e = 0; e < PER; ++e) {
                const int idx = t + e * NT;
                const int row = idx / Q;
                const int n2 = c * Q + idx % Q;
                const int yi = row * YROW + ypad<G>(n2);
                float2 v[CS];
#pragma unroll
                for (int n1 = 0; n1 < CS; ++n1) v[n1] = cl.map_shared_rank(Y, n1)[yi];
                dft_reg<CS, false>(v);
#pragma unroll
                for (int k1 = 0; k1 < CS; ++k1) {
                    const float2 z = (k1 == 0) ? v[0] : cmul(v[k1], tw_full(tw_half, n2 * k1, P));
                    cl.map_shared_rank(Z, k1)[yi] = z;
                }
            }
        }
        cl.sync();

        // ---- 3. PL-point FFT of the local Z rows; the last pass scatters ----
        // passes 0 .. n-2 in place in Z (the single-CTA pass code), last pass here
        fft_cluster_passes<CS, 0>(Z, tw, Y, cl, c);
        cl.sync();

        // ---- 4. store this CTA's contiguous bins ----
        {
            constexpr int V4 = SB * PL / 2 / NT;  // float4 (two bins) per thread
#pragma unroll
            for (int e = 0; e < V4; ++e) {
                const int idx = t + e * NT;        // float4 index in [0, SB*PL/2)
                const int row = idx / (PL / 2);
                const int col = (idx % (PL / 2)) * 2;
                if (row < nrows) {
                    const float2 x0 = Y[row * PL + col], x1 = Y[row * PL + col + 1];
                    __stcs(reinterpret_cast<float4 *>(d.out + (s0 + row) * P + c * PL + col),
                           make_float4(x0.x, x0.y, x1.x, x1.y));
                }
            }
        }
        __syncthreads();  // staging read complete before the next unit's FIR writes Y
    }
}

}  // namespace pfb
