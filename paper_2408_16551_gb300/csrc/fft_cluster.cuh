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

template <int CS, bool TC = false>
struct ClusterCfg {
    static constexpr int PL = 1024;          // branches per CTA
    static constexpr int P = CS * PL;
    static constexpr int NB = 2, SB = 8, MR = 16, G = 16;
    static constexpr int NT = PL / NB;        // 512 threads
    static constexpr int YROW = PL + PL / G;
    static constexpr int NTW = TC ? 0 : fft_tw_entries(PL, MR);
    // TC: the local PL-point DFT on the tensor cores (four-step, 32 x 32, the
    // same operand layouts as the warp-specialised kernel's TC mode)
    static constexpr int TC_P1 = 32, TC_LBO_A = 2064, TC_A2B = 8 * TC_LBO_A, TC_BTB = 64 * 64 * 2;
    static constexpr size_t OFF_A2 = (size_t)(2 * SB * YROW + NTW) * sizeof(float2);
    static constexpr size_t OFF_BT = OFF_A2 + (TC ? 2 * TC_A2B : 0);
    static constexpr size_t OFF_TWT = OFF_BT + (TC ? 2 * TC_BTB : 0);
    static constexpr size_t OFF_BAR = OFF_TWT + (TC ? TC_P1 * TC_P1 * 8 : 0);
    static constexpr size_t SMEM = OFF_BAR + (TC ? 32 : 0);
    static_assert(!TC || (OFF_A2 % 128 == 0 && OFF_BT % 128 == 0), "TC operand alignment");
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

// Local PL-point DFT of the 8 Z rows on the tensor cores (TC mode): two
// 128-row tiles of 4 spectra, each MMA 1 (32-point DFT over n1, A in TMEM),
// twiddle w_PL^(n2 k1), MMA 2 (32-point DFT over n2, A in shared memory); bin
// kk = k1 + 32 k2 goes to CTA k / PL (k = c + CS kk) as in the FFT route.
// Warp w: TMEM lane quarter q = w mod 4 (spectrum of the tile), column part
// w / 4 (8 of the 32 n1 / k1 / k2 columns).  Every wait is bounded; after a
// timeout the CTA records the error and keeps its cluster barriers.
template <class C>
__device__ __forceinline__ void cluster_tc_dft(const float2 *Z, float2 *stage, uint8_t *smem, uint32_t tmem,
                                               uint32_t mbar1, uint32_t mbar2, uint32_t &ph1, uint32_t &ph2,
                                               bool &tc_ok, cg::cluster_group &cl, int c) {
    constexpr int PL = C::PL, YROW = C::YROW, G = C::G, CS = C::P / C::PL, LBO_A = C::TC_LBO_A;
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int q = warp & 3, part = warp >> 2;
    const uint32_t trow = tmem + ((uint32_t)(32 * q) << 16);
    uint8_t *a2 = smem + C::OFF_A2;
    const uint32_t sA2 = smem_u32(a2), sBT = smem_u32(smem + C::OFF_BT);
    const float2 *twt = reinterpret_cast<const float2 *>(smem + C::OFF_TWT);
    const int a2_base = (lane >> 2) * LBO_A + (lane & 3) * 4 + (4 * q) * 128;
    auto mma_step = [&](bool step2, uint32_t bar, uint32_t &ph) {
        if (t == 0 && tc_ok) ws_tc_issue<C>(step2, tmem, sA2, sBT, bar);
        bool w = true;
        if (tc_ok) {
            w = mbar_wait(bar, ph & 1);
            ++ph;
        }
        if (__syncthreads_or(!w)) tc_ok = false;
        tc_fence_after();
    };
#pragma unroll 1
    for (int tile = 0; tile < 2; ++tile) {
        // ---- MMA 1 operand: row (q, n2 = lane), K = (n1, re/im), columns n1 in this warp's part ----
        const float2 *zr = Z + (4 * tile + q) * YROW;
        uint32_t vh[8], vl[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) split_bf16x2(zr[ypad<G>(32 * (8 * part + j) + lane)], vh[j], vl[j]);
        tmem_st<8>(trow + kTcColA1 + 8 * part, vh);
        tmem_st<8>(trow + kTcColA1 + 32 + 8 * part, vl);
        tmem_wait_st();
        tc_fence_before();
        __syncthreads();
        if (t == 0) tc_fence_after();
        mma_step(false, mbar1, ph1);
        // ---- twiddle, split, transposed store: MMA 2 operand row (q, k1), K = (n2 = lane, re/im) ----
        {
            float2 w8[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) w8[j] = twt[(8 * part + j) * C::TC_P1 + lane];
            uint32_t r[16];
            tmem_ld16(trow + kTcColD1 + 16 * part, r);
            tmem_wait_ld();
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int k1 = 8 * part + j;
                const float2 z = cmul(make_float2(__uint_as_float(r[2 * j]), __uint_as_float(r[2 * j + 1])), w8[j]);
                uint32_t hi, lo;
                split_bf16x2(z, hi, lo);
                const int off = a2_base + (k1 >> 3) * 128 + (k1 & 7) * 16;
                *reinterpret_cast<uint32_t *>(a2 + off) = hi;
                *reinterpret_cast<uint32_t *>(a2 + C::TC_A2B + off) = lo;
            }
        }
        fence_proxy_async_smem();
        tc_fence_before();
        __syncthreads();
        if (t == 0) tc_fence_after();
        mma_step(true, mbar2, ph2);
        // ---- bins kk = k1 + 32 k2 (thread k1 = lane, k2 in this warp's part) -> owner CTA ----
        {
            uint32_t r[16];
            tmem_ld16(trow + kTcColD2 + 16 * part, r);
            tmem_wait_ld();
            const int row = 4 * tile + q;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int k = c + CS * (lane + 32 * (8 * part + j));
                cl.map_shared_rank(stage, k / PL)[row * PL + (k % PL)] =
                    make_float2(__uint_as_float(r[2 * j]), __uint_as_float(r[2 * j + 1]));
            }
        }
        tc_fence_before();
    }
}

template <int CS, int TT, int IN, bool TC = false>
__global__ void __launch_bounds__(ClusterCfg<CS, TC>::NT, 1) k_fft_cluster(const __grid_constant__ LaunchArgs a) {
    using C = ClusterCfg<CS, TC>;
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
    // TC: DFT-matrix tiles and twiddles (from a.tw), TMEM, MMA barriers
    uint8_t *smem8 = reinterpret_cast<uint8_t *>(csm);
    uint64_t *tcbar = reinterpret_cast<uint64_t *>(smem8 + C::OFF_BAR);
    volatile uint32_t *tmem_slot = reinterpret_cast<volatile uint32_t *>(tcbar + 2);
    uint32_t ph1 = 0, ph2 = 0;
    bool tc_ok = true;
    if constexpr (TC) {
        const int4 *src = reinterpret_cast<const int4 *>(a.tw);
        int4 *dst = reinterpret_cast<int4 *>(smem8 + C::OFF_BT);
        constexpr int NV = (2 * C::TC_BTB + C::TC_P1 * C::TC_P1 * 8) / 16;
        for (int i = t; i < NV; i += NT) dst[i] = src[i];
        if (t == 0) {
            mbar_init(smem_u32(&tcbar[0]), 1);
            mbar_init(smem_u32(&tcbar[1]), 1);
            mbar_init_fence();
        }
        if (t < 32) tmem_alloc(smem_u32((const void *)tmem_slot), kTcCols);
        fence_proxy_async_smem();
        tc_fence_before();
    }

    const int64_t cid = blockIdx.x / CS;
    const int64_t u0 = cid * a.units_per_cta;
    const int64_t u1 = min(u0 + (int64_t)a.units_per_cta, a.nunits);
    int cur = -1;
    float h[TT][NB];
    __syncthreads();
    if constexpr (TC) tc_fence_after();
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

        // ---- 3. PL-point DFT of the local Z rows; the last step scatters ----
        if constexpr (TC) {
            cluster_tc_dft<C>(Z, Y, smem8, *tmem_slot, smem_u32(&tcbar[0]), smem_u32(&tcbar[1]), ph1, ph2, tc_ok,
                              cl, c);
        } else {
            // passes 0 .. n-2 in place in Z (the single-CTA pass code), last pass here
            fft_cluster_passes<CS, 0>(Z, tw, Y, cl, c);
        }
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
                    __stcs(reinterpret_cast<float4 *>(d.out + (s0 + row) * d.ldo + c * PL + col),
                           make_float4(x0.x, x0.y, x1.x, x1.y));
                }
            }
        }
        __syncthreads();  // staging read complete before the next unit's FIR writes Y
    }
    if constexpr (TC) {
        // a commit whose completion was not observed: let it land before TMEM is freed
        if (!tc_ok && t == 0) {
            mbar_wait(smem_u32(&tcbar[0]), (ph1 + 1) & 1);
            mbar_wait(smem_u32(&tcbar[1]), (ph2 + 1) & 1);
        }
        if (!tc_ok && t == 0) report_error(a.err, KERR_TIMEOUT);
        tc_fence_before();
        __syncthreads();
        if (t < 32) {
            tc_fence_after();
            tmem_dealloc(*tmem_slot, kTcCols);
        }
    }
}

}  // namespace pfb
