// Synthesis (inverse) filter bank, FP32, warp-specialised and fed by the TMA
// engine: the adjoint of the analysis channeliser, up to the IDFT's 1/P.
//
//   y~[s,p]   = (1/P) sum_{k<P} X[s,k] exp(+2 pi i p k / P)   (Sec. 4.2, the
//               inverse Fourier-matrix product)
//   xh[fP+p]  = sum_{m<T} h[mP+p] y~[f-m, p],  f < S + T - 1,  y~ = 0 outside
//               0 <= s < S (each branch value goes back to the T frames the
//               per-branch FIR of Sec. 5.2 took it from)
//
// P = 4Q (Q = 128 or 256).  The inverse DFT is decimated in time once,
// k = 4m + k1:
//   V_k1[t]        = sum_{m<Q} X[4m + k1] exp(+2 pi i t m / Q)       IFFT warps
//   U_k1[t]        = exp(+2 pi i t k1 / P) V_k1[t]                   FIR warps
//   y~[t + Q kk]   = (1/P) sum_{k1<4} i^(kk k1) U_k1[t]              FIR warps
// and the 1/P is folded into the taps (exact: P is a power of two).  The IFFT
// warps run the forward Stockham passes on conjugated values (V = conj(FFT(
// conj X))).  Roles:
//   producer (lane 0 of warp PRODW): 1-D bulk copies of the spectrum rows into
//       a ring of NSLOT slots;
//   IFFT warps (128 threads): batches of SB rows; pass 0 (radix 16) reads the
//       four interleaved sub-rows straight from the ring, pass 1 finishes the
//       Q-point transforms and writes V into a double-buffered batch buffer;
//   FIR warps (Q threads, branches t + Q kk): the twiddles (three complex
//       products per row; each thread's t is fixed), the radix-4 step, then the
//       synthesis FIR with the T-1 pending output frames in registers (slot
//       rotation at compile time, as in the analysis kernel); every row
//       completes one output frame, stored with coalesced streaming stores.
// A CTA owns a contiguous range of output frames [fA, fB) per stream; it
// needs spectra fA-T+1 .. fB-1 (rows outside [0, S) are zero).
#pragma once

#include "fft_fast.cuh"  // ypad, and (via fft_ws.cuh) ws_next_segment, named_bar_or

namespace pfb {

template <int P, int TT>
struct SyCfg {
    static constexpr int Q = P / 4;
    static constexpr int NB = 4;                     // branches per FIR thread: t + Q kk
    static constexpr int NFT = Q;
    static constexpr int NFIRW = NFT / 32;
    static constexpr int NIFW = 4;
    static constexpr int NIFT = NIFW * 32;
    static constexpr int PRODW = NFIRW + NIFW;
    static constexpr int NTHREADS = NFT + NIFT + 128;
    static constexpr int SB = 4;                     // spectra per IFFT batch
    static constexpr int MR = 16, G = 16;
    static constexpr int R0 = fft_radix(Q, 0, MR), R1 = fft_radix(Q, 1, MR);
    static constexpr int STRIDE0 = Q / R0, STRIDE1 = Q / R1;
    static constexpr int SROW = Q + Q / G + 8;       // pass-0 output sub-row (padded)
    static constexpr int NSLOT = 8;
    static constexpr int FB = P * 8;                 // bytes per spectrum row
    static constexpr int NTQ = fft_tw_entries(Q, MR);
    static constexpr int NTW = NTQ + 3 * Q;          // pass list, then w_P^(t k1), k1 = 1..3
    static constexpr int OFF_RING = 0;
    static constexpr int OFF_W = OFF_RING + NSLOT * FB;
    static constexpr int OFF_U = OFF_W + SB * 4 * SROW * 8;
    static constexpr int OFF_TW = OFF_U + 2 * SB * 4 * Q * 8;
    static constexpr int OFF_BAR = OFF_TW + NTW * 8;
    static constexpr int NBAR = 2 * NSLOT + 4;       // full, empty, ufull[2], uempty[2]
    static constexpr int SMEM = OFF_BAR + NBAR * 8 + 16;
    static constexpr int REG_FIR = 208, REG_IF = 72, REG_PROD = 24;
    static_assert(P == 512 || P == 1024, "P = 4Q with Q = 128 or 256");
    static_assert(fft_npasses(Q, MR) == 2 && R0 == G && STRIDE1 == 16, "two passes, radix 16 first");
    static_assert(NFT % 128 == 0, "FIR warps form whole warpgroups");
    static_assert(NFT * REG_FIR + NIFT * REG_IF + 128 * REG_PROD <= 65536, "register split");
    static_assert(SMEM <= 232448, "shared memory");
};

__device__ __forceinline__ float2 conjf2(float2 v) { return make_float2(v.x, -v.y); }

// real spectrum rows [rA, rB) of a segment of output frames [fA, fB)
__device__ __forceinline__ void sy_rows(int64_t fA, int64_t fB, int T, int64_t nrows, int64_t &rA, int64_t &rB) {
    rA = max((int64_t)0, fA - T + 1);
    rB = min(nrows, fB);
}

template <int P, int TT>
__global__ void __launch_bounds__(SyCfg<P, TT>::NTHREADS, 1) k_synth_ws(const __grid_constant__ LaunchArgs a) {
    using C = SyCfg<P, TT>;
    constexpr int Q = C::Q, NB = C::NB, SB = C::SB, NSLOT = C::NSLOT, G = C::G, SROW = C::SROW;
    extern __shared__ __align__(128) uint8_t sy_smem[];
    uint8_t *ring = sy_smem + C::OFF_RING;
    float2 *W = reinterpret_cast<float2 *>(sy_smem + C::OFF_W);
    float2 *U = reinterpret_cast<float2 *>(sy_smem + C::OFF_U);
    float2 *tw = reinterpret_cast<float2 *>(sy_smem + C::OFF_TW);
    uint64_t *bars = reinterpret_cast<uint64_t *>(sy_smem + C::OFF_BAR);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(bars + C::NBAR);
    const uint32_t full0 = smem_u32(&bars[0]), empty0 = smem_u32(&bars[NSLOT]);
    const uint32_t ufull0 = smem_u32(&bars[2 * NSLOT]), uempty0 = smem_u32(&bars[2 * NSLOT + 2]);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int i = 0; i < NSLOT; ++i) {
            mbar_init(full0 + 8 * i, 1);
            mbar_init(empty0 + 8 * i, 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(ufull0 + 8 * i, 1);
            mbar_init(uempty0 + 8 * i, C::NFIRW);
        }
        mbar_init_fence();
        *abort_flag = 0;
    }
    // twiddles from the FP64-generated table w_P^r (r < P/2): the Q-point pass
    // list, then w_P^(t k1) for t < Q, k1 = 1..3
    {
        const float2 *tw_half = static_cast<const float2 *>(a.aux);
        auto wP = [&](int r) {
            r %= P;
            const float2 w = __ldg(tw_half + (r < P / 2 ? r : r - P / 2));
            return r < P / 2 ? w : make_float2(-w.x, -w.y);
        };
        for (int i = threadIdx.x; i < C::NTQ; i += C::NTHREADS) {
            // the only pass with Ns > 1 is pass 1 (Ns = 16, R = R1)
            const int jj = i / (C::R1 - 1), r = i % (C::R1 - 1) + 1;
            tw[i] = wP(r * jj * (P / (16 * C::R1)));
        }
        for (int i = threadIdx.x; i < 3 * Q; i += C::NTHREADS) tw[C::NTQ + i] = wP((i % Q) * (i / Q + 1));
    }
    __syncthreads();

    WsRange range;
    range.u = (int64_t)blockIdx.x * a.units_per_cta;
    range.u1 = min(range.u + (int64_t)a.units_per_cta, a.nunits);

    if (warp < C::NFIRW) {
        // ======================= FIR warps =======================
        asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(C::REG_FIR) : "memory");
        const int t = threadIdx.x;
        float hs[TT][NB];
        float2 pend[TT][NB];
        // this thread's twiddles w_P^(t k1), k1 = 1..3, in shared memory (read per
        // row: holding them in registers spills the FIR state); U_k1 = conj(w) V_k1
        const float2 *wt = tw + C::NTQ + t;
        int cur = -1;
        uint32_t bc = 0;   // batches consumed
        int urow = 0;      // rows consumed from the current batch
        bool ok = true;
        int si;
        int64_t fA, fB;
        while (ok && ws_next_segment(a, range, si, fA, fB)) {
            const StreamDesc &d = a.s[si];
            if (si != cur) {
                cur = si;
                const float inv_p = 1.0f / (float)P;  // exact: P is a power of two
#pragma unroll
                for (int m = 0; m < TT; ++m)
#pragma unroll
                    for (int kk = 0; kk < NB; ++kk) hs[m][kk] = __ldg(d.taps + m * P + t + Q * kk) * inv_p;
            }
            int64_t rA, rB;
            sy_rows(fA, fB, TT, d.n_frames, rA, rB);
            const int64_t s_first = fA - TT + 1;
            // segment-relative counters fit 32 bits: a segment is at most one
            // CTA's range of output frames (units_per_cta, checked on the host)
            const int nfr = (int)(fB - s_first);             // rows s_first .. fB-1
            const int iA = (int)(rA - s_first), iB = (int)(rB - s_first);  // rows that exist
            int batch_rows = (int)min((int64_t)SB, rB - rA);   // rows of the current batch
            int done_rows = 0;                                 // real rows consumed in this segment
            float2 *o_seg = d.out + s_first * (int64_t)P + t;
#pragma unroll 1
            for (int i0 = 0; i0 < nfr && ok; i0 += TT) {
#pragma unroll
                for (int k = 0; k < TT; ++k) {
                    const int i = i0 + k;
                    if (i < nfr) {
                        float2 yv[NB];
#pragma unroll
                        for (int kk = 0; kk < NB; ++kk) yv[kk] = make_float2(0.f, 0.f);
                        if (i >= iA && i < iB) {
                            if (urow == 0 &&
                                !__all_sync(0xffffffffu, mbar_wait(ufull0 + 8 * (bc & 1), (bc >> 1) & 1))) {
                                *abort_flag = 1;
                                ok = false;
                                break;
                            }
                            {
                                const float2 *ur = U + ((bc & 1) * SB + urow) * 4 * Q + t;
                                const float2 u0 = ur[0], u1 = cmul(ur[Q], conjf2(wt[0])),
                                             u2 = cmul(ur[2 * Q], conjf2(wt[Q])), u3 = cmul(ur[3 * Q], conjf2(wt[2 * Q]));
                                // y~[t + Q kk] = sum_k1 i^(kk k1) U_k1[t]
                                const float2 a0 = cadd2(u0, u2), a1 = csub2(u0, u2);
                                const float2 a2 = cadd2(u1, u3), a3 = csub2(u1, u3);
                                const float2 ia3 = make_float2(-a3.y, a3.x);  // i a3
                                yv[0] = cadd2(a0, a2);
                                yv[1] = cadd2(a1, ia3);
                                yv[2] = csub2(a0, a2);
                                yv[3] = csub2(a1, ia3);
                                ++done_rows;
                                if (++urow == batch_rows) {
                                    // the batch's values are in registers: hand the buffer back
                                    __syncwarp();
                                    if (lane == 0) mbar_arrive(uempty0 + 8 * (bc & 1));
                                    ++bc;
                                    urow = 0;
                                    batch_rows = min(SB, iB - iA - done_rows);
                                }
                            }
                        }
                        // row s reaches output frames s .. s + TT - 1 (register slot (i + m) mod TT);
                        // frame s + TT - 1 starts here, frame s completes
#pragma unroll
                        for (int kk = 0; kk < NB; ++kk)
                            pend[(k + TT - 1) % TT][kk] = make_float2(hs[TT - 1][kk] * yv[kk].x, hs[TT - 1][kk] * yv[kk].y);
#pragma unroll
                        for (int m = TT - 2; m >= 0; --m) {
                            const int js = (k + m) % TT;
#pragma unroll
                            for (int kk = 0; kk < NB; ++kk)
                                pend[js][kk] = fma2(make_float2(hs[m][kk], hs[m][kk]), yv[kk], pend[js][kk]);
                        }
                        if (i >= TT - 1) {  // frame s_first + i = fA + (i - TT + 1) is complete
                            float2 *o = o_seg + (int64_t)i * P;
#pragma unroll
                            for (int kk = 0; kk < NB; ++kk) store_cs(o + Q * kk, pend[k][kk]);
                        }
                    }
                }
            }
        }
    } else if (warp < C::PRODW) {
        // ======================= IFFT warps =======================
        asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(C::REG_IF) : "memory");
        const int ft = threadIdx.x - C::NFT;
        uint32_t pc = 0, bc = 0;
        bool ok = true;
        int si;
        int64_t fA, fB;
        auto fail_any = [&](bool w) { return named_bar_or<1>(C::NIFT, !w); };
        while (ok && ws_next_segment(a, range, si, fA, fB)) {
            const StreamDesc &d = a.s[si];
            int64_t rA, rB;
            sy_rows(fA, fB, TT, d.n_frames, rA, rB);
            for (int64_t r0 = rA; r0 < rB && ok; r0 += SB, ++bc) {
                const int nr = (int)min((int64_t)SB, rB - r0);
                // the batch's rows have landed in the ring
                bool w = true;
                for (int r = 0; r < nr; ++r) w = w && mbar_wait(full0 + 8 * ((pc + r) % NSLOT), ((pc + r) / NSLOT) & 1);
                if (fail_any(w)) {
                    *abort_flag = 1;
                    ok = false;
                    break;
                }
                // ---- pass 0 (radix 16) on the conjugated sub-rows X[4m + k1] ----
                constexpr int NBF0 = SB * 4 * C::STRIDE0;
#pragma unroll 1
                for (int b = ft; b < NBF0; b += C::NIFT) {
                    const int k1 = b & 3, j = (b >> 2) % C::STRIDE0, row = (b >> 2) / C::STRIDE0;
                    if (row >= nr) continue;
                    const float2 *x = reinterpret_cast<const float2 *>(ring + ((pc + row) % NSLOT) * C::FB);
                    float2 v[C::R0];
#pragma unroll
                    for (int r = 0; r < C::R0; ++r) v[r] = conjf2(x[4 * (j + r * C::STRIDE0) + k1]);
                    dft_reg<C::R0, true>(v);
                    float2 *dst = W + (4 * row + k1) * SROW + (G + 1) * j;
#pragma unroll
                    for (int r = 0; r < C::R0; ++r) dst[r] = v[r];
                }
                named_bar_sync<1>(C::NIFT);
                // the ring rows are consumed (their values are in W): back to the producer
                if (ft == 0)
                    for (int r = 0; r < nr; ++r) mbar_arrive(empty0 + 8 * ((pc + r) % NSLOT));
                pc += nr;
                // U buffer (bc & 1) is free once the FIR warps used batch bc - 2
                if (bc >= 2 && fail_any(mbar_wait(uempty0 + 8 * (bc & 1), ((bc >> 1) + 1) & 1))) {
                    *abort_flag = 1;
                    ok = false;
                    break;
                }
                // ---- pass 1: finish the Q-point transforms, conjugate ----
                constexpr int NBF1 = SB * 4 * C::STRIDE1;
                const float2 *twp = tw + fft_tw_offset(Q, 1, C::MR);
                float2 *ub = U + (bc & 1) * SB * 4 * Q;
#pragma unroll 1
                for (int b = ft; b < NBF1; b += C::NIFT) {
                    const int j = b % C::STRIDE1, k1 = (b / C::STRIDE1) & 3, row = b / (4 * C::STRIDE1);
                    if (row >= nr) continue;
                    const float2 *src = W + (4 * row + k1) * SROW + ypad<G>(j);
                    float2 v[C::R1];
#pragma unroll
                    for (int r = 0; r < C::R1; ++r) v[r] = src[r * (C::STRIDE1 + C::STRIDE1 / G)];
                    const float2 *w = twp + j * (C::R1 - 1);
#pragma unroll
                    for (int r = 1; r < C::R1; ++r) v[r] = cmul(v[r], w[r - 1]);
                    dft_reg<C::R1, true>(v);
                    float2 *u = ub + (row * 4 + k1) * Q + j;
#pragma unroll
                    for (int r = 0; r < C::R1; ++r) u[16 * r] = conjf2(v[r]);  // V_k1; the FIR warps twiddle it
                }
                named_bar_sync<1>(C::NIFT);  // U written, W free for the next pass 0
                if (ft == 0) mbar_arrive(ufull0 + 8 * (bc & 1));
            }
        }
    } else {
        // ======================= producer warp(group) =======================
        asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(C::REG_PROD) : "memory");
        if (warp == C::PRODW && lane == 0) {
            uint32_t pc = 0;
            bool ok = true;
            int si;
            int64_t fA, fB;
            while (ok && ws_next_segment(a, range, si, fA, fB)) {
                const StreamDesc &d = a.s[si];
                int64_t rA, rB;
                sy_rows(fA, fB, TT, d.n_frames, rA, rB);
                const uint8_t *in = static_cast<const uint8_t *>(d.in);
                for (int64_t s = rA; s < rB && ok; ++s, ++pc) {
                    const uint32_t slot = pc % NSLOT;
                    if (pc >= NSLOT && !mbar_wait(empty0 + 8 * slot, ((pc / NSLOT) + 1) & 1)) {
                        *abort_flag = 1;
                        ok = false;
                        break;
                    }
                    mbar_expect_tx(full0 + 8 * slot, C::FB);
                    bulk_g2s(smem_u32(ring + slot * C::FB), in + s * (int64_t)C::FB, C::FB, full0 + 8 * slot);
                }
            }
            const uint32_t first = pc > NSLOT ? pc - NSLOT : 0;
            for (uint32_t q = first; q < pc; ++q) {
                if (!mbar_wait(full0 + 8 * (q % NSLOT), (q / NSLOT) & 1)) *abort_flag = 1;
            }
        }
        __syncwarp();
    }
    __syncthreads();
    if (threadIdx.x == 0 && *abort_flag) report_error(a.err, KERR_TIMEOUT);
}

}  // namespace pfb
