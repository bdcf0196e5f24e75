// Fused polyphase FIR + FFT for P = CS * 1024 (P = 2048, 4096) on a cluster
// of CS CTAs, warp-specialised and fed by the TMA engine (variant 1 of the
// cluster FFT family).
//
//   y[s,p] = sum_{m<T} h[m*P+p] * x[(s+m)*P+p]     (Sec. 5.2 / Sec. 4.3)
//   X[s,k] = sum_p y[s,p] exp(-2 pi i p k / P)       (Sec. 4.1)
//
// CTA c (cluster rank) owns branches p = c*PL + n, n < PL = 1024, and the
// DFT is factored (four-step form, decimation in frequency across the CTAs):
//   Z_k1[n]           = w_P^(n k1) * sum_{n1<CS} y[n1*PL + n] w_CS^(n1 k1)
//   X[k1 + CS*kk]     = sum_{n<PL} Z_k1[n] w_PL^(n kk)
// and CTA k1 computes the PL-point DFT of Z_k1, itself split once more by a
// radix-4 decimation in frequency (n = n' + Q j, Q = PL/4) as in the
// single-CTA warp-specialised kernel.  Roles in every CTA:
//   producer (lane 0 of warp PRODW): 1-D bulk copies of the CTA's contiguous
//       slice of each frame (PL samples) into a ring of NSLOT slots;
//   FIR warps (256 threads, branches n = t + Q j, j < 4): streaming FIR state
//       in registers; the four branch sums of a finished spectrum go straight
//       to the CTA d = t / QC that owns n' = t in the cross step, as two
//       16-byte asynchronous stores into its double-buffered gather buffer X
//       whose completion is counted in bytes on d's mbarrier;
//   FFT warps (128 threads), per batch of SB spectra:
//     1. cross step: for each of this CTA's QC values n' and j < 4, the CS
//        branch sums y[n1*PL + n' + Q j] (from X), a CS-point DFT, the twiddle
//        w_P^(n k1), a radix-4 butterfly over j; the four sub-row values go to
//        CTA k1's Z buffer, again as byte-counted asynchronous stores;
//     2. once all of this CTA's Z has landed: pass 1 of the four Q-point sub-
//        transforms (pre-twiddles w_PL^(n' k1')), Z -> W;
//     3. pass 2, W -> bins k = c + CS*(4m + k1') of the output rows.
// Data hand-overs between CTAs are byte-counted on the receiver's mbarrier
// (no release fence on the sender's side; the receiver's CTA-scope wait on
// its own barrier sees the bytes); buffer hand-backs are relaxed remote
// arrivals, issued after the values were consumed.  Every wait is
// bounded (1 s of %globaltimer); a timeout sets the launch's error word and
// the roles wind down; all threads of all CTAs meet at a final cluster
// barrier, so no CTA exits while a peer may still touch its shared memory.
// The branch sums never leave the chip.
#pragma once

#include "fft_cluster.cuh"

namespace pfb {

template <int CS, int TT, int IN, bool TC = false>
struct WcCfg {
    static constexpr int PL = 1024;                 // branches per CTA
    static constexpr int P = CS * PL;
    static constexpr int Q = PL / 4;                // sub-transform length of the local radix-4 split
    static constexpr int NB = 4;                    // branches per FIR thread: t + Q j
    static constexpr int NFT = Q;                   // FIR threads
    static constexpr int NFIRW = NFT / 32;
    static constexpr int NFFTW = 4;
    static constexpr int NFFTT = NFFTW * 32;
    static constexpr int PRODW = NFIRW + NFFTW;     // producer warp (its warpgroup: 3 idle warps)
    static constexpr int NTHREADS = NFT + NFFTT + 128;
    static constexpr int SB = 4;                    // spectra per batch
    static constexpr int MR = 16, G = 16;
    static constexpr int SROW = Q + Q / G + 8;      // radix-4 sub-row
    static constexpr int YROW = PL + PL / G;        // TC: natural-order Z row (padded)
    static constexpr int ZBUF = TC ? SB * YROW : SB * 4 * SROW;  // float2 per Z (and W) buffer
    static constexpr int QC = Q / CS;               // cross-step n' per CTA
    static constexpr int NSLOT = 8;
    static constexpr int ESZ = IN == PFB_IN_C64 ? 8 : (IN == PFB_IN_R32 ? 4 : 2);
    static constexpr int FB = PL * ESZ;             // bytes of the CTA's slice of a frame
    static constexpr int NTQ = fft_tw_entries(Q, MR);
    // pass list, pre-twiddles w_PL^(n' k1'), then the cross-step twiddles
    // w_P^(n k1) of this CTA's n = c*QC + nl + Q j, as [k1 - 1][j][nl]
    static constexpr int NTX = (CS - 1) * 4 * QC;
    static constexpr int NTW = (TC ? 0 : NTQ + 3 * Q) + NTX;
    static constexpr int OFF_TWX = TC ? 0 : NTQ + 3 * Q;  // cross-step twiddles within the table
    // TC (local 1024-point DFT on the tensor cores, P1 = 32): the step-2 A
    // operand (bf16 hi and lo, K-major, 128 rows x 64), the 32-point DFT matrix
    // in real block form (bf16 hi and lo, 64 x 64), twiddles w_1024^(k1 n2)
    static constexpr int TC_P1 = 32, TC_LBO_A = 2064, TC_A2B = 8 * TC_LBO_A, TC_BTB = 64 * 64 * 2;
    // gather buffer X of the cross step: [s][n1][j pair][n' - c*QC], 16 bytes
    // (two branch sums, j = 2 jp and 2 jp + 1) per entry
    static constexpr int XBUF = SB * CS * 2 * QC;   // 16-byte entries per buffer
    static constexpr uint32_t BYTES_X = XBUF * 16;  // bytes landing per batch
    static constexpr uint32_t BYTES_Z = SB * 4 * Q * 8;
    static constexpr int OFF_RING = 0;
    static constexpr int OFF_X = OFF_RING + NSLOT * FB;
    static constexpr int OFF_Z = OFF_X + 2 * XBUF * 16;
    static constexpr int OFF_W = OFF_Z + ZBUF * 8;
    static constexpr int OFF_A2 = OFF_W + (TC ? 0 : ZBUF * 8);
    static constexpr int OFF_BT = OFF_A2 + (TC ? 2 * TC_A2B : 0);
    static constexpr int OFF_TWT = OFF_BT + (TC ? 2 * TC_BTB : 0);
    static constexpr int OFF_TW = OFF_TWT + (TC ? TC_P1 * TC_P1 * 8 : 0);
    static constexpr int OFF_BAR = OFF_TW + NTW * 8;
    // full[NSLOT], empty[NSLOT], xfull[2], xempty[2], zfull, zempty;
    // TC: MMA 1 / MMA 2 complete, step-1 / step-2 operand written
    static constexpr int NBAR = 2 * NSLOT + 6 + (TC ? 4 : 0);
    static constexpr int SMEM = OFF_BAR + NBAR * 8 + 16;
    static constexpr int REG_FIR = TC ? 200 : 208, REG_FFT = TC ? 88 : 72, REG_PROD = 24;
    static_assert(!TC || (OFF_A2 % 128 == 0 && OFF_BT % 128 == 0), "TC operand alignment");
    static_assert(!TC || PL == TC_P1 * TC_P1, "TC: PL = 32 x 32, 4 spectra per 128-row tile");
    static_assert(NFT % 128 == 0 && NTHREADS % 128 == 0, "roles are whole warpgroups");
    static_assert(NFT * REG_FIR + NFFTT * REG_FFT + 128 * REG_PROD <= 65536, "register split");
    static_assert(fft_npasses(Q, MR) == 2, "two local passes after the radix-4 split");
    static_assert(QC * CS == Q, "cross-step share");
    static_assert(SMEM <= 232448, "shared memory");
    static_assert(BYTES_X == (uint32_t)SB * PL * 8, "every branch sum of a batch lands once");
};

// distributed shared memory: 8-byte load / store at a shared::cluster address
__device__ __forceinline__ float2 ld_dsmem_f2(uint32_t addr) {
    float2 v;
    asm volatile("ld.shared::cluster.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(addr) : "memory");
    return v;
}
__device__ __forceinline__ void st_dsmem_f2(uint32_t addr, float2 v) {
    asm volatile("st.shared::cluster.v2.f32 [%0], {%1, %2};" ::"r"(addr), "f"(v.x), "f"(v.y) : "memory");
}

// Last pass of the four Q-point sub-transforms (radix-4 split of the CTA's
// PL-point DFT): local bin 4m + k1' is global bin c + CS*(4m + k1').
template <int Q, int SB, int SROW, int G, int CS>
__device__ __forceinline__ void wc_dif4_last(const float2 *src, const float2 *tw, float2 *out_row0, int nrows,
                                             int ft, int nft, int c, int64_t ldo) {
    constexpr int MR = 16;
    constexpr int PASS = fft_npasses(Q, MR) - 1;
    constexpr int R = fft_radix(Q, PASS, MR);
    constexpr int NS = fft_ns(Q, PASS, MR);
    constexpr int STRIDE = Q / R;
    static_assert(STRIDE == NS && STRIDE % G == 0, "last pass");
    constexpr int NBF = SB * 4 * STRIDE;
    constexpr int P = CS * 4 * Q;
    const float2 *twp = tw + fft_tw_offset(Q, PASS, MR);
#pragma unroll 1
    for (int b = ft; b < NBF; b += nft) {
        const int k1 = b & 3;
        const int j = (b >> 2) % STRIDE;
        const int row = (b >> 2) / STRIDE;
        const float2 *s = src + (4 * row + k1) * SROW + ypad<G>(j);
        float2 v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = s[r * (STRIDE + STRIDE / G)];
        const float2 *w = twp + j * (R - 1);
#pragma unroll
        for (int r = 1; r < R; ++r) v[r] = cmul(v[r], w[r - 1]);
        dft_reg<R, true>(v);
        if (row < nrows) {
            float2 *o = out_row0 + row * ldo + c + CS * (4 * j + k1);
#pragma unroll
            for (int r = 0; r < R; ++r) store_cs(o + CS * 4 * NS * r, v[r]);
        }
    }
}

template <int CS, int TT, int IN, bool TC = false>
__global__ void __launch_bounds__(WcCfg<CS, TT, IN, TC>::NTHREADS, 1)
    k_fft_ws_cluster(const __grid_constant__ LaunchArgs a) {
    using C = WcCfg<CS, TT, IN, TC>;
    constexpr int PL = C::PL, P = C::P, Q = C::Q, QC = C::QC, NB = C::NB, SB = C::SB, NSLOT = C::NSLOT;
    constexpr int SROW = C::SROW, G = C::G, NFT = C::NFT, NFFTT = C::NFFTT;
    extern __shared__ __align__(128) uint8_t wc_smem[];
    uint8_t *ring = wc_smem + C::OFF_RING;
    const float4 *X = reinterpret_cast<const float4 *>(wc_smem + C::OFF_X);
    float2 *Z = reinterpret_cast<float2 *>(wc_smem + C::OFF_Z);
    float2 *W = reinterpret_cast<float2 *>(wc_smem + C::OFF_W);
    float2 *tw = reinterpret_cast<float2 *>(wc_smem + C::OFF_TW);
    uint64_t *bars = reinterpret_cast<uint64_t *>(wc_smem + C::OFF_BAR);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(bars + C::NBAR);
    volatile uint32_t *tmem_slot = reinterpret_cast<volatile uint32_t *>(abort_flag + 1);
    const uint32_t mbar1 = smem_u32(&bars[2 * NSLOT + 6]), mbar2 = smem_u32(&bars[2 * NSLOT + 7]);
    const uint32_t op1 = smem_u32(&bars[2 * NSLOT + 8]), op2 = smem_u32(&bars[2 * NSLOT + 9]);
    const uint32_t full0 = smem_u32(&bars[0]), empty0 = smem_u32(&bars[NSLOT]);
    const uint32_t xfull0 = smem_u32(&bars[2 * NSLOT]), xempty0 = smem_u32(&bars[2 * NSLOT + 2]);
    const uint32_t zfull = smem_u32(&bars[2 * NSLOT + 4]), zempty = smem_u32(&bars[2 * NSLOT + 5]);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t crank = cluster_ctarank();

    WsRange range;
    range.u = (int64_t)(blockIdx.x / CS) * a.units_per_cta;
    range.u1 = min(range.u + (int64_t)a.units_per_cta, a.nunits);
    // batches of this cluster's range (the same in every CTA of the cluster)
    uint32_t nbatch = 0;
    {
        WsRange r = range;
        int si;
        int64_t sA, sB;
        while (ws_next_segment(a, r, si, sA, sB)) nbatch += (uint32_t)((sB - sA + SB - 1) / SB);
    }

    if (threadIdx.x == 0) {
        for (int i = 0; i < NSLOT; ++i) {
            mbar_init(full0 + 8 * i, 1);
            mbar_init(empty0 + 8 * i, C::NFIRW);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(xfull0 + 8 * i, 1);               // own arrive + BYTES_X from every CTA's FIR warps
            mbar_init(xempty0 + 8 * i, CS * C::NFFTW);  // every CTA's FFT warps consumed their X buffer i
        }
        mbar_init(zfull, 1);                            // own arrive + BYTES_Z from every CTA's cross step
        mbar_init(zempty, CS * C::NFFTW);               // every CTA finished reading its Z
        if constexpr (TC) {
            mbar_init(mbar1, 1);                        // MMA 1 complete (tcgen05.commit)
            mbar_init(mbar2, 1);                        // MMA 2 complete
            mbar_init(op1, C::NFFTT);                   // step-1 operand written (TMEM)
            mbar_init(op2, C::NFFTT);                   // step-2 operand written (shared memory)
        }
        mbar_init_fence();
        // arm the first use of each byte-counted barrier
        for (uint32_t i = 0; i < 2 && i < nbatch; ++i) mbar_expect_tx(xfull0 + 8 * i, C::BYTES_X);
        if (nbatch > 0) mbar_expect_tx(zfull, C::BYTES_Z);
        *abort_flag = 0;
    }
    // twiddles of the local transform, from the FP64-generated table w_P^r
    // (r < P/2): the Q-point pass list, then w_PL^(n k1') = w_P^(CS n k1')
    {
        const float2 *tw_half = static_cast<const float2 *>(a.aux);
        for (int i = threadIdx.x; i < (TC ? 0 : C::NTQ); i += C::NTHREADS) {
            int off = 0, e = 0;
#pragma unroll
            for (int ps = 0; ps < fft_npasses(Q, C::MR); ++ps) {
                const int ns = fft_ns(Q, ps, C::MR), R = fft_radix(Q, ps, C::MR);
                if (ns > 1 && i >= off && i < off + ns * (R - 1)) {
                    const int jj = (i - off) / (R - 1), r = (i - off) % (R - 1) + 1;
                    e = r * jj * (P / (ns * R));
                }
                if (ns > 1) off += ns * (R - 1);
            }
            tw[i] = tw_full(tw_half, e % P, P);
        }
        for (int i = threadIdx.x; i < (TC ? 0 : 3 * Q); i += C::NTHREADS)
            tw[C::NTQ + i] = tw_full(tw_half, CS * (i % Q) * (i / Q + 1), P);
        for (int i = threadIdx.x; i < C::NTX; i += C::NTHREADS) {
            const int nl = i % QC, j = (i / QC) % 4, k1 = i / (4 * QC) + 1;
            tw[C::OFF_TWX + i] = tw_full(tw_half, ((int)crank * QC + nl + Q * j) * k1, P);
        }
    }
    if constexpr (TC) {
        // 32-point DFT-matrix tiles (hi, lo) and the twiddles w_1024^(k1 n2), 16-byte vectors
        const int4 *src = reinterpret_cast<const int4 *>(a.tw);
        int4 *dst = reinterpret_cast<int4 *>(wc_smem + C::OFF_BT);
        constexpr int NV = (2 * C::TC_BTB + C::TC_P1 * C::TC_P1 * 8) / 16;
        for (int i = threadIdx.x; i < NV; i += C::NTHREADS) dst[i] = src[i];
        if (warp == C::NFIRW) tmem_alloc(smem_u32((const void *)tmem_slot), kTcCols);
        fence_proxy_async_smem();  // the tables are read by the tensor core
        tc_fence_before();
    }
    __syncthreads();
    cluster_sync_all();
    if constexpr (TC) tc_fence_after();  // barriers of every CTA initialised and armed before any remote traffic

    if (warp < C::NFIRW) {
        // ======================= FIR warps =======================
        asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(C::REG_FIR) : "memory");
        const int t = threadIdx.x;
        // the cross-step owner of n' = t, and this thread's entries of its X buffer
        const uint32_t owner = (uint32_t)(t / QC);
        const uint32_t x_base = mapa_shared(smem_u32(X) + (uint32_t)((crank * 2) * QC + t % QC) * 16u, owner);
        float h[TT][NB];
        float2 pend[TT][NB];
        int cur = -1;
        uint32_t pc = 0, bc = 0;
        int brow = 0;
        bool ok = true;
        int si;
        int64_t sA, sB;
        // two 16-byte stores of this thread's branch sums (j = 0, 1 and j = 2, 3) of batch row `row`
        auto push = [&](int row, float2 y0, float2 y1, float2 y2, float2 y3) {
            const uint32_t e = x_base + (bc & 1) * (C::XBUF * 16u) + (uint32_t)(row * CS * 2 * QC) * 16u;
            const uint32_t fb = mapa_shared(xfull0 + 8 * (bc & 1), owner);
            st_async_v4(e, make_float4(y0.x, y0.y, y1.x, y1.y), fb);
            st_async_v4(e + QC * 16u, make_float4(y2.x, y2.y, y3.x, y3.y), fb);
        };
        while (ok && ws_next_segment(a, range, si, sA, sB)) {
            const StreamDesc &d = a.s[si];
            if (si != cur) {
                cur = si;
#pragma unroll
                for (int m = 0; m < TT; ++m)
#pragma unroll
                    for (int j = 0; j < NB; ++j) h[m][j] = __ldg(d.taps + m * P + crank * PL + t + Q * j);
            }
            // segment-relative counters fit 32 bits: a segment is at most one
            // cluster's range (units_per_cta, checked on the host)
            const int nspec = (int)(sB - sA);
            const int nfr = nspec + TT - 1;
            for (int i0 = 0; i0 < nfr && ok; i0 += TT) {
#pragma unroll
                for (int k = 0; k < TT; ++k) {
                    const int i = i0 + k;
                    if (i < nfr) {
                        const uint32_t slot = pc % NSLOT;
                        if (!__all_sync(0xffffffffu, mbar_wait(full0 + 8 * slot, (pc / NSLOT) & 1))) {
                            *abort_flag = 1;
                            ok = false;
                            break;
                        }
                        float2 v[NB];
                        {
                            const uint8_t *fr = ring + slot * C::FB;
                            const float sc = d.scale;
#pragma unroll
                            for (int j = 0; j < NB; ++j) {
                                const int q = t + Q * j;
                                if constexpr (IN == PFB_IN_C64) v[j] = reinterpret_cast<const float2 *>(fr)[q];
                                else if constexpr (IN == PFB_IN_R32)
                                    v[j] = make_float2(reinterpret_cast<const float *>(fr)[q], 0.f);
                                else {
                                    const char2 c2 = reinterpret_cast<const char2 *>(fr)[q];
                                    v[j] = make_float2((float)c2.x * sc, (float)c2.y * sc);
                                }
                            }
                            // the previous frame's ring slot goes back to the producer now:
                            // every lane has used the values it loaded from it (a TMA refill
                            // must not overtake a shared-memory read still in flight)
                            __syncwarp();
                            if (lane == 0 && pc > 0) mbar_arrive(empty0 + 8 * ((pc - 1) % NSLOT));
                        }
                        ++pc;
                        // frame i contributes h[m] * x to spectrum i - m (register slot (i - m) mod TT)
#pragma unroll
                        for (int j = 0; j < NB; ++j) pend[k][j] = make_float2(h[0][j] * v[j].x, h[0][j] * v[j].y);
#pragma unroll
                        for (int m = 1; m < TT; ++m) {
                            const int js = ((k - m) % TT + TT) % TT;
#pragma unroll
                            for (int j = 0; j < NB; ++j)
                                pend[js][j] = fma2(make_float2(h[m][j], h[m][j]), v[j], pend[js][j]);
                        }
                        const int jspec = i - (TT - 1);
                        if (jspec >= 0) {
                            const int jslot = (k + 1) % TT;
                            // every CTA's cross step consumed this X buffer's previous batch
                            if (brow == 0 && bc >= 2 &&
                                !__all_sync(0xffffffffu,
                                            mbar_wait(xempty0 + 8 * (bc & 1), ((bc >> 1) + 1) & 1))) {
                                *abort_flag = 1;
                                ok = false;
                                break;
                            }
                            push(brow, pend[jslot][0], pend[jslot][1], pend[jslot][2], pend[jslot][3]);
                            if (++brow == SB) {
                                ++bc;
                                brow = 0;
                            }
                        }
                    }
                }
            }
            if (ok && brow > 0) {
                // a short batch at the end of a segment still delivers SB rows:
                // the receiver counts bytes
                const float2 z0 = make_float2(0.f, 0.f);
#pragma unroll 1
                for (int r = brow; r < SB; ++r) push(r, z0, z0, z0, z0);
                ++bc;
                brow = 0;
            }
        }
    } else if (warp < C::PRODW) {
        // ======================= FFT warps =======================
        asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(C::REG_FFT) : "memory");
        const int ft = threadIdx.x - NFT;
        const float2 *twx = tw + C::OFF_TWX;  // cross-step twiddles [k1 - 1][j][nl]
        const uint32_t zloc = smem_u32(Z);
        uint32_t bc = 0;
        bool ok = true;
        int si;
        int64_t sA, sB;
        auto fail_any = [&](bool w) { return named_bar_or<1>(NFFTT, !w); };
        // TC: warp w owns spectrum q = w mod 4 of a 4-spectrum batch (TMEM lane quarter q)
        const int q = warp & 3;
        const uint32_t tmem = TC ? *tmem_slot : 0u;
        const uint32_t trow = tmem + ((uint32_t)(32 * q) << 16);
        uint32_t ph1 = 0, ph2 = 0;  // MMA completions observed
        auto wait_mma = [&](uint32_t bar, uint32_t &ph) {
            const bool w = mbar_wait(bar, ph & 1);
            ++ph;
            const bool failed = named_bar_or<2>(NFFTT, !w);
            tc_fence_after();
            return !failed;
        };
        bool have_prev = false;
        float2 *prev_rows = nullptr;
        int prev_nrows = 0;
        // TC epilogue: bins k1 + 32 k2 (k1 = lane) of spectrum q, global bin c + CS (k1 + 32 k2)
        auto epilogue = [&](float2 *rows, int nrows, int64_t ldo) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                uint32_t r[32];
                tmem_ld32(trow + kTcColD2 + 32 * h, r);
                tmem_wait_ld();
                if (q < nrows) {
                    float2 *o = rows + q * ldo + crank + CS * (lane + 32 * (16 * h));
#pragma unroll
                    for (int j = 0; j < 16; ++j)
                        store_cs(o + CS * 32 * j, make_float2(__uint_as_float(r[2 * j]), __uint_as_float(r[2 * j + 1])));
                }
            }
        };
        int64_t ldo_prev = 0;
        while (ok && ws_next_segment(a, range, si, sA, sB)) {
            const StreamDesc &d = a.s[si];
            const int64_t nspec = sB - sA;
            const int64_t nb = (nspec + SB - 1) / SB;
            for (int64_t qb = 0; qb < nb && ok; ++qb, ++bc) {
                float2 *out_rows = d.out + (sA + qb * SB) * d.ldo;
                const int nrows = (int)min((int64_t)SB, nspec - qb * SB);
                // every CTA's branch sums for this batch have landed in our X buffer
                if (fail_any(mbar_wait(xfull0 + 8 * (bc & 1), (bc >> 1) & 1))) {
                    *abort_flag = 1;
                    ok = false;
                    break;
                }
                if (ft == 0 && bc + 2 < nbatch) mbar_expect_tx(xfull0 + 8 * (bc & 1), C::BYTES_X);  // next use
                // every CTA finished pass 1 of the previous batch: all Z buffers are free
                if (bc >= 1 && fail_any(mbar_wait(zempty, (bc - 1) & 1))) {
                    *abort_flag = 1;
                    ok = false;
                    break;
                }
                // ---- 1. cross step ----
                const float4 *xb = X + (bc & 1) * C::XBUF;
                const uint32_t zf_base = zfull;
#pragma unroll 1
                for (int it = ft; it < SB * QC; it += NFFTT) {
                    const int s = it / QC, nl = it % QC;
                    const int np = (int)crank * QC + nl;
                    float2 z[CS][4];
#pragma unroll
                    for (int jp = 0; jp < 2; ++jp) {
                        float4 e[CS];
#pragma unroll
                        for (int n1 = 0; n1 < CS; ++n1) e[n1] = xb[((s * CS + n1) * 2 + jp) * QC + nl];
#pragma unroll
                        for (int h2 = 0; h2 < 2; ++h2) {
                            const int j = 2 * jp + h2;
                            float2 u[CS];
#pragma unroll
                            for (int n1 = 0; n1 < CS; ++n1)
                                u[n1] = h2 == 0 ? make_float2(e[n1].x, e[n1].y) : make_float2(e[n1].z, e[n1].w);
                            dft_reg<CS, true>(u);
                            z[0][j] = u[0];
#pragma unroll
                            for (int k1 = 1; k1 < CS; ++k1) z[k1][j] = cmul(u[k1], twx[((k1 - 1) * 4 + j) * QC + nl]);
                        }
                    }
                    if constexpr (TC) {
                        // natural order: Z_k1[n' + Q j] into row s of CTA k1
#pragma unroll
                        for (int k1 = 0; k1 < CS; ++k1) {
                            const uint32_t zfb = mapa_shared(zf_base, k1);
#pragma unroll
                            for (int j = 0; j < 4; ++j)
                                st_async_v2(mapa_shared(zloc + (uint32_t)(s * C::YROW + ypad<G>(np + Q * j)) * 8u, k1),
                                            z[k1][j], zfb);
                        }
                        continue;
                    }
                    const uint32_t zoff = (uint32_t)(4 * s * SROW + ypad<G>(np)) * 8u;
#pragma unroll
                    for (int k1 = 0; k1 < CS; ++k1) {
                        // radix-4 butterfly over j (the twiddles w_PL^(n' k1') come in pass 1)
                        const float2 a0 = cadd2(z[k1][0], z[k1][2]), a1 = csub2(z[k1][0], z[k1][2]);
                        const float2 a2 = cadd2(z[k1][1], z[k1][3]), a3 = csub2(z[k1][1], z[k1][3]);
                        const float2 mi_a3 = make_float2(a3.y, -a3.x);  // -i a3
                        const uint32_t zb = mapa_shared(zloc + zoff, k1);
                        const uint32_t zfb = mapa_shared(zf_base, k1);
                        st_async_v2(zb, cadd2(a0, a2), zfb);
                        st_async_v2(zb + SROW * 8u, cadd2(a1, mi_a3), zfb);
                        st_async_v2(zb + 2u * SROW * 8u, csub2(a0, a2), zfb);
                        st_async_v2(zb + 3u * SROW * 8u, csub2(a1, mi_a3), zfb);
                    }
                }
                // our X buffer has been read: hand it back to every CTA's FIR warps
                __syncwarp();
                if (lane == 0) {
#pragma unroll
                    for (int r = 0; r < CS; ++r) mbar_arrive_cluster_relaxed(mapa_shared(xempty0 + 8 * (bc & 1), r));
                }
                // ---- 2. this CTA's Z has landed: pass 1, Z -> W ----
                if (fail_any(mbar_wait(zfull, bc & 1))) {
                    *abort_flag = 1;
                    ok = false;
                    break;
                }
                if (ft == 0 && bc + 1 < nbatch) mbar_expect_tx(zfull, C::BYTES_Z);  // next batch
                if constexpr (TC) {
                    // ---- 2. MMA 1 operand: row (q, n2 = lane), K = (n1, re/im), into TMEM ----
                    const float2 *zrow = Z + q * C::YROW;
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        uint32_t vh[16], vl[16];
#pragma unroll
                        for (int j = 0; j < 16; ++j) split_bf16x2(zrow[ypad<G>(32 * (16 * h + j) + lane)], vh[j], vl[j]);
                        tmem_st<16>(trow + kTcColA1 + 16 * h, vh);
                        tmem_st<16>(trow + kTcColA1 + 32 + 16 * h, vl);
                    }
                    tmem_wait_st();
                    // Z read: every CTA may send its next batch
                    __syncwarp();
                    if (lane == 0) {
#pragma unroll
                        for (int r = 0; r < CS; ++r) mbar_arrive_cluster_relaxed(mapa_shared(zempty, r));
                    }
                    tc_fence_before();
                    mbar_arrive(op1);
                    // ---- while MMA 1 runs: the previous batch's bins ----
                    if (have_prev) {
                        if (!wait_mma(mbar2, ph2)) {
                            *abort_flag = 1;
                            ok = false;
                            break;
                        }
                        epilogue(prev_rows, prev_nrows, ldo_prev);
                        have_prev = false;
                    }
                    if (!wait_mma(mbar1, ph1)) {
                        *abort_flag = 1;
                        ok = false;
                        break;
                    }
                    // ---- 3. twiddle w_1024^(n2 k1), split, transposed store: MMA 2 operand ----
                    uint8_t *a2 = wc_smem + C::OFF_A2;
                    const float2 *twt = reinterpret_cast<const float2 *>(wc_smem + C::OFF_TWT);
                    const int a2_base = (lane >> 2) * C::TC_LBO_A + (lane & 3) * 4 + (4 * q) * 128;
#pragma unroll
                    for (int h = 0; h < 4; ++h) {  // 8 k1 per TMEM load
                        float2 w8[8];
#pragma unroll
                        for (int j = 0; j < 8; ++j) w8[j] = twt[(8 * h + j) * C::TC_P1 + lane];
                        uint32_t r[16];
                        tmem_ld16(trow + kTcColD1 + 16 * h, r);
                        tmem_wait_ld();
#pragma unroll
                        for (int j = 0; j < 8; ++j) {
                            const int k1 = 8 * h + j;
                            const float2 zz =
                                cmul(make_float2(__uint_as_float(r[2 * j]), __uint_as_float(r[2 * j + 1])), w8[j]);
                            uint32_t hi, lo;
                            split_bf16x2(zz, hi, lo);
                            const int off = a2_base + (k1 >> 3) * 128 + (k1 & 7) * 16;
                            *reinterpret_cast<uint32_t *>(a2 + off) = hi;
                            *reinterpret_cast<uint32_t *>(a2 + C::TC_A2B + off) = lo;
                        }
                    }
                    fence_proxy_async_smem();
                    tc_fence_before();
                    mbar_arrive(op2);
                    prev_rows = out_rows;
                    prev_nrows = nrows;
                    ldo_prev = d.ldo;
                    have_prev = true;
                    continue;
                }
                ws_pass<Q, C::MR, 4 * SB, 0, false, SROW, G, true>(Z, W, tw, nullptr, 0, ft, NFFTT, tw + C::NTQ);
                named_bar_sync<1>(NFFTT);
                if (lane == 0) {
#pragma unroll
                    for (int r = 0; r < CS; ++r) mbar_arrive_cluster_relaxed(mapa_shared(zempty, r));
                }
                // ---- 3. pass 2, W -> bins c + CS (4m + k1') ----
                wc_dif4_last<Q, SB, SROW, G, CS>(W, tw, out_rows, nrows, ft, NFFTT, (int)crank, d.ldo);
                named_bar_sync<1>(NFFTT);  // W free before the next pass 1
            }
        }
        if constexpr (TC) {
            if (ok && have_prev) {
                if (wait_mma(mbar2, ph2)) epilogue(prev_rows, prev_nrows, ldo_prev);
                else *abort_flag = 1;
            }
        }
    } else {
        // ======================= producer warp(group) =======================
        asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(C::REG_PROD) : "memory");
        if constexpr (TC) {
            if (warp == C::PRODW + 1 && lane == 0)
                ws_tc_mma_thread<C>(a, range, wc_smem, op1, op2, mbar1, mbar2, *tmem_slot, abort_flag);
        }
        if (warp == C::PRODW && lane == 0) {
            uint32_t pc = 0;
            bool ok = true;
            int si;
            int64_t sA, sB;
            while (ok && ws_next_segment(a, range, si, sA, sB)) {
                const StreamDesc &d = a.s[si];
                const int64_t f_end = sB + TT - 1;
                for (int64_t f = sA; f < f_end && ok; ++f, ++pc) {
                    const uint32_t slot = pc % NSLOT;
                    if (pc >= NSLOT && !mbar_wait(empty0 + 8 * slot, ((pc / NSLOT) + 1) & 1)) {
                        *abort_flag = 1;
                        ok = false;
                        break;
                    }
                    const uint8_t *src;
                    if (f < d.n_state) src = static_cast<const uint8_t *>(d.state) + f * (int64_t)P * C::ESZ;
                    else src = static_cast<const uint8_t *>(d.in) + (f - d.n_state) * (int64_t)P * C::ESZ;
                    src += (int64_t)crank * C::FB;
                    mbar_expect_tx(full0 + 8 * slot, C::FB);
                    bulk_g2s(smem_u32(ring + slot * C::FB), src, C::FB, full0 + 8 * slot);
                }
            }
            // every copy issued has landed before the CTA exits
            const uint32_t first = pc > NSLOT ? pc - NSLOT : 0;
            for (uint32_t q = first; q < pc; ++q) {
                if (!mbar_wait(full0 + 8 * (q % NSLOT), (q / NSLOT) & 1)) *abort_flag = 1;
            }
        }
        __syncwarp();
    }
    // no CTA leaves while a peer may still store into its X or Z buffers or
    // arrive on its barriers
    if constexpr (TC) tc_fence_before();
    cluster_sync_all();
    if constexpr (TC) {
        if (warp == C::NFIRW) {
            tc_fence_after();
            tmem_dealloc(*tmem_slot, kTcCols);
        }
    }
    if (threadIdx.x == 0 && *abort_flag) report_error(a.err, KERR_TIMEOUT);
}

}  // namespace pfb
