// Fused polyphase FIR + FFT for P = CS * 1024 (P = 2048, 4096) on a cluster
// of CS CTAs, warp-specialised, fed by the TMA engine, with ONE exchange of
// partial transforms between the CTAs (variant 2 of the cluster FFT family).
//
//   y[s,p] = sum_{m<T} h[m*P+p] * x[(s+m)*P+p]     (Sec. 5.2 / Sec. 4.3)
//   X[s,k] = sum_p y[s,p] exp(-2 pi i p k / P)       (Sec. 4.1)
//
// Branch ownership: FIR thread t of CTA c (cluster rank) owns the four
// branches p = (P/4) j + n, j < 4, n = 256 c + t.  The DFT is split twice by
// decimation in frequency:
//   stage 1 (FIR warps of the sender):
//       Z_k1[n] = w_P^(n k1) sum_j y[(P/4) j + n] w_4^(j k1),
//       X[k1 + 4 kk] = sum_{n < P/4} Z_k1[n] w_(P/4)^(n kk);
//       the thread's four branch sums give Z_k1[n] for k1 < 4 at once; Z_k1
//       belongs to CTA k1 CS / 4 (CS = 4: one P/4-point sub-transform per
//       CTA; CS = 2: two per CTA), where it goes as an 8-byte asynchronous
//       store into that spectrum's receive slot, whose mbarrier counts the
//       bytes; this is the only exchange between the CTAs;
//   stage 2 (FFT warps of the receiver, first pass of a batch): with
//       n = 256 c + t the P/4-point transform of Z_k1 splits once more over
//       the source CTA c (radix CS),
//       V[t] = w_(P/4)^(t k2) sum_c Z_k1[256 c + t] w_CS^(c k2),
//       X[k1 + 4 (k2 + (4/CS) m)] = sum_t V[t] w_256^(t m),
//       read straight from the receive slots into four 256-point sub-rows;
//   then two radix-16 Stockham passes of those sub-transforms (W0 -> W1 ->
//       HBM), the single-CTA kernel's passes; bin m of sub-row q is global
//       bin base(q) + (P/256) m.
// Roles in every CTA:
//   producer (lane 0 of warp PRODW): four 1-D bulk copies per frame (the
//       CTA's 256-sample chunk of each quarter of the frame) into a ring of
//       NSLOT slots;
//   FIR warps (256 threads): streaming FIR state in registers (T slots per
//       branch, rotated at compile time), stage 1 and the send;
//   FFT warps (128 threads): per batch of SB spectra, stage 2 and the passes.
// Hand-over discipline: NR receive slots, one per spectrum in flight, each
// with a byte-counting "full" mbarrier (armed by the receiving FFT warps for
// every use, before they hand the slot back) and an "empty" mbarrier in every
// sender (count CS: the FFT warps of every receiving CTA hand the slot back
// with a relaxed remote arrival once its values are read).  A FIR warp waits
// for "empty" only when it reuses a slot, so the FIR warps run up to NR - SB
// spectra ahead of the slowest receiver and never wait for remote data.
// Every wait is bounded (the launch's wait_ns); a timeout sets the error
// word and the roles wind down; all threads of all CTAs meet at a final
// cluster barrier, so no CTA exits while a peer may still touch its shared
// memory.  The branch sums and partial transforms never leave the chip.
#pragma once

#include "fft_ws_cluster.cuh"

namespace pfb {

template <int CS, int TT, int IN>
struct Wc2Cfg {
    static constexpr int P = CS * 1024;
    static constexpr int E = 4 / CS;                 // sub-transforms of stage 1 per CTA
    static constexpr int Q = 256;                    // length of the FFT warps' sub-transforms
    static constexpr int NFT = 256, NFIRW = NFT / 32;
    static constexpr int NFFTW = 4, NFFTT = NFFTW * 32;
    static constexpr int PRODW = NFIRW + NFFTW;      // producer warp (its warpgroup: 3 idle warps)
    static constexpr int NTHREADS = NFT + NFFTT + 128;
    static constexpr int SB = 4;                     // spectra per FFT batch
    static constexpr int MR = 16, G = 16;
    static constexpr int SROW = Q + Q / G + 8;       // sub-row stride (float2), 16 banks apart
    static constexpr int WBUF = SB * 4 * SROW;       // float2 per W buffer
    static constexpr int NSLOT = 6;                  // input ring slots (frames)
    static constexpr int NR = 12;                    // receive slots (spectra)
    static constexpr int ESZ = IN == PFB_IN_C64 ? 8 : (IN == PFB_IN_R32 ? 4 : 2);
    static constexpr int CB = 256 * ESZ;             // bytes of one 256-branch chunk
    static constexpr int FB = 4 * CB;                // bytes of the CTA's four chunks of a frame
    static constexpr int RB = 4 * 256 * 8;           // bytes of one receive slot: [row][t] float2
    static constexpr int NTQ = fft_tw_entries(Q, MR);
    static constexpr int NT2 = 3 * 256;              // stage-2 twiddles w_P^(4 t k2), [k2 - 1][t]
    static constexpr int OFF_RING = 0;
    static constexpr int OFF_R = OFF_RING + NSLOT * FB;
    static constexpr int OFF_W0 = OFF_R + NR * RB;
    static constexpr int OFF_W1 = OFF_W0 + WBUF * 8;
    static constexpr int OFF_TW = OFF_W1 + WBUF * 8;
    static constexpr int OFF_TW2 = OFF_TW + NTQ * 8;
    static constexpr int OFF_BAR = OFF_TW2 + NT2 * 8;
    // full[NSLOT], empty[NSLOT], rfull[NR], rempty[NR]
    static constexpr int NBAR = 2 * NSLOT + 2 * NR;
    static constexpr int SMEM = OFF_BAR + NBAR * 8 + 16;
    static constexpr int REG_FIR = 208, REG_FFT = 72, REG_PROD = 24;
    static_assert(CS == 2 || CS == 4, "P = 2048 or 4096");
    static_assert(NR >= 2 * SB, "receive slots for at least two batches");
    static_assert(NFT * REG_FIR + NFFTT * REG_FFT + 128 * REG_PROD <= 65536, "register split");
    static_assert(fft_npasses(Q, MR) == 2, "two FFT passes");
    static_assert(CB % 16 == 0 && OFF_R % 16 == 0 && OFF_W0 % 16 == 0, "bulk-copy and st.async alignment");
    static_assert(SMEM <= 232448, "shared memory");
};

// Last pass of the four 256-point sub-transforms of each spectrum: bin m of
// sub-row q is global bin base(q) + STR m, STR = P / 256, with
//   CS = 4: base(q) = c + 4 q;   CS = 2: base(q) = 2 c + (q >> 1) + 4 (q & 1).
template <int CS, int SB, int SROW, int G>
__device__ __forceinline__ void wc2_last(const float2 *src, const float2 *tw, float2 *out_row0, int nrows, int ft,
                                         int nft, int c, int64_t ldo) {
    constexpr int Q = 256, MR = 16;
    constexpr int PASS = fft_npasses(Q, MR) - 1;
    constexpr int R = fft_radix(Q, PASS, MR);
    constexpr int NS = fft_ns(Q, PASS, MR);
    constexpr int STRIDE = Q / R;
    constexpr int STR = CS * 4;  // P / 256
    static_assert(STRIDE == NS && STRIDE % G == 0, "last pass");
    constexpr int NBF = SB * 4 * STRIDE;
    const float2 *twp = tw + fft_tw_offset(Q, PASS, MR);
#pragma unroll 1
    for (int b = ft; b < NBF; b += nft) {
        const int q = b & 3;
        const int j = (b >> 2) % STRIDE;
        const int row = (b >> 2) / STRIDE;
        const float2 *s = src + (4 * row + q) * SROW + ypad<G>(j);
        float2 v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = s[r * (STRIDE + STRIDE / G)];
        const float2 *w = twp + j * (R - 1);
#pragma unroll
        for (int r = 1; r < R; ++r) v[r] = cmul(v[r], w[r - 1]);
        dft_reg<R, true>(v);
        if (row < nrows) {
            const int base = CS == 4 ? c + 4 * q : 2 * c + (q >> 1) + 4 * (q & 1);
            float2 *o = out_row0 + row * ldo + base + STR * j;
#pragma unroll
            for (int r = 0; r < R; ++r) store_cs(o + STR * NS * r, v[r]);
        }
    }
}

template <int CS, int TT, int IN>
__global__ void __launch_bounds__(Wc2Cfg<CS, TT, IN>::NTHREADS, 1)
    k_fft_wc2(const __grid_constant__ LaunchArgs a) {
    using C = Wc2Cfg<CS, TT, IN>;
    constexpr int P = C::P, SB = C::SB, NSLOT = C::NSLOT, NR = C::NR, G = C::G;
    constexpr int SROW = C::SROW, NFIRW = C::NFIRW;
    extern __shared__ __align__(128) uint8_t w2_smem[];
    uint8_t *ring = w2_smem + C::OFF_RING;
    float2 *W0 = reinterpret_cast<float2 *>(w2_smem + C::OFF_W0);
    float2 *W1 = reinterpret_cast<float2 *>(w2_smem + C::OFF_W1);
    float2 *tw = reinterpret_cast<float2 *>(w2_smem + C::OFF_TW);
    const float2 *tw2 = reinterpret_cast<const float2 *>(w2_smem + C::OFF_TW2);
    uint64_t *bars = reinterpret_cast<uint64_t *>(w2_smem + C::OFF_BAR);
    volatile int *flags = reinterpret_cast<volatile int *>(bars + C::NBAR);  // [0] abort, [1] FFT broadcast
    volatile int *abort_flag = flags;
    const uint32_t full0 = smem_u32(&bars[0]), empty0 = smem_u32(&bars[NSLOT]);
    const uint32_t rfull0 = smem_u32(&bars[2 * NSLOT]), rempty0 = smem_u32(&bars[2 * NSLOT + NR]);
    const uint32_t r_base = smem_u32(w2_smem + C::OFF_R);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t crank = cluster_ctarank();
    const float2 *tw_half = static_cast<const float2 *>(a.aux);  // w_P^r, r < P/2 (FP64-generated)

    if (threadIdx.x == 0) {
        for (int i = 0; i < NSLOT; ++i) {
            mbar_init(full0 + 8 * i, 1);
            mbar_init(empty0 + 8 * i, NFIRW);
        }
        for (int i = 0; i < NR; ++i) {
            mbar_init(rfull0 + 8 * i, 1);    // the receiver's arm + RB bytes from the CS senders
            mbar_init(rempty0 + 8 * i, CS);  // the FFT warps of every receiving CTA handed the slot back
        }
        mbar_init_fence();
        // arm the first use of every receive slot (later uses: by the receiving FFT warps)
        for (int i = 0; i < NR; ++i) mbar_expect_tx(rfull0 + 8 * i, C::RB);
        flags[0] = 0;
        flags[1] = 0;
    }
    // twiddles from the FP64-generated table: the 256-point pass list
    // (w_256^e = w_P^(e P/256)) and the stage-2 table w_P^(4 t k2)
    for (int i = threadIdx.x; i < C::NTQ; i += C::NTHREADS) {
        int off = 0, e = 0;
#pragma unroll
        for (int ps = 0; ps < fft_npasses(C::Q, C::MR); ++ps) {
            const int ns = fft_ns(C::Q, ps, C::MR), R = fft_radix(C::Q, ps, C::MR);
            if (ns > 1 && i >= off && i < off + ns * (R - 1)) {
                const int jj = (i - off) / (R - 1), r = (i - off) % (R - 1) + 1;
                e = r * jj * (C::Q / (ns * R));
            }
            if (ns > 1) off += ns * (R - 1);
        }
        tw[i] = tw_full(tw_half, (e * (P / C::Q)) % P, P);
    }
    for (int i = threadIdx.x; i < C::NT2; i += C::NTHREADS)
        reinterpret_cast<float2 *>(w2_smem + C::OFF_TW2)[i] = tw_full(tw_half, (4 * (i % 256) * (i / 256 + 1)) % P, P);
    __syncthreads();
    cluster_sync_all();  // every CTA's barriers initialised and armed before any remote traffic

    WsRange range;
    range.u = (int64_t)(blockIdx.x / CS) * a.units_per_cta;
    range.u1 = min(range.u + (int64_t)a.units_per_cta, a.nunits);

    if (warp < NFIRW) {
        // ======================= FIR warps =======================
        asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(C::REG_FIR) : "memory");
        const int t = threadIdx.x;
        const uint32_t wns = (uint32_t)a.wait_ns;  // at most 4 s (checked on the host)
        const int n = 256 * (int)crank + t;        // stage-1 index of this thread's branches (P/4) j + n
        float h[TT][4];
        float2 pend[TT][4];
        float2 wt1[3];  // w_P^(n k1), k1 = 1..3
#pragma unroll
        for (int k1 = 1; k1 < 4; ++k1) wt1[k1 - 1] = tw_full(tw_half, (n * k1) % P, P);
        // this thread's entry of row r of a receive slot: r_loc + slot * RB + r * 2048
        const uint32_t r_loc = r_base + (uint32_t)t * 8u;
        int cur = -1;
        uint32_t pc = 0;  // frames consumed
        uint32_t g0 = 0;  // spectra of the earlier segments (receive-slot sequence)
        bool ok = true;
        int si;
        int64_t sA, sB;
        while (ok && ws_next_segment(a, range, si, sA, sB)) {
            const StreamDesc &d = a.s[si];
            if (si != cur) {
                cur = si;
#pragma unroll
                for (int m = 0; m < TT; ++m)
#pragma unroll
                    for (int j = 0; j < 4; ++j) h[m][j] = __ldg(d.taps + m * P + (P / 4) * j + n);
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
                        if (!__all_sync(0xffffffffu, mbar_wait32(full0 + 8 * slot, (pc / NSLOT) & 1, wns))) {
                            *abort_flag = 1;
                            ok = false;
                            break;
                        }
                        float2 v[4];
                        {
                            const uint8_t *fr = ring + slot * C::FB;
                            const float sc = d.scale;
#pragma unroll
                            for (int j = 0; j < 4; ++j) {
                                const int q = 256 * j + t;
                                if constexpr (IN == PFB_IN_C64) v[j] = reinterpret_cast<const float2 *>(fr)[q];
                                else if constexpr (IN == PFB_IN_R32)
                                    v[j] = make_float2(reinterpret_cast<const float *>(fr)[q], 0.f);
                                else {
                                    const char2 c2 = reinterpret_cast<const char2 *>(fr)[q];
                                    v[j] = make_float2((float)c2.x * sc, (float)c2.y * sc);
                                }
                            }
                            // the previous frame's ring slot goes back to the producer now:
                            // every lane has used the values it loaded from it
                            __syncwarp();
                            if (lane == 0 && pc > 0) mbar_arrive(empty0 + 8 * ((pc - 1) % NSLOT));
                        }
                        ++pc;
                        // frame i contributes h[m] * x to spectrum i - m (register slot (i - m) mod TT)
#pragma unroll
                        for (int j = 0; j < 4; ++j) pend[k][j] = make_float2(h[0][j] * v[j].x, h[0][j] * v[j].y);
#pragma unroll
                        for (int m = 1; m < TT; ++m) {
                            const int js = ((k - m) % TT + TT) % TT;
#pragma unroll
                            for (int j = 0; j < 4; ++j) pend[js][j] = fma2(make_float2(h[m][j], h[m][j]), v[j], pend[js][j]);
                        }
                        const int jspec = i - (TT - 1);
                        if (jspec >= 0) {
                            // ---- stage 1 and the send of spectrum g ----
                            const int jslot = (k + 1) % TT;
                            const uint32_t g = g0 + (uint32_t)jspec;
                            const uint32_t rs = g % NR;
                            // the FFT warps of every receiver handed this slot's previous use back
                            if (g >= NR &&
                                !__all_sync(0xffffffffu, mbar_wait32(rempty0 + 8u * rs, ((g / NR) - 1) & 1, wns))) {
                                *abort_flag = 1;
                                ok = false;
                                break;
                            }
                            const float2 a0 = cadd2(pend[jslot][0], pend[jslot][2]);
                            const float2 a1 = csub2(pend[jslot][0], pend[jslot][2]);
                            const float2 a2 = cadd2(pend[jslot][1], pend[jslot][3]);
                            const float2 a3 = csub2(pend[jslot][1], pend[jslot][3]);
                            const float2 mi_a3 = make_float2(a3.y, -a3.x);  // -i a3
                            float2 z[4];
                            z[0] = cadd2(a0, a2);
                            z[1] = cmul(cadd2(a1, mi_a3), wt1[0]);
                            z[2] = cmul(csub2(a0, a2), wt1[1]);
                            z[3] = cmul(csub2(a1, mi_a3), wt1[2]);
                            const uint32_t e_loc = r_loc + rs * (uint32_t)C::RB;
                            const uint32_t b_loc = rfull0 + 8u * rs;
#pragma unroll
                            for (int k1 = 0; k1 < 4; ++k1) {
                                const uint32_t dst = (uint32_t)(k1 * CS / 4);  // owner CTA of sub-transform k1
                                const uint32_t row = crank * C::E + (uint32_t)(k1 % C::E);
                                st_async_v2(mapa_shared(e_loc + row * 2048u, dst), z[k1], mapa_shared(b_loc, dst));
                            }
                        }
                    }
                }
            }
            g0 += (uint32_t)nspec;
        }
    } else if (warp < C::PRODW) {
        // ======================= FFT warps =======================
        asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(C::REG_FFT) : "memory");
        const int ft = threadIdx.x - C::NFT;
        const uint32_t wns = (uint32_t)a.wait_ns;
        uint32_t g0 = 0;
        bool ok = true;
        int si;
        int64_t sA, sB;
        while (ok && ws_next_segment(a, range, si, sA, sB)) {
            const StreamDesc &d = a.s[si];
            const int nspec = (int)(sB - sA);
            for (int s0 = 0; s0 < nspec && ok; s0 += SB) {
                const int nrows = min(SB, nspec - s0);
                const uint32_t gb = g0 + (uint32_t)s0;
                // one thread waits for the batch's receive slots (and arms their
                // next use); the decision is broadcast so that every FFT thread
                // reaches the same named barriers
                if (ft == 0) {
                    bool w = true;
                    for (int r = 0; r < nrows && w; ++r) {
                        const uint32_t g = gb + (uint32_t)r, rs = g % NR;
                        w = mbar_wait32(rfull0 + 8u * rs, (g / NR) & 1, wns);
                        if (w) mbar_expect_tx(rfull0 + 8u * rs, C::RB);
                    }
                    flags[1] = w ? 1 : 0;
                }
                named_bar_sync<1>(C::NFFTT);
                if (!flags[1]) {
                    *abort_flag = 1;
                    ok = false;
                    break;
                }
                // ---- stage 2: radix CS over the source CTA, receive slots -> W0 ----
#pragma unroll 1
                for (int it = ft; it < SB * 256; it += C::NFFTT) {
                    const int row = it >> 8, t = it & 255;
                    if (row >= nrows) continue;  // (the sub-rows of missing rows are never stored)
                    const uint32_t rs = (gb + (uint32_t)row) % NR;
                    const float2 *src = reinterpret_cast<const float2 *>(w2_smem + C::OFF_R + rs * C::RB) + t;
                    float2 zz[4];
#pragma unroll
                    for (int r = 0; r < 4; ++r) zz[r] = src[r * 256];
                    float2 *ysub = W0 + row * 4 * SROW + ypad<G>(t);
                    if constexpr (CS == 4) {
                        const float2 a0 = cadd2(zz[0], zz[2]), a1 = csub2(zz[0], zz[2]);
                        const float2 a2 = cadd2(zz[1], zz[3]), a3 = csub2(zz[1], zz[3]);
                        const float2 mi_a3 = make_float2(a3.y, -a3.x);
                        ysub[0] = cadd2(a0, a2);
                        ysub[SROW] = cmul(cadd2(a1, mi_a3), tw2[t]);
                        ysub[2 * SROW] = cmul(csub2(a0, a2), tw2[256 + t]);
                        ysub[3 * SROW] = cmul(csub2(a1, mi_a3), tw2[512 + t]);
                    } else {
                        // rows r = 2 c + e: radix 2 over c for each sub-transform e, sub-row q = 2 e + k2
                        const float2 w = tw2[t];
#pragma unroll
                        for (int e = 0; e < 2; ++e) {
                            ysub[(2 * e) * SROW] = cadd2(zz[e], zz[2 + e]);
                            ysub[(2 * e + 1) * SROW] = cmul(csub2(zz[e], zz[2 + e]), w);
                        }
                    }
                }
                named_bar_sync<1>(C::NFFTT);
                // the batch's receive slots have been read: hand them back to every sender
                if (ft < nrows) {
                    const uint32_t eb = rempty0 + 8u * ((gb + (uint32_t)ft) % NR);
#pragma unroll
                    for (int r = 0; r < CS; ++r) mbar_arrive_cluster_relaxed(mapa_shared(eb, (uint32_t)r));
                }
                // ---- two radix-16 passes: W0 -> W1 -> bins base(q) + (P/256) m ----
                ws_pass<C::Q, C::MR, 4 * SB, 0, false, SROW, G>(W0, W1, tw, nullptr, 0, ft, C::NFFTT);
                named_bar_sync<1>(C::NFFTT);
                wc2_last<CS, SB, SROW, G>(W1, tw, d.out + (sA + s0) * d.ldo, nrows, ft, C::NFFTT, (int)crank, d.ldo);
                named_bar_sync<1>(C::NFFTT);  // W0 and W1 free before the next batch
            }
            g0 += (uint32_t)nspec;
        }
    } else {
        // ======================= producer warp(group) =======================
        asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(C::REG_PROD) : "memory");
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
                    if (pc >= NSLOT && !mbar_wait(empty0 + 8 * slot, ((pc / NSLOT) + 1) & 1, a.wait_ns)) {
                        *abort_flag = 1;
                        ok = false;
                        break;
                    }
                    const uint8_t *src;
                    if (f < d.n_state) src = static_cast<const uint8_t *>(d.state) + f * (int64_t)P * C::ESZ;
                    else src = static_cast<const uint8_t *>(d.in) + (f - d.n_state) * (int64_t)P * C::ESZ;
                    src += (int64_t)crank * C::CB;
                    const uint32_t dst = smem_u32(ring + slot * C::FB);
                    mbar_expect_tx(full0 + 8 * slot, C::FB);
#pragma unroll
                    for (int j = 0; j < 4; ++j)
                        bulk_g2s(dst + j * C::CB, src + (int64_t)j * (P / 4) * C::ESZ, C::CB, full0 + 8 * slot);
                }
            }
            // every copy issued has landed before the CTA exits
            const uint32_t first = pc > NSLOT ? pc - NSLOT : 0;
            for (uint32_t q = first; q < pc; ++q) {
                if (!mbar_wait(full0 + 8 * (q % NSLOT), (q / NSLOT) & 1, a.wait_ns)) *abort_flag = 1;
            }
        }
        __syncwarp();
    }
    // no CTA leaves while a peer may still store into its receive slots or
    // arrive on its barriers
    cluster_sync_all();
    if (threadIdx.x == 0 && *abort_flag) report_error(a.err, KERR_TIMEOUT);
}

}  // namespace pfb
