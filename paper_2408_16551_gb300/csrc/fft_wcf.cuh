// Fused polyphase FIR + FFT for P = 4096 on a cluster of four CTAs in
// four-step form, P = 64 x 64 (variant 3 of the cluster FFT family).
//
//   y[s,p] = sum_{m<T} h[m*P+p] * x[(s+m)*P+p]     (Sec. 5.2 / Sec. 4.3)
//   X[s,k] = sum_p y[s,p] exp(-2 pi i p k / P)       (Sec. 4.1)
//
// With p = 64 p1 + p2 and k = k1 + 64 k2 (all four indices < 64):
//   B_p2[k1]          = sum_{p1} y[64 p1 + p2] w_64^(p1 k1)
//   X[k1 + 64 k2]     = sum_{p2} w_64^(p2 k2) w_P^(p2 k1) B_p2[k1].
// CTA c (cluster rank) owns the columns p2 = 16 c + u (u < 16) in the first
// step and the rows k1 = 16 c + kl (kl < 16) in the second, so that it reads
// its input as 64 runs of 16 consecutive samples per frame and writes its
// bins as 64 runs of 16 consecutive bins per spectrum; one exchange between
// the CTAs carries B_p2[k1] from the column owner to the row owner.
//   FIR warps, thread t = 16 t1 + u: the four branches p1 = 16 j + t1 (j < 4)
//       of column p2, the T - 1 pending spectra in registers (a spectrum takes
//       its last tap and is consumed in the slot the next one starts in); on
//       completion the first radix-4 step of the 64-point
//       DFT over p1 (decimation in frequency):
//       Z_a[t1] = w_64^(t1 a) sum_j y[64 (16 j + t1) + p2] w_4^(j a),  a < 4;
//   FFT warps, pass A: B_p2[a + 4 b] = sum_{t1} Z_a[t1] w_16^(t1 b); each
//       value goes as an 8-byte asynchronous store into the receive slot of
//       CTA (a + 4 b) / 16, whose mbarrier counts the bytes;
//   combine in the receiver (even spectra: FIR warps, thread t = 16 kl + u,
//       DR spectra later; odd spectra: FFT warps, one batch after pass A):
//       the radix-4 step over the source CTA c of the 64-point DFT over p2 =
//       16 c + u, with k2 = k2a + 4 k2b:
//       S_k2a = w_P^(u (k1 + 64 k2a)) sum_c w_4^(c k2a) w_256^(c k1) B_(16c+u)[k1],
//       in place in the receive slot;
//   FFT warps, pass B, LAG batches after pass A:
//       X[k1 + 64 (k2a + 4 k2b)] = sum_u S_k2a[u] w_16^(u k2b).
// Roles in every CTA: the producer warpgroup (16-byte asynchronous copies of
// the 64 runs of a frame; one bulk copy per run was bound by the copy
// engine's request rate) fills a ring of NSLOT frames; 8 FIR warps; 4 FFT
// warps, each independent of the others (every hand-over is an mbarrier, no
// named barrier).  Hand-overs: ring full/empty (producer <-> FIR), Y
// full/empty per batch of SB spectra (FIR -> pass A), receive slot rfull
// (bytes from the four senders; armed by the pass-B warps for its next use
// before they hand it back), r2full (combine done -> pass B) and rempty
// in every sender (the pass-B warps of every receiver hand the slot back
// with relaxed remote arrivals).  Every wait is bounded (the launch's
// wait_ns); a timeout sets the error word and the roles wind down; all
// threads of all CTAs meet at a final cluster barrier, so no CTA exits while
// a peer may still touch its shared memory.  The branch sums and partial
// transforms never leave the chip.
#pragma once

#include "fft_ws_cluster.cuh"

namespace pfb {

template <int TT, int IN>
struct WcfCfg {
    static constexpr int P = 4096, CS = 4;
    static constexpr int NFT = 256, NFIRW = NFT / 32;
    static constexpr int NFFTW = 4, NFFTT = NFFTW * 32;
    static constexpr int PRODW = NFIRW + NFFTW;      // first warp of the producer warpgroup
    static constexpr int NTHREADS = NFT + NFFTT + 128;
    static constexpr int SB = 2;                     // spectra per batch (one pass-A / pass-B butterfly per FFT thread)
    static constexpr int LAG = 2;                    // batches from a batch's pass A to its pass B
    static constexpr int DR = 4;                     // spectra from a spectrum's send to its combine in the FIR warps
    static constexpr int NSLOT = 8;                  // input ring slots (frames)
    static constexpr int NR = 10;                    // receive slots (spectra)
    static constexpr int ESZ = IN == PFB_IN_C64 ? 8 : (IN == PFB_IN_R32 ? 4 : 2);
    static constexpr int RUN = 16 * ESZ;             // bytes of one 16-sample run
    static constexpr int FB = 1024 * ESZ;            // bytes of the CTA's 64 runs of a frame
    static constexpr int NCP = FB / 16 / 128;        // 16-byte copies per producer thread and frame
    static constexpr int YBUF = SB * 1024;           // float2 per Y buffer: [row][a][t1][u]
    static constexpr int RK = 17;                    // receive-slot row kl, padded (float2)
    static constexpr int RS = 16 * RK;               // one source CTA c (or one k2a) of a slot
    static constexpr int RSLOT = 4 * RS;             // float2 per receive slot
    static constexpr uint32_t RB = 1024 * 8;         // bytes landing per use of a slot
    static constexpr int NTWF = 3 * 16;              // w_64^(t1 a), [a - 1][t1]
    static constexpr int NTWR = 7 * 256;             // combine twiddles, [i][16 kl + u]
    static constexpr int OFF_RING = 0;
    static constexpr int OFF_Y = OFF_RING + NSLOT * FB;
    static constexpr int OFF_R = OFF_Y + 2 * YBUF * 8;
    static constexpr int OFF_TWF = OFF_R + NR * RSLOT * 8;
    static constexpr int OFF_TWR = OFF_TWF + NTWF * 8;
    static constexpr int OFF_META = OFF_TWR + NTWR * 8;   // [FFT warp][4] batch records, 32 bytes each
    static constexpr int OFF_BAR = OFF_META + NFFTW * 4 * 32;
    // full[NSLOT], empty[NSLOT], yfull[2], yempty[2], rfull[NR], r2full[NR], rempty[NR]
    static constexpr int NBAR = 2 * NSLOT + 4 + 3 * NR;
    static constexpr int SMEM = OFF_BAR + NBAR * 8 + 16;
    // register split (setmaxnreg), measured on 64 x 2^20 samples: 200/80/32 ran
    // 1.3 % faster than 208/72/24 (FIR 192 spills and ran 27 % slower)
    static constexpr int REG_FIR = 200, REG_FFT = 80, REG_PROD = 32;
    static_assert(NFT * REG_FIR + NFFTT * REG_FFT + 128 * REG_PROD <= 65536, "register split");
    static_assert(TT >= 2, "pending-spectrum slots");
    static_assert(DR >= SB && LAG * SB >= DR, "a combine needs its batch sent; pass B needs its combines");
    static_assert(NR > (LAG + 1) * SB + DR / SB, "receive slots for the spectra between a send and its hand-back");
    static_assert(NCP * 16 * 128 == FB, "whole 16-byte pieces per producer thread");
    static_assert(RUN % 16 == 0 && OFF_Y % 16 == 0 && OFF_R % 16 == 0 && (RSLOT * 8) % 16 == 0, "alignment");
    static_assert(SMEM <= 232448, "shared memory");
};

struct WcfMeta {
    float2 *out;
    int64_t ldo;
    int32_t nrows;
    uint32_t g;  // cluster sequence number of the batch's first spectrum
    int64_t pad_;
};

template <int TT, int IN>
__global__ void __launch_bounds__(WcfCfg<TT, IN>::NTHREADS, 1) k_fft_wcf(const __grid_constant__ LaunchArgs a) {
    using C = WcfCfg<TT, IN>;
    constexpr int P = C::P, SB = C::SB, NSLOT = C::NSLOT, NR = C::NR, RS = C::RS, RK = C::RK;
    extern __shared__ __align__(128) uint8_t wf_smem[];
    uint8_t *ring = wf_smem + C::OFF_RING;
    float2 *Y = reinterpret_cast<float2 *>(wf_smem + C::OFF_Y);
    float2 *R = reinterpret_cast<float2 *>(wf_smem + C::OFF_R);
    float2 *twf = reinterpret_cast<float2 *>(wf_smem + C::OFF_TWF);
    float2 *twr = reinterpret_cast<float2 *>(wf_smem + C::OFF_TWR);
    WcfMeta *meta = reinterpret_cast<WcfMeta *>(wf_smem + C::OFF_META);
    uint64_t *bars = reinterpret_cast<uint64_t *>(wf_smem + C::OFF_BAR);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(bars + C::NBAR);
    const uint32_t full0 = smem_u32(&bars[0]), empty0 = smem_u32(&bars[NSLOT]);
    const uint32_t yfull0 = smem_u32(&bars[2 * NSLOT]), yempty0 = smem_u32(&bars[2 * NSLOT + 2]);
    const uint32_t rfull0 = smem_u32(&bars[2 * NSLOT + 4]), r2full0 = smem_u32(&bars[2 * NSLOT + 4 + NR]);
    const uint32_t rempty0 = smem_u32(&bars[2 * NSLOT + 4 + 2 * NR]);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int crank = (int)cluster_ctarank();
    const float2 *tw_half = static_cast<const float2 *>(a.aux);  // w_P^r, r < P/2 (FP64-generated)

    if (threadIdx.x == 0) {
        for (int i = 0; i < NSLOT; ++i) {
            mbar_init(full0 + 8 * i, 128);  // one copy-completion arrival per producer thread
            mbar_init(empty0 + 8 * i, C::NFIRW);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(yfull0 + 8 * i, C::NFIRW);
            mbar_init(yempty0 + 8 * i, C::NFFTW);
        }
        for (int i = 0; i < NR; ++i) {
            mbar_init(rfull0 + 8 * i, 1);        // the receiver's arm + RB bytes from the four senders
            mbar_init(r2full0 + 8 * i, C::NFIRW);  // 8 FIR warps, or 4 FFT warps arriving with count 2
            mbar_init(rempty0 + 8 * i, 2 * 4);   // the two pass-B warps of the slot's row in each receiver
        }
        mbar_init_fence();
        for (int i = 0; i < NR; ++i) mbar_expect_tx(rfull0 + 8 * i, C::RB);  // first use of every receive slot
        *abort_flag = 0;
    }
    // twiddles from the FP64-generated table w_P^e
    for (int i = threadIdx.x; i < C::NTWF; i += C::NTHREADS) twf[i] = tw_full(tw_half, (64 * (i & 15) * (i / 16 + 1)) % P, P);
    for (int i = threadIdx.x; i < C::NTWR; i += C::NTHREADS) {
        const int idx = i >> 8, tt = i & 255, kl = tt >> 4, u = tt & 15;
        const int k1 = 16 * crank + kl;
        const int e = idx < 3 ? 16 * (idx + 1) * k1 : u * (k1 + 64 * (idx - 3));
        twr[i] = tw_full(tw_half, e % P, P);
    }
    __syncthreads();
    cluster_sync_all();  // every CTA's barriers initialised and armed before any remote traffic

    WsRange range;
    range.u = (int64_t)(blockIdx.x / C::CS) * a.units_per_cta;
    range.u1 = min(range.u + (int64_t)a.units_per_cta, a.nunits);

    if (warp < C::NFIRW) {
        // ======================= FIR warps =======================
        asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(C::REG_FIR) : "memory");
        const int t = threadIdx.x;
        const uint32_t wns = (uint32_t)a.wait_ns;  // at most 4 s (checked on the host)
        const int pcol = 64 * (t >> 4) + 16 * crank + (t & 15);  // branch 1024 j + pcol
        float h[TT][4];
        constexpr int NS = TT - 1;  // register slots of pending spectra
        float2 pend[NS][4];
        int cur = -1;
        uint32_t pc = 0;  // frames consumed
        uint32_t bc = 0;  // batches handed to pass A
        uint32_t g0 = 0;  // spectra of the earlier segments
        uint32_t rc = 0;  // spectra combined
        bool ok = true;
        // combine of received spectrum rc (thread t = 16 kl + u), in place
        auto combine = [&]() -> bool {
            const uint32_t rs = rc % NR;
            if (!__all_sync(0xffffffffu, mbar_wait32(rfull0 + 8u * rs, (rc / NR) & 1, wns))) return false;
            float2 *q = R + rs * C::RSLOT + RK * (t >> 4) + (t & 15);
            const float2 r0 = q[0];
            const float2 r1 = cmul(q[RS], twr[t]);
            const float2 r2 = cmul(q[2 * RS], twr[256 + t]);
            const float2 r3 = cmul(q[3 * RS], twr[512 + t]);
            const float2 a0 = cadd2(r0, r2), a1 = csub2(r0, r2);
            const float2 a2 = cadd2(r1, r3), a3 = csub2(r1, r3);
            const float2 mi_a3 = make_float2(a3.y, -a3.x);  // -i a3
            q[0] = cmul(cadd2(a0, a2), twr[768 + t]);
            q[RS] = cmul(cadd2(a1, mi_a3), twr[1024 + t]);
            q[2 * RS] = cmul(csub2(a0, a2), twr[1280 + t]);
            q[3 * RS] = cmul(csub2(a1, mi_a3), twr[1536 + t]);
            __syncwarp();
            if (lane == 0) mbar_arrive(r2full0 + 8u * rs);
            ++rc;
            return true;
        };
        // the FIR warps combine the even spectra, the FFT warps the odd ones
        auto combine_or_skip = [&]() -> bool {
            if (rc & 1) {
                ++rc;
                return true;
            }
            return combine();
        };
        int si;
        int64_t sA, sB;
        while (ok && ws_next_segment(a, range, si, sA, sB)) {
            const StreamDesc &d = a.s[si];
            if (si != cur) {
                cur = si;
#pragma unroll
                for (int m = 0; m < TT; ++m)
#pragma unroll
                    for (int j = 0; j < 4; ++j) h[m][j] = __ldg(d.taps + m * P + 1024 * j + pcol);
            }
            // segment-relative counters fit 32 bits: a segment is at most one
            // cluster's range (units_per_cta, checked on the host)
            const int nspec = (int)(sB - sA);
            const int nfr = nspec + TT - 1;
            // NS = TT - 1 register slots: spectrum s lives in slot s mod NS; at
            // frame i the slot of spectrum i - NS takes its last tap and is
            // consumed before spectrum i starts in it
            for (int i0 = 0; i0 < nfr && ok; i0 += NS) {
#pragma unroll
                for (int k = 0; k < NS; ++k) {
                    const int i = i0 + k;
                    if (i < nfr) {
                        const uint32_t slot = pc % NSLOT;
                        if (!__all_sync(0xffffffffu, mbar_wait32(full0 + 8 * slot, (pc / NSLOT) & 1, wns))) {
                            ok = false;
                            break;
                        }
                        float2 v[4];
                        {
                            const uint8_t *fr = ring + slot * C::FB;
                            const float sc = d.scale;
#pragma unroll
                            for (int j = 0; j < 4; ++j) {
                                const int q = 256 * j + t;  // run 16 j + t1, sample u
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
                        // frame i contributes h[m] * x to spectrum i - m, slot (i - m) mod NS
#pragma unroll
                        for (int m = 1; m < NS; ++m) {
                            const int js = ((k - m) % NS + NS) % NS;
#pragma unroll
                            for (int j = 0; j < 4; ++j) pend[js][j] = fma2(make_float2(h[m][j], h[m][j]), v[j], pend[js][j]);
                        }
                        const int jspec = i - NS;
                        if (jspec >= 0) {
                            // ---- spectrum jspec completes in slot k: radix-4 over j into Y ----
#pragma unroll
                            for (int j = 0; j < 4; ++j) pend[k][j] = fma2(make_float2(h[NS][j], h[NS][j]), v[j], pend[k][j]);
                            const int brow = jspec % SB;
                            if (brow == 0 && bc >= 2 &&
                                !__all_sync(0xffffffffu, mbar_wait32(yempty0 + 8 * (bc & 1), ((bc >> 1) + 1) & 1, wns))) {
                                ok = false;
                                break;
                            }
                            float2 *ys = Y + (bc & 1) * C::YBUF + brow * 1024 + t;
                            const float2 a0 = cadd2(pend[k][0], pend[k][2]);
                            const float2 a1 = csub2(pend[k][0], pend[k][2]);
                            const float2 a2 = cadd2(pend[k][1], pend[k][3]);
                            const float2 a3 = csub2(pend[k][1], pend[k][3]);
                            const float2 mi_a3 = make_float2(a3.y, -a3.x);  // -i a3
                            const int t1 = t >> 4;
                            ys[0] = cadd2(a0, a2);
                            ys[256] = cmul(cadd2(a1, mi_a3), twf[t1]);
                            ys[512] = cmul(csub2(a0, a2), twf[16 + t1]);
                            ys[768] = cmul(csub2(a1, mi_a3), twf[32 + t1]);
                            if (brow == SB - 1 || jspec == nspec - 1) {
                                __syncwarp();
                                if (lane == 0) mbar_arrive(yfull0 + 8 * (bc & 1));
                                ++bc;
                            }
                        }
                        // spectrum i starts in slot k
#pragma unroll
                        for (int j = 0; j < 4; ++j) pend[k][j] = make_float2(h[0][j] * v[j].x, h[0][j] * v[j].y);
                        // ---- combine of the spectrum sent DR spectra earlier ----
                        if (jspec >= 0 && g0 + (uint32_t)jspec >= rc + C::DR && !combine_or_skip()) {
                            ok = false;
                            break;
                        }
                    }
                }
            }
            g0 += (uint32_t)nspec;
        }
        while (ok && rc < g0) ok = combine_or_skip();  // the last DR spectra of the range
        if (!ok) *abort_flag = 1;
    } else if (warp < C::PRODW) {
        // ======================= FFT warps =======================
        asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(C::REG_FFT) : "memory");
        const int w = warp - C::NFIRW;
        const int row = w >> 1;                     // batch row of this warp
        const int hf = 2 * (w & 1) + (lane >> 4);   // pass A: a; pass B: k2a
        const int l16 = lane & 15;                  // pass A: u; pass B: kl
        WcfMeta *mym = meta + w * 4;
        const uint32_t wns = (uint32_t)a.wait_ns;  // at most 4 s (checked on the host)
        uint32_t nA = 0, nB = 0, nC = 0, gA = 0;
        bool ok = true, more = true;
        int si = 0;
        int64_t sA = 0, sB = 0;
        int s0 = 0, nspec = 0;  // segment-relative (a segment is at most one cluster's range)
        const uint32_t r_loc = smem_u32(R);
        while (ok) {
            while (more && s0 >= nspec) {
                if (ws_next_segment(a, range, si, sA, sB)) {
                    s0 = 0;
                    nspec = (int)(sB - sA);
                } else {
                    more = false;
                }
            }
            if (more) {
                // ---- pass A of batch nA: 16-point DFTs over t1, sent to the row owners ----
                const StreamDesc &d = a.s[si];
                const int nrows = min(SB, nspec - s0);
                if (lane == 0) {
                    WcfMeta m;
                    m.out = d.out + (sA + s0) * d.ldo;
                    m.ldo = d.ldo;
                    m.nrows = nrows;
                    m.g = gA;
                    m.pad_ = 0;
                    mym[nA & 3] = m;
                }
                if (!__all_sync(0xffffffffu, mbar_wait32(yfull0 + 8 * (nA & 1), (nA >> 1) & 1, wns))) {
                    ok = false;
                    break;
                }
                if (row < nrows) {
                    const uint32_t g = gA + (uint32_t)row, rs = g % NR;
                    // every receiver handed this slot's previous use back
                    if (g >= NR &&
                        !__all_sync(0xffffffffu, mbar_wait32(rempty0 + 8u * rs, ((g / NR) + 1) & 1, wns))) {
                        ok = false;
                        break;
                    }
                    const float2 *ys = Y + (nA & 1) * C::YBUF + row * 1024 + hf * 256 + l16;
                    float2 v[16];
#pragma unroll
                    for (int t1 = 0; t1 < 16; ++t1) v[t1] = ys[16 * t1];
                    dft_reg<16, true>(v);
                    // B_p2[hf + 4 b] -> CTA b / 4, entry [c][kl = hf + 4 (b mod 4)][u]
                    const uint32_t e_loc = r_loc + (uint32_t)(rs * C::RSLOT + crank * RS + RK * hf + l16) * 8u;
                    const uint32_t b_loc = rfull0 + 8u * rs;
                    // one address translation per destination CTA: a CTA's shared memory
                    // is one contiguous range of the cluster window
#pragma unroll
                    for (int dst = 0; dst < 4; ++dst) {
                        const uint32_t e_rem = mapa_shared(e_loc, (uint32_t)dst);
                        const uint32_t b_rem = mapa_shared(b_loc, (uint32_t)dst);
#pragma unroll
                        for (int be = 0; be < 4; ++be) st_async_v2(e_rem + (uint32_t)(RK * 4 * be) * 8u, v[4 * dst + be], b_rem);
                    }
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(yempty0 + 8 * (nA & 1));
                s0 += SB;
                gA += (uint32_t)nrows;
                ++nA;
            }
            if (nC < nA && (!more || nA - nC > 1)) {
                // ---- combine of the odd spectra of batch nC (the FIR warps take the even ones) ----
                __syncwarp();
                const WcfMeta m = mym[nC & 3];
#pragma unroll 1
                for (int row2 = 0; row2 < m.nrows && ok; ++row2) {
                    const uint32_t g = m.g + (uint32_t)row2, rs = g % NR;
                    if ((g & 1) == 0) continue;
                    if (!__all_sync(0xffffffffu, mbar_wait32(rfull0 + 8u * rs, (g / NR) & 1, wns))) {
                        ok = false;
                        break;
                    }
#pragma unroll
                    for (int hh = 0; hh < 2; ++hh) {
                        const int tt = 32 * w + lane + 128 * hh;  // 16 kl + u
                        float2 *q = R + rs * C::RSLOT + RK * (tt >> 4) + (tt & 15);
                        const float2 r0 = q[0];
                        const float2 r1 = cmul(q[RS], twr[tt]);
                        const float2 r2 = cmul(q[2 * RS], twr[256 + tt]);
                        const float2 r3 = cmul(q[3 * RS], twr[512 + tt]);
                        const float2 a0 = cadd2(r0, r2), a1 = csub2(r0, r2);
                        const float2 a2 = cadd2(r1, r3), a3 = csub2(r1, r3);
                        const float2 mi_a3 = make_float2(a3.y, -a3.x);  // -i a3
                        q[0] = cmul(cadd2(a0, a2), twr[768 + tt]);
                        q[RS] = cmul(cadd2(a1, mi_a3), twr[1024 + tt]);
                        q[2 * RS] = cmul(csub2(a0, a2), twr[1280 + tt]);
                        q[3 * RS] = cmul(csub2(a1, mi_a3), twr[1536 + tt]);
                    }
                    __syncwarp();
                    if (lane == 0) mbar_arrive_n(r2full0 + 8u * rs, 2);  // 4 FFT warps x 2 = the 8 FIR arrivals
                }
                if (!ok) break;
                ++nC;
            }
            if (nB < nC && (!more || nA - nB > (uint32_t)C::LAG)) {
                // ---- pass B of batch nB: 16-point DFTs over u, bins to HBM ----
                __syncwarp();
                const WcfMeta m = mym[nB & 3];
                if (row < m.nrows) {
                    const uint32_t g = m.g + (uint32_t)row, rs = g % NR;
                    if (!__all_sync(0xffffffffu, mbar_wait32(r2full0 + 8u * rs, (g / NR) & 1, wns))) {
                        ok = false;
                        break;
                    }
                    const float2 *q = R + rs * C::RSLOT + hf * RS + RK * l16;
                    float2 v[16];
#pragma unroll
                    for (int u = 0; u < 16; ++u) v[u] = q[u];
                    dft_reg<16, true>(v);
                    float2 *o = m.out + row * m.ldo + 16 * crank + l16 + 64 * hf;
#pragma unroll
                    for (int k2b = 0; k2b < 16; ++k2b) store_cs(o + 256 * k2b, v[k2b]);
                    // hand the slot back: arm its next use, then tell every sender
                    if ((w & 1) == 0 && lane == 0) mbar_expect_tx(rfull0 + 8u * rs, C::RB);
                    __syncwarp();
                    if (lane < 4) mbar_arrive_cluster_relaxed(mapa_shared(rempty0 + 8u * rs, (uint32_t)lane));
                }
                ++nB;
            } else if (!more && nB == nA) {
                break;
            }
        }
        if (!ok) *abort_flag = 1;
    } else {
        // ======================= producer warpgroup =======================
        // 128 threads gather the CTA's 64 runs of a frame with 16-byte
        // asynchronous copies; each thread's arrival on the slot's "full"
        // barrier fires once its own copies have landed
        asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(C::REG_PROD) : "memory");
        const int pt = threadIdx.x - C::PRODW * 32;
        uint32_t pc = 0;
        bool ok = true;
        int si;
        int64_t sA, sB;
        while (ok && ws_next_segment(a, range, si, sA, sB)) {
            const StreamDesc &d = a.s[si];
            const int64_t f_end = sB + TT - 1;
            for (int64_t f = sA; f < f_end; ++f, ++pc) {
                const uint32_t slot = pc % NSLOT;
                if (pc >= NSLOT && !mbar_wait(empty0 + 8 * slot, ((pc / NSLOT) + 1) & 1, a.wait_ns)) {
                    ok = false;
                    break;
                }
                const uint8_t *src;
                if (f < d.n_state) src = static_cast<const uint8_t *>(d.state) + f * (int64_t)P * C::ESZ;
                else src = static_cast<const uint8_t *>(d.in) + (f - d.n_state) * (int64_t)P * C::ESZ;
                src += (int64_t)crank * C::RUN;
                const uint32_t dst = smem_u32(ring + slot * C::FB);
                // 16-byte piece q of the slot: run q / (RUN / 16) (samples 64 r + 16 c ..), piece q mod (RUN / 16)
#pragma unroll
                for (int i = 0; i < C::NCP; ++i) {
                    const int q = pt + 128 * i;
                    const int r = q / (C::RUN / 16), pe = q % (C::RUN / 16);
                    cp_async16(dst + q * 16, src + (int64_t)r * 64 * C::ESZ + pe * 16);
                }
                cp_async_arrive_noinc(full0 + 8 * slot);
            }
        }
        // every copy issued has landed before the CTA exits
        asm volatile("cp.async.wait_all;" ::: "memory");
        if (!ok) *abort_flag = 1;
    }
    // no CTA leaves while a peer may still store into its receive slots or
    // arrive on its barriers
    cluster_sync_all();
    if (threadIdx.x == 0 && *abort_flag) report_error(a.err, KERR_TIMEOUT);
}

}  // namespace pfb
