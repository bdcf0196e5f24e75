// Fused polyphase FIR + FFT, FP32, warp-specialised and fed by the TMA engine
// (variant 5 of the fast FFT family).
//
//   y[s,p] = sum_{m<T} h[m*P+p] * x[(s+m)*P+p]     (Sec. 5.2 per-branch FIR,
//                                                    Sec. 4.3 correlation form)
//   X[s,k] = sum_p y[s,p] exp(-2 pi i p k / P)       (Sec. 4.1, the DFT)
//
// One CTA per SM walks a contiguous range of spectra.  Its warps have roles:
//   producer (1 warp, lane 0): 1-D bulk copies of whole input frames into a
//       ring of NSLOT shared-memory slots (mbarrier complete_tx), in frame
//       order, so every input byte is read from HBM exactly once per CTA
//       (an L2 prefetch running ahead of the ring measured slower);
//   FIR warps (P/NB threads, NB consecutive branches each): stream the frames
//       out of the ring; the branch sums of the T spectra a frame feeds live in
//       registers (slot (s mod T), rotated at compile time by unrolling the
//       frame loop T times), so each frame costs T fp32x2 FMAs per branch and
//       one spectrum of branch sums completes per frame; rows go to a
//       double-buffered batch buffer Y in shared memory (SB spectra);
//   FFT warps (128 threads): radix-16 Stockham passes, out of place
//       (Y -> W0 -> W1 -> HBM), natural-order bins stored straight from
//       registers; they release Y as soon as the first pass has read it.
// Roles hand over through mbarriers; every wait is bounded (1 s of
// %globaltimer) and a timeout sets the launch's error word and winds down.
// For P = 1024 (4 branches per FIR thread, 16 taps) the FIR warpgroups take
// 208 registers, the FFT warpgroup 72 and the producer warpgroup 24
// (setmaxnreg): 256*208 + 128*72 + 128*24 = 512*128 registers at launch.
// P = 1024 splits the DFT once more (decimation in frequency by 4): FIR thread
// t owns branches t + k*P/4 (k = 0..3) and hands over the radix-4 butterfly
// of its four branch sums, output k1 already multiplied by w_P^(t k1); the
// FFT warps finish four P/4-point transforms (Y -> W -> HBM), bin 4m + k1
// coming from sub-transform k1.  Otherwise thread t owns the branch
// pairs (2t, 2t+1) + k*P/NPAIR.  Either way its ring reads and branch-sum
// writes are contiguous across the warp (no shared-memory bank conflicts).
#pragma once

#include "devutil.cuh"
#include "fftplan.h"
#include "internal.h"
#include "sync.cuh"
#include "tc.cuh"

namespace pfb {

template <int P, int TT, int IN, bool TC = false>
struct WsCfg {
    static constexpr int NB = P >= 1024 ? 4 : (P >= 512 ? 2 : 1);  // branches per FIR thread
    static constexpr int NPAIR = NB >= 2 ? NB / 2 : 1;              // branch pairs (2t, 2t+1) + k P/NPAIR
    // P = 1024: thread t owns branches t + k*P/4 and applies the first radix-4
    // decimation-in-frequency butterfly before handing over; the FFT warps
    // apply its twiddles in their first pass and run four P/4-point
    // transforms per spectrum
    static constexpr bool DIF4 = (P == 1024) && !TC;
    static constexpr int Q = P / 4;                                  // sub-transform length (DIF4)
    static constexpr int SROW = Q + Q / 16 + 8;                      // sub-row stride (float2), 16 banks apart
    static constexpr int NFT = P / NB;                               // FIR threads
    static constexpr int NFIRW = NFT / 32;
    static constexpr bool SETMAXNREG = (P >= 1024);
    static constexpr int NFFTW = 4;                                  // FFT warps (one per SM sub-partition)
    static constexpr int NFFTT = NFFTW * 32;
    static constexpr int PRODW = NFIRW + NFFTW;                      // producer warp index
    // with setmaxnreg the producer sits in a warpgroup of its own (3 idle warps)
    static constexpr int NTHREADS = NFT + NFFTT + (SETMAXNREG ? 128 : 32);
    static constexpr int SB = 4;                                     // spectra per FFT batch
    static_assert(TT % SB == 0, "batch rows follow the frame loop's unrolling");
    static constexpr int MR = 16;
    static constexpr int G = 16;
    static constexpr int YROW = P + P / G;
    static constexpr int NSLOT = 8;
    static constexpr int ESZ = IN == PFB_IN_C64 ? 8 : (IN == PFB_IN_R32 ? 4 : 2);
    static constexpr int FB = P * ESZ;                               // frame bytes
    // pass twiddles: the P-point list, or (DIF4) the Q-point list, which is a
    // prefix of the P-point table, followed by w_P^(t k), k = 1..3, t < Q
    static constexpr int NTW = DIF4 ? fft_tw_entries(Q, MR) + 3 * Q : fft_tw_entries(P, MR);
    static constexpr int NPASS = DIF4 ? fft_npasses(Q, MR) : fft_npasses(P, MR);
    // shared memory layout (bytes); DIF4 needs one W buffer (two passes)
    static constexpr int OFF_RING = 0;
    static constexpr int OFF_Y = OFF_RING + NSLOT * FB;
    static constexpr int YBUF = DIF4 ? SB * 4 * SROW * 8 : SB * YROW * 8;
    static constexpr int OFF_W = OFF_Y + 2 * YBUF;
    static constexpr int OFF_TW = OFF_W + (TC ? 0 : (DIF4 ? 1 : 2) * YBUF);
    // TC (tensor-core four-step DFT, P = 32 x 32): the step-2 A operand
    // (bf16 hi and lo, K-major, 128 rows x 64), the 32-point DFT matrix in
    // real block form (bf16 hi and lo, K-major tile of 64 x 64) and the
    // twiddles w_P^(k1 n2) as a [k1][n2] table
    static constexpr int TC_P1 = 32;
    static constexpr int TC_LBO_A = 2064;                            // K-group stride: 16 B off 128 -> 4 banks
    static constexpr int TC_A2B = 8 * TC_LBO_A;                      // bytes of one A2 term
    static constexpr int TC_BTB = 64 * 64 * 2;                       // bytes of one B term
    static constexpr int OFF_A2 = OFF_TW;
    static constexpr int OFF_BT = OFF_A2 + (TC ? 2 * TC_A2B : 0);
    static constexpr int OFF_TWT = OFF_BT + (TC ? 2 * TC_BTB : 0);
    static constexpr int OFF_META = TC ? OFF_TWT + TC_P1 * TC_P1 * 8 : OFF_TW + (NTW > 0 ? NTW : 1) * 8;
    static constexpr int OFF_BAR = OFF_META + 3 * 32;
    static constexpr int NBAR = 2 * NSLOT + 4 + (TC ? 4 : 0);  // TC: MMA 1/2 done, operand 1/2 ready
    static constexpr int SMEM = OFF_BAR + NBAR * 8 + 16;
    static_assert(!TC || (P == TC_P1 * TC_P1 && SB * TC_P1 == 128), "TC: P = 32 x 32, 4 spectra per 128-row tile");
    static_assert(!TC || (OFF_A2 % 128 == 0 && OFF_BT % 128 == 0), "TC operand alignment");
    static_assert(!TC || SETMAXNREG, "TC: the MMA issuer is a warp of the producer warpgroup");
    static_assert(NFT % 128 == 0 || !SETMAXNREG, "FIR warps form whole warpgroups");
    static_assert(!DIF4 || (NB == 4 && NFT == Q && fft_npasses(Q, MR) == 2), "DIF4 layout");
    static_assert(NFIRW * 32 + NFFTT + (SETMAXNREG ? 128 : 32) == NTHREADS, "layout");
    // register split (setmaxnreg): FIR 208, FFT 72, producer warpgroup 24; the
    // tensor-core DFT warps (TC) keep more live values, their FIR is lighter
    static constexpr int REG_FIR = TC ? 200 : 208, REG_FFT = TC ? 88 : 72, REG_PROD = 24;
    static_assert(!SETMAXNREG || NFT * REG_FIR + NFFTT * REG_FFT + 128 * REG_PROD <= NTHREADS * (65536 / NTHREADS),
                  "registers");
};

struct WsMeta {
    float2 *out;   // first output row of the batch
    int64_t ldo;   // output row stride (complex64 elements)
    int nrows;
    int pad[3];
};

// one out-of-place Stockham pass over a batch of SB rows, run by the FFT warps
// PRETW: rows are the DIF4 sub-rows (row mod 4 = k1) and element n of sub-row
// k1 is first multiplied by pre[(k1 - 1) * P + n] = w_{4P}^(n k1) (k1 > 0)
template <int P, int MR, int SB, int PASS, bool LAST, int YROW, int G, bool PRETW = false>
__device__ __forceinline__ void ws_pass(const float2 *src, float2 *dst, const float2 *tw, float2 *out_row0, int nrows,
                                        int ft, int nft, const float2 *pre = nullptr, int64_t ldo = P) {
    constexpr int R = fft_radix(P, PASS, MR);
    constexpr int NS = fft_ns(P, PASS, MR);
    constexpr int STRIDE = P / R;
    constexpr int NBF = SB * STRIDE;  // butterflies in the batch
    const float2 *twp = tw + fft_tw_offset(P, PASS, MR);
#pragma unroll 1
    for (int b = ft; b < NBF; b += nft) {
        const int row = b / STRIDE, j = b % STRIDE;
        float2 v[R];
        const float2 *s = src + row * YROW;
        if constexpr (STRIDE % G == 0) {
            s += ypad<G>(j);
#pragma unroll
            for (int r = 0; r < R; ++r) v[r] = s[r * (STRIDE + STRIDE / G)];
        } else {
#pragma unroll
            for (int r = 0; r < R; ++r) v[r] = s[ypad<G>(j + r * STRIDE)];
        }
        if constexpr (PRETW) {
            const int k1 = row & 3;
            if (k1 != 0) {
                const float2 *w = pre + (k1 - 1) * P + j;
#pragma unroll
                for (int r = 0; r < R; ++r) v[r] = cmul(v[r], w[r * STRIDE]);
            }
        }
        if constexpr (NS > 1) {
            const float2 *w = twp + (j % NS) * (R - 1);
#pragma unroll
            for (int r = 1; r < R; ++r) v[r] = cmul(v[r], w[r - 1]);
        }
        dft_reg<R, true>(v);
        if constexpr (!LAST) {
            float2 *d = dst + row * YROW;
            if constexpr (NS == 1) {
                static_assert(R == G, "first pass radix equals the padding period");
                d += (G + 1) * j;
#pragma unroll
                for (int r = 0; r < R; ++r) d[r] = v[r];
            } else {
                d += ypad<G>((j / NS) * NS * R + (j % NS));
#pragma unroll
                for (int r = 0; r < R; ++r) d[r * (NS + NS / G)] = v[r];
            }
        } else {
            if (row < nrows) {
                float2 *o = out_row0 + row * ldo + j;
#pragma unroll
                for (int r = 0; r < R; ++r) store_cs(o + r * NS, v[r]);
            }
        }
    }
}

template <int P, int MR, int SB, int PASS, int YROW, int G>
__device__ __forceinline__ void ws_passes(float2 *Y, float2 *W0, float2 *W1, const float2 *tw, float2 *out_row0,
                                          int nrows, int ft, int nft, uint32_t yempty_bar, int nfftt, int64_t ldo) {
    constexpr int NPASS = fft_npasses(P, MR);
    constexpr bool LAST = (PASS == NPASS - 1);
    const float2 *src = (PASS == 0) ? Y : ((PASS % 2 == 1) ? W0 : W1);
    float2 *dst = (PASS % 2 == 0) ? W0 : W1;
    ws_pass<P, MR, SB, PASS, LAST, YROW, G>(src, dst, tw, out_row0, nrows, ft, nft, nullptr, ldo);
    if constexpr (!LAST) {
        named_bar_sync<1>(nfftt);
        if (PASS == 0 && ft == 0) mbar_arrive(yempty_bar);  // Y has been read: the FIR warps may refill it
        ws_passes<P, MR, SB, PASS + 1, YROW, G>(Y, W0, W1, tw, out_row0, nrows, ft, nft, yempty_bar, nfftt, ldo);
    } else if constexpr (PASS == 0) {
        // single-pass transform (not used for P >= 64)
        if (ft == 0) mbar_arrive(yempty_bar);
    }
}

// Last pass of the four Q-point sub-transforms of each spectrum (DIF4): sub-
// transform k1 of row `row` sits at sub-row 4*row + k1; its bin m is the
// spectrum's bin 4m + k1.  k1 varies fastest across threads, so each store
// instruction writes 32 consecutive bins.
template <int Q, int SB, int SROW, int G>
__device__ __forceinline__ void ws_dif4_last(const float2 *src, const float2 *tw, float2 *out_row0, int nrows, int ft,
                                             int nft, int64_t ldo) {
    constexpr int MR = 16;
    constexpr int PASS = fft_npasses(Q, MR) - 1;
    constexpr int R = fft_radix(Q, PASS, MR);
    constexpr int NS = fft_ns(Q, PASS, MR);
    constexpr int STRIDE = Q / R;
    static_assert(STRIDE == NS && STRIDE % G == 0, "last pass");
    constexpr int NBF = SB * 4 * STRIDE;
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
            float2 *o = out_row0 + row * ldo + 4 * j + k1;
#pragma unroll
            for (int r = 0; r < R; ++r) store_cs(o + 4 * NS * r, v[r]);
        }
    }
}

// named barrier that also ORs a predicate over the participating threads
template <int ID>
__device__ __forceinline__ bool named_bar_or(int nthreads, bool v) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\tbar.red.or.pred q, %2, %3, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)v), "n"(ID), "r"(nthreads)
        : "memory");
    return r != 0;
}

// iterate the CTA's spectra range as (stream, [sA, sB)) segments
struct WsRange {
    int64_t u, u1;
};

__device__ __forceinline__ bool ws_next_segment(const LaunchArgs &a, WsRange &r, int &si, int64_t &sA, int64_t &sB) {
    if (r.u >= r.u1) return false;
    si = find_stream(a, r.u);
    const StreamDesc &d = a.s[si];
    const int64_t end = min(r.u1, d.unit0 + d.S);
    sA = r.u - d.unit0;
    sB = end - d.unit0;
    r.u = end;
    return true;
}

// ---------------------------------------------------------------------------
// Tensor-core DFT warps (TC): the DFT of Sec. 4.1 as two 32-point DFT-matrix
// products on the tensor cores (four-step form, P = 32 x 32, p = 32 n1 + n2,
// k = k1 + 32 k2), split-bf16 operands (hi = RN(v), lo = RN(v - hi); three
// products hi*hi + hi*lo + lo*hi), FP32 accumulation in TMEM:
//   Z[n2][k1]       = sum_{n1} y[32 n1 + n2] w_32^(n1 k1)        (MMA 1)
//   X[k1 + 32 k2]   = sum_{n2} (Z[n2][k1] w_P^(n2 k1)) w_32^(n2 k2)  (MMA 2)
// One batch = 4 spectra = one 128-row tile; warp w (TMEM lane quarter w mod 4)
// owns spectrum w mod 4 of the batch.  MMA 1: A = branch sums in TMEM (row
// (s, n2), K = (n1, re/im)), written by tcgen05.st; MMA 2: A in shared memory
// (row (s, k1), K = (n2, re/im)), written transposed from the MMA 1 result
// after the twiddle; B = the real block form [[Re, Im], [-Im, Re]] of the
// 32-point DFT matrix, the same for both.  Bins leave straight from TMEM.
// ---------------------------------------------------------------------------
constexpr uint32_t kTcCols = 256;                  // A1 [0, 64), D1 [64, 128), D2 [128, 192)
constexpr uint32_t kTcColA1 = 0, kTcColD1 = 64, kTcColD2 = 128;

// MMA issue for one batch: step 1 (A in TMEM) or step 2 (A in shared memory),
// 4 K-steps x 3 split products, then a commit to `bar`
template <class C>
__device__ __forceinline__ void ws_tc_issue(bool step2, uint32_t tmem, uint32_t sA2, uint32_t sBT, uint32_t bar) {
    constexpr uint32_t IDESC = tc_idesc_bf16(128, 64);
    constexpr int LBO_A = C::TC_LBO_A;
#pragma unroll 1
    for (int ks = 0; ks < 4; ++ks) {  // K = 64 in steps of 16
        const uint64_t bh = tc_desc_kmajor(sBT + ks * 256, 128, 1024);
        const uint64_t bl = tc_desc_kmajor(sBT + C::TC_BTB + ks * 256, 128, 1024);
        if (!step2) {
            const uint32_t d = tmem + kTcColD1, ah = tmem + kTcColA1 + 8 * ks, al = ah + 32;
            tc_mma_ts(d, ah, bh, IDESC, ks > 0);
            tc_mma_ts(d, ah, bl, IDESC, 1u);
            tc_mma_ts(d, al, bh, IDESC, 1u);
        } else {
            const uint32_t d = tmem + kTcColD2;
            const uint64_t ah = tc_desc_kmajor(sA2 + ks * 2 * LBO_A, LBO_A, 128);
            const uint64_t al = tc_desc_kmajor(sA2 + C::TC_A2B + ks * 2 * LBO_A, LBO_A, 128);
            tc_mma_ss(d, ah, bh, IDESC, ks > 0);
            tc_mma_ss(d, ah, bl, IDESC, 1u);
            tc_mma_ss(d, al, bh, IDESC, 1u);
        }
    }
    tc_commit(bar);
}

// The MMA issuer (one thread of the producer warpgroup): per batch, waits for
// the DFT warps' step-1 operand, issues MMA 1, waits for the step-2 operand,
// issues MMA 2.  Keeps the tensor-core issue off the DFT warps' path.
template <class C>
__device__ __forceinline__ void ws_tc_mma_thread(const LaunchArgs &a, WsRange range, uint8_t *ws_smem, uint32_t op1,
                                                 uint32_t op2, uint32_t mbar1, uint32_t mbar2, uint32_t tmem,
                                                 volatile int *abort_flag) {
    constexpr int SB = C::SB;
    const uint32_t sA2 = smem_u32(ws_smem + C::OFF_A2), sBT = smem_u32(ws_smem + C::OFF_BT);
    uint32_t bc = 0, issued1 = 0, issued2 = 0;
    bool ok = true;
    int si;
    int64_t sA, sB;
    while (ok && ws_next_segment(a, range, si, sA, sB)) {
        const int64_t nb = (sB - sA + SB - 1) / SB;
        for (int64_t qb = 0; qb < nb && ok; ++qb, ++bc) {
            if (!mbar_wait(op1, bc & 1, a.wait_ns)) {
                ok = false;
                break;
            }
            tc_fence_after();
            ws_tc_issue<C>(false, tmem, sA2, sBT, mbar1);
            ++issued1;
            if (!mbar_wait(op2, bc & 1, a.wait_ns)) {
                ok = false;
                break;
            }
            tc_fence_after();
            ws_tc_issue<C>(true, tmem, sA2, sBT, mbar2);
            ++issued2;
        }
    }
    if (!ok) *abort_flag = 1;
    // everything issued has completed before the CTA frees TMEM
    if (issued1 && !mbar_wait(mbar1, (issued1 - 1) & 1, a.wait_ns)) *abort_flag = 1;
    if (issued2 && !mbar_wait(mbar2, (issued2 - 1) & 1, a.wait_ns)) *abort_flag = 1;
}

template <class C>
__device__ __forceinline__ void ws_tc_dft(const LaunchArgs &a, WsRange range, uint8_t *ws_smem, WsMeta *meta,
                                          uint32_t yfull0, uint32_t yempty0, uint32_t op1, uint32_t op2,
                                          uint32_t mbar1, uint32_t mbar2, uint32_t tmem, volatile int *abort_flag,
                                          int ft, int warp, int lane) {
    constexpr int SB = C::SB, YROW = C::YROW, G = C::G, P = C::TC_P1 * C::TC_P1, NT = C::NFFTT;
    constexpr int LBO_A = C::TC_LBO_A;
    const int q = warp & 3;  // spectrum of the batch = TMEM lane quarter
    const uint32_t trow = tmem + ((uint32_t)(32 * q) << 16);
    uint8_t *a2 = ws_smem + C::OFF_A2;
    const float2 *twt = reinterpret_cast<const float2 *>(ws_smem + C::OFF_TWT);
    const float2 *Y = reinterpret_cast<const float2 *>(ws_smem + C::OFF_Y);
    // a2 byte offset of this thread's (re, im) pair in row m = 32 q + k1, K = (n2 = lane, re/im)
    const int a2_base = (lane >> 2) * LBO_A + (lane & 3) * 4 + (4 * q) * 128;
    // every DFT thread waits; the barrier ORs the failures so all take the same path
    uint32_t ph1 = 0, ph2 = 0;  // completions observed on mbar1 / mbar2
    auto wait_mma = [&](uint32_t bar, uint32_t &ph) {
        const bool w = mbar_wait(bar, ph & 1, a.wait_ns);
        ++ph;
        const bool fail = named_bar_or<2>(NT, !w);
        tc_fence_after();
        return !fail;
    };
    // bins k1 + 32 k2 of spectrum q of a finished batch (thread k1 = lane)
    auto epilogue = [&](const WsMeta &mt) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            uint32_t r[32];
            tmem_ld32(trow + kTcColD2 + 32 * h, r);
            tmem_wait_ld();
            if (q < mt.nrows) {
                float2 *o = mt.out + q * mt.ldo + lane + 32 * (16 * h);
#pragma unroll
                for (int j = 0; j < 16; ++j)
                    store_cs(o + 32 * j, make_float2(__uint_as_float(r[2 * j]), __uint_as_float(r[2 * j + 1])));
            }
        }
    };
    uint32_t bc = 0;
    bool ok = true, have_prev = false;
    WsMeta mt_prev;
    int si;
    int64_t sA, sB;
    // Pipeline over batches b: T1(b) | MMA 1(b) under epilogue(b-1) ; T2(b) | MMA 2(b) under T1(b+1)
    while (ok && ws_next_segment(a, range, si, sA, sB)) {
        const int64_t nb = (sB - sA + SB - 1) / SB;
        for (int64_t qb = 0; qb < nb && ok; ++qb, ++bc) {
            if (ft == 0) meta[2].nrows = mbar_wait(yfull0 + 8 * (bc & 1), (bc >> 1) & 1, a.wait_ns) ? 1 : 0;
            named_bar_sync<1>(NT);
            if (!meta[2].nrows) {
                *abort_flag = 1;
                ok = false;
                break;
            }
            const WsMeta mt = meta[bc & 1];
            // ---- MMA 1 operand: row (q, n2 = lane), K = (n1, re/im), into TMEM ----
            const float2 *yrow = Y + (bc & 1) * (SB * YROW) + q * YROW;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                uint32_t vh[16], vl[16];
#pragma unroll
                for (int j = 0; j < 16; ++j) split_bf16x2(yrow[ypad<G>(32 * (16 * h + j) + lane)], vh[j], vl[j]);
                tmem_st<16>(trow + kTcColA1 + 16 * h, vh);
                tmem_st<16>(trow + kTcColA1 + 32 + 16 * h, vl);
            }
            tmem_wait_st();
            mbar_arrive(yempty0 + 8 * (bc & 1));  // this thread is done with Y
            tc_fence_before();
            mbar_arrive(op1);
            // ---- while MMA 1 runs: the previous batch's bins ----
            if (have_prev) {
                if (!wait_mma(mbar2, ph2)) {
                    *abort_flag = 1;
                    ok = false;
                    break;
                }
                epilogue(mt_prev);
                have_prev = false;
            }
            if (!wait_mma(mbar1, ph1)) {
                *abort_flag = 1;
                ok = false;
                break;
            }
            // ---- twiddle, split, transposed store: MMA 2 operand row (q, k1), K = (n2 = lane, re/im) ----
#pragma unroll
            for (int h = 0; h < 4; ++h) {  // 8 k1 per TMEM load
                // the twiddles first: the operand stores below may alias them for the compiler
                float2 w8[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) w8[j] = twt[(8 * h + j) * C::TC_P1 + lane];
                uint32_t r[16];
                tmem_ld16(trow + kTcColD1 + 16 * h, r);
                tmem_wait_ld();
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int k1 = 8 * h + j;
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
            mbar_arrive(op2);
            mt_prev = mt;
            have_prev = true;
        }
    }
    if (ok && have_prev) {
        if (wait_mma(mbar2, ph2)) epilogue(mt_prev);
        else *abort_flag = 1;
    }
}

template <int P, int TT, int IN, bool TC = false>
__global__ void __launch_bounds__(WsCfg<P, TT, IN, TC>::NTHREADS, 1) k_fft_ws(const __grid_constant__ LaunchArgs a) {
    using C = WsCfg<P, TT, IN, TC>;
    constexpr int NB = C::NB, SB = C::SB, NSLOT = C::NSLOT, YROW = C::YROW, G = C::G;
    extern __shared__ __align__(128) uint8_t ws_smem[];
    uint8_t *ring = ws_smem + C::OFF_RING;
    float2 *Y = reinterpret_cast<float2 *>(ws_smem + C::OFF_Y);
    float2 *W = reinterpret_cast<float2 *>(ws_smem + C::OFF_W);
    float2 *tw = reinterpret_cast<float2 *>(ws_smem + C::OFF_TW);
    WsMeta *meta = reinterpret_cast<WsMeta *>(ws_smem + C::OFF_META);
    uint64_t *bars = reinterpret_cast<uint64_t *>(ws_smem + C::OFF_BAR);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(bars + C::NBAR);
    const uint32_t full0 = smem_u32(&bars[0]), empty0 = smem_u32(&bars[NSLOT]);
    const uint32_t yfull0 = smem_u32(&bars[2 * NSLOT]), yempty0 = smem_u32(&bars[2 * NSLOT + 2]);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int i = 0; i < NSLOT; ++i) {
            mbar_init(full0 + 8 * i, 1);
            mbar_init(empty0 + 8 * i, C::NFIRW);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(yfull0 + 8 * i, C::NFIRW);
            mbar_init(yempty0 + 8 * i, TC ? C::NFFTT : 1);  // TC: every DFT thread releases Y
        }
        if constexpr (TC) {
            mbar_init(smem_u32(&bars[2 * NSLOT + 4]), 1);         // MMA 1 complete (tcgen05.commit)
            mbar_init(smem_u32(&bars[2 * NSLOT + 5]), 1);         // MMA 2 complete
            mbar_init(smem_u32(&bars[2 * NSLOT + 6]), C::NFFTT);  // step-1 operand written
            mbar_init(smem_u32(&bars[2 * NSLOT + 7]), C::NFFTT);  // step-2 operand written
        }
        mbar_init_fence();
        *abort_flag = 0;
    }
    // twiddle tables into shared memory (all threads, before the roles split)
    if constexpr (C::DIF4) {
        constexpr int NTQ = fft_tw_entries(C::Q, C::MR);
        const float2 *tw_half = static_cast<const float2 *>(a.aux);  // w_P^r, r < P/2
        for (int i = threadIdx.x; i < NTQ; i += C::NTHREADS) tw[i] = a.tw[i];
        for (int i = threadIdx.x; i < 3 * C::Q; i += C::NTHREADS) {
            const int r = (i / C::Q + 1) * (i % C::Q);  // w_P^(t k1), t = i mod Q, k1 = i / Q + 1
            const float2 w = tw_half[r % (P / 2)];
            tw[NTQ + i] = r < P / 2 ? w : make_float2(-w.x, -w.y);
        }
    } else if constexpr (TC) {
        // DFT matrix hi/lo tiles and twiddles, 16-byte vectors
        const int4 *src = static_cast<const int4 *>(a.aux);
        int4 *dst = reinterpret_cast<int4 *>(ws_smem + C::OFF_BT);
        constexpr int NV = (2 * C::TC_BTB + C::TC_P1 * C::TC_P1 * 8) / 16;
        for (int i = threadIdx.x; i < NV; i += C::NTHREADS) dst[i] = src[i];
    } else {
        for (int i = threadIdx.x; i < C::NTW; i += C::NTHREADS) tw[i] = a.tw[i];
    }
    volatile uint32_t *tmem_slot = reinterpret_cast<volatile uint32_t *>(abort_flag + 1);
    if constexpr (TC) {
        if (warp == C::NFIRW) tmem_alloc(smem_u32((const void *)tmem_slot), kTcCols);
        fence_proxy_async_smem();  // the tables are read by the tensor core
        tc_fence_before();
    }
    __syncthreads();
    if constexpr (TC) tc_fence_after();

    WsRange range;
    range.u = (int64_t)blockIdx.x * a.units_per_cta;
    range.u1 = min(range.u + (int64_t)a.units_per_cta, a.nunits);

    if (warp < C::NFIRW) {
        // ======================= FIR warps =======================
        if constexpr (C::SETMAXNREG) asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(C::REG_FIR) : "memory");
        const int t = threadIdx.x;
        constexpr int NPAIR = C::NPAIR;
        constexpr int PSTRIDE = P / NPAIR;   // distance between this thread's branch pairs
        // branch of (pair k, b): k * PSTRIDE + 2t + b   (NB = 1: branch t)
        auto branch = [&](int k, int b) {
            if constexpr (C::DIF4) return (2 * k + b) * C::Q + t;
            else return NB == 1 ? t : k * PSTRIDE + 2 * t + b;
        };
        float h[TT][NB];
        float2 pend[TT][NB];
        // DIF4: this thread's twiddles w_P^(t k1), k1 = 1..3, applied to the
        // butterfly outputs before they are handed over
        float2 wt[3];
        if constexpr (C::DIF4) {
#pragma unroll
            for (int k1 = 1; k1 < 4; ++k1) wt[k1 - 1] = tw[fft_tw_entries(C::Q, C::MR) + (k1 - 1) * C::Q + t];
        }
        int cur = -1;
        uint32_t pc = 0;   // frames consumed
        uint32_t bc = 0;   // batches produced
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
                    for (int b = 0; b < NB; ++b) h[m][b] = __ldg(d.taps + m * P + branch(b >> 1, b & 1));
            }
            // segment-relative counters fit 32 bits: a segment is at most one
            // CTA's range (units_per_cta, checked on the host)
            const int nspec = (int)(sB - sA);
            const int nfr = nspec + TT - 1;
            float2 *out_seg = d.out + sA * d.ldo;
            for (int i0 = 0; i0 < nfr && ok; i0 += TT) {
#pragma unroll
                for (int k = 0; k < TT; ++k) {
                    const int i = i0 + k;
                    if (i < nfr) {
                        // ---- frame i of the segment from the ring ----
                        const uint32_t slot = pc % NSLOT;
                        // warp-uniform decision: every lane takes the same path
                        if (!__all_sync(0xffffffffu, mbar_wait(full0 + 8 * slot, (pc / NSLOT) & 1, a.wait_ns))) {
                            *abort_flag = 1;
                            ok = false;
                            break;
                        }
                        float2 v[NB];
                        {
                            const uint8_t *fr = ring + slot * C::FB;
                            const float sc = d.scale;
#pragma unroll
                            for (int k2 = 0; k2 < NPAIR; ++k2) {
                                if constexpr (C::DIF4) {
#pragma unroll
                                    for (int b = 0; b < 2; ++b) {
                                        const int q = branch(k2, b);
                                        if constexpr (IN == PFB_IN_C64) v[2 * k2 + b] = reinterpret_cast<const float2 *>(fr)[q];
                                        else if constexpr (IN == PFB_IN_R32)
                                            v[2 * k2 + b] = make_float2(reinterpret_cast<const float *>(fr)[q], 0.f);
                                        else {
                                            const char2 c2 = reinterpret_cast<const char2 *>(fr)[q];
                                            v[2 * k2 + b] = make_float2((float)c2.x * sc, (float)c2.y * sc);
                                        }
                                    }
                                } else if constexpr (NB == 1) {
                                    if constexpr (IN == PFB_IN_C64) v[0] = reinterpret_cast<const float2 *>(fr)[t];
                                    else if constexpr (IN == PFB_IN_R32)
                                        v[0] = make_float2(reinterpret_cast<const float *>(fr)[t], 0.f);
                                    else {
                                        const char2 c2 = reinterpret_cast<const char2 *>(fr)[t];
                                        v[0] = make_float2((float)c2.x * sc, (float)c2.y * sc);
                                    }
                                } else {
                                    const int q = branch(k2, 0);   // even branch of the pair
                                    if constexpr (IN == PFB_IN_C64) {
                                        const float4 w4 = reinterpret_cast<const float4 *>(fr)[q >> 1];
                                        v[2 * k2] = make_float2(w4.x, w4.y);
                                        v[2 * k2 + 1] = make_float2(w4.z, w4.w);
                                    } else if constexpr (IN == PFB_IN_R32) {
                                        const float2 w2 = reinterpret_cast<const float2 *>(fr)[q >> 1];
                                        v[2 * k2] = make_float2(w2.x, 0.f);
                                        v[2 * k2 + 1] = make_float2(w2.y, 0.f);
                                    } else {
                                        const char4 c4 = reinterpret_cast<const char4 *>(fr)[q >> 1];
                                        v[2 * k2] = make_float2((float)c4.x * sc, (float)c4.y * sc);
                                        v[2 * k2 + 1] = make_float2((float)c4.z * sc, (float)c4.w * sc);
                                    }
                                }
                            }
                            // the previous frame's ring slot goes back to the producer now:
                            // every lane has used the values it loaded from it (a TMA refill
                            // must not overtake a shared-memory read still in flight)
                            __syncwarp();
                            if (lane == 0 && pc > 0) mbar_arrive(empty0 + 8 * ((pc - 1) % NSLOT));
                        }
                        ++pc;
                        // ---- feed the T spectra this frame belongs to ----
                        // frame i contributes h[m] * x to spectrum i - m; slot (i - m) mod TT
#pragma unroll
                        for (int b = 0; b < NB; ++b) pend[k][b] = make_float2(h[0][b] * v[b].x, h[0][b] * v[b].y);
#pragma unroll
                        for (int m = 1; m < TT; ++m) {
                            const int js = ((k - m) % TT + TT) % TT;
#pragma unroll
                            for (int b = 0; b < NB; ++b)
                                pend[js][b] = fma2(make_float2(h[m][b], h[m][b]), v[b], pend[js][b]);
                        }
                        // ---- spectrum i - TT + 1 is complete ----
                        const int jspec = i - (TT - 1);
                        if (jspec >= 0) {
                            const int jslot = ((k + 1) % TT);
                            // row of the batch: every segment's batches start at its spectrum 0
                            // and SB divides TT, so the row is (k + 1) mod SB, fixed at compile time
                            const int brow = (k + 1) % SB;
                            // new batch: wait until the FFT warps have released this Y buffer
                            if (brow == 0 && bc >= 2 &&
                                !__all_sync(0xffffffffu, mbar_wait(yempty0 + 8 * (bc & 1), ((bc >> 1) + 1) & 1, a.wait_ns))) {
                                *abort_flag = 1;
                                ok = false;
                                break;
                            }
                            if constexpr (C::DIF4) {
                                // radix-4 DIF butterfly on y[t + k Q], k = 0..3
                                float2 *ysub = reinterpret_cast<float2 *>(ws_smem + C::OFF_Y + (bc & 1) * C::YBUF) +
                                               brow * 4 * C::SROW + ypad<G>(t);
                                const float2 a0 = cadd2(pend[jslot][0], pend[jslot][2]);
                                const float2 a1 = csub2(pend[jslot][0], pend[jslot][2]);
                                const float2 a2 = cadd2(pend[jslot][1], pend[jslot][3]);
                                const float2 a3 = csub2(pend[jslot][1], pend[jslot][3]);
                                const float2 mi_a3 = make_float2(a3.y, -a3.x);  // -i a3
                                ysub[0] = cadd2(a0, a2);
                                ysub[C::SROW] = cmul(cadd2(a1, mi_a3), wt[0]);
                                ysub[2 * C::SROW] = cmul(csub2(a0, a2), wt[1]);
                                ysub[3 * C::SROW] = cmul(csub2(a1, mi_a3), wt[2]);
                            } else {
                                float2 *yrow = Y + (bc & 1) * (SB * YROW) + brow * YROW;
#pragma unroll
                                for (int b = 0; b < NB; ++b) yrow[ypad<G>(branch(b >> 1, b & 1))] = pend[jslot][b];
                            }
                            if (brow == SB - 1 || jspec == nspec - 1) {
                                if (t == 0) {
                                    meta[bc & 1].out = out_seg + (int64_t)(jspec - brow) * d.ldo;
                                    meta[bc & 1].ldo = d.ldo;
                                    meta[bc & 1].nrows = brow + 1;
                                }
                                __syncwarp();
                                if (lane == 0) mbar_arrive(yfull0 + 8 * (bc & 1));
                                ++bc;
                            }
                        }
                    }
                }
            }
        }
    } else if (warp < C::PRODW) {
        // ======================= FFT warps =======================
        if constexpr (C::SETMAXNREG) asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(C::REG_FFT) : "memory");
        const int ft = threadIdx.x - C::NFT;
        if constexpr (TC) {
            ws_tc_dft<C>(a, range, ws_smem, meta, yfull0, yempty0, smem_u32(&bars[2 * NSLOT + 6]),
                         smem_u32(&bars[2 * NSLOT + 7]), smem_u32(&bars[2 * NSLOT + 4]),
                         smem_u32(&bars[2 * NSLOT + 5]), *tmem_slot, abort_flag, ft, warp, lane);
        } else {
        uint32_t bc = 0;
        bool ok = true;
        int si;
        int64_t sA, sB;
        while (ok && ws_next_segment(a, range, si, sA, sB)) {
            const int64_t nb = (sB - sA + SB - 1) / SB;
            for (int64_t q = 0; q < nb && ok; ++q, ++bc) {
                // one thread waits, the decision is broadcast so that every FFT
                // thread reaches the same named barriers
                if (ft == 0) meta[2].nrows = mbar_wait(yfull0 + 8 * (bc & 1), (bc >> 1) & 1, a.wait_ns) ? 1 : 0;
                named_bar_sync<1>(C::NFFTT);
                if (!meta[2].nrows) {
                    *abort_flag = 1;
                    ok = false;
                    break;
                }
                const WsMeta mt = meta[bc & 1];
                float2 *Yb = Y + (bc & 1) * (SB * YROW);
                if constexpr (C::DIF4) {
                    Yb = reinterpret_cast<float2 *>(ws_smem + C::OFF_Y + (bc & 1) * C::YBUF);
                    ws_pass<C::Q, C::MR, 4 * SB, 0, false, C::SROW, G>(Yb, W, tw, nullptr, 0, ft, C::NFFTT);
                    named_bar_sync<1>(C::NFFTT);
                    if (ft == 0) mbar_arrive(yempty0 + 8 * (bc & 1));  // Y has been read
                    ws_dif4_last<C::Q, SB, C::SROW, G>(W, tw, mt.out, mt.nrows, ft, C::NFFTT, mt.ldo);
                } else {
                    ws_passes<P, C::MR, SB, 0, YROW, G>(Yb, W, W + SB * YROW, tw, mt.out, mt.nrows, ft, C::NFFTT,
                                                        yempty0 + 8 * (bc & 1), C::NFFTT, mt.ldo);
                }
                named_bar_sync<1>(C::NFFTT);  // W buffers free before the next batch
            }
        }
        }
    } else {
        // ======================= producer warp(group) =======================
        if constexpr (C::SETMAXNREG) asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(C::REG_PROD) : "memory");
        if constexpr (TC) {
            if (warp == C::PRODW + 1 && lane == 0)
                ws_tc_mma_thread<C>(a, range, ws_smem, smem_u32(&bars[2 * NSLOT + 6]), smem_u32(&bars[2 * NSLOT + 7]),
                                    smem_u32(&bars[2 * NSLOT + 4]), smem_u32(&bars[2 * NSLOT + 5]), *tmem_slot,
                                    abort_flag);
        }
        if (warp == C::PRODW && lane == 0) {
            uint32_t pc = 0;
            // error-reporting test hook: with FAULT_NO_COPIES the producer
            // issues no copies at all, so every consumer's bounded wait runs
            // out, the roles wind down and the error word is set
            bool ok = TC || a.fault != FAULT_NO_COPIES;
            int si;
            int64_t sA, sB;
            while (ok && ws_next_segment(a, range, si, sA, sB)) {
                const StreamDesc &d = a.s[si];
                const int64_t f_end = sB + TT - 1;
                const uint8_t *in = static_cast<const uint8_t *>(d.in);
                for (int64_t f = sA; f < f_end && ok; ++f, ++pc) {
                    const uint32_t slot = pc % NSLOT;
                    if (pc >= NSLOT && !mbar_wait(empty0 + 8 * slot, ((pc / NSLOT) + 1) & 1, a.wait_ns)) {
                        *abort_flag = 1;
                        ok = false;
                        break;
                    }
                    const uint8_t *src;
                    if (f < d.n_state) src = static_cast<const uint8_t *>(d.state) + f * (int64_t)C::FB;
                    else src = in + (f - d.n_state) * (int64_t)C::FB;
                    mbar_expect_tx(full0 + 8 * slot, C::FB);
                    bulk_g2s(smem_u32(ring + slot * C::FB), src, C::FB, full0 + 8 * slot);
                }
            }
            // drain: every copy issued must have landed before the CTA exits
            const uint32_t first = pc > NSLOT ? pc - NSLOT : 0;
            for (uint32_t q = first; q < pc; ++q) {
                if (!mbar_wait(full0 + 8 * (q % NSLOT), (q / NSLOT) & 1, a.wait_ns)) *abort_flag = 1;
            }
        }
        __syncwarp();
    }
    if constexpr (TC) tc_fence_before();
    __syncthreads();
    if constexpr (TC) {
        if (warp == C::NFIRW) {
            tc_fence_after();
            tmem_dealloc(*tmem_slot, kTcCols);
        }
    }
    if (threadIdx.x == 0 && *abort_flag) report_error(a.err, KERR_TIMEOUT);
}

// rows of the launch: one work unit per spectrum
template <int P, int TT, int IN, bool TC = false>
static pfb_status launch_fft_ws_k(LaunchArgs &a, cudaStream_t stream) {
    using C = WsCfg<P, TT, IN, TC>;
    auto k = k_fft_ws<P, TT, IN, TC>;
    static int grid_cap = 0;
    if (grid_cap == 0) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
        if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(k_fft_ws)");
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        grid_cap = sms;
    }
    int64_t grid = a.nunits < grid_cap ? a.nunits : grid_cap;
    if (grid < 1) return PFB_OK;
    if ((a.nunits + grid - 1) / grid > INT32_MAX - 64)  // segment counters are 32-bit in the kernel
        return fail(PFB_ERR_INVALID, "too many spectra for one launch of k_fft_ws");
    a.units_per_cta = (int32_t)((a.nunits + grid - 1) / grid);
    grid = (a.nunits + a.units_per_cta - 1) / a.units_per_cta;
    k<<<(unsigned)grid, C::NTHREADS, C::SMEM, stream>>>(a);
    g_launches++;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "launch k_fft_ws");
    return PFB_OK;
}

}  // namespace pfb
