// Split-bf16 DFT-matrix product in two passes (variant 2 of the split-bf16
// family, P = 1024, 2048, 4096, T <= 16): the literal DFT-as-GEMM of
// Sec. 4.1 with the branch sums of Sec. 5.2 computed once.
//
// Pass 1 (k_fir_tiles_ring, CUDA cores): the polyphase FIR for every spectrum,
//   y[s,p] = sum_{m<T} h[m*P+p] x[(s+m)*P+p], split into bf16 hi = RN(y) and
//   lo = RN(y - hi) and written to a workspace already in the tensor core's
//   operand order: per 128-spectrum M tile and 64-real K block one 16 KB
//   chunk of 8 x 8 core matrices (8 rows x 16 bytes each, K-major), so that
//   pass 2 moves each operand with one bulk copy.
// Pass 2 (k_gemm_tiles, tcgen05): X = [Yr|Yi] B with B the real block form of
//   the DFT matrix (pre-tiled hi and lo, the table of variant 0), three
//   products per K step (hi*hi + hi*lo + lo*hi), M = 128, N = 128, K = 16 per
//   MMA, operands in shared memory, FP32 accumulation in TMEM.  One producer
//   thread fills a 3-stage ring with four bulk copies per K block, one thread
//   issues the MMAs, four epilogue warps drain the accumulator.  Accumulation
//   is two-level as in variant 0: the tensor core sums chunks of 8 K blocks in
//   one of two TMEM accumulators (double-buffered, so the MMAs continue while
//   the other one is drained), and the epilogue adds every chunk into a
//   running FP32 sum in registers (round to nearest); the tensor core's own
//   accumulation drifts by about 1.8e-8 of the result per MMA step, which the
//   chunking bounds independently of P.
// Tiles run in blocks of 8 M tiles x 16 N tiles, so that the operand slabs
// the grid works on at one time stay in L2.  Every wait is bounded (the
// launch's wait_ns); on expiry the kernel records KERR_TIMEOUT, waits
// (bounded) for what it issued and frees its TMEM.
#include <cuda_bf16.h>

#include "devutil.cuh"
#include "internal.h"
#include "sync.cuh"
#include "tc.cuh"

namespace pfb {

constexpr int Y2_M = 128, Y2_KB = 64;                 // reals per workspace chunk: rows x K block
constexpr int Y2_CHUNK_ELEMS = Y2_M * Y2_KB;          // bf16 elements per chunk (16 KB)
constexpr int F2_THREADS = 256, F2_BR = 4;             // FIR pass: threads, branches per thread

int64_t gemm2p_units(const Plan &plan, int64_t S) { return ((S + Y2_M - 1) / Y2_M) * (plan.P / 64); }

// hi and lo halves: 128-spectrum tiles x (2P / 64) K blocks x 16 KB chunks each
size_t gemm2p_workspace_bytes(const Plan &plan, int64_t nunits) {
    const int64_t ntm = nunits / (plan.P / 64);
    return 2 * (size_t)ntm * (2 * plan.P / Y2_KB) * Y2_CHUNK_ELEMS * sizeof(__nv_bfloat16);
}

bool gemm2p_supported(const Plan &plan) {
    return (plan.P == 1024 || plan.P == 2048 || plan.P == 4096) && plan.T <= 16 &&
           (plan.TT == 4 || plan.TT == 8 || plan.TT == 16);
}

// Pass 1: work item w = (global M tile, chunk of 1024 branches).  A producer
// warpgroup gathers the item's 128 + T - 1 frame slices with 16-byte
// asynchronous copies (one arrival per thread on the slot's barrier) into a
// ring of R2_NSLOT slots; FIR thread t owns branches chunk * 1024 + 4t .. + 3
// and streams the frames through T pending sums per branch in registers
// (register split FIR 224 / producer 56).  Reading the frames straight from
// global memory instead ran pass 1 about 2.7 % of the two passes slower.
constexpr int R2_NSLOT = 8, R2_THREADS = F2_THREADS + 128;
template <int IN>
struct R2Cfg {
    static constexpr int ESZ = IN == PFB_IN_C64 ? 8 : (IN == PFB_IN_R32 ? 4 : 2);
    static constexpr int FB = F2_THREADS * F2_BR * ESZ;  // bytes of the CTA's 1024 branches of a frame
    static constexpr int NCP = FB / 16 / 128;            // 16-byte copies per producer thread and frame
    static constexpr int SMEM = R2_NSLOT * FB + 2 * R2_NSLOT * 8 + 16;
    static_assert(NCP * 16 * 128 == FB, "whole 16-byte pieces per producer thread");
};

template <int IN, int TT>
__global__ void __launch_bounds__(R2_THREADS, 1)
    k_fir_tiles_ring(const __grid_constant__ LaunchArgs a, int P, int64_t ntiles, __nv_bfloat16 *yhi,
                     __nv_bfloat16 *ylo) {
    using C = R2Cfg<IN>;
    extern __shared__ __align__(128) uint8_t r2_smem[];
    uint64_t *bars = reinterpret_cast<uint64_t *>(r2_smem + R2_NSLOT * C::FB);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(bars + 2 * R2_NSLOT);
    const uint32_t full0 = smem_u32(&bars[0]), empty0 = smem_u32(&bars[R2_NSLOT]);
    const int nchunk = P / (F2_THREADS * F2_BR), NTL = P / 64, KBLK = 2 * P / Y2_KB;
    constexpr int NFR = Y2_M + TT - 1;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t wns = (uint32_t)a.wait_ns;
    if (threadIdx.x == 0) {
        for (int i = 0; i < R2_NSLOT; ++i) {
            mbar_init(full0 + 8 * i, 128);             // one copy-completion arrival per producer thread
            mbar_init(empty0 + 8 * i, F2_THREADS / 32);  // every FIR warp has read the slot
        }
        mbar_init_fence();
        *abort_flag = 0;
    }
    __syncthreads();
    if (warp < F2_THREADS / 32) {
        // ---------------- FIR warps ----------------
        asm volatile("setmaxnreg.inc.sync.aligned.u32 224;" ::: "memory");
        const int t = threadIdx.x;
        uint32_t pc = 0;
        bool ok = true;
        for (int64_t w = blockIdx.x; w < ntiles * nchunk && ok; w += gridDim.x) {
            const int64_t gmt = w / nchunk;
            const int chunk = (int)(w % nchunk);
            const int si = find_stream(a, gmt * NTL);
            const StreamDesc &d = a.s[si];
            const int p0 = chunk * (F2_THREADS * F2_BR) + F2_BR * t;
            float h[TT][4];
#pragma unroll
            for (int m = 0; m < TT; ++m)
#pragma unroll
                for (int j = 0; j < 4; ++j) h[m][j] = __ldg(d.taps + m * P + p0 + j);
            const int kk0 = 2 * p0, kb = kk0 / Y2_KB, kg = (kk0 % Y2_KB) / 8;
            const int64_t cbase = (gmt * KBLK + kb) * (int64_t)Y2_CHUNK_ELEMS + kg * 64;
            const float sc = d.scale;
            float2 pend[TT][4];
            for (int i0 = 0; i0 < NFR && ok; i0 += TT) {
#pragma unroll
                for (int k = 0; k < TT; ++k) {
                    const int i = i0 + k;
                    if (i < NFR) {
                        const uint32_t slot = pc % R2_NSLOT;
                        if (!__all_sync(0xffffffffu, mbar_wait32(full0 + 8 * slot, (pc / R2_NSLOT) & 1, wns))) {
                            ok = false;
                            break;
                        }
                        const uint8_t *fr = r2_smem + slot * C::FB;
                        float2 v[4];
                        if constexpr (IN == PFB_IN_C64) {
                            const float4 a0 = reinterpret_cast<const float4 *>(fr)[2 * t];
                            const float4 a1 = reinterpret_cast<const float4 *>(fr)[2 * t + 1];
                            v[0] = make_float2(a0.x, a0.y);
                            v[1] = make_float2(a0.z, a0.w);
                            v[2] = make_float2(a1.x, a1.y);
                            v[3] = make_float2(a1.z, a1.w);
                        } else if constexpr (IN == PFB_IN_R32) {
                            const float4 a0 = reinterpret_cast<const float4 *>(fr)[t];
                            v[0] = make_float2(a0.x, 0.f);
                            v[1] = make_float2(a0.y, 0.f);
                            v[2] = make_float2(a0.z, 0.f);
                            v[3] = make_float2(a0.w, 0.f);
                        } else {
                            const int2 a0 = reinterpret_cast<const int2 *>(fr)[t];
                            const char4 lo = *reinterpret_cast<const char4 *>(&a0.x);
                            const char4 hi = *reinterpret_cast<const char4 *>(&a0.y);
                            v[0] = make_float2((float)lo.x * sc, (float)lo.y * sc);
                            v[1] = make_float2((float)lo.z * sc, (float)lo.w * sc);
                            v[2] = make_float2((float)hi.x * sc, (float)hi.y * sc);
                            v[3] = make_float2((float)hi.z * sc, (float)hi.w * sc);
                        }
                        // the previous frame's slot goes back: every lane has used its values
                        __syncwarp();
                        if (lane == 0 && pc > 0) mbar_arrive(empty0 + 8 * ((pc - 1) % R2_NSLOT));
                        ++pc;
#pragma unroll
                        for (int j = 0; j < 4; ++j) pend[k][j] = make_float2(h[0][j] * v[j].x, h[0][j] * v[j].y);
#pragma unroll
                        for (int m = 1; m < TT; ++m) {
                            const int js = ((k - m) % TT + TT) % TT;
#pragma unroll
                            for (int j = 0; j < 4; ++j) pend[js][j] = fma2(make_float2(h[m][j], h[m][j]), v[j], pend[js][j]);
                        }
                        const int r = i - (TT - 1);
                        if (r >= 0) {
                            const int js = (k + 1) % TT;
                            uint4 hv, lv;
                            split_bf16x2(pend[js][0], hv.x, lv.x);
                            split_bf16x2(pend[js][1], hv.y, lv.y);
                            split_bf16x2(pend[js][2], hv.z, lv.z);
                            split_bf16x2(pend[js][3], hv.w, lv.w);
                            const int64_t off = cbase + (r >> 3) * 512 + (r & 7) * 8;
                            *reinterpret_cast<uint4 *>(yhi + off) = hv;
                            *reinterpret_cast<uint4 *>(ylo + off) = lv;
                        }
                    }
                }
            }
        }
        if (!ok) *abort_flag = 1;
    } else {
        // ---------------- producer warpgroup ----------------
        asm volatile("setmaxnreg.dec.sync.aligned.u32 56;" ::: "memory");
        const int pt = threadIdx.x - F2_THREADS;
        uint32_t pc = 0;
        bool ok = true;
        for (int64_t w = blockIdx.x; w < ntiles * nchunk && ok; w += gridDim.x) {
            const int64_t gmt = w / nchunk;
            const int chunk = (int)(w % nchunk);
            const int si = find_stream(a, gmt * NTL);
            const StreamDesc &d = a.s[si];
            const int64_t s0 = (gmt - d.unit0 / NTL) * Y2_M;
            for (int i = 0; i < NFR; ++i, ++pc) {
                const uint32_t slot = pc % R2_NSLOT;
                if (pc >= R2_NSLOT && !mbar_wait32(empty0 + 8 * slot, ((pc / R2_NSLOT) + 1) & 1, wns)) {
                    ok = false;
                    break;
                }
                const uint32_t dst = smem_u32(r2_smem + slot * C::FB);
                const int64_t f = s0 + i;
                if (f < d.n_frames) {
                    int64_t smp;
                    const uint8_t *src = static_cast<const uint8_t *>(frame_source(d, f, P, smp)) +
                                         (smp + (int64_t)chunk * F2_THREADS * F2_BR) * C::ESZ;
#pragma unroll
                    for (int q = 0; q < C::NCP; ++q) cp_async16(dst + (pt + 128 * q) * 16, src + (pt + 128 * q) * 16);
                    cp_async_arrive_noinc(full0 + 8 * slot);
                } else {
                    // past the end of the stream: zero frames (rows that are computed, never stored)
#pragma unroll
                    for (int q = 0; q < C::NCP; ++q)
                        *reinterpret_cast<uint4 *>(r2_smem + slot * C::FB + (pt + 128 * q) * 16) = make_uint4(0, 0, 0, 0);
                    mbar_arrive(full0 + 8 * slot);
                }
            }
        }
        asm volatile("cp.async.wait_all;" ::: "memory");
        if (!ok) *abort_flag = 1;
    }
    __syncthreads();
    if (threadIdx.x == 0 && *abort_flag) report_error(a.err, KERR_TIMEOUT);
}

// ---------------------------------------------------------------------------
// Pass 2: the product
// ---------------------------------------------------------------------------
// The MMAs read both operands from shared memory, into which the bulk copies
// also write: per K block of 64 reals and M = 128 the shared-memory traffic is
// the stage's bytes written plus 4 K steps x 3 products x (A + B tile) read.
// At N = 128 that is 64 KB + 96 KB against 12 MMAs of 64 cycles each at the
// tensor core's rate, which caps the tensor pipe near 60 % at 128 bytes per
// cycle; at N = 256 it is 96 KB + 144 KB against 12 MMAs of 128 cycles,
// about 80 %.  So an N tile is 256 reals (128 bins): the full width of one
// tile of the variant-0 table, in two stages of 96 KB.
template <int BN>
struct G2Cfg {
    static constexpr int N = BN;                             // reals per N tile
    static constexpr int NST = BN == 256 ? 2 : 3;            // ring stages
    static constexpr int OPA = Y2_CHUNK_ELEMS * 2;           // bytes of one A chunk (128 x 64 bf16)
    static constexpr int OPB = BN * Y2_KB * 2;               // bytes of one B chunk (BN x 64 bf16)
    static constexpr int STAGE = 2 * OPA + 2 * OPB;          // A hi, A lo, B hi, B lo
    static constexpr int EPIW = BN / 32;                     // epilogue warps: 4 TMEM lane quarters x BN / 128 column halves
    static constexpr int PRODW = EPIW, MMAW = EPIW + 1, THREADS = (EPIW + 2) * 32;
    static constexpr int SMEM = NST * STAGE + 256 + 1024;    // + barriers, + alignment slack
    static constexpr uint32_t TMEM_COLS = 2 * BN;            // two accumulators
    static constexpr uint32_t IDESC = tc_idesc_bf16(128, BN);
    static constexpr int MB = 8, NB = 2048 / BN;             // tile blocks kept together (L2): 8 M tiles x 2048 reals
    static_assert(SMEM <= 232448, "shared memory");
    static_assert(STAGE < (1 << 20), "transaction count of one stage");
};
constexpr int G2_BN = 256;
constexpr int G2_CHUNK = 8;                                  // K blocks per TMEM accumulation chunk

// tile w of the blocked order -> (global M tile, N tile)
template <int BN>
__device__ __forceinline__ void g2_tile(int64_t w, int64_t ntm, int ntn, int64_t &gmt, int &nt) {
    using C = G2Cfg<BN>;
    const int nb = ntn < C::NB ? ntn : C::NB;
    const int64_t bm = w / ((int64_t)C::MB * ntn);
    const int64_t idx = w - bm * C::MB * ntn;
    const int64_t mrows = min((int64_t)C::MB, ntm - bm * C::MB);
    const int64_t bn = idx / (mrows * nb), r = idx % (mrows * nb);
    gmt = bm * C::MB + r / nb;
    nt = (int)(bn * nb + r % nb);
}

template <int BN>
__global__ void __launch_bounds__(G2Cfg<BN>::THREADS, 1)
    k_gemm_tiles(const __grid_constant__ LaunchArgs a, int P, int64_t ntm, const __nv_bfloat16 *yhi,
                 const __nv_bfloat16 *ylo) {
    using C = G2Cfg<BN>;
    constexpr int NST = C::NST;
    extern __shared__ __align__(1024) uint8_t g2_raw[];
    uint8_t *sm = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(g2_raw) + 1023) & ~uintptr_t(1023));
    uint64_t *bars = reinterpret_cast<uint64_t *>(sm + NST * C::STAGE);
    // full[NST], empty[NST], dfull[2], dfree[2], then the TMEM address and the abort flag
    const uint32_t full0 = smem_u32(&bars[0]), empty0 = smem_u32(&bars[NST]);
    const uint32_t dfull0 = smem_u32(&bars[2 * NST]), dfree0 = smem_u32(&bars[2 * NST + 2]);
    volatile uint32_t *tmem_slot = reinterpret_cast<volatile uint32_t *>(bars + 2 * NST + 4);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(bars + 2 * NST + 5);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint64_t wns = a.wait_ns;
    if (threadIdx.x == 0) {
        for (int i = 0; i < NST; ++i) {
            mbar_init(full0 + 8 * i, 1);   // the producer's arrive.expect_tx + the copies' bytes
            mbar_init(empty0 + 8 * i, 1);  // the MMA thread's commit
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(dfull0 + 8 * i, 1);        // the MMA thread's commit at the end of a chunk
            mbar_init(dfree0 + 8 * i, C::EPIW);  // every epilogue warp has read its part of the accumulator
        }
        mbar_init_fence();
        *abort_flag = 0;
    }
    if (warp == C::MMAW) tmem_alloc(smem_u32((const void *)tmem_slot), C::TMEM_COLS);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    const int ntn = 2 * P / BN, KBLK = 2 * P / Y2_KB;
    const int nchunks = (KBLK + G2_CHUNK - 1) / G2_CHUNK;
    const int64_t ntiles = ntm * ntn;
    const __nv_bfloat16 *Bhi = static_cast<const __nv_bfloat16 *>(a.aux);
    // the variant-0 table: tiles (N tile of 256 reals, K block) of 256 x 64, hi then lo; a
    // 128-real N tile is one contiguous half of one of them
    const __nv_bfloat16 *Blo = Bhi + (int64_t)(P / 128) * KBLK * (2 * Y2_CHUNK_ELEMS);
    const uint32_t sA = smem_u32(sm);

    if (warp == C::PRODW) {
        // ---------------- producer: four bulk copies per K block ----------------
        if (lane == 0) {
            uint32_t g = 0;
            bool ok = true;
            for (int64_t w = blockIdx.x; w < ntiles && ok; w += gridDim.x) {
                int64_t gmt;
                int nt;
                g2_tile<BN>(w, ntm, ntn, gmt, nt);
                for (int kb = 0; kb < KBLK; ++kb, ++g) {
                    const uint32_t st = g % NST;
                    if (g >= NST && !mbar_wait(empty0 + 8 * st, ((g / NST) + 1) & 1, wns)) {
                        ok = false;
                        break;
                    }
                    const uint32_t fb = full0 + 8 * st, dst = sA + st * C::STAGE;
                    mbar_expect_tx(fb, C::STAGE);
                    const int64_t ao = (gmt * KBLK + kb) * (int64_t)Y2_CHUNK_ELEMS;
                    const int64_t bo = BN == 256 ? ((int64_t)nt * KBLK + kb) * (2 * Y2_CHUNK_ELEMS)
                                                 : ((int64_t)(nt >> 1) * KBLK + kb) * (2 * Y2_CHUNK_ELEMS) +
                                                       (nt & 1) * Y2_CHUNK_ELEMS;
                    bulk_g2s(dst, yhi + ao, C::OPA, fb);
                    bulk_g2s(dst + C::OPA, ylo + ao, C::OPA, fb);
                    bulk_g2s(dst + 2 * C::OPA, Bhi + bo, C::OPB, fb);
                    bulk_g2s(dst + 2 * C::OPA + C::OPB, Blo + bo, C::OPB, fb);
                }
            }
            if (!ok) *abort_flag = 1;
            // every copy issued has landed before the CTA exits
            const uint32_t first = g > NST ? g - NST : 0;
            for (uint32_t q = first; q < g; ++q)
                if (!mbar_wait(full0 + 8 * (q % NST), (q / NST) & 1, wns)) *abort_flag = 1;
        }
        __syncwarp();
    } else if (warp == C::MMAW) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            uint32_t g = 0, c = 0;
            bool ok = true, issued = false;
            for (int64_t w = blockIdx.x; w < ntiles && ok; w += gridDim.x) {
                for (int kb = 0; kb < KBLK && ok; ++kb, ++g) {
                    const uint32_t buf = c & 1;
                    if (kb % G2_CHUNK == 0 && c >= 2 && !mbar_wait(dfree0 + 8 * buf, ((c >> 1) + 1) & 1, wns)) {
                        ok = false;
                        break;
                    }
                    const uint32_t st = g % NST;
                    if (!mbar_wait(full0 + 8 * st, (g / NST) & 1, wns)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t d_t = tmem + buf * BN;
                    const uint32_t ah = sA + st * C::STAGE, al = ah + C::OPA, bh = ah + 2 * C::OPA, bl = bh + C::OPB;
#pragma unroll
                    for (int ks = 0; ks < Y2_KB / 16; ++ks) {
                        const uint64_t dah = tc_desc_kmajor(ah + ks * 256, 128, 1024);
                        const uint64_t dal = tc_desc_kmajor(al + ks * 256, 128, 1024);
                        const uint64_t dbh = tc_desc_kmajor(bh + ks * 256, 128, 1024);
                        const uint64_t dbl = tc_desc_kmajor(bl + ks * 256, 128, 1024);
                        tc_mma_ss(d_t, dah, dbh, C::IDESC, (kb % G2_CHUNK > 0 || ks > 0) ? 1u : 0u);
                        tc_mma_ss(d_t, dah, dbl, C::IDESC, 1u);
                        tc_mma_ss(d_t, dal, dbh, C::IDESC, 1u);
                    }
                    tc_commit(empty0 + 8 * st);  // the stage is free once these MMAs are done
                    issued = true;
                    if (kb % G2_CHUNK == G2_CHUNK - 1 || kb == KBLK - 1) {
                        tc_commit(dfull0 + 8 * buf);  // the chunk's sum is in the accumulator
                        ++c;
                    }
                }
            }
            if (!ok) *abort_flag = 1;
            // every MMA issued has completed before TMEM is freed
            if (issued && !ok) {
                const uint32_t gl = g - 1;
                if (!mbar_wait(empty0 + 8 * (gl % NST), (gl / NST) & 1, wns)) *abort_flag = 1;
            }
        }
        __syncwarp();
    } else {
        // ---------------- epilogue warps: TMEM lane quarter warp % 4, columns 128 (warp / 4) .. + 127 ----------------
        float sacc[128];
        uint32_t c = 0;
        bool ok = true;
        const int quarter = warp & 3, half = warp >> 2;
        const uint32_t trow = tmem + ((uint32_t)(32 * quarter) << 16) + 128u * half;
        for (int64_t w = blockIdx.x; w < ntiles && ok; w += gridDim.x) {
            int64_t gmt;
            int nt;
            g2_tile<BN>(w, ntm, ntn, gmt, nt);
#pragma unroll
            for (int i = 0; i < 128; ++i) sacc[i] = 0.f;
            for (int cc = 0; cc < nchunks; ++cc, ++c) {
                const uint32_t buf = c & 1;
                if (!__all_sync(0xffffffffu, mbar_wait(dfull0 + 8 * buf, (c >> 1) & 1, wns))) {
                    ok = false;
                    break;
                }
                tc_fence_after();
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    uint32_t r[32];
                    tmem_ld32(trow + buf * BN + 32 * q, r);
                    tmem_wait_ld();
#pragma unroll
                    for (int i = 0; i < 32; ++i) sacc[32 * q + i] += __uint_as_float(r[i]);
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(dfree0 + 8 * buf);
            }
            if (!ok) break;
            const int si = find_stream(a, gmt * (P / 64));
            const StreamDesc &d = a.s[si];
            const int64_t s = (gmt - d.unit0 / (P / 64)) * Y2_M + 32 * quarter + lane;
            if (s < d.S) {
                float4 *o = reinterpret_cast<float4 *>(reinterpret_cast<float *>(d.out) + s * 2 * d.ldo +
                                                       (int64_t)nt * BN + 128 * half);
#pragma unroll
                for (int i = 0; i < 32; ++i)
                    __stcs(o + i, make_float4(sacc[4 * i], sacc[4 * i + 1], sacc[4 * i + 2], sacc[4 * i + 3]));
            }
        }
        if (!ok) *abort_flag = 1;
    }
    // ---------------- teardown ----------------
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == C::MMAW) tmem_dealloc(tmem, C::TMEM_COLS);
    if (threadIdx.x == 0 && *abort_flag) report_error(a.err, KERR_TIMEOUT);
}

// ---------------------------------------------------------------------------
// launch: workspace, pass 1, pass 2 (same stream)
// ---------------------------------------------------------------------------
template <int IN, int TT>
static pfb_status launch_fir_tiles(const Plan &plan, const LaunchArgs &a, int64_t ntm, __nv_bfloat16 *yhi,
                                   __nv_bfloat16 *ylo, cudaStream_t stream) {
    const int64_t work = ntm * (plan.P / (F2_THREADS * F2_BR));
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    using C = R2Cfg<IN>;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_fir_tiles_ring<IN, TT>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
        if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(k_fir_tiles_ring)");
        attr = true;
    }
    const int64_t grid = work < (int64_t)sms ? work : (int64_t)sms;  // one CTA per SM (registers)
    k_fir_tiles_ring<IN, TT><<<(unsigned)grid, R2_THREADS, C::SMEM, stream>>>(a, plan.P, ntm, yhi, ylo);
    g_launches++;
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? PFB_OK : cuda_fail(e, "launch k_fir_tiles_ring");
}

template <int IN>
static pfb_status launch_fir_tiles_t(const Plan &plan, const LaunchArgs &a, int64_t ntm, __nv_bfloat16 *yhi,
                                     __nv_bfloat16 *ylo, cudaStream_t stream) {
    switch (plan.TT) {
    case 4: return launch_fir_tiles<IN, 4>(plan, a, ntm, yhi, ylo, stream);
    case 8: return launch_fir_tiles<IN, 8>(plan, a, ntm, yhi, ylo, stream);
    default: return launch_fir_tiles<IN, 16>(plan, a, ntm, yhi, ylo, stream);
    }
}

// The workspace (hi and lo branch sums, 4 x P bytes per padded spectrum) is
// the plan's and grows on demand: launches of one plan in this variant must
// not overlap, and a CUDA-graph capture needs it grown beforehand (by an
// earlier launch of the size, or by pfb_batch_create).
pfb_status launch_gemm_bf16x3_2p(const Plan &plan, LaunchArgs &a, cudaStream_t stream) {
    if (!gemm2p_supported(plan)) return fail(PFB_ERR_UNSUPPORTED, "split-bf16 variant 2 needs P in {1024, 2048, 4096}, T <= 16");
    if (a.nunits <= 0) return PFB_OK;
    if (!plan.d_dft) return fail(PFB_ERR_INTERNAL, "split-bf16 DFT matrix not built");
    const int ntn = plan.P / 64;
    const int64_t ntm = a.nunits / ntn;
    const size_t half = gemm2p_workspace_bytes(plan, a.nunits) / 2;
    pfb_status wst = grow_plan_workspace(plan, 2 * half, stream);
    if (wst != PFB_OK) return wst;
    Plan &mp = const_cast<Plan &>(plan);
    __nv_bfloat16 *yhi = static_cast<__nv_bfloat16 *>(mp.d_ws2);
    __nv_bfloat16 *ylo = yhi + half / sizeof(__nv_bfloat16);
    pfb_status st;
    switch (plan.in_dtype) {
    case PFB_IN_C64: st = launch_fir_tiles_t<PFB_IN_C64>(plan, a, ntm, yhi, ylo, stream); break;
    case PFB_IN_R32: st = launch_fir_tiles_t<PFB_IN_R32>(plan, a, ntm, yhi, ylo, stream); break;
    case PFB_IN_CI8: st = launch_fir_tiles_t<PFB_IN_CI8>(plan, a, ntm, yhi, ylo, stream); break;
    default: return fail(PFB_ERR_INVALID, "bad dtype");
    }
    if (st != PFB_OK) return st;
    using GC = G2Cfg<G2_BN>;
    static int grid_cap = 0;
    if (grid_cap == 0) {
        cudaError_t e = cudaFuncSetAttribute(k_gemm_tiles<G2_BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, GC::SMEM);
        if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(k_gemm_tiles)");
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        grid_cap = sms;  // one CTA per SM (about 198 KB of shared memory)
    }
    const int64_t ntiles = ntm * (2 * plan.P / G2_BN);
    const int64_t grid = ntiles < grid_cap ? ntiles : grid_cap;
    k_gemm_tiles<G2_BN><<<(unsigned)grid, GC::THREADS, GC::SMEM, stream>>>(a, plan.P, ntm, yhi, ylo);
    g_launches++;
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? PFB_OK : cuda_fail(e, "launch k_gemm_tiles");
}

}  // namespace pfb
