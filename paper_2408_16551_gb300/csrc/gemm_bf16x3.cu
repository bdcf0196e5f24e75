// Fused polyphase FIR + DFT as a product with the Fourier matrix on the
// tensor cores (tcgen05, sm_103a), split-bf16 with FP32 accumulation.
//
// The DFT of Sec. 4.1 (Z = X F) is run in real block form: with the branch
// sums y[s,p] interleaved (re, im) along K = 2P and the output interleaved
// along N = 2P,
//     X[s, 2k+d] = sum_{2p+c} y[s, 2p+c] * B[2p+c, 2k+d]
//     B[2p,2k] = B[2p+1,2k+1] = cos(th),  B[2p+1,2k] = sin(th),  B[2p,2k+1] = -sin(th)
// with th = 2 pi (p k mod P) / P.  Both operands are split into bf16 hi + lo
// (hi = RN(v), lo = RN(v - hi); B from its FP64 value, y from its fp32 value)
// and three products are accumulated in FP32:  hi*hi + hi*lo + lo*hi.
//
// CTA = 9 warps, one CTA per SM (all 512 TMEM columns):
//   warps 0-7: the FIR of Sec. 5.2 for a 128-spectrum x 32-branch slice per
//              K block: warp w covers the 32 spectra of TMEM lane quarter w%4
//              and 16 of the 32 branches (w/4); lane = (branch, half of the
//              spectra), register window over 16 spectra, packed fp32x2 FMAs,
//              coalesced loads; a warp-local transpose through shared memory
//              to lane = spectrum, the hi/lo split, tcgen05.st into the A stage
//              in TMEM; the accumulator drains and the epilogue (tcgen05.ld ->
//              HBM) are split the same way (column halves);
//   warp 8:    lane 0 bulk-copies the pre-tiled B_hi/B_lo tiles of the K block
//              into shared memory (mbarrier complete_tx) and issues the
//              3 x 4 tcgen05.mma (M=128, N=256, K=16, A from TMEM, B from
//              shared memory, no swizzle) and the tcgen05.commit.
// Two stages (A in TMEM, B in shared memory) let the FIR of K block g+1 run
// while the tensor core works on block g.
// Accumulation is two-level: the tensor core accumulates K2_CHUNK K blocks
// (3 x 4 x K2_CHUNK MMAs) in TMEM, then the epilogue warps drain the
// accumulator and add it, in FP32 with round-to-nearest on the CUDA cores,
// into the output tile (the tile in HBM/L2 is the running sum).  The tensor
// core's FP32 accumulation adds a small bias per MMA step (about 1.8e-8 of
// the result per step, measured); chunking bounds it independently of P.  Every mbarrier wait is bounded
// (1 s of %globaltimer); on expiry the kernel records KERR_TIMEOUT, drains
// what it issued (bounded) and frees its TMEM.
#include <cuda_bf16.h>

#include "devutil.cuh"
#include "internal.h"
#include "sync.cuh"
#include "tc.cuh"

namespace pfb {

constexpr int K2_M = 128, K2_N = 256, K2_KB = 64;  // reals per tile: M rows, N cols, K block
constexpr int K2_FIRW = 8, K2_WARPS = K2_FIRW + 1, K2_THREADS = K2_WARPS * 32;
constexpr int K2_TILE_ELEMS = K2_N * K2_KB;  // bf16 elements per B tile (32 KB)
constexpr int K2_TILE_BYTES = K2_TILE_ELEMS * 2;
constexpr int K2_SMEM_B = 2 * 2 * K2_TILE_BYTES;  // 2 stages x (hi, lo)
constexpr int K2_TR = 17;                          // transpose row stride (float2)
constexpr int K2_SMEM_TR = K2_FIRW * 32 * K2_TR * 8;
constexpr int K2_SMEM_BAR = 64;
constexpr int K2_SMEM = K2_SMEM_B + K2_SMEM_TR + K2_SMEM_BAR + 1024;  // + alignment slack
constexpr uint32_t K2_TMEM_COLS = 512;
constexpr uint32_t K2_COL_A = 256;                 // A stages start after the 256-column accumulator
constexpr int K2_CHUNK = 8;                        // K blocks per TMEM accumulation chunk

// instruction descriptor, kind::f16: D=f32, A=B=bf16, K-major A and B, N=256, M=128
constexpr uint32_t K2_IDESC = tc_idesc_bf16(K2_M, K2_N);

// variant 0: (128-spectrum M tile, 128-bin N tile) pairs; variant 1 (factored): spectra
int64_t cluster_units(int64_t S);

int64_t gemm_bf16x3_units(const Plan &plan, int64_t S) {
    if (plan.variant == 2) return gemm2p_units(plan, S);
    if (plan.variant == 1) return (plan.P == 1024 || ws_cluster_supported(plan)) ? S : cluster_units(S);
    return ((S + K2_M - 1) / K2_M) * (plan.P / (K2_N / 2));
}

// ---------------------------------------------------------------------------
// table: pre-tiled B_hi / B_lo, tile (nt, kb) = 256 (N) x 64 (K) bf16 in the
// K-major no-swizzle core-matrix order: core matrix (ng, kg) of 8 rows x 8
// elements at element offset (ng*8 + kg)*64, row r at +8r, element e at +e
// (leading-dimension byte offset 128 B along K, stride 1024 B along N).
// ---------------------------------------------------------------------------
// conj = 1: the conjugate matrix (exponent +2 pi i pk/P), for the inverse DFT
__global__ void gen_dft_bf16x3_kernel(__nv_bfloat16 *Bhi, __nv_bfloat16 *Blo, int P, int conj) {
    const int64_t total = (int64_t)2 * P * 2 * P;
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= total) return;
    const int KBLK = (2 * P) / K2_KB;
    const int64_t tile = i / K2_TILE_ELEMS;
    const int w = (int)(i % K2_TILE_ELEMS);
    const int nt = (int)(tile / KBLK), kb = (int)(tile % KBLK);
    const int cm = w / 64, within = w % 64;
    const int ng = cm / 8, kg = cm % 8, r = within / 8, e = within % 8;
    const int n = nt * K2_N + ng * 8 + r;   // output column 2k + d
    const int kk = kb * K2_KB + kg * 8 + e; // reduction index 2p + c
    const int k = n >> 1, dsel = n & 1, p = kk >> 1, csel = kk & 1;
    const int64_t ex = ((int64_t)p * k) % P;
    double s, c;
    sincospi(2.0 * (double)ex / (double)P, &s, &c);
    if (conj) s = -s;
    double v;
    if (csel == dsel) v = c;
    else if (csel == 1) v = s;   // B[2p+1][2k]
    else v = -s;                 // B[2p][2k+1]
    const __nv_bfloat16 hi = __double2bfloat16(v);
    const __nv_bfloat16 lo = __double2bfloat16(v - (double)__bfloat162float(hi));
    Bhi[i] = hi;
    Blo[i] = lo;
}

static pfb_status build_table(Plan &plan, int conj) {
    const int64_t n = (int64_t)2 * plan.P * 2 * plan.P;
    plan.dft_bytes = 2 * n * sizeof(__nv_bfloat16);
    PFB_CUDA_TRY(cudaMalloc(&plan.d_dft, plan.dft_bytes));
    __nv_bfloat16 *hi = static_cast<__nv_bfloat16 *>(plan.d_dft);
    gen_dft_bf16x3_kernel<<<(unsigned)((n + 255) / 256), 256>>>(hi, hi + n, plan.P, conj);
    g_launches++;
    PFB_CUDA_TRY(cudaGetLastError());
    return PFB_OK;
}

pfb_status build_gemm_bf16x3_table(Plan &plan) { return build_table(plan, 0); }

// the conjugate DFT matrix, for the synthesis bank's inverse DFT
pfb_status build_gemm_bf16x3_table_conj(Plan &plan) { return build_table(plan, 1); }

pfb_status build_gemm_f32_table(Plan &plan);

// tables a variant needs that plan creation did not build
pfb_status ensure_variant_tables(Plan &plan) {
    if (plan.family == FAM_GEMM_BF16X3 && (plan.variant == 0 || plan.variant == 2) && !plan.d_dft &&
        plan.P >= K2_N / 2 && plan.T <= 16) {
        pfb_status st = build_gemm_bf16x3_table(plan);
        if (st != PFB_OK) return st;
        PFB_CUDA_TRY(cudaDeviceSynchronize());
    }
    return PFB_OK;
}

pfb_status build_gemm_tables(Plan &plan) {
    if (plan.family == FAM_GEMM_F32) return build_gemm_f32_table(plan);
    if (plan.family == FAM_GEMM_BF16X3) {
        if (plan.P < K2_N / 2 || plan.T > 16) return PFB_OK;  // no kernel; execute reports UNSUPPORTED
        if (tcf_supported(plan)) {
            // the dense DFT matrix (16 MB at P = 1024, 256 MB at P = 4096) is
            // built only when its variant is selected (ensure_variant_tables)
            return build_tcf_table(plan);
        }
        return build_gemm_bf16x3_table(plan);
    }
    return PFB_OK;
}

// ---------------------------------------------------------------------------
// PTX helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
    // B tiles: LBO = 128 B (K direction), SBO = 1024 B (N direction)
    return tc_desc_kmajor(addr, 128, 1024);
}

__device__ __forceinline__ void mma_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t b_desc, uint32_t accumulate) {
    tc_mma_ts(d_tmem, a_tmem, b_desc, K2_IDESC, accumulate);
}

__device__ __forceinline__ void named_sync() { asm volatile("bar.sync 1, %0;" ::"r"(K2_THREADS) : "memory"); }

// Move 128 columns (this warp's half) of this thread's accumulator row into
// the output tile row: first chunk stores, later chunks add (FP32, RN).
__device__ __forceinline__ void drain_row(uint32_t trow, float *orow, bool valid, bool first, bool last) {
#pragma unroll 1
    for (int c = 0; c < K2_N / 64; ++c) {
        uint32_t r[32];
        tmem_ld32(trow + 32 * c, r);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (valid) {
            float4 *o = reinterpret_cast<float4 *>(orow + 32 * c);
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                float4 v = make_float4(__uint_as_float(r[4 * q]), __uint_as_float(r[4 * q + 1]),
                                       __uint_as_float(r[4 * q + 2]), __uint_as_float(r[4 * q + 3]));
                if (!first) {
                    const float4 prev = o[q];
                    v.x += prev.x; v.y += prev.y; v.z += prev.z; v.w += prev.w;
                }
                if (last) __stcs(o + q, v);
                else o[q] = v;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// kernel
// ---------------------------------------------------------------------------
template <int IN, int TT>
__global__ void __launch_bounds__(K2_THREADS, 1) k_gemm_bf16x3(const __grid_constant__ LaunchArgs a, int P) {
    extern __shared__ __align__(1024) uint8_t k2_smem_raw[];
    uint8_t *sm = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(k2_smem_raw) + 1023) & ~uintptr_t(1023));
    float2 *tr_all = reinterpret_cast<float2 *>(sm + K2_SMEM_B);
    uint64_t *bars = reinterpret_cast<uint64_t *>(sm + K2_SMEM_B + K2_SMEM_TR);  // bfull[0..1], mdone[0..1]
    volatile uint32_t *tmem_slot = reinterpret_cast<volatile uint32_t *>(bars + 4);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(bars + 5);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t bfull0 = smem_u32(&bars[0]), mdone0 = smem_u32(&bars[2]);

    if (threadIdx.x == 0) {
        for (int i = 0; i < 4; ++i)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bars[i])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        *abort_flag = 0;
    }
    if (warp == K2_FIRW) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32((const void *)tmem_slot)),
                     "r"(K2_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    const int KBLK = (2 * P) / K2_KB;
    const int NTL = P / (K2_N / 2);
    const __nv_bfloat16 *Bhi = static_cast<const __nv_bfloat16 *>(a.aux);
    const __nv_bfloat16 *Blo = Bhi + (int64_t)NTL * KBLK * K2_TILE_ELEMS;
    const uint32_t sB = smem_u32(sm);

    uint32_t g = 0;                 // K blocks this CTA has gone through (stage = g & 1)
    int64_t last_commit = -1;       // last K block whose MMAs were committed (issuer only)
    int64_t last_copy = -1;         // last K block whose B copies were issued (issuer only)
    int64_t last_waited_full = -1;  // last K block whose B copies were waited for (issuer only)
    bool aborted = false;

    for (int64_t u = blockIdx.x; u < a.nunits && !aborted; u += gridDim.x) {
        const int si = find_stream(a, u);
        const StreamDesc &d = a.s[si];
        const int64_t lu = u - d.unit0;
        const int64_t s0 = (lu / NTL) * K2_M;
        const int nt = (int)(lu % NTL);
        for (int kb = 0; kb < KBLK; ++kb, ++g) {
            const uint32_t stage = g & 1;
            const bool need_wait = g >= 2;
            const uint32_t wpar = ((g >> 1) + 1) & 1;  // completion (g-2)/2 of mdone[stage]
            if (warp == K2_FIRW) {
                if (lane == 0) {
                    if (need_wait && !mbar_wait(mdone0 + 8 * stage, wpar)) {
                        *abort_flag = 1;
                    } else {
                        const uint32_t bf = bfull0 + 8 * stage;
                        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bf),
                                     "r"(2 * K2_TILE_BYTES)
                                     : "memory");
                        const int64_t toff = ((int64_t)nt * KBLK + kb) * K2_TILE_ELEMS;
                        asm volatile(
                            "cp.async.bulk.shared::cta.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                                sB + stage * 2 * K2_TILE_BYTES),
                            "l"(Bhi + toff), "r"(K2_TILE_BYTES), "r"(bf)
                            : "memory");
                        asm volatile(
                            "cp.async.bulk.shared::cta.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                                sB + stage * 2 * K2_TILE_BYTES + K2_TILE_BYTES),
                            "l"(Blo + toff), "r"(K2_TILE_BYTES), "r"(bf)
                            : "memory");
                        last_copy = g;
                    }
                }
            } else {
                // ---------------- FIR warps ----------------
                bool ok = true;
                if (need_wait) ok = mbar_wait(mdone0 + 8 * stage, wpar);
                if (!ok) *abort_flag = 1;
                tc_fence_after();
                if (ok) {
                    const int q = warp & 3, hb = warp >> 2;      // lane quarter, branch half
                    const int bl = lane & 15, rh = lane >> 4;    // branch in the half, spectra half
                    const int p = kb * 32 + 16 * hb + bl;        // this lane's branch
                    const int64_t f0 = s0 + 32 * q + 16 * rh;    // first frame of the window
                    float h[TT];
#pragma unroll
                    for (int m = 0; m < TT; ++m) h[m] = __ldg(d.taps + m * P + p);
                    float2 acc[16];
#pragma unroll
                    for (int j = 0; j < 16; ++j) acc[j] = make_float2(0.f, 0.f);
                    const bool interior = f0 >= d.n_state && f0 + 16 + TT - 1 <= d.n_frames;
                    if (interior) {
                        const int64_t base = (f0 - d.n_state) * P + p;
#pragma unroll
                        for (int i = 0; i < 16 + TT - 1; ++i) {
                            const float2 v = Loader<IN>::load1(d.in, base + (int64_t)i * P, d.scale);
#pragma unroll
                            for (int j = 0; j < 16; ++j) {
                                const int m = i - j;
                                if (m >= 0 && m < TT) acc[j] = fma2(make_float2(h[m], h[m]), v, acc[j]);
                            }
                        }
                    } else {
#pragma unroll
                        for (int i = 0; i < 16 + TT - 1; ++i) {
                            const int64_t f = f0 + i;
                            float2 v = make_float2(0.f, 0.f);
                            if (f < d.n_frames) {
                                int64_t smp;
                                const void *src = frame_source(d, f, P, smp);
                                v = Loader<IN>::load1(src, smp + p, d.scale);
                            }
#pragma unroll
                            for (int j = 0; j < 16; ++j) {
                                const int m = i - j;
                                if (m >= 0 && m < TT) acc[j] = fma2(make_float2(h[m], h[m]), v, acc[j]);
                            }
                        }
                    }
                    // transpose: lane = (branch, spectra half) -> lane = spectrum row
                    float2 *tr = tr_all + warp * 32 * K2_TR;
#pragma unroll
                    for (int j = 0; j < 16; ++j) tr[(16 * rh + j) * K2_TR + bl] = acc[j];
                    __syncwarp();
                    uint32_t vh[16], vl[16];
#pragma unroll
                    for (int c = 0; c < 16; ++c) {
                        const float2 y = tr[lane * K2_TR + c];
                        const __nv_bfloat162 hi = __floats2bfloat162_rn(y.x, y.y);
                        const float2 hf = __bfloat1622float2(hi);
                        const __nv_bfloat162 lo = __floats2bfloat162_rn(y.x - hf.x, y.y - hf.y);
                        vh[c] = bf16x2_bits(hi);
                        vl[c] = bf16x2_bits(lo);
                    }
                    __syncwarp();
                    const uint32_t trow = tmem + ((uint32_t)(32 * q) << 16);
                    const uint32_t acol = K2_COL_A + 64 * stage + 16 * hb;
                    tmem_st<16>(trow + acol, vh);
                    tmem_st<16>(trow + acol + 32, vl);
                    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
                    if (kb > 0 && kb % K2_CHUNK == 0) {
                        // chunk boundary: the previous K block's MMAs end the chunk; move the
                        // accumulator into the output tile before this chunk's first MMA
                        const uint32_t gp = g - 1;
                        ok = mbar_wait(mdone0 + 8 * (gp & 1), (gp >> 1) & 1);
                        if (!ok) *abort_flag = 1;
                        tc_fence_after();
                        if (ok) {
                            const int row = 32 * q + lane;
                            const int64_t s = s0 + row;
                            float *orow = reinterpret_cast<float *>(d.out) + s * 2 * d.ldo + (int64_t)nt * K2_N;
                            drain_row(trow + 128 * hb, orow + 128 * hb, s < d.S, kb == K2_CHUNK, false);
                        }
                    }
                }
                tc_fence_before();
            }
            named_sync();
            if (*abort_flag) {
                aborted = true;
                break;
            }
            if (warp == K2_FIRW && lane == 0) {
                tc_fence_after();
                if (!mbar_wait(bfull0 + 8 * stage, (g >> 1) & 1)) {
                    *abort_flag = 1;
                } else {
                    last_waited_full = g;
                    const uint32_t a_hi = tmem + K2_COL_A + 64 * stage, a_lo = a_hi + 32;
                    const uint32_t b_hi = sB + stage * 2 * K2_TILE_BYTES, b_lo = b_hi + K2_TILE_BYTES;
#pragma unroll
                    for (int ks = 0; ks < K2_KB / 16; ++ks) {
                        const uint64_t dh = smem_desc(b_hi + ks * 256), dl = smem_desc(b_lo + ks * 256);
                        mma_ts(tmem, a_hi + 8 * ks, dh, (kb % K2_CHUNK > 0 || ks > 0) ? 1u : 0u);
                        mma_ts(tmem, a_hi + 8 * ks, dl, 1u);
                        mma_ts(tmem, a_lo + 8 * ks, dh, 1u);
                    }
                    asm volatile(
                        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                            mdone0 + 8 * stage)
                        : "memory");
                    last_commit = g;
                }
            }
        }
        if (aborted) break;
        // ---------------- epilogue: accumulator -> HBM ----------------
        if (warp < K2_FIRW) {
            const int q = warp & 3, hb = warp >> 2;
            const uint32_t gl = g - 1;
            bool ok = mbar_wait(mdone0 + 8 * (gl & 1), (gl >> 1) & 1);
            if (!ok) *abort_flag = 1;
            tc_fence_after();
            if (ok) {
                const int row = 32 * q + lane;
                const int64_t s = s0 + row;
                float *orow = reinterpret_cast<float *>(d.out) + s * 2 * d.ldo + (int64_t)nt * K2_N;
                const uint32_t trow = tmem + ((uint32_t)(32 * q) << 16);
                drain_row(trow + 128 * hb, orow + 128 * hb, s < d.S, KBLK <= K2_CHUNK, true);
            }
            tc_fence_before();
        }
        // all warps: the epilogue's tcgen05.ld are complete before the next
        // unit's first MMA overwrites the accumulator, and every warp takes
        // the same abort decision
        named_sync();
        if (*abort_flag) aborted = true;
    }

    // ---------------- teardown ----------------
    __syncthreads();
    if (warp == K2_FIRW) {
        if (lane == 0) {
            bool ok = true;
            if (last_commit >= 0) ok = mbar_wait(mdone0 + 8 * (last_commit & 1), (last_commit >> 1) & 1) && ok;
            if (last_copy > last_waited_full)
                ok = mbar_wait(bfull0 + 8 * (last_copy & 1), (last_copy >> 1) & 1) && ok;
            if (!ok || *abort_flag) report_error(a.err, KERR_TIMEOUT);
        }
        __syncwarp();
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(K2_TMEM_COLS)
                     : "memory");
    }
}

template <int IN, int TT>
static pfb_status launch_k2(const Plan &plan, LaunchArgs &a, cudaStream_t stream) {
    auto k = k_gemm_bf16x3<IN, TT>;
    static int grid_cap = 0;
    if (grid_cap == 0) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, K2_SMEM);
        if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(k_gemm_bf16x3)");
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        grid_cap = sms;  // one CTA per SM: it takes all 512 TMEM columns
    }
    int64_t grid = a.nunits < grid_cap ? a.nunits : grid_cap;
    if (grid < 1) return PFB_OK;
    a.units_per_cta = 0;
    k<<<(unsigned)grid, K2_THREADS, K2_SMEM, stream>>>(a, plan.P);
    g_launches++;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "launch k_gemm_bf16x3");
    return PFB_OK;
}

template <int IN>
static pfb_status launch_k2_t(const Plan &plan, LaunchArgs &a, cudaStream_t stream) {
    switch (plan.TT) {
    case 4: return launch_k2<IN, 4>(plan, a, stream);
    case 8: return launch_k2<IN, 8>(plan, a, stream);
    default: return launch_k2<IN, 16>(plan, a, stream);
    }
}

pfb_status launch_gemm_bf16x3(const Plan &plan, LaunchArgs &a, cudaStream_t stream) {
    if (plan.variant == 1) return launch_gemm_bf16x3_tcf(plan, a, stream);
    if (plan.variant == 2) return launch_gemm_bf16x3_2p(plan, a, stream);
    if (plan.P < K2_N / 2) return fail(PFB_ERR_UNSUPPORTED, "split-bf16 DFT-GEMM path needs P >= 128");
    if (plan.T > 16) return fail(PFB_ERR_UNSUPPORTED, "split-bf16 DFT-GEMM path needs T <= 16");
    if (a.nunits > 0 && !plan.d_dft) return fail(PFB_ERR_INTERNAL, "split-bf16 DFT matrix not built");
    switch (plan.in_dtype) {
    case PFB_IN_C64: return launch_k2_t<PFB_IN_C64>(plan, a, stream);
    case PFB_IN_R32: return launch_k2_t<PFB_IN_R32>(plan, a, stream);
    case PFB_IN_CI8: return launch_k2_t<PFB_IN_CI8>(plan, a, stream);
    default: return fail(PFB_ERR_INVALID, "bad dtype");
    }
}

}  // namespace pfb
