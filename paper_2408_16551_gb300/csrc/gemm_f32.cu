// Polyphase FIR + DFT as a product with the Fourier matrix, FP32 on the SIMT
// cores (the "plain FP32 form" of the DFT-as-matrix-product, Sec. 4.1:
// Z(m,n) = sum_l X(m,l) F(l,n) with F = the P x P DFT matrix).
//
//   A = y[s, p]      (branch sums, the FIR of Sec. 5.2)
//   B = W[p, k] = exp(-2 pi i (p k mod P) / P)   (complex64, built in FP64)
//   X[s, k] = sum_p A[s, p] B[p, k]               (complex FMA, FP32 accumulation)
//
// Two routes.
// P a multiple of 128 (two passes): k_fir_rows_f32 computes the FIR once into
//   a plan-owned workspace, 128-spectrum row blocks of [128][P] complex64 (rows
//   past a stream's end are zero); k_cgemm_f32 multiplies: a work unit is a
//   128-spectrum x 128-bin output tile, 256 threads each accumulating an 8 x 8
//   complex micro-tile (rows ty + 16 i, bin pairs 2 tx + 32 j: 16-byte shared
//   reads of two branches of A and of two bins of W, conflict-free, and
//   16-byte coalesced stores), the K loop walks 16 branches at a time through
//   a 3-stage ring of 16-byte cp.async copies of the A and W slices.
// Other P (fused): a work unit is a 64-spectrum x BN-bin output tile (BN = 128,
//   or 64 for P = 64); 256 threads, each accumulating a 4 x BN/16 complex
//   micro-tile; the K loop walks 16 branches at a time: the FIR computes the
//   64 x 16 slice of A in the kernel (four spectra per thread: each input
//   frame is loaded once per thread), the matching 16 x BN slice of W comes
//   from HBM/L2.
// Units are dealt round-robin so CTAs running at the same time share M-tiles
// (input rows) and W stays hot in L2.  Both routes add the products over p in
// the same order.
#include "devutil.cuh"
#include "internal.h"

namespace pfb {

constexpr int G3_BM = 64, G3_BK = 16, G3_THREADS = 256;
static int g3_bn(int P) { return P >= 128 ? 128 : 64; }

// two-pass route: tile 128 x 128, K slices of 16 branches, 3 stages
constexpr int G4_BM = 128, G4_BN = 128, G4_BK = 16, G4_NST = 3, G4_THREADS = 256, G4_FB = 256;
constexpr int G4_ASTR = G4_BK + 2;                               // A row stride (float2): 144 bytes
constexpr int G4_STAGE = G4_BM * G4_ASTR + G4_BK * G4_BN;        // float2 per stage (A, then W)
constexpr int G4_SMEM = G4_NST * G4_STAGE * 8;
static bool g4_two_pass(const Plan &plan) { return plan.P >= 128 && plan.P % 128 == 0; }

size_t gemm_f32_workspace_bytes(const Plan &plan, int64_t nunits) {
    if (!g4_two_pass(plan)) return 0;
    return (size_t)(nunits / (plan.P / G4_BN)) * G4_BM * plan.P * sizeof(float2);
}

int64_t gemm_f32_units(const Plan &plan, int64_t S) {
    if (g4_two_pass(plan)) return ((S + G4_BM - 1) / G4_BM) * (plan.P / G4_BN);
    return ((S + G3_BM - 1) / G3_BM) * (plan.P / g3_bn(plan.P));
}

// W[p][k] = exp(-2 pi i (p k mod P) / P) in FP64, rounded to complex64
__global__ void gen_dft_f32_kernel(float2 *W, int P) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= (int64_t)P * P) return;
    const int64_t p = i / P, k = i % P;
    const int64_t e = (p * k) % P;
    double s, c;
    sincospi(2.0 * (double)e / (double)P, &s, &c);
    W[i] = make_float2((float)c, (float)-s);
}

template <int IN, int G3_BN>
__global__ void __launch_bounds__(G3_THREADS) k_gemm_f32(const __grid_constant__ LaunchArgs a, int P) {
    using L = Loader<IN>;
    constexpr int G3_NJ = G3_BN / 16;  // bins per thread
    __shared__ float2 As[G3_BK][G3_BM + 1];
    __shared__ float2 Bs[G3_BK][G3_BN];
    const float2 *W = static_cast<const float2 *>(a.aux);
    const int t = threadIdx.x, tx = t & 15, ty = t >> 4;
    const int NT = P / G3_BN;
    for (int64_t u = blockIdx.x; u < a.nunits; u += gridDim.x) {
        const int si = find_stream(a, u);
        const StreamDesc &d = a.s[si];
        const int64_t lu = u - d.unit0;
        const int64_t s0 = (lu / NT) * G3_BM;
        const int k0 = (int)(lu % NT) * G3_BN;
        float2 acc[4][G3_NJ];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < G3_NJ; ++j) acc[i][j] = make_float2(0.f, 0.f);
        for (int pc = 0; pc < P; pc += G3_BK) {
            __syncthreads();
            // A slice: FIR of 64 spectra x 16 branches.  Thread (kk, g) computes
            // spectra 4g .. 4g+3 of branch pc + kk: it streams the T + 3 frames they
            // share once, keeping the last four taps in registers (tap i meets
            // spectrum 4g + r at frame 4g + r + i)
            {
                const int kk = t & 15, g = t >> 4;
                const int p = pc + kk;
                const int64_t sg = s0 + 4 * g;
                float2 y0 = make_float2(0.f, 0.f), y1 = y0, y2 = y0, y3 = y0;
                float h0 = 0.f, h1 = 0.f, h2 = 0.f, h3 = 0.f;
                if (sg < d.S) {
#pragma unroll 2
                    for (int i = 0; i < d.T + 3; ++i) {
                        h3 = h2; h2 = h1; h1 = h0;
                        h0 = i < d.T ? __ldg(d.taps + i * P + p) : 0.f;
                        const int64_t f = sg + i;
                        float2 v = make_float2(0.f, 0.f);
                        if (f < d.n_frames) {
                            int64_t smp;
                            const void *src = frame_source(d, f, P, smp);
                            v = L::load1(src, smp + p, d.scale);
                        }
                        // frame sg + i: tap i of spectrum sg, tap i-1 of sg+1, ...
                        y0.x = fmaf(h0, v.x, y0.x); y0.y = fmaf(h0, v.y, y0.y);
                        y1.x = fmaf(h1, v.x, y1.x); y1.y = fmaf(h1, v.y, y1.y);
                        y2.x = fmaf(h2, v.x, y2.x); y2.y = fmaf(h2, v.y, y2.y);
                        y3.x = fmaf(h3, v.x, y3.x); y3.y = fmaf(h3, v.y, y3.y);
                    }
                }
                As[kk][4 * g] = y0;
                As[kk][4 * g + 1] = sg + 1 < d.S ? y1 : make_float2(0.f, 0.f);
                As[kk][4 * g + 2] = sg + 2 < d.S ? y2 : make_float2(0.f, 0.f);
                As[kk][4 * g + 3] = sg + 3 < d.S ? y3 : make_float2(0.f, 0.f);
            }
            // B slice: 16 x 128 of W
#pragma unroll
            for (int e = 0; e < G3_BK * G3_BN / G3_THREADS; ++e) {
                const int idx = t + e * G3_THREADS;
                const int kk = idx / G3_BN, c = idx % G3_BN;
                Bs[kk][c] = __ldg(W + (int64_t)(pc + kk) * P + k0 + c);
            }
            __syncthreads();
#pragma unroll
            for (int kk = 0; kk < G3_BK; ++kk) {
                float2 av[4], bv[G3_NJ];
#pragma unroll
                for (int i = 0; i < 4; ++i) av[i] = As[kk][ty + 16 * i];
#pragma unroll
                for (int j = 0; j < G3_NJ; ++j) bv[j] = Bs[kk][tx + 16 * j];
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < G3_NJ; ++j) {
                        acc[i][j].x = fmaf(av[i].x, bv[j].x, acc[i][j].x);
                        acc[i][j].x = fmaf(-av[i].y, bv[j].y, acc[i][j].x);
                        acc[i][j].y = fmaf(av[i].x, bv[j].y, acc[i][j].y);
                        acc[i][j].y = fmaf(av[i].y, bv[j].x, acc[i][j].y);
                    }
            }
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int64_t s = s0 + ty + 16 * i;
            if (s < d.S) {
#pragma unroll
                for (int j = 0; j < G3_NJ; ++j) store_cs(d.out + s * d.ldo + k0 + tx + 16 * j, acc[i][j]);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// two-pass route, pass 1: the FIR into 128-spectrum row blocks
// ---------------------------------------------------------------------------
// Work item = (global row block gmb, 256 branches); thread t owns branch
// p = 256 * chunk + t and the block's 32 groups of four spectra: group g
// streams the T + 3 frames its four spectra share once, with the last four
// taps in registers (the A-slice FIR of the fused kernel).
template <int IN>
__global__ void __launch_bounds__(G4_THREADS) k_fir_rows_f32(const __grid_constant__ LaunchArgs a, int P, float2 *Y) {
    using L = Loader<IN>;
    const int NT = P / G4_BN;
    const int nbb = (P + G4_FB - 1) / G4_FB;
    const int64_t nmb = a.nunits / NT;
    for (int64_t w = blockIdx.x; w < nmb * nbb; w += gridDim.x) {
        const int64_t gmb = w / nbb;
        const int p = (int)(w % nbb) * G4_FB + threadIdx.x;
        if (p >= P) continue;
        const int si = find_stream(a, gmb * NT);
        const StreamDesc &d = a.s[si];
        const int64_t s0 = (gmb - d.unit0 / NT) * G4_BM;
        float2 *yb = Y + gmb * (int64_t)G4_BM * P + p;
        for (int g = 0; g < G4_BM / 4; ++g) {
            const int64_t sg = s0 + 4 * g;
            float2 y0 = make_float2(0.f, 0.f), y1 = y0, y2 = y0, y3 = y0;
            float h0 = 0.f, h1 = 0.f, h2 = 0.f, h3 = 0.f;
            if (sg < d.S) {
#pragma unroll 2
                for (int i = 0; i < d.T + 3; ++i) {
                    h3 = h2; h2 = h1; h1 = h0;
                    h0 = i < d.T ? __ldg(d.taps + i * P + p) : 0.f;
                    const int64_t f = sg + i;
                    float2 v = make_float2(0.f, 0.f);
                    if (f < d.n_frames) {
                        int64_t smp;
                        const void *src = frame_source(d, f, P, smp);
                        v = L::load1(src, smp + p, d.scale);
                    }
                    // frame sg + i: tap i of spectrum sg, tap i-1 of sg+1, ...
                    y0.x = fmaf(h0, v.x, y0.x); y0.y = fmaf(h0, v.y, y0.y);
                    y1.x = fmaf(h1, v.x, y1.x); y1.y = fmaf(h1, v.y, y1.y);
                    y2.x = fmaf(h2, v.x, y2.x); y2.y = fmaf(h2, v.y, y2.y);
                    y3.x = fmaf(h3, v.x, y3.x); y3.y = fmaf(h3, v.y, y3.y);
                }
            }
            const float2 z = make_float2(0.f, 0.f);
            yb[(int64_t)(4 * g) * P] = sg < d.S ? y0 : z;
            yb[(int64_t)(4 * g + 1) * P] = sg + 1 < d.S ? y1 : z;
            yb[(int64_t)(4 * g + 2) * P] = sg + 2 < d.S ? y2 : z;
            yb[(int64_t)(4 * g + 3) * P] = sg + 3 < d.S ? y3 : z;
        }
    }
}

// ---------------------------------------------------------------------------
// two-pass route, pass 2: X = Y W, 128 x 128 tiles
// ---------------------------------------------------------------------------
__device__ __forceinline__ void g4_cp16(uint32_t dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void g4_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void g4_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

// the A slice (128 rows x 16 branches: 8 pieces of 16 bytes per row) and the
// W slice (16 rows x 128 bins: 64 pieces per row) of K step kb into stage st
__device__ __forceinline__ void g4_load(uint32_t sbase, int st, const float2 *ya, const float2 *W, int P, int k0,
                                        int kb, int t) {
    const uint32_t as = sbase + (uint32_t)(st * G4_STAGE) * 8u;
    const uint32_t bs = as + (uint32_t)(G4_BM * G4_ASTR) * 8u;
    const int pc = kb * G4_BK;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const int q = t + G4_THREADS * e;  // A piece: row q / 8, piece q % 8
        const int m = q >> 3, c = q & 7;
        g4_cp16(as + (uint32_t)(m * G4_ASTR + 2 * c) * 8u, ya + (int64_t)m * P + pc + 2 * c);
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const int q = t + G4_THREADS * e;  // W piece: row q / 64, piece q % 64
        const int kk = q >> 6, c = q & 63;
        g4_cp16(bs + (uint32_t)(kk * G4_BN + 2 * c) * 8u, W + (int64_t)(pc + kk) * P + k0 + 2 * c);
    }
}

__global__ void __launch_bounds__(G4_THREADS, 1) k_cgemm_f32(const __grid_constant__ LaunchArgs a, int P,
                                                            const float2 *__restrict__ Y) {
    extern __shared__ __align__(16) float2 g4_smem[];
    const float2 *W = static_cast<const float2 *>(a.aux);
    const int t = threadIdx.x, tx = t & 15, ty = t >> 4;
    const int NT = P / G4_BN, NK = P / G4_BK;
    const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(g4_smem);
    for (int64_t u = blockIdx.x; u < a.nunits; u += gridDim.x) {
        const int64_t gmb = u / NT;
        const int k0 = (int)(u % NT) * G4_BN;
        const int si = find_stream(a, u);
        const StreamDesc &d = a.s[si];
        const int64_t s0 = (gmb - d.unit0 / NT) * G4_BM;
        const float2 *ya = Y + gmb * (int64_t)G4_BM * P;
        float2 acc[8][8];
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[i][j] = make_float2(0.f, 0.f);
        __syncthreads();  // the previous tile's last stage has been read by every thread
        g4_load(sbase, 0, ya, W, P, k0, 0, t);
        g4_commit();
        if (NK > 1) g4_load(sbase, 1, ya, W, P, k0, 1, t);
        g4_commit();
        for (int kb = 0; kb < NK; ++kb) {
            g4_wait1();        // this thread's copies of step kb have landed
            __syncthreads();   // everyone's have; stage (kb + 2) mod 3 is no longer read
            if (kb + 2 < NK) g4_load(sbase, (kb + 2) % G4_NST, ya, W, P, k0, kb + 2, t);
            g4_commit();
            const float2 *As = g4_smem + (kb % G4_NST) * G4_STAGE;
            const float2 *Bs = As + G4_BM * G4_ASTR;
#pragma unroll
            for (int kk = 0; kk < G4_BK; kk += 2) {
                float4 av[8];  // rows ty + 16 i, branches kk and kk + 1
#pragma unroll
                for (int i = 0; i < 8; ++i) av[i] = *reinterpret_cast<const float4 *>(As + (ty + 16 * i) * G4_ASTR + kk);
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    float4 bq[4];  // bins 2 tx + 32 j .. + 1
#pragma unroll
                    for (int j = 0; j < 4; ++j) bq[j] = *reinterpret_cast<const float4 *>(Bs + (kk + h) * G4_BN + 2 * tx + 32 * j);
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        const float ax = h ? av[i].z : av[i].x, ay = h ? av[i].w : av[i].y;
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            float2 &c0 = acc[i][2 * j], &c1 = acc[i][2 * j + 1];
                            c0.x = fmaf(ax, bq[j].x, c0.x); c0.x = fmaf(-ay, bq[j].y, c0.x);
                            c0.y = fmaf(ax, bq[j].y, c0.y); c0.y = fmaf(ay, bq[j].x, c0.y);
                            c1.x = fmaf(ax, bq[j].z, c1.x); c1.x = fmaf(-ay, bq[j].w, c1.x);
                            c1.y = fmaf(ax, bq[j].w, c1.y); c1.y = fmaf(ay, bq[j].z, c1.y);
                        }
                    }
                }
            }
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int64_t s = s0 + ty + 16 * i;
            if (s < d.S) {
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    __stcs(reinterpret_cast<float4 *>(d.out + s * d.ldo + k0 + 2 * tx + 32 * j),
                           make_float4(acc[i][2 * j].x, acc[i][2 * j].y, acc[i][2 * j + 1].x, acc[i][2 * j + 1].y));
            }
        }
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
}

template <int IN>
static pfb_status launch_g4(const Plan &plan, LaunchArgs &a, cudaStream_t stream) {
    static int grid_cap = 0, fir_cap = 0;
    if (grid_cap == 0) {
        cudaError_t e = cudaFuncSetAttribute(k_cgemm_f32, cudaFuncAttributeMaxDynamicSharedMemorySize, G4_SMEM);
        if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(k_cgemm_f32)");
        int dev = 0, sms = 0, per_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fir_rows_f32<IN>, G4_THREADS, 0);
        if (e != cudaSuccess || per_sm < 1) return cuda_fail(e, "occupancy(k_fir_rows_f32)");
        fir_cap = sms * per_sm;
        grid_cap = sms;  // one CTA per SM (registers of the 8 x 8 complex micro-tile)
    }
    if (a.nunits <= 0) return PFB_OK;
    const int NT = plan.P / G4_BN;
    const int64_t nmb = a.nunits / NT;
    pfb_status wst = grow_plan_workspace(plan, gemm_f32_workspace_bytes(plan, a.nunits), stream);
    if (wst != PFB_OK) return wst;
    Plan &mp = const_cast<Plan &>(plan);
    float2 *Y = static_cast<float2 *>(mp.d_ws2);
    a.units_per_cta = 0;
    const int64_t fwork = nmb * ((plan.P + G4_FB - 1) / G4_FB);
    const int64_t fgrid = fwork < fir_cap ? fwork : fir_cap;
    k_fir_rows_f32<IN><<<(unsigned)fgrid, G4_THREADS, 0, stream>>>(a, plan.P, Y);
    g_launches++;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "launch k_fir_rows_f32");
    const int64_t grid = a.nunits < grid_cap ? a.nunits : grid_cap;
    k_cgemm_f32<<<(unsigned)grid, G4_THREADS, G4_SMEM, stream>>>(a, plan.P, Y);
    g_launches++;
    e = cudaGetLastError();
    return e == cudaSuccess ? PFB_OK : cuda_fail(e, "launch k_cgemm_f32");
}

template <int IN, int BN>
static pfb_status launch_g3(const Plan &plan, LaunchArgs &a, cudaStream_t stream) {
    auto k = k_gemm_f32<IN, BN>;
    static int grid_cap = 0;
    if (grid_cap == 0) {
        int dev = 0, sms = 0, per_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, G3_THREADS, 0);
        if (e != cudaSuccess || per_sm < 1) return cuda_fail(e, "occupancy(k_gemm_f32)");
        grid_cap = sms * per_sm;
    }
    int64_t grid = a.nunits < grid_cap ? a.nunits : grid_cap;
    if (grid < 1) return PFB_OK;
    a.units_per_cta = 0;
    k<<<(unsigned)grid, G3_THREADS, 0, stream>>>(a, plan.P);
    g_launches++;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "launch k_gemm_f32");
    return PFB_OK;
}

pfb_status launch_gemm_f32(const Plan &plan, LaunchArgs &a, cudaStream_t stream) {
    if (plan.P < 64) return fail(PFB_ERR_UNSUPPORTED, "FP32 DFT-GEMM path needs P >= 64");
    if (g4_two_pass(plan)) {
        switch (plan.in_dtype) {
        case PFB_IN_C64: return launch_g4<PFB_IN_C64>(plan, a, stream);
        case PFB_IN_R32: return launch_g4<PFB_IN_R32>(plan, a, stream);
        case PFB_IN_CI8: return launch_g4<PFB_IN_CI8>(plan, a, stream);
        default: return fail(PFB_ERR_INVALID, "bad dtype");
        }
    }
    const bool wide = g3_bn(plan.P) == 128;
    switch (plan.in_dtype) {
    case PFB_IN_C64: return wide ? launch_g3<PFB_IN_C64, 128>(plan, a, stream) : launch_g3<PFB_IN_C64, 64>(plan, a, stream);
    case PFB_IN_R32: return wide ? launch_g3<PFB_IN_R32, 128>(plan, a, stream) : launch_g3<PFB_IN_R32, 64>(plan, a, stream);
    case PFB_IN_CI8: return wide ? launch_g3<PFB_IN_CI8, 128>(plan, a, stream) : launch_g3<PFB_IN_CI8, 64>(plan, a, stream);
    default: return fail(PFB_ERR_INVALID, "bad dtype");
    }
}

pfb_status build_gemm_f32_table(Plan &plan) {
    const int64_t n = (int64_t)plan.P * plan.P;
    plan.dft_bytes = n * sizeof(float2);
    PFB_CUDA_TRY(cudaMalloc(&plan.d_dft, plan.dft_bytes));
    gen_dft_f32_kernel<<<(unsigned)((n + 255) / 256), 256>>>(static_cast<float2 *>(plan.d_dft), plan.P);
    g_launches++;
    PFB_CUDA_TRY(cudaGetLastError());
    return PFB_OK;
}

}  // namespace pfb
