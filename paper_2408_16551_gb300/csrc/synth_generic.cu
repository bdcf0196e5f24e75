// Synthesis (inverse) filter bank for every plan the fused synthesis kernel
// does not take (any P, any T <= 64, any DFT path, hop P), in two steps:
//   1. the inverse DFT of Sec. 4.2 of every spectrum,
//        y~[s,p] = (1/P) sum_k X[s,k] exp(+2 pi i p k / P),
//      into a plan-owned device buffer, either by a radix-2 Stockham FFT in
//      shared memory with conjugated FP64-built twiddles (FP32 paths) or, for
//      split-bf16 plans, as the product with the conjugate DFT matrix on the
//      tensor cores: the dense split-bf16 DFT-matrix product of the analysis
//      (in two passes for P = 1024, 2048, 4096, else fused) run through an
//      internal one-tap plan (taps 1/P, exact in binary) whose DFT-matrix
//      table is built with the opposite sign;
//   2. the adjoint of the per-branch FIR of Sec. 5.2,
//        xh[f*P + p] = sum_{m<T, 0 <= f-m < S} h'[m*P + p] y~[f-m, p],
//      one output sample per thread, coalesced across p.
#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "devutil.cuh"
#include "internal.h"

namespace pfb {

constexpr int kSyThreads = 256;

static inline int sy_rows(int P) { return P >= 2048 ? 1 : 2048 / P; }

// step 1, FP32: rows [u*RB, u*RB + RB) of X -> y~ (times 1/P), radix-2 Stockham
// passes ping-ponging between two shared buffers, twiddles conj(w_P^r)
__global__ void __launch_bounds__(kSyThreads) k_synth_idft(const float2 *__restrict__ X, float2 *__restrict__ y,
                                                           const float2 *__restrict__ tw_r2, int64_t S, int P,
                                                           int RB) {
    extern __shared__ __align__(16) float2 sy_sm[];
    float2 *buf0 = sy_sm;
    float2 *buf1 = sy_sm + (size_t)RB * P;
    const int t = threadIdx.x;
    const float inv = 1.0f / (float)P;  // a power of two: exact
    const int64_t nunits = (S + RB - 1) / RB;
    for (int64_t u = blockIdx.x; u < nunits; u += gridDim.x) {
        const int64_t s0 = u * RB;
        const int nrows = (int)min((int64_t)RB, S - s0);
        __syncthreads();  // buffers free
        for (int idx = t; idx < nrows * P; idx += kSyThreads) buf0[idx] = __ldg(X + s0 * P + idx);
        __syncthreads();
        float2 *in = buf0, *out = buf1;
        const int half = P >> 1;
        for (int Ns = 1; Ns < P; Ns <<= 1) {
            const bool last = (Ns << 1) == P;
            for (int idx = t; idx < nrows * half; idx += kSyThreads) {
                const int row = idx / half, j = idx - row * half;
                const int jj = j & (Ns - 1);
                const float2 w = __ldg(tw_r2 + jj * (P / (2 * Ns)));
                const float2 x0 = in[row * P + j];
                const float2 x1 = cmul(in[row * P + j + half], make_float2(w.x, -w.y));
                const int base = ((j - jj) << 1) + jj;
                float2 a = cadd(x0, x1), b = csub(x0, x1);
                if (last) {
                    float2 *o = y + (s0 + row) * P;
                    o[base] = make_float2(a.x * inv, a.y * inv);
                    o[base + Ns] = make_float2(b.x * inv, b.y * inv);
                } else {
                    out[row * P + base] = a;
                    out[row * P + base + Ns] = b;
                }
            }
            __syncthreads();
            float2 *tmp = in;
            in = out;
            out = tmp;
        }
    }
}

// step 2: the adjoint per-branch FIR, xh[f, p] for f < S + T - 1
__global__ void __launch_bounds__(kSyThreads) k_synth_fir(const float2 *__restrict__ y, float2 *__restrict__ xh,
                                                          const float *__restrict__ taps, int64_t S, int P, int T) {
    const int64_t F = S + T - 1;
    const int64_t total = F * P;
    for (int64_t i = blockIdx.x * (int64_t)kSyThreads + threadIdx.x; i < total; i += (int64_t)gridDim.x * kSyThreads) {
        const int64_t f = i / P;
        const int p = (int)(i - f * P);
        const int m0 = f >= S ? (int)(f - S + 1) : 0;   // spectra f - m < S
        const int m1 = f < T - 1 ? (int)f : T - 1;      // spectra f - m >= 0
        float2 acc = make_float2(0.f, 0.f);
        for (int m = m0; m <= m1; ++m) {
            const float hv = __ldg(taps + (int64_t)m * P + p);
            const float2 v = __ldg(y + (f - m) * P + p);
            acc.x = fmaf(hv, v.x, acc.x);
            acc.y = fmaf(hv, v.y, acc.y);
        }
        store_cs(xh + i, acc);
    }
}

static int device_sms() {
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms < 1) sms = 1;
    }
    return sms;
}

pfb_status build_gemm_bf16x3_table_conj(Plan &plan);

// The internal one-tap plan of the tensor-core inverse DFT (built on first use).
static pfb_status ensure_inverse_plan(Plan &p) {
    if (p.inv) return PFB_OK;
    Plan *q = new (std::nothrow) Plan();
    if (!q) return fail(PFB_ERR_OOM, "host allocation");
    q->desc = p.desc;
    q->desc.T = 1;
    q->desc.window = PFB_WIN_USER;
    q->desc.in_dtype = PFB_IN_C64;
    q->desc.hop = 0;
    q->desc.tap_order = PFB_TAPS_CORRELATION;
    q->device = p.device;
    q->P = p.P;
    q->T = 1;
    q->TT = fft_fast_tt(1);
    q->in_dtype = PFB_IN_C64;
    q->path = PFB_DFT_GEMM_BF16X3;
    q->family = FAM_GEMM_BF16X3;
    q->esize = 8;
    q->hop = p.P;
    q->R = 1;
    // the dense DFT-matrix product: in two passes (a one-tap FIR pass into the
    // pre-tiled workspace, then the pipelined GEMM) where that kernel exists,
    // else fused
    q->variant = gemm2p_supported(*q) ? 2 : 0;
    q->h_err = p.h_err;  // report into the parent plan's error word
    q->d_err = p.d_err;
    q->wait_ns = p.wait_ns;
    pfb_status st = PFB_OK;
    // taps: 1/P in row 0, zero in the padded rows
    std::vector<float> taps((size_t)q->TT * q->P, 0.0f);
    for (int i = 0; i < q->P; ++i) taps[i] = 1.0f / (float)q->P;
    if (cudaMalloc(&q->d_taps_pad, sizeof(float) * taps.size()) != cudaSuccess) st = fail(PFB_ERR_OOM, "inverse taps");
    if (st == PFB_OK &&
        cudaMemcpy(q->d_taps_pad, taps.data(), sizeof(float) * taps.size(), cudaMemcpyHostToDevice) != cudaSuccess)
        st = fail(PFB_ERR_CUDA, "inverse taps copy");
    if (st == PFB_OK) st = build_gemm_bf16x3_table_conj(*q);
    if (st == PFB_OK && cudaDeviceSynchronize() != cudaSuccess) st = fail(PFB_ERR_CUDA, "inverse table");
    if (st == PFB_OK) st = prepare_family(*q);
    if (st != PFB_OK) {
        cudaFree(q->d_taps_pad);
        cudaFree(q->d_dft);
        free_plan_workspaces(*q);
        delete q;
        return st;
    }
    p.inv = q;
    return PFB_OK;
}

void free_inverse_plan(Plan &p) {
    if (!p.inv) return;
    cudaFree(p.inv->d_taps_pad);
    cudaFree(p.inv->d_dft);
    free_plan_workspaces(*p.inv);
    delete p.inv;
    p.inv = nullptr;
}

bool synth_generic_supported(const Plan &p) {
    if (p.R != 1) return false;
    if (p.family == FAM_GEMM_BF16X3) return p.P >= 128 && p.P <= 4096;
    return true;
}

pfb_status launch_synth_generic(Plan &p, const float2 *X, int64_t S, float2 *xh, cudaStream_t stream) {
    const size_t ybytes = (size_t)S * p.P * sizeof(float2);
    {
        std::lock_guard<std::mutex> lk(p.stage_mu);
        if (p.synth_y_bytes < ybytes) {
            cudaFree(p.d_synth_y);
            p.d_synth_y = nullptr;
            p.synth_y_bytes = 0;
            if (cudaMalloc(&p.d_synth_y, ybytes) != cudaSuccess) {
                cudaGetLastError();
                return fail(PFB_ERR_OOM, "synthesis buffer");
            }
            p.synth_y_bytes = ybytes;
        }
        if (p.family == FAM_GEMM_BF16X3) {
            pfb_status st = ensure_inverse_plan(p);
            if (st != PFB_OK) return st;
        }
    }
    float2 *y = static_cast<float2 *>(p.d_synth_y);
    if (p.family == FAM_GEMM_BF16X3) {
        // the spectra as a one-tap "stream" of S frames: spectrum s of the
        // inverse plan is (1/P) X[s] times the conjugate DFT matrix
        StreamDesc d;
        std::memset(&d, 0, sizeof(d));
        d.in = X;
        d.out = y;
        d.n_frames = S;
        d.S = S;
        d.ldo = p.P;
        d.taps = p.inv->d_taps_pad;
        d.scale = 1.0f;
        d.T = 1;
        pfb_status st = launch_family(*p.inv, &d, 1, stream);
        if (st != PFB_OK) return st;
    } else {
        const int RB = sy_rows(p.P);
        const size_t smem = 2 * (size_t)RB * p.P * sizeof(float2);
        static bool attr = false;
        if (!attr) {
            cudaError_t e = cudaFuncSetAttribute(k_synth_idft, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024);
            if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(k_synth_idft)");
            attr = true;
        }
        const int64_t units = (S + RB - 1) / RB;
        const unsigned grid = (unsigned)std::min<int64_t>(units, (int64_t)device_sms() * 4);
        k_synth_idft<<<grid, kSyThreads, smem, stream>>>(X, y, p.d_tw_r2, S, p.P, RB);
        g_launches++;
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e, "launch k_synth_idft");
    }
    const int64_t total = (S + p.T - 1) * p.P;
    const unsigned grid = (unsigned)std::min<int64_t>((total + kSyThreads - 1) / kSyThreads, (int64_t)device_sms() * 8);
    k_synth_fir<<<grid, kSyThreads, 0, stream>>>(y, xh, p.d_taps, S, p.P, p.T);
    g_launches++;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "launch k_synth_fir");
    return PFB_OK;
}

}  // namespace pfb
