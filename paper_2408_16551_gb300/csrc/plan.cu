// Plan creation: validation, FP64 table generation on the GPU, plan lifetime.
//
// Everything here runs once per plan.  FP64 is used on the GPU only in these
// generators: the windowed-sinc prototype (the branch taps of Sec. 5.2), the
// FFT twiddles and the DFT matrix (the Fourier matrix of Sec. 4.1).
#include <cmath>
#include <cstring>
#include <new>

#include "fftplan.h"
#include "internal.h"

namespace pfb {

bool is_pow2(int64_t v) { return v > 0 && (v & (v - 1)) == 0; }
int ilog2(int64_t v) {
    int r = 0;
    while ((int64_t(1) << r) < v) ++r;
    return r;
}

int64_t out_spectra(const Plan &p, int64_t n_samples) {
    if (n_samples < 0) return -1;
    if (p.R > 1) {  // hop D < P: windows start at s*D and span P*T samples
        const int64_t L = (int64_t)p.P * p.T;
        return n_samples < L ? 0 : (n_samples - L) / p.hop + 1;
    }
    int64_t F = n_samples / p.P;
    int64_t S = F - p.T + 1;
    return S > 0 ? S : 0;
}

// ---------------------------------------------------------------------------
// FP64 generators
// ---------------------------------------------------------------------------

// Symmetric window over L points times sinc((n-c)/P), c = (L-1)/2.
__global__ void gen_prototype_kernel(double *h, int P, int L, int window) {
    int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= L) return;
    double w = 1.0;
    if (L > 1) {
        double a = 2.0 * (double)n / (double)(L - 1);  // angle / pi
        switch (window) {
        case PFB_WIN_HANN: w = 0.5 - 0.5 * cospi(a); break;
        case PFB_WIN_HAMMING: w = 0.54 - 0.46 * cospi(a); break;
        case PFB_WIN_BLACKMAN: w = 0.42 - 0.5 * cospi(a) + 0.08 * cospi(2.0 * a); break;
        default: break;
        }
    }
    double u = ((double)n - 0.5 * (double)(L - 1)) / (double)P;
    double s = (u == 0.0) ? 1.0 : sinpi(u) / (3.14159265358979323846 * u);
    h[n] = w * s;
}

// One block: deterministic FP64 sum, then h /= sum.
__global__ void normalise_kernel(double *h, int L) {
    __shared__ double part[1024];
    double acc = 0.0;
    for (int i = threadIdx.x; i < L; i += blockDim.x) acc += h[i];
    part[threadIdx.x] = acc;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
        __syncthreads();
    }
    double sum = part[0];
    for (int i = threadIdx.x; i < L; i += blockDim.x) h[i] = h[i] / sum;
}

// taps[m][p] = h[m*P+p] (fp32) and the zero-extended copy used by the fast
// FFT family: pad[m][p] = h[m*P+p] for m < T, 0 for T <= m < TT.
// fp32 tap tables [T][P] (and the zero-extended [TT][P] copy); with the
// convolution tap order, row m of branch p holds h[(T-1-m)*P + p]
__global__ void taps_to_f32_kernel(const double *h, int P, int T, int TT, int reverse, float *taps, float *pad) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P * (TT > T ? TT : T)) return;
    const int m = i / P, p = i % P;
    const float v = (m < T) ? (float)h[(reverse ? (T - 1 - m) : m) * P + p] : 0.0f;
    if (i < P * T) taps[i] = v;
    if (pad && i < P * TT) pad[i] = v;
}

// exp(-2 pi i e / M) in FP64, rounded to fp32.
__device__ __forceinline__ float2 twiddle64(int64_t e, int64_t M) {
    e %= M;
    double s, c;
    sincospi(2.0 * (double)e / (double)M, &s, &c);
    return make_float2((float)c, (float)-s);
}

// radix-2 table: w^r = exp(-2 pi i r / P), r < P/2
__global__ void gen_tw_r2_kernel(float2 *tw, int P) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < P / 2) tw[r] = twiddle64(r, P);
}

// Stockham pass tables of the fast FFT family: for each pass (Ns, R) with
// Ns > 1, entries [(j mod Ns)*(R-1) + r-1] = exp(-2 pi i r j / (Ns R)).
__global__ void gen_tw_pass_kernel(float2 *tw, int Ns, int R) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= Ns * (R - 1)) return;
    int j = i / (R - 1), r = i % (R - 1) + 1;
    tw[i] = twiddle64((int64_t)r * j, (int64_t)Ns * R);
}

// ---------------------------------------------------------------------------
// fast-FFT family twiddles (pass list in fftplan.h)
// ---------------------------------------------------------------------------
pfb_status grow_plan_workspace(const Plan &plan, size_t bytes, cudaStream_t stream) {
    Plan &mp = const_cast<Plan &>(plan);
    std::lock_guard<std::mutex> lk(mp.ws2_mu);
    if (mp.ws2_bytes >= bytes) return PFB_OK;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    const cudaError_t ce = cudaStreamIsCapturing(stream, &cs);
    if (ce != cudaSuccess) cudaGetLastError();
    else if (cs != cudaStreamCaptureStatusNone)
        return fail(PFB_ERR_UNSUPPORTED, "the plan's workspace would grow inside a stream capture: run a launch "
                                         "of this size before capturing it");
    if (mp.d_ws2) mp.ws2_retired.push_back(mp.d_ws2);  // a captured graph may still read it
    mp.d_ws2 = nullptr;
    mp.ws2_bytes = 0;
    if (cudaMalloc(&mp.d_ws2, bytes) != cudaSuccess) {
        cudaGetLastError();
        return fail(PFB_ERR_OOM, "plan workspace");
    }
    mp.ws2_bytes = bytes;
    return PFB_OK;
}

void free_plan_workspaces(Plan &plan) {
    cudaFree(plan.d_ws2);
    plan.d_ws2 = nullptr;
    plan.ws2_bytes = 0;
    for (void *q : plan.ws2_retired) cudaFree(q);
    plan.ws2_retired.clear();
}

static pfb_status build_pass_table(int P, int MR, float2 **out) {
    const int total = fft_tw_entries(P, MR);
    PFB_CUDA_TRY(cudaMalloc(out, (total > 0 ? total : 1) * sizeof(float2)));
    for (int i = 0; i < fft_npasses(P, MR); ++i) {
        const int Ns = fft_ns(P, i, MR), R = fft_radix(P, i, MR);
        if (Ns == 1) continue;
        const int n = Ns * (R - 1);
        gen_tw_pass_kernel<<<(n + 255) / 256, 256>>>(*out + fft_tw_offset(P, i, MR), Ns, R);
        g_launches++;
    }
    PFB_CUDA_TRY(cudaGetLastError());
    return PFB_OK;
}

// tables for the radix-16 and radix-32 pass lists (variants pick one)
pfb_status build_fft_fast_twiddles(Plan &plan) {
    pfb_status st = build_pass_table(plan.P, 16, &plan.d_tw);
    if (st != PFB_OK) return st;
    return build_pass_table(plan.P, 32, &plan.d_tw32);
}

// ---------------------------------------------------------------------------
// plan lifetime
// ---------------------------------------------------------------------------

static_assert(sizeof(pfb_plan_desc) == 48, "pfb_plan_desc layout (the Python binding mirrors it)");

static pfb_status validate(const pfb_plan_desc *d) {
    if (!d) return fail(PFB_ERR_INVALID, "descriptor is NULL");
    if (!is_pow2(d->P) || d->P < 4 || d->P > 4096)
        return fail(PFB_ERR_INVALID, "P must be a power of two in [4, 4096]");
    if (d->T < 1 || d->T > 64) return fail(PFB_ERR_INVALID, "T must be in [1, 64]");
    if (d->in_dtype < PFB_IN_R32 || d->in_dtype > PFB_IN_CI8) return fail(PFB_ERR_INVALID, "bad in_dtype");
    if (d->window < PFB_WIN_HANN || d->window > PFB_WIN_USER) return fail(PFB_ERR_INVALID, "bad window");
    if (d->window == PFB_WIN_USER && !d->user_taps_host)
        return fail(PFB_ERR_INVALID, "window USER needs user_taps_host");
    if (d->window != PFB_WIN_USER && d->user_taps_host)
        return fail(PFB_ERR_INVALID, "user_taps_host given without window USER");
    if (d->path < PFB_DFT_FFT_F32 || d->path > PFB_DFT_GEMM_BF16X3) return fail(PFB_ERR_INVALID, "bad path");
    if (d->in_dtype == PFB_IN_CI8 && !std::isfinite(d->in_scale))
        return fail(PFB_ERR_INVALID, "in_scale must be finite");
    if (d->reserved != 0) return fail(PFB_ERR_INVALID, "reserved field must be 0");
    if (d->tap_order != PFB_TAPS_CORRELATION && d->tap_order != PFB_TAPS_CONVOLUTION)
        return fail(PFB_ERR_INVALID, "bad tap_order");
    if (d->hop != 0 && d->hop != d->P) {
        const int esize = d->in_dtype == PFB_IN_R32 ? 4 : d->in_dtype == PFB_IN_C64 ? 8 : 2;
        if (d->hop < 1 || d->hop > d->P || d->P % d->hop != 0) return fail(PFB_ERR_INVALID, "hop must divide P");
        if (d->P / d->hop > kMaxOversampling) return fail(PFB_ERR_INVALID, "oversampling P/hop above 32");
        if ((d->hop * esize) % 16 != 0)
            return fail(PFB_ERR_INVALID, "hop * bytes per sample must be a multiple of 16");
    }
    return PFB_OK;
}

static void free_plan(Plan *p) {
    if (!p) return;
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(p->device);
    cudaFree(p->d_h64);
    cudaFree(p->d_taps);
    cudaFree(p->d_taps_pad);
    cudaFree(p->d_tw);
    cudaFree(p->d_tw_r2);
    cudaFree(p->d_tw32);
    cudaFree(p->d_dft);
    cudaFree(p->d_tcf);
    free_error_words(p->h_err);
    if (p->s_copy_in) cudaStreamDestroy(p->s_copy_in);
    if (p->s_copy_out) cudaStreamDestroy(p->s_copy_out);
    for (cudaEvent_t e : p->ev_pipe)
        if (e) cudaEventDestroy(e);
    cudaFree(p->d_stage_in);
    cudaFree(p->d_stage_out);
    cudaFree(p->d_synth_y);
    free_plan_workspaces(*p);
    free_inverse_plan(*p);
    if (prev >= 0) cudaSetDevice(prev);
    delete p;
}

static pfb_status create_impl(const pfb_plan_desc *desc, Plan *p) {
    p->desc = *desc;
    p->desc.user_taps_host = nullptr;
    p->P = desc->P;
    p->T = desc->T;
    p->in_dtype = desc->in_dtype;
    p->path = desc->path;
    p->esize = desc->in_dtype == PFB_IN_R32 ? 4 : desc->in_dtype == PFB_IN_C64 ? 8 : 2;
    p->hop = desc->hop ? desc->hop : desc->P;
    p->R = desc->P / p->hop;
    if (desc->path == PFB_DFT_FFT_F32) {
        p->family = fft_fast_supported(p->P, p->T)      ? FAM_FFT_FAST
                    : fft_cluster_supported(p->P, p->T) ? FAM_FFT_CLUSTER
                                                        : FAM_FFT_GENERIC;
    } else if (desc->path == PFB_DFT_GEMM_F32) {
        p->family = FAM_GEMM_F32;
    } else {
        p->family = FAM_GEMM_BF16X3;
    }
    const bool padded = p->family == FAM_FFT_FAST || p->family == FAM_FFT_CLUSTER ||
                        (p->family == FAM_GEMM_BF16X3 && p->T <= 16);
    p->TT = padded ? fft_fast_tt(p->T) : p->T;
    p->variant = default_variant(*p);

    const int P = p->P, T = p->T, L = P * T;
    {
        pfb_status est = alloc_error_words(1, &p->h_err, &p->d_err);
        if (est != PFB_OK) return est;
    }
    PFB_CUDA_TRY(cudaMalloc(&p->d_h64, sizeof(double) * L));
    if (desc->window == PFB_WIN_USER) {
        PFB_CUDA_TRY(cudaMemcpy(p->d_h64, desc->user_taps_host, sizeof(double) * L, cudaMemcpyHostToDevice));
    } else {
        gen_prototype_kernel<<<(L + 255) / 256, 256>>>(p->d_h64, P, L, desc->window);
        normalise_kernel<<<1, 1024>>>(p->d_h64, L);
        g_launches += 2;
    }
    PFB_CUDA_TRY(cudaMalloc(&p->d_taps, sizeof(float) * L));
    if (padded) PFB_CUDA_TRY(cudaMalloc(&p->d_taps_pad, sizeof(float) * P * p->TT));
    int nconv = P * (p->TT > T ? p->TT : T);
    taps_to_f32_kernel<<<(nconv + 255) / 256, 256>>>(p->d_h64, P, T, p->TT, desc->tap_order == PFB_TAPS_CONVOLUTION,
                                                     p->d_taps, p->d_taps_pad);
    g_launches++;

    PFB_CUDA_TRY(cudaMalloc(&p->d_tw_r2, sizeof(float2) * (P / 2)));
    gen_tw_r2_kernel<<<(P / 2 + 255) / 256, 256>>>(p->d_tw_r2, P);
    g_launches++;
    if (p->family == FAM_FFT_FAST) {
        pfb_status st = build_fft_fast_twiddles(*p);
        if (st != PFB_OK) return st;
    }
    if (p->family == FAM_FFT_CLUSTER) {  // local 1024-point passes of the four-step FFT
        pfb_status st = build_pass_table(1024, 16, &p->d_tw);
        if (st != PFB_OK) return st;
    }
    if (p->family == FAM_GEMM_F32 || p->family == FAM_GEMM_BF16X3) {
        pfb_status st = build_gemm_tables(*p);
        if (st != PFB_OK) return st;
    }
    PFB_CUDA_TRY(cudaGetLastError());
    PFB_CUDA_TRY(cudaDeviceSynchronize());
    {
        // the static staging area of pfb_execute_host_noalloc is reserved and
        // its address cached now, not inside that entry point's first call
        pfb_status nst = noalloc_prepare(p->device);
        if (nst != PFB_OK) return nst;
    }
    {
        pfb_status pst = prepare_family(*p);
        if (pst != PFB_OK && pst != PFB_ERR_UNSUPPORTED) return pst;
        clear_error();
    }
    static const char *fam_names[] = {"pfb_fir_fft_f32", "pfb_fir_fft_f32_generic", "pfb_fir_dftgemm_f32",
                                      "pfb_fir_dftgemm_bf16x3", "pfb_fir_fft_f32_cluster"};
    p->kernel_name = fam_names[p->family];
    return PFB_OK;
}

}  // namespace pfb

using namespace pfb;

extern "C" pfb_status pfb_plan_create(const pfb_plan_desc *desc, pfb_plan_t *out_plan) {
    clear_error();
    if (!out_plan) return fail(PFB_ERR_INVALID, "out_plan is NULL");
    *out_plan = nullptr;
    pfb_status st = validate(desc);
    if (st != PFB_OK) return st;
    int dev = desc->device;
    int ndev = 0;
    PFB_CUDA_TRY(cudaGetDeviceCount(&ndev));
    int prev = 0;
    PFB_CUDA_TRY(cudaGetDevice(&prev));
    if (dev < 0) dev = prev;
    if (dev >= ndev) return fail(PFB_ERR_INVALID, "device ordinal out of range");
    Plan *p = new (std::nothrow) Plan();
    if (!p) return fail(PFB_ERR_OOM, "host allocation failed");
    p->device = dev;
    cudaSetDevice(dev);
    st = create_impl(desc, p);
    cudaSetDevice(prev);
    if (st != PFB_OK) {
        free_plan(p);
        return st;
    }
    *out_plan = reinterpret_cast<pfb_plan_t>(p);
    return PFB_OK;
}

extern "C" pfb_status pfb_plan_destroy(pfb_plan_t plan) {
    clear_error();
    free_plan(reinterpret_cast<Plan *>(plan));
    return PFB_OK;
}

extern "C" int64_t pfb_out_spectra(pfb_plan_t plan, int64_t n_samples) {
    if (!plan || n_samples < 0) return -1;
    return out_spectra(*reinterpret_cast<Plan *>(plan), n_samples);
}

extern "C" pfb_status pfb_plan_get_taps(pfb_plan_t plan, double *host_out, int64_t cap) {
    clear_error();
    if (!plan || !host_out) return fail(PFB_ERR_INVALID, "NULL argument");
    Plan *p = reinterpret_cast<Plan *>(plan);
    int64_t L = (int64_t)p->P * p->T;
    if (cap < L) return fail(PFB_ERR_INVALID, "cap < P*T");
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(p->device);
    cudaError_t e = cudaMemcpy(host_out, p->d_h64, sizeof(double) * L, cudaMemcpyDeviceToHost);
    cudaSetDevice(prev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy taps");
    return PFB_OK;
}

extern "C" const char *pfb_plan_kernel_name(pfb_plan_t plan) {
    if (!plan) return "";
    return reinterpret_cast<Plan *>(plan)->kernel_name.c_str();
}
