// Autotuner: picks the kernel variant (tile shape) of a plan's family by
// timing every candidate on the device, and caches the winner per
// (GPU name, P, T, dtype, family) -- in process, and in a JSON file when the
// environment variable PFB_AUTOTUNE_CACHE names one.  Plans created later
// for the same shape start from the cached choice.
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <map>
#include <sstream>

#include "internal.h"

namespace pfb {

int fast_spectra_per_unit(int variant);

static std::mutex g_tune_mu;
static std::map<std::string, int> g_tune_cache;
static bool g_tune_loaded = false;

static std::string gpu_name(int dev) {
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return "unknown";
    std::string n(prop.name);
    for (auto &c : n)
        if (c == '"' || c == '|') c = '_';
    return n;
}

static std::string key_of(const Plan &p) {
    std::ostringstream k;
    k << gpu_name(p.device) << "|P" << p.P << "|T" << p.T << "|d" << p.in_dtype << "|f" << p.family;
    return k.str();
}

// minimal reader/writer for a flat JSON object {"key": int, ...}
static void load_file_cache() {
    if (g_tune_loaded) return;
    g_tune_loaded = true;
    const char *path = std::getenv("PFB_AUTOTUNE_CACHE");
    if (!path) return;
    std::ifstream f(path);
    if (!f) return;
    std::stringstream ss;
    ss << f.rdbuf();
    const std::string s = ss.str();
    size_t i = 0;
    while (true) {
        size_t a = s.find('"', i);
        if (a == std::string::npos) break;
        size_t b = s.find('"', a + 1);
        if (b == std::string::npos) break;
        size_t c = s.find(':', b);
        if (c == std::string::npos) break;
        g_tune_cache[s.substr(a + 1, b - a - 1)] = std::atoi(s.c_str() + c + 1);
        i = s.find_first_of(",}", c);
        if (i == std::string::npos) break;
    }
}

static void save_file_cache() {
    const char *path = std::getenv("PFB_AUTOTUNE_CACHE");
    if (!path) return;
    std::ofstream f(std::string(path) + ".tmp");
    f << "{";
    bool first = true;
    for (auto &kv : g_tune_cache) {
        f << (first ? "\n  " : ",\n  ") << '"' << kv.first << "\": " << kv.second;
        first = false;
    }
    f << "\n}\n";
    f.close();
    std::rename((std::string(path) + ".tmp").c_str(), path);
}

// fast FFT family: 6 tile shapes; split-bf16 family: 0 = dense DFT-matrix
// product, 1 = factored (four-step) tensor-core DFT, 2 = dense product in two
// passes (FIR to a pre-tiled workspace, then a pipelined tcgen05 GEMM); cluster FFT family:
// 0 = synchronous, 1 = warp-specialised with the cross-CTA step in the FFT
// warps, 2 = warp-specialised with one exchange from the FIR warps' radix-4
// step to the receiving FFT warps, 3 = four-step 64 x 64 (P = 4096)
int family_variants(const Plan &plan) {
    if (plan.family == FAM_FFT_FAST) return 6;
    if (plan.family == FAM_GEMM_BF16X3) return 3;
    if (plan.family == FAM_FFT_CLUSTER) return 4;
    return 1;
}

// variant 5 of the fast FFT family needs P >= 128 and T equal to its tap count;
// the factored split-bf16 DFT needs P = 1024 and T equal to its tap count
static bool variant_supported(const Plan &plan, int v) {
    if (plan.family == FAM_FFT_FAST && v == 5) return plan.P >= 128 && plan.T == plan.TT;
    if (plan.family == FAM_GEMM_BF16X3 && v == 1) return tcf_supported(plan);
    if (plan.family == FAM_GEMM_BF16X3 && v == 2) return gemm2p_supported(plan);
    if (plan.family == FAM_FFT_CLUSTER && v == 3) return wcf_supported(plan);
    if (plan.family == FAM_FFT_CLUSTER && v >= 1) return v < 3 && ws_cluster_supported(plan);
    return v >= 0 && v < family_variants(plan);
}

int default_variant(const Plan &plan) {
    if (family_variants(plan) <= 1) return 0;
    if (plan.family == FAM_GEMM_BF16X3) return tcf_supported(plan) ? 1 : gemm2p_supported(plan) ? 2 : 0;
    if (plan.family == FAM_FFT_CLUSTER) return wcf_supported(plan) ? 3 : ws_cluster_supported(plan) ? 2 : 0;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    load_file_cache();
    auto it = g_tune_cache.find(key_of(plan));
    if (it != g_tune_cache.end() && it->second >= 0 && it->second < family_variants(plan)) return it->second;
    if (const char *v = std::getenv("PFB_FFT_VARIANT")) {
        int x = std::atoi(v);
        if (x >= 0 && x < family_variants(plan)) return x;
    }
    // built-in choice (fastest in a GB300 sweep over P = 64..1024, T = 16):
    // 2 branches per thread, 8 spectra per unit, radix 16, scalar fp32
    return 0;
}

}  // namespace pfb

using namespace pfb;

extern "C" int32_t pfb_plan_variant(pfb_plan_t plan) {
    return plan ? reinterpret_cast<Plan *>(plan)->variant : -1;
}

extern "C" int32_t pfb_plan_num_variants(pfb_plan_t plan) {
    return plan ? family_variants(*reinterpret_cast<Plan *>(plan)) : -1;
}

extern "C" pfb_status pfb_plan_set_variant(pfb_plan_t plan, int32_t variant) {
    clear_error();
    if (!plan) return fail(PFB_ERR_INVALID, "plan is NULL");
    Plan &p = *reinterpret_cast<Plan *>(plan);
    if (variant < 0 || variant >= family_variants(p)) return fail(PFB_ERR_INVALID, "variant out of range");
    if (!variant_supported(p, variant)) return fail(PFB_ERR_UNSUPPORTED, "variant not available for this P/T");
    p.variant = variant;
    pfb_status st = ensure_variant_tables(p);
    if (st != PFB_OK) return st;
    return prepare_family(p);
}

extern "C" pfb_status pfb_plan_autotune(pfb_plan_t plan, int64_t n_samples, void *cuda_stream, double *out_best_ms) {
    clear_error();
    if (!plan) return fail(PFB_ERR_INVALID, "plan is NULL");
    Plan &p = *reinterpret_cast<Plan *>(plan);
    const int nv = family_variants(p);
    const int64_t S = out_spectra(p, n_samples);
    if (S <= 0) return fail(PFB_ERR_INVALID, "n_samples gives no spectra");
    int prev_dev = 0;
    cudaGetDevice(&prev_dev);
    cudaSetDevice(p.device);
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    void *din = nullptr, *dout = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    pfb_status st = PFB_OK;
    const size_t in_bytes = (size_t)n_samples * p.esize, out_bytes = (size_t)S * p.P * sizeof(float2);
    if (cudaMalloc(&din, in_bytes) != cudaSuccess || cudaMalloc(&dout, out_bytes) != cudaSuccess) {
        st = fail(PFB_ERR_OOM, "autotune buffers");
    }
    if (st == PFB_OK && (cudaMemsetAsync(din, 0x3c, in_bytes, s) != cudaSuccess ||
                         cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess))
        st = fail(PFB_ERR_CUDA, "autotune setup");
    int best = p.variant;
    float best_ms = 1e30f;
    const int saved = p.variant;
    for (int v = 0; st == PFB_OK && v < nv; ++v) {
        if (!variant_supported(p, v)) continue;
        p.variant = v;
        st = ensure_variant_tables(p);
        if (st == PFB_OK) st = prepare_family(p);
        if (st != PFB_OK) break;
        for (int w = 0; w < 2 && st == PFB_OK; ++w) st = pfb_execute(plan, din, n_samples, dout, S, s);
        if (st != PFB_OK) break;
        cudaEventRecord(e0, s);
        const int reps = 5;
        for (int r = 0; r < reps && st == PFB_OK; ++r) st = pfb_execute(plan, din, n_samples, dout, S, s);
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess) st = fail(PFB_ERR_CUDA, "autotune sync");
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        ms /= reps;
        if (st == PFB_OK && ms < best_ms) {
            best_ms = ms;
            best = v;
        }
    }
    p.variant = (st == PFB_OK) ? best : saved;
    if (st == PFB_OK) {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        load_file_cache();
        g_tune_cache[key_of(p)] = best;
        save_file_cache();
        if (out_best_ms) *out_best_ms = best_ms;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(din);
    cudaFree(dout);
    cudaSetDevice(prev_dev);
    return st;
}
