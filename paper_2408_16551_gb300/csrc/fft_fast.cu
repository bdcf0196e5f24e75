// Dispatcher of the fast fused FIR + FFT family (kernels in fft_fast.cuh,
// one translation unit per P).
#include "fft_fast.cuh"

namespace pfb {

template <> pfb_status launch_fft_fast_p<64>(const Plan &, LaunchArgs &, cudaStream_t);
template <> pfb_status launch_fft_fast_p<128>(const Plan &, LaunchArgs &, cudaStream_t);
template <> pfb_status launch_fft_fast_p<256>(const Plan &, LaunchArgs &, cudaStream_t);
template <> pfb_status launch_fft_fast_p<512>(const Plan &, LaunchArgs &, cudaStream_t);
template <> pfb_status launch_fft_fast_p<1024>(const Plan &, LaunchArgs &, cudaStream_t);

bool fft_fast_supported(int P, int T) { return P >= 64 && P <= 1024 && T >= 1 && T <= 16; }
int fft_fast_tt(int T) { return T <= 4 ? 4 : (T <= 8 ? 8 : 16); }

pfb_status launch_fft_fast(const Plan &plan, LaunchArgs &a, cudaStream_t stream) {
    switch (plan.P) {
    case 64: return launch_fft_fast_p<64>(plan, a, stream);
    case 128: return launch_fft_fast_p<128>(plan, a, stream);
    case 256: return launch_fft_fast_p<256>(plan, a, stream);
    case 512: return launch_fft_fast_p<512>(plan, a, stream);
    case 1024: return launch_fft_fast_p<1024>(plan, a, stream);
    default: return fail(PFB_ERR_UNSUPPORTED, "fast FFT family: P outside [64, 1024]");
    }
}

}  // namespace pfb

namespace pfb {
// spectra per work unit of each variant (see launch_fft_fast_v)
int fast_spectra_per_unit(int variant) {
    static const int sb[] = {8, 8, 4, 4, 16, 1};
    return sb[variant];
}
int64_t fast_units(const Plan &plan, int64_t S) {
    const int sb = fast_spectra_per_unit(plan.variant);
    return (S + sb - 1) / sb;
}
}  // namespace pfb
