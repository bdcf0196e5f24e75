// Instantiation of the fused FIR + FFT kernels for P = 1024 (see fft_fast.cuh).
#include "fft_fast.cuh"

namespace pfb {
PFB_DEFINE_FFT_FAST_P(1024)
}  // namespace pfb
