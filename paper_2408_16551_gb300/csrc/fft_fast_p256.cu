// Instantiation of the fused FIR + FFT kernels for P = 256 (see fft_fast.cuh).
#include "fft_fast.cuh"

namespace pfb {
PFB_DEFINE_FFT_FAST_P(256)
}  // namespace pfb
