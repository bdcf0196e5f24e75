// Instantiation of the fused FIR + FFT kernels for P = 512 (see fft_fast.cuh).
#include "fft_fast.cuh"

namespace pfb {
PFB_DEFINE_FFT_FAST_P(512)
}  // namespace pfb
