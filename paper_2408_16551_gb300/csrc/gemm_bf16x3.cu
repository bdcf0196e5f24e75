// Fused polyphase FIR + DFT-matrix product on the tensor cores (split bf16).
#include "internal.h"

namespace pfb {
int64_t gemm_bf16x3_units(const Plan &plan, int64_t S) { return 0; }
pfb_status launch_gemm_bf16x3(const Plan &plan, LaunchArgs &a, cudaStream_t stream) {
    return fail(PFB_ERR_UNSUPPORTED, "split-bf16 DFT-GEMM path not built yet");
}
}  // namespace pfb
