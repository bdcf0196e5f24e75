// Fused polyphase FIR + DFT-matrix product in FP32 on the SIMT cores.
#include "internal.h"

namespace pfb {
int64_t gemm_f32_units(const Plan &plan, int64_t S) { return 0; }
pfb_status launch_gemm_f32(const Plan &plan, LaunchArgs &a, cudaStream_t stream) {
    return fail(PFB_ERR_UNSUPPORTED, "FP32 DFT-GEMM path not built yet");
}
pfb_status build_gemm_tables(Plan &plan) { return PFB_OK; }
}  // namespace pfb
