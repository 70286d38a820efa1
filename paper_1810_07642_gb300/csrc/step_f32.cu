// FP32 instantiations of the fused step (tflbm_step.cuh).
#include "tflbm_step.cuh"

namespace tflbm {

cudaError_t launch_step_f32(const float* fin, float* fout, const float* kappa, const Geom& G,
                            const Consts<float>& C, const Shape& S, cudaStream_t st)
{
    switch (S.block_x) {
        case 64: return launch_step_bx<float, float, 64>(fin, fout, kappa, G, C, S.rows, st);
        case 128: return launch_step_bx<float, float, 128>(fin, fout, kappa, G, C, S.rows, st);
        case 256: return launch_step_bx<float, float, 256>(fin, fout, kappa, G, C, S.rows, st);
        default: return cudaErrorInvalidValue;
    }
}

int step_blocks_per_sm_f32(int block_x, bool omega1, bool kfield)
{
    switch (block_x) {
        case 64: return blocks_per_sm_bx<float, float, 64>(omega1, kfield);
        case 128: return blocks_per_sm_bx<float, float, 128>(omega1, kfield);
        case 256: return blocks_per_sm_bx<float, float, 256>(omega1, kfield);
        default: return 0;
    }
}

}  // namespace tflbm
