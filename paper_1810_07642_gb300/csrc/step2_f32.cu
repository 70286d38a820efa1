// Two-column fused step (tflbm_step2.cuh) with FP32 moving populations;
// one translation unit per storage type keeps the build parallel.
#include "tflbm_step2.cuh"

namespace tflbm {

cudaError_t pair_step_f32(int block_x, const void* fin, void* fout, const void* kappa, const Geom& G,
                         const Consts<float>& C, int bands, cudaStream_t st)
{
    return pair_step<float>(block_x, fin, fout, kappa, G, C, bands, st);
}

int pair_blocks_per_sm_f32(int block_x, bool omega1, bool kfield)
{
    return pair_blocks_per_sm<float>(block_x, omega1, kfield);
}

cudaError_t pair_step_batch_f32(const BatchLaunch& L, cudaStream_t st)
{
    return pair_step_batch<float>(L, st);
}

}  // namespace tflbm
