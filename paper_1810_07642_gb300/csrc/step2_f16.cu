// Two-column fused step (tflbm_step2.cuh) with FP16 moving populations;
// one translation unit per storage type keeps the build parallel.
#include "tflbm_step2.cuh"

namespace tflbm {

cudaError_t pair_step_f16(int block_x, const void* fin, void* fout, const void* kappa, const Geom& G,
                         const Consts<float>& C, int bands, cudaStream_t st)
{
    return pair_step<__half>(block_x, fin, fout, kappa, G, C, bands, st);
}

int pair_blocks_per_sm_f16(int block_x, bool omega1, bool kfield)
{
    return pair_blocks_per_sm<__half>(block_x, omega1, kfield);
}

cudaError_t pair_step_batch_f16(const BatchLaunch& L, cudaStream_t st)
{
    return pair_step_batch<__half>(L, st);
}

}  // namespace tflbm
