// Two-column fused step (tflbm_step2.cuh) with BF16 moving populations;
// one translation unit per storage type keeps the build parallel.
#include "tflbm_step2.cuh"

namespace tflbm {

cudaError_t pair_step_bf16(int block_x, const void* fin, void* fout, const void* kappa, const Geom& G,
                         const Consts<float>& C, int bands, cudaStream_t st)
{
    return pair_step<__nv_bfloat16>(block_x, fin, fout, kappa, G, C, bands, st);
}

int pair_blocks_per_sm_bf16(int block_x, bool omega1, bool kfield)
{
    return pair_blocks_per_sm<__nv_bfloat16>(block_x, omega1, kfield);
}

cudaError_t pair_step_batch_bf16(const BatchLaunch& L, cudaStream_t st)
{
    return pair_step_batch<__nv_bfloat16>(L, st);
}

}  // namespace tflbm
