// Instantiations of the one-column fused step (tflbm_step.cuh) with the 8
// moving populations stored in FP16 or BF16 and all arithmetic in FP32.
#include "tflbm_step.cuh"

namespace tflbm {

template <typename SM>
static cudaError_t launch_n(const void* fin, void* fout, const void* kappa, const Geom& G,
                            const Consts<float>& C, const Shape& S, cudaStream_t st)
{
    const float* f0 = (const float*)fin;
    const SM* fm = (const SM*)((const char*)fin + G.plane * sizeof(float));
    float* g0 = (float*)fout;
    SM* gm = (SM*)((char*)fout + G.plane * sizeof(float));
    const float* k = (const float*)kappa;
    switch (S.block_x) {
        case 64: return launch_step_bx<SM, float, 64>(S.pipeline, f0, fm, g0, gm, k, G, C, launch_bands(S, G.ny), st);
        case 128: return launch_step_bx<SM, float, 128>(S.pipeline, f0, fm, g0, gm, k, G, C, launch_bands(S, G.ny), st);
        case 256: return launch_step_bx<SM, float, 256>(S.pipeline, f0, fm, g0, gm, k, G, C, launch_bands(S, G.ny), st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_step_narrow(int store, const void* fin, void* fout, const void* kappa,
                               const Geom& G, const Consts<float>& C, const Shape& S,
                               cudaStream_t st)
{
    if (store == kStoreF16) return launch_n<__half>(fin, fout, kappa, G, C, S, st);
    if (store == kStoreBF16) return launch_n<__nv_bfloat16>(fin, fout, kappa, G, C, S, st);
    return cudaErrorInvalidValue;
}

template <typename SM>
static int bps(int pipeline, int block_x, bool omega1, bool kfield)
{
    switch (block_x) {
        case 64: return blocks_per_sm_bx<SM, float, 64>(pipeline, omega1, kfield);
        case 128: return blocks_per_sm_bx<SM, float, 128>(pipeline, omega1, kfield);
        case 256: return blocks_per_sm_bx<SM, float, 256>(pipeline, omega1, kfield);
        default: return 0;
    }
}

int blocks_per_sm_narrow(int store, int pipeline, int block_x, bool omega1, bool kfield)
{
    if (store == kStoreF16) return bps<__half>(pipeline, block_x, omega1, kfield);
    if (store == kStoreBF16) return bps<__nv_bfloat16>(pipeline, block_x, omega1, kfield);
    return 0;
}

cudaError_t launch_batch_narrow(int store, const BatchLaunch& L, cudaStream_t st)
{
    if (store == kStoreF16) return launch_batch_typed<__half, float>(L, st);
    if (store == kStoreBF16) return launch_batch_typed<__nv_bfloat16, float>(L, st);
    return cudaErrorInvalidValue;
}

}  // namespace tflbm
