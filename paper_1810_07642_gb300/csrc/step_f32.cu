// FP32 and FP64 instantiations of the one-column fused step (tflbm_step.cuh)
// and the dispatch over storage types and pipelines.
#include "tflbm_step.cuh"

namespace tflbm {

cudaError_t launch_step_narrow(int store, const void* fin, void* fout, const void* kappa,
                               const Geom& G, const Consts<float>& C, const Shape& S,
                               cudaStream_t st);
int blocks_per_sm_narrow(int store, int pipeline, int block_x, bool omega1, bool kfield);
cudaError_t launch_batch_narrow(int store, const BatchLaunch& L, cudaStream_t st);

template <typename SM, typename T>
static cudaError_t launch_typed(const void* fin, void* fout, const void* kappa, const Geom& G,
                                const Consts<T>& C, const Shape& S, cudaStream_t st)
{
    const T* f0 = (const T*)fin;
    const SM* fm = (const SM*)((const char*)fin + G.plane * sizeof(T));
    T* g0 = (T*)fout;
    SM* gm = (SM*)((char*)fout + G.plane * sizeof(T));
    const T* k = (const T*)kappa;
    switch (S.block_x) {
        case 64: return launch_step_bx<SM, T, 64>(S.pipeline, f0, fm, g0, gm, k, G, C, launch_bands(S, G.ny), st);
        case 128: return launch_step_bx<SM, T, 128>(S.pipeline, f0, fm, g0, gm, k, G, C, launch_bands(S, G.ny), st);
        case 256: return launch_step_bx<SM, T, 256>(S.pipeline, f0, fm, g0, gm, k, G, C, launch_bands(S, G.ny), st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_step(int store, const void* fin, void* fout, const void* kappa, const Geom& G,
                        const Consts<float>* C32, const Consts<double>* C64, const Shape& S,
                        cudaStream_t st)
{
    if (S.pipeline == kPipePair) {
        switch (store) {
            case kStoreF32: return pair_step_f32(S.block_x, fin, fout, kappa, G, *C32, launch_bands(S, G.ny), st);
            case kStoreF16: return pair_step_f16(S.block_x, fin, fout, kappa, G, *C32, launch_bands(S, G.ny), st);
            case kStoreBF16: return pair_step_bf16(S.block_x, fin, fout, kappa, G, *C32, launch_bands(S, G.ny), st);
            default: return cudaErrorInvalidValue;
        }
    }
    switch (store) {
        case kStoreF32: return launch_typed<float, float>(fin, fout, kappa, G, *C32, S, st);
        case kStoreF64: return launch_typed<double, double>(fin, fout, kappa, G, *C64, S, st);
        default: return launch_step_narrow(store, fin, fout, kappa, G, *C32, S, st);
    }
}

int step_blocks_per_sm(int store, int pipeline, int block_x, bool omega1, bool kfield)
{
    if (pipeline == kPipePair) {
        switch (store) {
            case kStoreF32: return pair_blocks_per_sm_f32(block_x, omega1, kfield);
            case kStoreF16: return pair_blocks_per_sm_f16(block_x, omega1, kfield);
            case kStoreBF16: return pair_blocks_per_sm_bf16(block_x, omega1, kfield);
            default: return 0;
        }
    }
    if (store == kStoreF32 || store == kStoreF64) {
        const bool f = store == kStoreF32;
        switch (block_x) {
            case 64: return f ? blocks_per_sm_bx<float, float, 64>(pipeline, omega1, kfield)
                              : blocks_per_sm_bx<double, double, 64>(pipeline, omega1, kfield);
            case 128: return f ? blocks_per_sm_bx<float, float, 128>(pipeline, omega1, kfield)
                               : blocks_per_sm_bx<double, double, 128>(pipeline, omega1, kfield);
            case 256: return f ? blocks_per_sm_bx<float, float, 256>(pipeline, omega1, kfield)
                               : blocks_per_sm_bx<double, double, 256>(pipeline, omega1, kfield);
            default: return 0;
        }
    }
    return blocks_per_sm_narrow(store, pipeline, block_x, omega1, kfield);
}

cudaError_t launch_step_batch(int store, const BatchLaunch& L, cudaStream_t st)
{
    if (L.pair) {
        switch (store) {
            case kStoreF32: return pair_step_batch_f32(L, st);
            case kStoreF16: return pair_step_batch_f16(L, st);
            case kStoreBF16: return pair_step_batch_bf16(L, st);
            default: return cudaErrorInvalidValue;
        }
    }
    switch (store) {
        case kStoreF32: return launch_batch_typed<float, float>(L, st);
        case kStoreF64: return launch_batch_typed<double, double>(L, st);
        default: return launch_batch_narrow(store, L, st);
    }
}

}  // namespace tflbm
