// FP64 instantiations of the fused step (tflbm_step.cuh).
#include "tflbm_step.cuh"

namespace tflbm {

cudaError_t launch_step_f64(const double* fin, double* fout, const double* kappa, const Geom& G,
                            const Consts<double>& C, const Shape& S, cudaStream_t st)
{
    switch (S.block_x) {
        case 64: return launch_step_bx<double, double, 64>(fin, fout, kappa, G, C, S.rows, st);
        case 128: return launch_step_bx<double, double, 128>(fin, fout, kappa, G, C, S.rows, st);
        default: return cudaErrorInvalidValue;
    }
}

int step_blocks_per_sm_f64(int block_x, bool omega1, bool kfield)
{
    switch (block_x) {
        case 64: return blocks_per_sm_bx<double, double, 64>(omega1, kfield);
        case 128: return blocks_per_sm_bx<double, double, 128>(omega1, kfield);
        default: return 0;
    }
}

}  // namespace tflbm
