// Internal launch interface between the C-ABI layer (tflbm_api.cu) and the
// kernel translation units.  Not part of the public ABI.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace tflbm {

// Geometry of the population buffers: 9 planes of ny rows of `pitch`
// elements; only the first nx columns of a row are lattice nodes.
struct Geom {
    int nx, ny, pitch;
    long long plane;  // ny * pitch
};

// Per-run constants of the step, in the compute type T.
template <typename T>
struct Consts {
    T gamma;      // surface tension
    T g;          // gravity in the equilibria
    T delta;      // slip length
    T hstar;      // precursor thickness
    T nu6;        // 6 nu, nu = (tau - 1/2) / 3
    T omega;      // 1 / tau
    T gx, gy;     // tangential body acceleration
    T kappa_u;    // uniform kappa (used when no kappa field)
    T pi_sgn;     // +1 or -1
    T href;       // reference height: the rest population is stored as f_0 - href
    int n_exp, m_exp;
};

// Launch shape of the fused step.
struct Shape {
    int block_x;  // 32, 64, 128, 256
    int rows;     // rows per CTA
};

// fin: post-collision populations of step t (pre-streaming);
// fout: post-collision populations of step t + 1.  kappa: [ny][nx] or null.
cudaError_t launch_step_f32(const float* fin, float* fout, const float* kappa,
                            const Geom& G, const Consts<float>& C, const Shape& S,
                            cudaStream_t st);
cudaError_t launch_step_f64(const double* fin, double* fout, const double* kappa,
                            const Geom& G, const Consts<double>& C, const Shape& S,
                            cudaStream_t st);

// Storage convention: plane 0 holds f_0 - href, planes 1..8 hold f_l.  In
// this model the rest population carries almost all of h (f_0 ~ h, the moving
// populations are O(g h^2, h u)), so storing its deviation from a per-run
// reference height keeps rounding errors proportional to the perturbation
// rather than to h and removes the systematic mass drift of near-flat films.

// Resident CTAs per SM of the step kernel for a launch shape (0 if unknown).
int step_blocks_per_sm_f32(int block_x, bool omega1, bool kfield);
int step_blocks_per_sm_f64(int block_x, bool omega1, bool kfield);

// Auxiliary kernels, one set per storage type.
#define TFLBM_AUX_DECL(T, SUF)                                                             \
    cudaError_t launch_kappa_##SUF(T* kappa, const T* theta, int nx, int ny,               \
                                   int n_exp, int m_exp, double hstar, cudaStream_t st);   \
    cudaError_t launch_init_##SUF(T* f, const T* h0, const Geom& G, T g, T href,           \
                                  cudaStream_t st);                                      \
    cudaError_t launch_moments_##SUF(const T* f, T* h, T* ux, T* uy, const Geom& G,        \
                                     T href, cudaStream_t st);                            \
    cudaError_t launch_sum_##SUF(const T* x, long long n, double* partials, int nblocks,   \
                                 double* result, cudaStream_t st);                        \
    cudaError_t launch_pressure_force_##SUF(const T* f, const T* kappa, T* p, T* fx,       \
                                            T* fy, T* scratch_h, T* scratch_p,            \
                                            const Geom& G, const Consts<T>& C,            \
                                            cudaStream_t st);                             \
    cudaError_t launch_mass_##SUF(const T* f, const Geom& G, double* partials,             \
                                  int nblocks, double* result, cudaStream_t st);           \
    cudaError_t launch_check_##SUF(const T* f, const Geom& G, T href, int* flag,           \
                                   cudaStream_t st);                                      \
    cudaError_t launch_get_state_##SUF(const T* f, double* out, const Geom& G, T href,     \
                                       cudaStream_t st);                                  \
    cudaError_t launch_set_state_##SUF(T* f, const double* in, const Geom& G, T href,      \
                                       cudaStream_t st);

TFLBM_AUX_DECL(float, f32)
TFLBM_AUX_DECL(double, f64)
#undef TFLBM_AUX_DECL

// Number of partial sums the mass reduction writes (its grid size), and the
// number the plain field sum writes.
int mass_blocks(const Geom& G);
constexpr int kSumBlocks = 1184;

}  // namespace tflbm
