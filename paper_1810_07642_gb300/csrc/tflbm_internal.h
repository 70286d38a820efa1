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

// Step kernel variants: TMA bulk-copy pipeline (needs nx % 8 == 0, nx >= 16),
// or per-thread global loads (any size).
constexpr int kPipeTma = 0;
constexpr int kPipeLdg = 1;
constexpr int kPipeAsync = 2;  // per-thread cp.async staging (full-width storage only)
constexpr int kPipePair = 3;   // two columns per thread (FP32 compute type, nx even)
inline bool tma_pipeline_ok(int nx) { return nx % 8 == 0 && nx >= 16; }
inline bool pair_pipeline_ok(int nx, int store) { return nx % 2 == 0 && store != 1 /* kStoreF64 */; }

// Status bit a kernel sets when an mbarrier wait gave up (tf_lbm_check).
constexpr int kStatusTimeout = 4;
// Polls of one mbarrier before a bulk-copy kernel gives up (the default of
// Consts::wait_limit).
constexpr int kWaitLimit = 1 << 22;
// Status bit of the bounds-checked debug build (TFLBM_CHECK_BOUNDS): a step
// kernel computed an index outside the buffer it was meant for.
constexpr int kStatusBounds = 8;

// Index checks of the step kernels.  In a build with TFLBM_CHECK_BOUNDS
// defined, TFLBM_IDX(i, n, st) compares i with [0, n): outside it sets
// kStatusBounds in the status word st and yields 0 instead, so the access
// stays inside the buffer and nothing traps; TFLBM_CHECK(cond, st) sets the
// bit when cond is false.  In the normal build both compile to nothing.
#if defined(TFLBM_CHECK_BOUNDS) && defined(__CUDACC__)
__device__ __forceinline__ long long checked_index(long long i, long long n, int* status)
{
    if (i >= 0 && i < n) return i;
    if (status) atomicOr(status, kStatusBounds);
    return 0;
}
#define TFLBM_IDX(i, n, st) ((decltype(i))::tflbm::checked_index((long long)(i), (long long)(n), (st)))
#define TFLBM_CHECK(cond, st)                                  \
    do {                                                      \
        if (!(cond) && (st)) atomicOr((st), ::tflbm::kStatusBounds); \
    } while (0)
#else
#define TFLBM_IDX(i, n, st) (i)
#define TFLBM_CHECK(cond, st) \
    do {                      \
    } while (0)
#endif

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
    // 16-bit storage of the moving populations: q = (f_l - R_l) * mscale,
    // R_l = f_eq_l(href, 0) = r_axis (odd l) or r_diag (even l); minv = 1/mscale
    T mscale, minv, r_axis, r_diag;
    T nr_axis, nr_diag;  // -r_axis * mscale, -r_diag * mscale (exact: mscale is a power of 2)
    T r_sum;             // sum over the eight moving directions of R_l = 4 (r_axis + r_diag)
    int n_exp, m_exp;
    int* status;     // device word for kStatusTimeout (may be null)
    int wait_limit;  // polls of one mbarrier before giving up (<= 0: give up at once)
    int forcing;     // 0: Eq. (LBE) as printed; 1: second-order forcing
    int flip;        // 0 / 1, alternating from step to step: reverses every band's march
};

// Launch shape of the fused step.
struct Shape {
    int block_x;    // 64, 128, 256
    int rows;       // rows per CTA (band height)
    int pipeline;   // kPipeTma, kPipeLdg, kPipeAsync or kPipePair
    int bands = 0;  // balanced bands per launch; 0: ny / rows rounded up
};

// Bands of one launch of a step kernel for a shape (at most 65535, the grid's
// y limit; the kernels balance rows over the bands they are given).
inline int launch_bands(const Shape& S, int ny)
{
    long long b = S.bands > 0 ? S.bands : ((long long)ny + S.rows - 1) / S.rows;
    if (b > 65535) b = 65535;
    if (b < 1) b = 1;
    return (int)b;
}

// Storage of the 8 moving populations.
enum Store { kStoreF32 = 0, kStoreF64 = 1, kStoreF16 = 2, kStoreBF16 = 3 };

// fin: post-collision populations of step t (pre-streaming); fout: those of
// step t + 1.  A population buffer holds plane 0 (f_0 - href, compute type)
// followed by the 8 moving planes in the storage type, each `plane` elements.
// kappa: [ny][nx] or null.
cudaError_t launch_step(int store, const void* fin, void* fout, const void* kappa, const Geom& G,
                        const Consts<float>* C32, const Consts<double>* C64, const Shape& S,
                        cudaStream_t st);
// Resident CTAs per SM of the step kernel for a launch shape (0 if unknown).
int step_blocks_per_sm(int store, int pipeline, int block_x, bool omega1, bool kfield);
// The two-column step (pipeline kPipePair) per storage type (step2_*.cu),
// and its resident CTAs per SM.
cudaError_t pair_step_f32(int block_x, const void* fin, void* fout, const void* kappa, const Geom& G,
                          const Consts<float>& C, int bands, cudaStream_t st);
cudaError_t pair_step_f16(int block_x, const void* fin, void* fout, const void* kappa, const Geom& G,
                          const Consts<float>& C, int bands, cudaStream_t st);
cudaError_t pair_step_bf16(int block_x, const void* fin, void* fout, const void* kappa, const Geom& G,
                           const Consts<float>& C, int bands, cudaStream_t st);
int pair_blocks_per_sm_f32(int block_x, bool omega1, bool kfield);
int pair_blocks_per_sm_f16(int block_x, bool omega1, bool kfield);
int pair_blocks_per_sm_bf16(int block_x, bool omega1, bool kfield);

// One work item of the batched step: a band of a strip of one domain.
struct BatchItem {
    int dom, strip, band, nbands;
};
// One domain of a batch, as the batched step kernel reads it.
template <typename T>
struct BatchDomain {
    Geom G;
    Consts<T> C;
    void* buf[2];
    const T* kappa;  // [ny][nx] or null
};
// One batched step: `grid` CTAs of block_x threads over `nitems` items
// (grid == nitems without a queue).  doms points at BatchDomain<compute
// type>[count] in device memory; queue (2 ints, zero between launches) or
// null.  With query_occupancy set nothing is launched: the resident CTAs per
// SM of the selected kernel are written there instead.
struct BatchLaunch {
    int block_x;
    bool pair;  // the two-column kernel (nx even in every domain, FP32 compute type)
    bool omega1, kfield;
    const BatchItem* items;
    int nitems;
    const void* doms;
    int parity;
    int* queue;
    int grid;
    int* query_occupancy;
};
cudaError_t launch_step_batch(int store, const BatchLaunch& L, cudaStream_t st);
// The batched two-column step per storage type (step2_*.cu).
cudaError_t pair_step_batch_f32(const BatchLaunch& L, cudaStream_t st);
cudaError_t pair_step_batch_f16(const BatchLaunch& L, cudaStream_t st);
cudaError_t pair_step_batch_bf16(const BatchLaunch& L, cudaStream_t st);

// Storage convention: plane 0 holds f_0 - href, planes 1..8 hold f_l (or its
// 16-bit encoding, see Consts).  In
// this model the rest population carries almost all of h (f_0 ~ h, the moving
// populations are O(g h^2, h u)), so storing its deviation from a per-run
// reference height keeps rounding errors proportional to the perturbation
// rather than to h and removes the systematic mass drift of near-flat films.

// Storage of one handle, as the auxiliary kernels need it (values in double;
// each kernel casts them to its compute type).
struct StoreDesc {
    int store;
    double href, mscale, minv, r_axis, r_diag;
};

// Auxiliary kernels, dispatched over the storage type.  Field buffers (h0,
// theta, kappa, moments, p, F, scratch) are in the compute type: double for
// kStoreF64, float otherwise.
cudaError_t aux_init(const StoreDesc& D, void* f, const void* h0, const Geom& G, double g, cudaStream_t st);
cudaError_t aux_moments(const StoreDesc& D, const void* f, void* h, void* ux, void* uy, const Geom& G,
                        cudaStream_t st);
cudaError_t aux_pressure_force(const StoreDesc& D, const void* f, const void* kappa, void* p, void* fx,
                               void* fy, void* sh, void* sp, const Geom& G, const Consts<float>* C32,
                               const Consts<double>* C64, cudaStream_t st);
cudaError_t aux_mass(const StoreDesc& D, const void* f, const Geom& G, double* partials, int nblocks,
                     double* result, cudaStream_t st);
cudaError_t aux_check(const StoreDesc& D, const void* f, const Geom& G, int* flag, cudaStream_t st);
cudaError_t aux_get_state(const StoreDesc& D, const void* f, double* out, const Geom& G, cudaStream_t st);
cudaError_t aux_set_state(const StoreDesc& D, void* f, const double* in, const Geom& G, cudaStream_t st);
// post-streaming populations in the compute type, [9][ny][nx]
// Film diagnostics of each domain of a BatchDomain table (buffer `parity`):
// out[d * kDiagOut ..] = the fields of tf_lbm_diag (wetted nodes: h > h_wet;
// Fourier sums at the integer modes (mx, my)).  partials holds
// diag_partials(ndom, nb) doubles.
constexpr int kDiagSums = 11;
constexpr int kDiagOut = kDiagSums + 1;
inline size_t diag_partials(int ndom, int nb) { return (size_t)ndom * nb * (2 * kDiagSums + 1); }
cudaError_t aux_diag(int store, const void* doms, int ndom, int parity, double h_wet, int mx, int my,
                     double* partials, int nb, double* out, cudaStream_t st);
// L2 norms (appendix, Eq. magnitude) of the x-components of the pressure,
// friction and dissipation terms into out[0..2]; scratch holds 5 fields of
// the compute type, partials 6 * nb doubles.
cudaError_t aux_term_norms(const StoreDesc& D, const void* f, const void* kappa, const Geom& G,
                           const Consts<float>* C32, const Consts<double>* C64, void* scratch, double* partials,
                           int nb, double* out, cudaStream_t st);
cudaError_t aux_export_state(const StoreDesc& D, const void* f, void* out, const Geom& G, cudaStream_t st);
cudaError_t aux_kappa(bool dbl, void* kappa, const void* theta, int nx, int ny, int ne, int me,
                      double hstar, cudaStream_t st);
// smallest of n values of the compute type into *result (double)
cudaError_t aux_min(bool dbl, const void* x, long long n, double* partials, int nblocks, double* result,
                    cudaStream_t st);


// Number of partial sums the mass reduction writes (its grid size), and the
// number the plain field sum writes.
int mass_blocks(const Geom& G);
constexpr int kSumBlocks = 1184;

}  // namespace tflbm
