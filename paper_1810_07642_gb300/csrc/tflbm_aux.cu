// Auxiliary kernels of the thin-film D2Q9 library: kappa field, initial
// populations, moments, film pressure and force (diagnostic), compensated
// mass, state scan and state import/export.  The stored buffer holds
// post-collision (pre-streaming) populations B_l, so the post-streaming
// populations of the current time are f_l(x) = B_l(x - c_l); plane 0 stores
// B_0 - href (the reference height convention of tflbm_internal.h).
#include <math.h>

#include "tflbm_internal.h"

namespace tflbm {
namespace {

__device__ __constant__ int kCx[9] = {0, 1, 1, 0, -1, -1, -1, 0, 1};
__device__ __constant__ int kCy[9] = {0, 0, 1, 1, 1, 0, -1, -1, -1};

__device__ __forceinline__ int wrapi(int i, int n)
{
    i %= n;
    return i < 0 ? i + n : i;
}

// Post-streaming populations at (x, y), with the rest population restored.
template <typename T>
__device__ __forceinline__ void pull_at(const T* __restrict__ f, const Geom& G, int x, int y,
                                        T href, T (&v)[9])
{
#pragma unroll
    for (int l = 0; l < 9; ++l) {
        const int xs = wrapi(x - kCx[l], G.nx), ys = wrapi(y - kCy[l], G.ny);
        v[l] = f[l * G.plane + (long long)ys * G.pitch + xs];
    }
    v[0] += href;
}

template <typename T>
__device__ __forceinline__ void moments9(const T (&v)[9], T& h, T& jx, T& jy)
{
    h = ((v[0] + v[1]) + (v[2] + v[3])) + ((v[4] + v[5]) + (v[6] + v[7])) + v[8];
    jx = ((v[1] + v[2]) + v[8]) - ((v[4] + v[5]) + v[6]);
    jy = ((v[2] + v[3]) + v[4]) - ((v[6] + v[7]) + v[8]);
}

// kappa(x) = (1 - cos theta)(n-1)(m-1)/((n-m) h_*), Eq. (disjoiningP), in double.
template <typename T>
__global__ void k_kappa(T* kappa, const T* theta, long long n, int ne, int me, double hstar)
{
    const double c = (double)(ne - 1) * (double)(me - 1) / ((double)(ne - me) * hstar);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        kappa[i] = T((1.0 - cos((double)theta[i])) * c);
}

// B_l(x) = f_eq_l(h0(x + c_l), u = 0), so that the pull gives f = f_eq(h0, 0).
template <typename T>
__global__ void k_init(T* f, const T* __restrict__ h0, Geom G, T g, T href)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= G.nx) return;
#pragma unroll
    for (int l = 0; l < 9; ++l) {
        const T h = h0[(long long)wrapi(y + kCy[l], G.ny) * G.nx + wrapi(x + kCx[l], G.nx)];
        const T gh2 = g * h * h;
        T v;
        if (l == 0) v = (h - href) - T(5.0 / 6.0) * gh2;
        else if (l & 1) v = gh2 * T(1.0 / 6.0);
        else v = gh2 * T(1.0 / 24.0);
        f[l * G.plane + (long long)y * G.pitch + x] = v;
    }
}

template <typename T>
__global__ void k_moments(const T* __restrict__ f, T* h, T* ux, T* uy, Geom G, T href)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= G.nx) return;
    T v[9], hh, jx, jy;
    pull_at(f, G, x, y, href, v);
    moments9(v, hh, jx, jy);
    const long long i = (long long)y * G.nx + x;
    if (h) h[i] = hh;
    if (ux) ux[i] = jx / hh;
    if (uy) uy[i] = jy / hh;
}

// Diagnostic film pressure and force, in three plain passes.
template <typename T>
__global__ void k_pf_h(const T* __restrict__ f, T* hbuf, Geom G, Consts<T> C)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= G.nx) return;
    T v[9], hh, jx, jy;
    pull_at(f, G, x, y, C.href, v);
    moments9(v, hh, jx, jy);
    hbuf[(long long)y * G.nx + x] = hh;
}

template <typename T>
__device__ __forceinline__ T ipow_(T r, int n)
{
    T o = T(1);
    for (int i = 0; i < n; ++i) o *= r;
    return o;
}

template <typename T>
__global__ void k_pf_p(const T* __restrict__ hbuf, const T* __restrict__ kappa, T* pbuf, Geom G,
                       Consts<T> C)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= G.nx) return;
    const int xm = wrapi(x - 1, G.nx), xp = wrapi(x + 1, G.nx);
    const int ym = wrapi(y - 1, G.ny), yp = wrapi(y + 1, G.ny);
    auto H = [&](int yy, int xx) { return hbuf[(long long)yy * G.nx + xx]; };
    const T h = H(y, x);
    const T axis = H(y, xm) + H(y, xp) + H(ym, x) + H(yp, x);
    const T diag = H(ym, xm) + H(ym, xp) + H(yp, xm) + H(yp, xp);
    T lap = (T(4) * axis + diag - T(20) * h) / T(6);
    const T kap = kappa ? kappa[(long long)y * G.nx + x] : C.kappa_u;
    const T r = C.hstar / h;
    lap += C.pi_sgn * kap * (ipow_(r, C.n_exp) - ipow_(r, C.m_exp));
    pbuf[(long long)y * G.nx + x] = -C.gamma * lap;
}

template <typename T>
__global__ void k_pf_f(const T* __restrict__ f, const T* __restrict__ pbuf, T* p, T* fx, T* fy,
                       Geom G, Consts<T> C)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= G.nx) return;
    const int xm = wrapi(x - 1, G.nx), xp = wrapi(x + 1, G.nx);
    const int ym = wrapi(y - 1, G.ny), yp = wrapi(y + 1, G.ny);
    auto P = [&](int yy, int xx) { return pbuf[(long long)yy * G.nx + xx]; };
    const T gpx = (P(y, xp) - P(y, xm)) / T(3) + (P(yp, xp) - P(yp, xm) + P(ym, xp) - P(ym, xm)) / T(12);
    const T gpy = (P(yp, x) - P(ym, x)) / T(3) + (P(yp, xp) - P(ym, xp) + P(yp, xm) - P(ym, xm)) / T(12);
    T v[9], hh, jx, jy;
    pull_at(f, G, x, y, C.href, v);
    moments9(v, hh, jx, jy);
    const T fr = C.nu6 / (T(2) * hh * hh + T(6) * C.delta * hh + T(3) * C.delta * C.delta);
    const long long i = (long long)y * G.nx + x;
    if (p) p[i] = P(y, x);
    if (fx) fx[i] = -hh * gpx - fr * jx + hh * C.gx;
    if (fy) fy[i] = -hh * gpy - fr * jy + hh * C.gy;
}

// Neumaier pair (s, c): value s + c.
struct Comp {
    double s, c;
};

__device__ __forceinline__ void comp_add(Comp& a, double v)
{
    const double t = a.s + v;
    if (fabs(a.s) >= fabs(v)) a.c += (a.s - t) + v;
    else a.c += (v - t) + a.s;
    a.s = t;
}

__device__ __forceinline__ void comp_merge(Comp& a, const Comp& b)
{
    comp_add(a, b.s);
    a.c += b.c;
}

__device__ __forceinline__ Comp warp_reduce(Comp a)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        Comp b;
        b.s = __shfl_down_sync(0xffffffffu, a.s, off);
        b.c = __shfl_down_sync(0xffffffffu, a.c, off);
        comp_merge(a, b);
    }
    return a;
}

constexpr int kMassThreads = 256;

// Sum of every stored population (the total liquid volume: streaming only
// permutes populations on the periodic lattice).  One (s, c) pair per block.
template <typename T>
__global__ void __launch_bounds__(kMassThreads) k_mass_partial(const T* __restrict__ f, Geom G,
                                                               double* partials)
{
    Comp a{0.0, 0.0};
    const long long nrows = 9LL * G.ny;
    for (long long row = blockIdx.x; row < nrows; row += gridDim.x) {
        const T* p = f + row * G.pitch;  // plane l, row y: l * plane + y * pitch = row * pitch
        for (int x = threadIdx.x; x < G.nx; x += blockDim.x) comp_add(a, (double)p[x]);
    }
    a = warp_reduce(a);
    __shared__ Comp sm[kMassThreads / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sm[wid] = a;
    __syncthreads();
    if (wid == 0) {
        Comp b = lane < kMassThreads / 32 ? sm[lane] : Comp{0.0, 0.0};
        b = warp_reduce(b);
        if (lane == 0) {
            partials[2 * blockIdx.x] = b.s;
            partials[2 * blockIdx.x + 1] = b.c;
        }
    }
}

// Plain compensated sum of n values (used for the mean initial height).
template <typename T>
__global__ void __launch_bounds__(kMassThreads) k_sum_partial(const T* __restrict__ x, long long n,
                                                              double* partials)
{
    Comp a{0.0, 0.0};
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        comp_add(a, (double)x[i]);
    a = warp_reduce(a);
    __shared__ Comp sm[kMassThreads / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sm[wid] = a;
    __syncthreads();
    if (wid == 0) {
        Comp b = lane < kMassThreads / 32 ? sm[lane] : Comp{0.0, 0.0};
        b = warp_reduce(b);
        if (lane == 0) {
            partials[2 * blockIdx.x] = b.s;
            partials[2 * blockIdx.x + 1] = b.c;
        }
    }
}

__global__ void __launch_bounds__(kMassThreads) k_mass_final(const double* partials, int n, double* out)
{
    Comp a{0.0, 0.0};
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        comp_add(a, partials[2 * i]);
        a.c += partials[2 * i + 1];
    }
    a = warp_reduce(a);
    __shared__ Comp sm[kMassThreads / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sm[wid] = a;
    __syncthreads();
    if (wid == 0) {
        Comp b = lane < kMassThreads / 32 ? sm[lane] : Comp{0.0, 0.0};
        b = warp_reduce(b);
        if (lane == 0) *out = b.s + b.c;
    }
}

template <typename T>
__global__ void k_check(const T* __restrict__ f, Geom G, T href, int* flag)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    int bad = 0;
    if (x < G.nx) {
        T v[9], hh, jx, jy;
        pull_at(f, G, x, y, href, v);
        for (int l = 0; l < 9; ++l)
            if (!isfinite((double)v[l])) bad |= 1;
        moments9(v, hh, jx, jy);
        if (!isfinite((double)hh)) bad |= 1;
        else if (!(hh > T(0))) bad |= 2;
    }
    bad = __reduce_or_sync(0xffffffffu, bad);
    if (bad && (threadIdx.x & 31) == 0) atomicOr(flag, bad);
}

// State export in double: (f_0 - href) + href is exact in double for float
// storage, so an export / import round trip reproduces the stored bits.
template <typename T>
__global__ void k_get_state(const T* __restrict__ f, double* out, Geom G, T href)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= G.nx) return;
    const long long n = (long long)G.nx * G.ny, i = (long long)y * G.nx + x;
#pragma unroll
    for (int l = 0; l < 9; ++l) {
        const int xs = wrapi(x - kCx[l], G.nx), ys = wrapi(y - kCy[l], G.ny);
        const double v = (double)f[l * G.plane + (long long)ys * G.pitch + xs];
        out[l * n + i] = l == 0 ? v + (double)href : v;
    }
}

template <typename T>
__global__ void k_set_state(T* f, const double* __restrict__ in, Geom G, T href)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= G.nx) return;
    const long long n = (long long)G.nx * G.ny;
#pragma unroll
    for (int l = 0; l < 9; ++l) {
        const long long src = (long long)wrapi(y + kCy[l], G.ny) * G.nx + wrapi(x + kCx[l], G.nx);
        const double v = in[l * n + src];
        f[l * G.plane + (long long)y * G.pitch + x] = T(l == 0 ? v - (double)href : v);
    }
}

inline dim3 grid2d(const Geom& G, int bx) { return dim3((G.nx + bx - 1) / bx, G.ny); }

}  // namespace

int mass_blocks(const Geom& G)
{
    long long rows = 9LL * G.ny;
    return (int)(rows < 1184 ? rows : 1184);
}

#define TFLBM_AUX_DEF(T, SUF)                                                                   \
    cudaError_t launch_kappa_##SUF(T* kappa, const T* theta, int nx, int ny, int ne, int me,   \
                                   double hstar, cudaStream_t st)                              \
    {                                                                                           \
        long long n = (long long)nx * ny;                                                       \
        int blocks = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);                    \
        k_kappa<T><<<blocks, 256, 0, st>>>(kappa, theta, n, ne, me, hstar);                     \
        return cudaGetLastError();                                                              \
    }                                                                                           \
    cudaError_t launch_init_##SUF(T* f, const T* h0, const Geom& G, T g, T href,              \
                                  cudaStream_t st)                                             \
    {                                                                                           \
        k_init<T><<<grid2d(G, 128), 128, 0, st>>>(f, h0, G, g, href);                           \
        return cudaGetLastError();                                                              \
    }                                                                                           \
    cudaError_t launch_moments_##SUF(const T* f, T* h, T* ux, T* uy, const Geom& G,             \
                                     T href, cudaStream_t st)                                  \
    {                                                                                           \
        k_moments<T><<<grid2d(G, 128), 128, 0, st>>>(f, h, ux, uy, G, href);                    \
        return cudaGetLastError();                                                              \
    }                                                                                           \
    cudaError_t launch_sum_##SUF(const T* x, long long n, double* partials, int nblocks,        \
                                 double* result, cudaStream_t st)                              \
    {                                                                                           \
        k_sum_partial<T><<<nblocks, kMassThreads, 0, st>>>(x, n, partials);                     \
        k_mass_final<<<1, kMassThreads, 0, st>>>(partials, nblocks, result);                    \
        return cudaGetLastError();                                                              \
    }                                                                                           \
    cudaError_t launch_pressure_force_##SUF(const T* f, const T* kappa, T* p, T* fx, T* fy,     \
                                            T* sh, T* sp, const Geom& G, const Consts<T>& C,    \
                                            cudaStream_t st)                                   \
    {                                                                                           \
        k_pf_h<T><<<grid2d(G, 128), 128, 0, st>>>(f, sh, G, C);                                 \
        k_pf_p<T><<<grid2d(G, 128), 128, 0, st>>>(sh, kappa, sp, G, C);                         \
        k_pf_f<T><<<grid2d(G, 128), 128, 0, st>>>(f, sp, p, fx, fy, G, C);                      \
        return cudaGetLastError();                                                              \
    }                                                                                           \
    cudaError_t launch_mass_##SUF(const T* f, const Geom& G, double* partials, int nblocks,     \
                                  double* result, cudaStream_t st)                             \
    {                                                                                           \
        k_mass_partial<T><<<nblocks, kMassThreads, 0, st>>>(f, G, partials);                    \
        k_mass_final<<<1, kMassThreads, 0, st>>>(partials, nblocks, result);                    \
        return cudaGetLastError();                                                              \
    }                                                                                           \
    cudaError_t launch_check_##SUF(const T* f, const Geom& G, T href, int* flag,               \
                                   cudaStream_t st)                                            \
    {                                                                                           \
        k_check<T><<<grid2d(G, 128), 128, 0, st>>>(f, G, href, flag);                           \
        return cudaGetLastError();                                                              \
    }                                                                                           \
    cudaError_t launch_get_state_##SUF(const T* f, double* out, const Geom& G, T href,         \
                                       cudaStream_t st)                                        \
    {                                                                                           \
        k_get_state<T><<<grid2d(G, 128), 128, 0, st>>>(f, out, G, href);                        \
        return cudaGetLastError();                                                              \
    }                                                                                           \
    cudaError_t launch_set_state_##SUF(T* f, const double* in, const Geom& G, T href,          \
                                       cudaStream_t st)                                        \
    {                                                                                           \
        k_set_state<T><<<grid2d(G, 128), 128, 0, st>>>(f, in, G, href);                         \
        return cudaGetLastError();                                                              \
    }

TFLBM_AUX_DEF(float, f32)
TFLBM_AUX_DEF(double, f64)

}  // namespace tflbm
