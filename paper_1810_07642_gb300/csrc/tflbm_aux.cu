// Auxiliary kernels of the thin-film D2Q9 library: kappa field, initial
// populations, moments, film pressure and force (diagnostic), compensated
// mass, state scan and state import/export.
//
// The stored buffer holds post-collision (pre-streaming) populations B_l, so
// the post-streaming populations of the current time are f_l(x) = B_l(x - c_l).
// Plane 0 stores B_0 - href in the compute type; the 8 moving planes follow in
// the storage type (the compute type, or a 16-bit encoding, see Consts in
// tflbm_internal.h).  All kernels here go through the Pops accessor below.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <math.h>

#include <type_traits>

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

__device__ __forceinline__ float cvt(float q) { return q; }
__device__ __forceinline__ double cvt(double q) { return q; }
__device__ __forceinline__ float cvt(__half q) { return __half2float(q); }
__device__ __forceinline__ float cvt(__nv_bfloat16 q) { return __bfloat162float(q); }
template <typename SM> __device__ __forceinline__ SM enc(float v);
template <> __device__ __forceinline__ __half enc<__half>(float v) { return __float2half_rn(v); }
template <> __device__ __forceinline__ __nv_bfloat16 enc<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }

// Read / write access to one population buffer.
template <typename T, typename SM>
struct Pops {
    T* f0;       // plane 0: f_0 - href
    SM* fm;      // moving planes 1..8
    long long plane;
    int pitch;
    T href, mscale, minv, r_axis, r_diag;

    __device__ __forceinline__ long long at(int y, int x) const { return (long long)y * pitch + x; }
    // the stored value of plane l at element i, decoded (plane 0: f_0 - href)
    __device__ __forceinline__ T raw(int l, long long i) const
    {
        if (l == 0) return f0[i];
        const SM q = fm[(l - 1) * plane + i];
        if constexpr (std::is_same<SM, T>::value) return q;
        else return fmaf(cvt(q), minv, (l & 1) ? r_axis : r_diag);
    }
    __device__ __forceinline__ T full(int l, long long i) const { return l == 0 ? raw(0, i) + href : raw(l, i); }
    // store the population value v (plane 0: v is f_0 - href)
    __device__ __forceinline__ void put(int l, long long i, T v) const
    {
        if (l == 0) f0[i] = v;
        else if constexpr (std::is_same<SM, T>::value) fm[(l - 1) * plane + i] = v;
        else fm[(l - 1) * plane + i] = enc<SM>((v - ((l & 1) ? r_axis : r_diag)) * mscale);
    }
};

template <typename T, typename SM>
Pops<T, SM> make_pops(const void* buf, const Geom& G, const StoreDesc& D)
{
    Pops<T, SM> P;
    P.f0 = (T*)buf;
    P.fm = (SM*)((char*)buf + G.plane * sizeof(T));
    P.plane = G.plane;
    P.pitch = G.pitch;
    P.href = T(D.href);
    P.mscale = T(D.mscale);
    P.minv = T(D.minv);
    P.r_axis = T(D.r_axis);
    P.r_diag = T(D.r_diag);
    return P;
}

// Post-streaming populations at (x, y).
template <typename T, typename SM>
__device__ __forceinline__ void pull_at(const Pops<T, SM>& P, const Geom& G, int x, int y, T (&v)[9])
{
#pragma unroll
    for (int l = 0; l < 9; ++l)
        v[l] = P.full(l, P.at(wrapi(y - kCy[l], G.ny), wrapi(x - kCx[l], G.nx)));
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
template <typename T, typename SM>
__global__ void k_init(Pops<T, SM> P, const T* __restrict__ h0, Geom G, T g)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= G.nx) return;
#pragma unroll
    for (int l = 0; l < 9; ++l) {
        const T h = h0[(long long)wrapi(y + kCy[l], G.ny) * G.nx + wrapi(x + kCx[l], G.nx)];
        const T gh2 = g * h * h;
        T v;
        if (l == 0) v = (h - P.href) - T(5.0 / 6.0) * gh2;
        else if (l & 1) v = gh2 * T(1.0 / 6.0);
        else v = gh2 * T(1.0 / 24.0);
        P.put(l, P.at(y, x), v);
    }
}

template <typename T, typename SM>
__global__ void k_moments(Pops<T, SM> P, T* h, T* ux, T* uy, Geom G)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= G.nx) return;
    T v[9], hh, jx, jy;
    pull_at(P, G, x, y, v);
    moments9(v, hh, jx, jy);
    const long long i = (long long)y * G.nx + x;
    if (h) h[i] = hh;
    if (ux) ux[i] = jx / hh;
    if (uy) uy[i] = jy / hh;
}

// Diagnostic film pressure and force, in three plain passes.
template <typename T, typename SM>
__global__ void k_pf_h(Pops<T, SM> P, T* hbuf, Geom G)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= G.nx) return;
    T v[9], hh, jx, jy;
    pull_at(P, G, x, y, v);
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

template <typename T, typename SM>
__global__ void k_pf_f(Pops<T, SM> P, const T* __restrict__ pbuf, T* p, T* fx, T* fy, Geom G,
                       Consts<T> C)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= G.nx) return;
    const int xm = wrapi(x - 1, G.nx), xp = wrapi(x + 1, G.nx);
    const int ym = wrapi(y - 1, G.ny), yp = wrapi(y + 1, G.ny);
    auto Pp = [&](int yy, int xx) { return pbuf[(long long)yy * G.nx + xx]; };
    const T gpx = (Pp(y, xp) - Pp(y, xm)) / T(3) + (Pp(yp, xp) - Pp(yp, xm) + Pp(ym, xp) - Pp(ym, xm)) / T(12);
    const T gpy = (Pp(yp, x) - Pp(ym, x)) / T(3) + (Pp(yp, xp) - Pp(ym, xp) + Pp(yp, xm) - Pp(ym, xm)) / T(12);
    T v[9], hh, jx, jy;
    pull_at(P, G, x, y, v);
    moments9(v, hh, jx, jy);
    const T fr = C.nu6 / (T(2) * hh * hh + T(6) * C.delta * hh + T(3) * C.delta * C.delta);
    const long long i = (long long)y * G.nx + x;
    if (p) p[i] = Pp(y, x);
    T Fx = -hh * gpx - fr * jx + hh * C.gx;
    T Fy = -hh * gpy - fr * jy + hh * C.gy;
    if (C.forcing) {
        // second-order forcing: friction at u = (j + F/2)/h, i.e.
        // h u (1 + fr/2) = j + F'/2 with F' the force without friction
        const T fpx = hh * (C.gx - gpx), fpy = hh * (C.gy - gpy);
        const T q = T(1) / (T(1) + T(0.5) * fr);
        Fx = fpx - fr * (jx + T(0.5) * fpx) * q;
        Fy = fpy - fr * (jy + T(0.5) * fpy) * q;
    }
    if (fx) fx[i] = Fx;
    if (fy) fy[i] = Fy;
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

__device__ __forceinline__ void block_store(Comp a, double* partials)
{
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

// Sum of every stored population, decoded (the total liquid volume minus
// nx*ny*href: streaming only permutes populations on the periodic lattice).
// With an FP32 compute type each thread keeps an error-free FP32 pair
// (sum, compensation; Knuth's TwoSum per element), which resolves the sum of
// its ~100 values to about 2^-48 and runs at FP32 rate; the pair goes to the
// double-precision block reduction once.  FP64 state sums in double.
template <typename T, typename SM>
__global__ void __launch_bounds__(kMassThreads) k_mass_partial(Pops<T, SM> P, Geom G, double* partials)
{
    Comp a{0.0, 0.0};
    float fs = 0.0f, fc = 0.0f;
    const long long nrows = 9LL * G.ny;
    for (long long row = blockIdx.x; row < nrows; row += gridDim.x) {
        const int l = (int)(row / G.ny), y = (int)(row % G.ny);
        for (int x = threadIdx.x; x < G.nx; x += blockDim.x) {
            const T v = P.raw(l, P.at(y, x));
            if constexpr (std::is_same<T, float>::value) {
                const float t = __fadd_rn(fs, v);
                const float bp = __fsub_rn(t, fs);
                fc = __fadd_rn(fc, __fadd_rn(__fsub_rn(fs, __fsub_rn(t, bp)), __fsub_rn(v, bp)));
                fs = t;
            } else {
                comp_add(a, (double)v);
            }
        }
    }
    if constexpr (std::is_same<T, float>::value) {
        comp_add(a, (double)fs);
        a.c += (double)fc;
    }
    block_store(a, partials);
}

// Thread 0 of the block receives the block's compensated sum / maximum.
__device__ __forceinline__ Comp block_sum(Comp a)
{
    __shared__ Comp sm[kMassThreads / 32];
    a = warp_reduce(a);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();  // sm may still be read from a previous call
    if (lane == 0) sm[wid] = a;
    __syncthreads();
    Comp b{0.0, 0.0};
    if (wid == 0) {
        b = lane < kMassThreads / 32 ? sm[lane] : Comp{0.0, 0.0};
        b = warp_reduce(b);
    }
    return b;
}

__device__ __forceinline__ double block_max(double v)
{
    __shared__ double sm[kMassThreads / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sm[wid] = v;
    __syncthreads();
    double b = -INFINITY;
    if (wid == 0) {
        b = lane < kMassThreads / 32 ? sm[lane] : -INFINITY;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) b = fmax(b, __shfl_xor_sync(0xffffffffu, b, o));
    }
    return b;
}

template <typename T, typename SM>
__device__ __forceinline__ Pops<T, SM> pops_of(const BatchDomain<T>& D, int parity)
{
    Pops<T, SM> P;
    P.f0 = (T*)D.buf[parity];
    P.fm = (SM*)((char*)D.buf[parity] + D.G.plane * sizeof(T));
    P.plane = D.G.plane;
    P.pitch = D.G.pitch;
    P.href = D.C.href;
    P.mscale = D.C.mscale;
    P.minv = D.C.minv;
    P.r_axis = D.C.r_axis;
    P.r_diag = D.C.r_diag;
    return P;
}

// Film diagnostics of domain blockIdx.y of a table (compensated sums in
// double): [0] h over the lattice; over the wetted nodes (h > h_wet) [1] h,
// [2] j_x, [3] j_y, [4] 1, [5] h cos(2 pi x / nx), [6] h sin(2 pi x / nx),
// [7] h cos(2 pi y / ny), [8] h sin(2 pi y / ny); over the lattice
// [9] h cos(phi), [10] h sin(phi) with phi = 2 pi (mx x / nx + my y / ny);
// and the largest h.  Block b writes kDiagPartial doubles at
// partials[(domain * gridDim.x + b) * kDiagPartial].
constexpr int kDiagPartial = 2 * kDiagSums + 1;
template <typename T, typename SM>
__global__ void __launch_bounds__(kMassThreads) k_diag_partial(const BatchDomain<T>* __restrict__ doms, int parity,
                                                               double h_wet, int mx, int my, double* partials)
{
    const BatchDomain<T>& D = doms[blockIdx.y];
    const Pops<T, SM> P = pops_of<T, SM>(D, parity);
    const Geom G = D.G;
    Comp a[kDiagSums];
#pragma unroll
    for (int k = 0; k < kDiagSums; ++k) a[k] = Comp{0.0, 0.0};
    double hmax = -INFINITY;
    const long long n = (long long)G.nx * G.ny;
    // integer wave numbers reduced modulo the lattice, so phases stay exact
    const long long kx = ((mx % G.nx) + G.nx) % G.nx, ky = ((my % G.ny) + G.ny) % G.ny;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(i % G.nx), y = (int)(i / G.nx);
        T v[9], hh, jx, jy;
        pull_at(P, G, x, y, v);
        moments9(v, hh, jx, jy);
        const double h = (double)hh;
        comp_add(a[0], h);
        const double q = (double)((kx * x) % G.nx) / G.nx + (double)((ky * y) % G.ny) / G.ny;
        double sp, cp;
        sincospi(2.0 * q, &sp, &cp);
        comp_add(a[9], h * cp);
        comp_add(a[10], h * sp);
        if (h > h_wet) {
            comp_add(a[1], h);
            comp_add(a[2], (double)jx);
            comp_add(a[3], (double)jy);
            a[4].s += 1.0;  // exact below 2^53
            double sx, cx, sy, cy;
            sincospi(2.0 * x / G.nx, &sx, &cx);
            sincospi(2.0 * y / G.ny, &sy, &cy);
            comp_add(a[5], h * cx);
            comp_add(a[6], h * sx);
            comp_add(a[7], h * cy);
            comp_add(a[8], h * sy);
        }
        hmax = fmax(hmax, h);
    }
    double* out = partials + ((long long)blockIdx.y * gridDim.x + blockIdx.x) * kDiagPartial;
#pragma unroll
    for (int k = 0; k < kDiagSums; ++k) {
        const Comp b = block_sum(a[k]);
        if (threadIdx.x == 0) {
            out[2 * k] = b.s;
            out[2 * k + 1] = b.c;
        }
    }
    const double m = block_max(hmax);
    if (threadIdx.x == 0) out[2 * kDiagSums] = m;
}

// One block per domain: reduce the partials of its nb blocks into
// out[domain * kDiagOut ..] in the order of tf_lbm_diag: sums 0..4, the
// maximum, sums 5..10.
__global__ void __launch_bounds__(kMassThreads) k_diag_final(const double* __restrict__ partials, int nb,
                                                             double* out)
{
    const double* p = partials + (long long)blockIdx.x * nb * kDiagPartial;
    double* o = out + (long long)blockIdx.x * kDiagOut;
    for (int k = 0; k < kDiagSums; ++k) {
        Comp a{0.0, 0.0};
        for (int i = threadIdx.x; i < nb; i += blockDim.x) {
            comp_add(a, p[i * kDiagPartial + 2 * k]);
            a.c += p[i * kDiagPartial + 2 * k + 1];
        }
        const Comp b = block_sum(a);
        if (threadIdx.x == 0) o[k < 5 ? k : k + 1] = b.s + b.c;
    }
    double m = -INFINITY;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) m = fmax(m, p[i * kDiagPartial + 2 * kDiagSums]);
    m = block_max(m);
    if (threadIdx.x == 0) o[5] = m;
}

// ---- term balance of the appendix (Eq. magnitude): fields h, j, p, div j
template <typename T, typename SM>
__global__ void k_tn_fields(Pops<T, SM> P, T* hb, T* jxb, T* jyb, Geom G)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= G.nx) return;
    T v[9], hh, jx, jy;
    pull_at(P, G, x, y, v);
    moments9(v, hh, jx, jy);
    const long long i = (long long)y * G.nx + x;
    hb[i] = hh;
    jxb[i] = jx;
    jyb[i] = jy;
}

// d/dx and d/dy of a field with the stencil of Eq. (derivative)
template <typename T>
struct Stencil {
    const T* f;
    Geom G;
    int x, y, xm, xp, ym, yp;
    __device__ Stencil(const T* f_, const Geom& G_, int x_, int y_) : f(f_), G(G_), x(x_), y(y_)
    {
        xm = wrapi(x - 1, G.nx);
        xp = wrapi(x + 1, G.nx);
        ym = wrapi(y - 1, G.ny);
        yp = wrapi(y + 1, G.ny);
    }
    __device__ T at(int yy, int xx) const { return f[(long long)yy * G.nx + xx]; }
    __device__ T dx() const
    {
        return (at(y, xp) - at(y, xm)) / T(3) + (at(yp, xp) - at(yp, xm) + at(ym, xp) - at(ym, xm)) / T(12);
    }
    __device__ T dy() const
    {
        return (at(yp, x) - at(ym, x)) / T(3) + (at(yp, xp) - at(ym, xp) + at(yp, xm) - at(ym, xm)) / T(12);
    }
    // Eq. (n_laplace) with the reading (1/6)[4 sum_axis + sum_diag - 20 phi]
    __device__ T lap() const
    {
        const T axis = at(y, xm) + at(y, xp) + at(ym, x) + at(yp, x);
        const T diag = at(ym, xm) + at(ym, xp) + at(yp, xm) + at(yp, xp);
        return (T(4) * axis + diag - T(20) * at(y, x)) / T(6);
    }
};

template <typename T>
__global__ void k_tn_div(const T* __restrict__ jx, const T* __restrict__ jy, T* div, Geom G)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= G.nx) return;
    div[(long long)y * G.nx + x] = Stencil<T>(jx, G, x, y).dx() + Stencil<T>(jy, G, x, y).dy();
}

// Sums of squares of the x-components of -h d_x p, -nu alpha(h) u_x and
// nu lap(j_x) + 2 nu d_x(div j) (three (s, c) pairs per block).
template <typename T>
__global__ void __launch_bounds__(kMassThreads) k_tn_terms(const T* __restrict__ hb, const T* __restrict__ jxb,
                                                           const T* __restrict__ pb, const T* __restrict__ db,
                                                           Geom G, Consts<T> C, double* partials)
{
    Comp a[3] = {{0.0, 0.0}, {0.0, 0.0}, {0.0, 0.0}};
    const long long n = (long long)G.nx * G.ny;
    const double nu = (double)C.nu6 / 6.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(i % G.nx), y = (int)(i / G.nx);
        const double h = (double)hb[i], jx = (double)jxb[i], d = (double)C.delta;
        const double tp = -h * (double)Stencil<T>(pb, G, x, y).dx();
        // nu alpha(h) u_x = 6 nu j_x / (2 h^2 + 6 delta h + 3 delta^2), Eqs. (forcefric, alphafric)
        const double tf = -6.0 * nu * jx / (2.0 * h * h + 6.0 * d * h + 3.0 * d * d);
        const double td = nu * (double)Stencil<T>(jxb, G, x, y).lap() + 2.0 * nu * (double)Stencil<T>(db, G, x, y).dx();
        comp_add(a[0], tp * tp);
        comp_add(a[1], tf * tf);
        comp_add(a[2], td * td);
    }
    for (int k = 0; k < 3; ++k) {
        const Comp b = block_sum(a[k]);
        if (threadIdx.x == 0) {
            partials[2 * (k * gridDim.x + blockIdx.x)] = b.s;
            partials[2 * (k * gridDim.x + blockIdx.x) + 1] = b.c;
        }
    }
}

__global__ void __launch_bounds__(kMassThreads) k_tn_final(const double* __restrict__ partials, int nb, double n,
                                                           double* out)
{
    for (int k = 0; k < 3; ++k) {
        Comp a{0.0, 0.0};
        for (int i = threadIdx.x; i < nb; i += blockDim.x) {
            comp_add(a, partials[2 * (k * nb + i)]);
            a.c += partials[2 * (k * nb + i) + 1];
        }
        const Comp b = block_sum(a);
        if (threadIdx.x == 0) out[k] = sqrt((b.s + b.c) / n);
    }
}

// Smallest of n values (NaNs ignored; +inf when there is none).
template <typename T>
__global__ void __launch_bounds__(kMassThreads) k_min_partial(const T* __restrict__ x, long long n,
                                                              double* partials)
{
    double m = -INFINITY;  // max of -x
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        m = fmax(m, -(double)x[i]);
    m = block_max(m);
    if (threadIdx.x == 0) partials[blockIdx.x] = m;
}

__global__ void __launch_bounds__(kMassThreads) k_min_final(const double* partials, int n, double* out)
{
    double m = -INFINITY;
    for (int i = threadIdx.x; i < n; i += blockDim.x) m = fmax(m, partials[i]);
    m = block_max(m);
    if (threadIdx.x == 0) *out = -m;
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

template <typename T, typename SM>
__global__ void k_check(Pops<T, SM> P, Geom G, int* flag)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    int bad = 0;
    if (x < G.nx) {
        T v[9], hh, jx, jy;
        pull_at(P, G, x, y, v);
        for (int l = 0; l < 9; ++l)
            if (!isfinite((double)v[l])) bad |= 1;
        moments9(v, hh, jx, jy);
        if (!isfinite((double)hh)) bad |= 1;
        else if (!(hh > T(0))) bad |= 2;
    }
    bad = __reduce_or_sync(0xffffffffu, bad);
    if (bad && (threadIdx.x & 31) == 0) atomicOr(flag, bad);
}

// State export in double: decoded values plus href in double are exact for
// float and 16-bit storage, so an export / import round trip reproduces the
// stored bits.
template <typename T, typename SM>
__global__ void k_get_state(Pops<T, SM> P, double* out, Geom G)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= G.nx) return;
    const long long n = (long long)G.nx * G.ny, i = (long long)y * G.nx + x;
#pragma unroll
    for (int l = 0; l < 9; ++l) {
        const double v = (double)P.raw(l, P.at(wrapi(y - kCy[l], G.ny), wrapi(x - kCx[l], G.nx)));
        out[l * n + i] = l == 0 ? v + (double)P.href : v;
    }
}

// Post-streaming populations in the compute type, [9][ny][nx] (adjoint input).
template <typename T, typename SM>
__global__ void k_export_state(Pops<T, SM> P, T* out, Geom G)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= G.nx) return;
    T v[9];
    pull_at(P, G, x, y, v);
    const long long n = (long long)G.nx * G.ny, i = (long long)y * G.nx + x;
#pragma unroll
    for (int l = 0; l < 9; ++l) out[l * n + i] = v[l];
}

template <typename T, typename SM>
__global__ void k_set_state(Pops<T, SM> P, const double* __restrict__ in, Geom G)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= G.nx) return;
    const long long n = (long long)G.nx * G.ny;
#pragma unroll
    for (int l = 0; l < 9; ++l) {
        const long long src = (long long)wrapi(y + kCy[l], G.ny) * G.nx + wrapi(x + kCx[l], G.nx);
        const double v = in[l * n + src];
        P.put(l, P.at(y, x), T(l == 0 ? v - (double)P.href : v));
    }
}

inline dim3 grid2d(const Geom& G, int bx) { return dim3((G.nx + bx - 1) / bx, G.ny); }

template <typename T, typename SM>
cudaError_t init_t(const StoreDesc& D, void* f, const void* h0, const Geom& G, double g, cudaStream_t st)
{
    k_init<T, SM><<<grid2d(G, 128), 128, 0, st>>>(make_pops<T, SM>(f, G, D), (const T*)h0, G, T(g));
    return cudaGetLastError();
}

template <typename T, typename SM>
cudaError_t moments_t(const StoreDesc& D, const void* f, void* h, void* ux, void* uy, const Geom& G,
                      cudaStream_t st)
{
    k_moments<T, SM><<<grid2d(G, 128), 128, 0, st>>>(make_pops<T, SM>(f, G, D), (T*)h, (T*)ux, (T*)uy, G);
    return cudaGetLastError();
}

template <typename T, typename SM>
cudaError_t pf_t(const StoreDesc& D, const void* f, const void* kappa, void* p, void* fx, void* fy,
                 void* sh, void* sp, const Geom& G, const Consts<T>& C, cudaStream_t st)
{
    const auto P = make_pops<T, SM>(f, G, D);
    k_pf_h<T, SM><<<grid2d(G, 128), 128, 0, st>>>(P, (T*)sh, G);
    k_pf_p<T><<<grid2d(G, 128), 128, 0, st>>>((const T*)sh, (const T*)kappa, (T*)sp, G, C);
    k_pf_f<T, SM><<<grid2d(G, 128), 128, 0, st>>>(P, (const T*)sp, (T*)p, (T*)fx, (T*)fy, G, C);
    return cudaGetLastError();
}

template <typename T, typename SM>
cudaError_t mass_t(const StoreDesc& D, const void* f, const Geom& G, double* partials, int nblocks,
                   double* result, cudaStream_t st)
{
    k_mass_partial<T, SM><<<nblocks, kMassThreads, 0, st>>>(make_pops<T, SM>(f, G, D), G, partials);
    k_mass_final<<<1, kMassThreads, 0, st>>>(partials, nblocks, result);
    return cudaGetLastError();
}

template <typename T, typename SM>
cudaError_t diag_t(const void* doms, int ndom, int parity, double h_wet, int mx, int my, double* partials, int nb,
                   double* out, cudaStream_t st)
{
    k_diag_partial<T, SM><<<dim3(nb, ndom), kMassThreads, 0, st>>>((const BatchDomain<T>*)doms, parity, h_wet,
                                                                  mx, my, partials);
    k_diag_final<<<ndom, kMassThreads, 0, st>>>(partials, nb, out);
    return cudaGetLastError();
}

template <typename T, typename SM>
cudaError_t term_norms_t(const StoreDesc& D, const void* f, const void* kappa, const Geom& G, const Consts<T>& C,
                         void* scratch, double* partials, int nb, double* out, cudaStream_t st)
{
    const long long n = (long long)G.nx * G.ny;
    T* hb = (T*)scratch;
    T* jxb = hb + n;
    T* jyb = jxb + n;
    T* pb = jyb + n;
    T* db = pb + n;
    k_tn_fields<T, SM><<<grid2d(G, 128), 128, 0, st>>>(make_pops<T, SM>(f, G, D), hb, jxb, jyb, G);
    k_pf_p<T><<<grid2d(G, 128), 128, 0, st>>>(hb, (const T*)kappa, pb, G, C);
    k_tn_div<T><<<grid2d(G, 128), 128, 0, st>>>(jxb, jyb, db, G);
    k_tn_terms<T><<<nb, kMassThreads, 0, st>>>(hb, jxb, pb, db, G, C, partials);
    k_tn_final<<<1, kMassThreads, 0, st>>>(partials, nb, (double)n, out);
    return cudaGetLastError();
}

template <typename T, typename SM>
cudaError_t check_t(const StoreDesc& D, const void* f, const Geom& G, int* flag, cudaStream_t st)
{
    k_check<T, SM><<<grid2d(G, 128), 128, 0, st>>>(make_pops<T, SM>(f, G, D), G, flag);
    return cudaGetLastError();
}

template <typename T, typename SM>
cudaError_t get_t(const StoreDesc& D, const void* f, double* out, const Geom& G, cudaStream_t st)
{
    k_get_state<T, SM><<<grid2d(G, 128), 128, 0, st>>>(make_pops<T, SM>(f, G, D), out, G);
    return cudaGetLastError();
}

template <typename T, typename SM>
cudaError_t export_t(const StoreDesc& D, const void* f, void* out, const Geom& G, cudaStream_t st)
{
    k_export_state<T, SM><<<grid2d(G, 128), 128, 0, st>>>(make_pops<T, SM>(f, G, D), (T*)out, G);
    return cudaGetLastError();
}

template <typename T, typename SM>
cudaError_t set_t(const StoreDesc& D, void* f, const double* in, const Geom& G, cudaStream_t st)
{
    k_set_state<T, SM><<<grid2d(G, 128), 128, 0, st>>>(make_pops<T, SM>(f, G, D), in, G);
    return cudaGetLastError();
}

}  // namespace

int mass_blocks(const Geom& G)
{
    long long rows = 9LL * G.ny;
    return (int)(rows < 1184 ? rows : 1184);
}

// Dispatch over the storage type: F32 and the 16-bit stores compute in float,
// F64 in double.
#define TFLBM_DISPATCH(D, CALL)                                                      \
    switch ((D).store) {                                                             \
        case kStoreF32: { using T = float; using SM = float; return CALL; }          \
        case kStoreF64: { using T = double; using SM = double; return CALL; }        \
        case kStoreF16: { using T = float; using SM = __half; return CALL; }         \
        case kStoreBF16: { using T = float; using SM = __nv_bfloat16; return CALL; } \
        default: return cudaErrorInvalidValue;                                       \
    }

cudaError_t aux_init(const StoreDesc& D, void* f, const void* h0, const Geom& G, double g, cudaStream_t st)
{
    TFLBM_DISPATCH(D, (init_t<T, SM>(D, f, h0, G, g, st)))
}

cudaError_t aux_moments(const StoreDesc& D, const void* f, void* h, void* ux, void* uy, const Geom& G,
                        cudaStream_t st)
{
    TFLBM_DISPATCH(D, (moments_t<T, SM>(D, f, h, ux, uy, G, st)))
}

cudaError_t aux_pressure_force(const StoreDesc& D, const void* f, const void* kappa, void* p, void* fx,
                               void* fy, void* sh, void* sp, const Geom& G, const Consts<float>* C32,
                               const Consts<double>* C64, cudaStream_t st)
{
    switch (D.store) {
        case kStoreF32: return pf_t<float, float>(D, f, kappa, p, fx, fy, sh, sp, G, *C32, st);
        case kStoreF64: return pf_t<double, double>(D, f, kappa, p, fx, fy, sh, sp, G, *C64, st);
        case kStoreF16: return pf_t<float, __half>(D, f, kappa, p, fx, fy, sh, sp, G, *C32, st);
        case kStoreBF16: return pf_t<float, __nv_bfloat16>(D, f, kappa, p, fx, fy, sh, sp, G, *C32, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t aux_mass(const StoreDesc& D, const void* f, const Geom& G, double* partials, int nblocks,
                     double* result, cudaStream_t st)
{
    TFLBM_DISPATCH(D, (mass_t<T, SM>(D, f, G, partials, nblocks, result, st)))
}

cudaError_t aux_diag(int store, const void* doms, int ndom, int parity, double h_wet, int mx, int my,
                     double* partials, int nb, double* out, cudaStream_t st)
{
    switch (store) {
        case kStoreF32: return diag_t<float, float>(doms, ndom, parity, h_wet, mx, my, partials, nb, out, st);
        case kStoreF64: return diag_t<double, double>(doms, ndom, parity, h_wet, mx, my, partials, nb, out, st);
        case kStoreF16: return diag_t<float, __half>(doms, ndom, parity, h_wet, mx, my, partials, nb, out, st);
        case kStoreBF16:
            return diag_t<float, __nv_bfloat16>(doms, ndom, parity, h_wet, mx, my, partials, nb, out, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t aux_term_norms(const StoreDesc& D, const void* f, const void* kappa, const Geom& G,
                           const Consts<float>* C32, const Consts<double>* C64, void* scratch, double* partials,
                           int nb, double* out, cudaStream_t st)
{
    switch (D.store) {
        case kStoreF32: return term_norms_t<float, float>(D, f, kappa, G, *C32, scratch, partials, nb, out, st);
        case kStoreF64: return term_norms_t<double, double>(D, f, kappa, G, *C64, scratch, partials, nb, out, st);
        case kStoreF16: return term_norms_t<float, __half>(D, f, kappa, G, *C32, scratch, partials, nb, out, st);
        case kStoreBF16:
            return term_norms_t<float, __nv_bfloat16>(D, f, kappa, G, *C32, scratch, partials, nb, out, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t aux_check(const StoreDesc& D, const void* f, const Geom& G, int* flag, cudaStream_t st)
{
    TFLBM_DISPATCH(D, (check_t<T, SM>(D, f, G, flag, st)))
}

cudaError_t aux_get_state(const StoreDesc& D, const void* f, double* out, const Geom& G, cudaStream_t st)
{
    TFLBM_DISPATCH(D, (get_t<T, SM>(D, f, out, G, st)))
}

cudaError_t aux_export_state(const StoreDesc& D, const void* f, void* out, const Geom& G, cudaStream_t st)
{
    TFLBM_DISPATCH(D, (export_t<T, SM>(D, f, out, G, st)))
}

cudaError_t aux_set_state(const StoreDesc& D, void* f, const double* in, const Geom& G, cudaStream_t st)
{
    TFLBM_DISPATCH(D, (set_t<T, SM>(D, f, in, G, st)))
}

cudaError_t aux_kappa(bool dbl, void* kappa, const void* theta, int nx, int ny, int ne, int me,
                      double hstar, cudaStream_t st)
{
    const long long n = (long long)nx * ny;
    const int blocks = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
    if (dbl) k_kappa<double><<<blocks, 256, 0, st>>>((double*)kappa, (const double*)theta, n, ne, me, hstar);
    else k_kappa<float><<<blocks, 256, 0, st>>>((float*)kappa, (const float*)theta, n, ne, me, hstar);
    return cudaGetLastError();
}

cudaError_t aux_min(bool dbl, const void* x, long long n, double* partials, int nblocks, double* result,
                    cudaStream_t st)
{
    if (dbl) k_min_partial<double><<<nblocks, kMassThreads, 0, st>>>((const double*)x, n, partials);
    else k_min_partial<float><<<nblocks, kMassThreads, 0, st>>>((const float*)x, n, partials);
    k_min_final<<<1, kMassThreads, 0, st>>>(partials, nblocks, result);
    return cudaGetLastError();
}


}  // namespace tflbm
