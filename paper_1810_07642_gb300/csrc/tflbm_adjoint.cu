// Discrete adjoint of the thin-film step and the checkpointed gradient tape.
//
// State: the post-streaming populations f(t), [9][ny][nx] in the compute
// type.  One step is f(t+1) = S(C(f(t))) with C the forced BGK collision of
// Eq. (LBE), using the force of Eq. (force) and the film pressure of
// Eqs. (pfilm, disjoiningP), and S the streaming.  Given a(t+1) = dL/df(t+1),
// the adjoint step returns a(t) = (d S C / d f(t))^T a(t+1) and adds
// (d S C / d kappa)^T a(t+1) to dL/dkappa.  Derivation, phase by phase
// (E_l are the equilibria of Eq. (equilibria) written in h and j = h u):
//   mu_l(x)  = a_l(x + c_l, t+1)                          streaming^T
//   aF       = sum_l 3 w_l c_l mu_l,  aE_l = omega mu_l    collision^T
//   aH       = sum_l aE_l dE_l/dh + aF.(G - grad p) - fr'(h) aF.j
//   aJ       = sum_l aE_l dE_l/dj - fr(h) aF,  ag = -h aF  force^T
//   ap(y)    = sum_l 3 w_l c_l . ag(y - c_l)               Eq. (derivative)^T
//   aPi = -gamma s ap: dL/dkappa += aPi (r^n - r^m), aH += aPi kappa (m r^m - n r^n)/h
//   aH      += lap(-gamma ap)                              Eq. (n_laplace) is symmetric
//   a_l(x,t) = aH + c_l . aJ + (1 - omega) mu_l            moments^T
// with r = h_*/h, fr = 6 nu / (2h^2 + 6 delta h + 3 delta^2).
//
// The gradient tape runs the forward from the handle's state, keeping a copy
// of the state every K steps (K ~ sqrt(T)); the backward pass restores each
// checkpoint in reverse order, recomputes the K states of that segment and
// runs the adjoint steps through them (sqrt(T) checkpoint-recompute).
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>
#include <vector>

#include "tflbm_adjoint_march.cuh"
#include "tflbm_handle.h"

namespace tflbm {
namespace {

__device__ __constant__ int aCx[9] = {0, 1, 1, 0, -1, -1, -1, 0, 1};
__device__ __constant__ int aCy[9] = {0, 0, 1, 1, 1, 0, -1, -1, -1};


template <typename T> __device__ __forceinline__ T wgt(int l) { return l == 0 ? T(4.0 / 9.0) : ((l & 1) ? T(1.0 / 9.0) : T(1.0 / 36.0)); }

struct Dims {
    int nx, ny;
    long long n;  // nx * ny
};

// Wrapped neighbourhood of node (x, y): row offsets of y-1, y, y+1 and
// columns x-1, x, x+1 (no integer division).
struct Nbr {
    long long r[3];
    int c[3];
    __device__ __forceinline__ Nbr(int x, int y, const Dims& D)
    {
        r[0] = (long long)(y == 0 ? D.ny - 1 : y - 1) * D.nx;
        r[1] = (long long)y * D.nx;
        r[2] = (long long)(y + 1 == D.ny ? 0 : y + 1) * D.nx;
        c[0] = x == 0 ? D.nx - 1 : x - 1;
        c[1] = x;
        c[2] = x + 1 == D.nx ? 0 : x + 1;
    }
    // index of node (x + dx, y + dy), dx, dy in {-1, 0, 1}
    __device__ __forceinline__ long long at(int dy, int dx) const { return r[dy + 1] + c[dx + 1]; }
};

// h, j of the state f at every node
template <typename T>
__global__ void k_adj_moments(const T* __restrict__ f, T* h, T* jx, T* jy, Dims D)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= D.nx) return;
    const long long i = (long long)y * D.nx + x;
    T s = 0, sx = 0, sy = 0;
#pragma unroll
    for (int l = 0; l < 9; ++l) {
        const T v = f[l * D.n + i];
        s += v;
        sx += T(aCx[l]) * v;
        sy += T(aCy[l]) * v;
    }
    h[i] = s;
    jx[i] = sx;
    jy[i] = sy;
}

// film pressure p = -gamma (lap h + s kappa (r^n - r^m))
template <typename T>
__global__ void k_adj_pressure(const T* __restrict__ h, const T* __restrict__ kappa, T* p, Dims D,
                               Consts<T> C)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= D.nx) return;
    const Nbr nb(x, y, D);
    auto H = [&](int dy, int dx) { return h[nb.at(dy, dx)]; };
    const T axis = H(0, -1) + H(0, 1) + H(-1, 0) + H(1, 0);
    const T diag = H(-1, -1) + H(-1, 1) + H(1, -1) + H(1, 1);
    const T hh = H(0, 0);
    T lap = (T(4) * axis + diag - T(20) * hh) / T(6);
    const long long i = (long long)y * D.nx + x;
    const T kap = kappa ? kappa[i] : C.kappa_u;
    const T r = C.hstar / hh;
    T rn = 1, rm = 1;
    for (int k = 0; k < C.n_exp; ++k) rn *= r;
    for (int k = 0; k < C.m_exp; ++k) rm *= r;
    p[i] = -C.gamma * (lap + C.pi_sgn * kap * (rn - rm));
}

// collision and force adjoint at every node
template <typename T>
__global__ void k_adj_collide(const T* __restrict__ h, const T* __restrict__ jx, const T* __restrict__ jy,
                              const T* __restrict__ p, const T* __restrict__ a_next, T* aH, T* aJx,
                              T* aJy, T* agx, T* agy, Dims D, Consts<T> C)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= D.nx) return;
    const long long i = (long long)y * D.nx + x;
    const Nbr nb(x, y, D);
    auto Pp = [&](int dy, int dx) { return p[nb.at(dy, dx)]; };
    // Eq. (derivative) at the node
    const T gpx = (Pp(0, 1) - Pp(0, -1)) / T(3) + (Pp(1, 1) - Pp(1, -1) + Pp(-1, 1) - Pp(-1, -1)) / T(12);
    const T gpy = (Pp(1, 0) - Pp(-1, 0)) / T(3) + (Pp(1, 1) - Pp(-1, 1) + Pp(1, -1) - Pp(-1, -1)) / T(12);
    const T hh = h[i], Jx = jx[i], Jy = jy[i], j2 = Jx * Jx + Jy * Jy, g = C.g, w = C.omega;
    T aFx = 0, aFy = 0, ah = 0, ajx = 0, ajy = 0;
#pragma unroll
    for (int l = 0; l < 9; ++l) {
        const T m = a_next[l * D.n + nb.at(aCy[l], aCx[l])];
        aFx += T(3) * wgt<T>(l) * T(aCx[l]) * m;
        aFy += T(3) * wgt<T>(l) * T(aCy[l]) * m;
        const T am = w * m;
        const T cj = T(aCx[l]) * Jx + T(aCy[l]) * Jy;
        T dh, djx, djy;
        if (l == 0) {
            dh = T(1) - T(5) * g * hh / T(3) + T(2) * j2 / (T(3) * hh * hh);
            djx = -T(4) * Jx / (T(3) * hh);
            djy = -T(4) * Jy / (T(3) * hh);
        } else if (l & 1) {
            dh = g * hh / T(3) - cj * cj / (T(2) * hh * hh) + j2 / (T(6) * hh * hh);
            djx = T(aCx[l]) / T(3) + cj * T(aCx[l]) / hh - Jx / (T(3) * hh);
            djy = T(aCy[l]) / T(3) + cj * T(aCy[l]) / hh - Jy / (T(3) * hh);
        } else {
            dh = g * hh / T(12) - cj * cj / (T(8) * hh * hh) + j2 / (T(24) * hh * hh);
            djx = T(aCx[l]) / T(12) + cj * T(aCx[l]) / (T(4) * hh) - Jx / (T(12) * hh);
            djy = T(aCy[l]) / T(12) + cj * T(aCy[l]) / (T(4) * hh) - Jy / (T(12) * hh);
        }
        ah += am * dh;
        ajx += am * djx;
        ajy += am * djy;
    }
    const T den = T(2) * hh * hh + C.delta * (T(6) * hh + T(3) * C.delta);
    const T nu6 = C.nu6;
    const T fr = nu6 / den;
    const T dfr = -nu6 * (T(4) * hh + T(6) * C.delta) / (den * den);
    ah += aFx * (C.gx - gpx) + aFy * (C.gy - gpy) - dfr * (aFx * Jx + aFy * Jy);
    aH[i] = ah;
    aJx[i] = ajx - fr * aFx;
    aJy[i] = ajy - fr * aFy;
    agx[i] = -hh * aFx;
    agy[i] = -hh * aFy;
}

// transpose of the gradient stencil, then the film-pressure adjoint
template <typename T>
__global__ void k_adj_pressure_t(const T* __restrict__ agx, const T* __restrict__ agy,
                                 const T* __restrict__ h, const T* __restrict__ kappa, T* aH, T* alap,
                                 T* grad_kappa, Dims D, Consts<T> C)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= D.nx) return;
    const long long i = (long long)y * D.nx + x;
    const Nbr nb(x, y, D);
    T ap = 0;
#pragma unroll
    for (int l = 0; l < 9; ++l) {
        const long long k = nb.at(-aCy[l], -aCx[l]);
        ap += T(3) * wgt<T>(l) * (T(aCx[l]) * agx[k] + T(aCy[l]) * agy[k]);
    }
    alap[i] = -C.gamma * ap;
    const T api = -C.gamma * C.pi_sgn * ap;
    const T hh = h[i];
    const T r = C.hstar / hh;
    T rn = 1, rm = 1;
    for (int k = 0; k < C.n_exp; ++k) rn *= r;
    for (int k = 0; k < C.m_exp; ++k) rm *= r;
    const T kap = kappa ? kappa[i] : C.kappa_u;
    grad_kappa[i] += api * (rn - rm);
    aH[i] += api * kap * (T(C.m_exp) * rm - T(C.n_exp) * rn) / hh;
}

// Laplacian (symmetric) and the moments' transpose
template <typename T>
__global__ void k_adj_out(const T* __restrict__ aH, const T* __restrict__ alap, const T* __restrict__ aJx,
                          const T* __restrict__ aJy, const T* __restrict__ a_next, T* a, Dims D,
                          Consts<T> C)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= D.nx) return;
    const long long i = (long long)y * D.nx + x;
    const Nbr nb(x, y, D);
    auto Ls = [&](int dy, int dx) { return alap[nb.at(dy, dx)]; };
    const T axis = Ls(0, -1) + Ls(0, 1) + Ls(-1, 0) + Ls(1, 0);
    const T diag = Ls(-1, -1) + Ls(-1, 1) + Ls(1, -1) + Ls(1, 1);
    const T ah = aH[i] + (T(4) * axis + diag - T(20) * Ls(0, 0)) / T(6);
    const T jx = aJx[i], jy = aJy[i], om = T(1) - C.omega;
#pragma unroll
    for (int l = 0; l < 9; ++l) {
        const T m = a_next[l * D.n + nb.at(aCy[l], aCx[l])];
        a[l * D.n + i] = ah + T(aCx[l]) * jx + T(aCy[l]) * jy + om * m;
    }
}

// dL/dh0 = sum_l a_l(0) dE_l(h0, 0)/dh0; dL/dtheta = dL/dkappa sin(theta) c
template <typename T>
__global__ void k_adj_init(const T* __restrict__ h0, const T* __restrict__ a0, T* gh0, const T* __restrict__ gk,
                           const T* __restrict__ theta, T* gth, Dims D, Consts<T> C, T kc, T theta_u)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= D.n) return;
    if (gh0) {
        const T hh = h0[i];
        T s = a0[i] * (T(1) - T(5) * C.g * hh / T(3));
#pragma unroll
        for (int l = 1; l < 9; ++l) s += a0[l * D.n + i] * C.g * hh * ((l & 1) ? T(1.0 / 3.0) : T(1.0 / 12.0));
        gh0[i] = s;
    }
    if (gth) gth[i] = gk[i] * sin(theta ? theta[i] : theta_u) * kc;
}

template <typename T>
__global__ void k_seed(const T* __restrict__ gh, T* a, Dims D)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= D.n) return;
    const T v = gh[i];
#pragma unroll
    for (int l = 0; l < 9; ++l) a[l * D.n + i] = v;  // h = sum_l f_l
}

inline dim3 g2(const Dims& D) { return dim3((D.nx + 127) / 128, D.ny); }
inline int g1(const Dims& D) { return (int)((D.n + 255) / 256); }

template <typename T>
cudaError_t adjoint_t(tf_lbm_handle* H, const void* f, const void* an, void* a, void* gk, cudaStream_t st)
{
    Dims D{H->G.nx, H->G.ny, (long long)H->G.nx * H->G.ny};
    T* s = (T*)H->adj;
    T *h = s, *jx = s + D.n, *jy = s + 2 * D.n, *p = s + 3 * D.n, *aH = s + 4 * D.n, *aJx = s + 5 * D.n,
      *aJy = s + 6 * D.n, *agx = s + 7 * D.n, *agy = s + 8 * D.n, *alap = s + 9 * D.n;
    const Consts<T> C = make_consts<T>(H);
    const T* kap = (const T*)H->kappa;
    k_adj_moments<T><<<g2(D), 128, 0, st>>>((const T*)f, h, jx, jy, D);
    k_adj_pressure<T><<<g2(D), 128, 0, st>>>(h, kap, p, D, C);
    k_adj_collide<T><<<g2(D), 128, 0, st>>>(h, jx, jy, p, (const T*)an, aH, aJx, aJy, agx, agy, D, C);
    k_adj_pressure_t<T><<<g2(D), 128, 0, st>>>(agx, agy, h, kap, aH, alap, (T*)gk, D, C);
    k_adj_out<T><<<g2(D), 128, 0, st>>>(aH, alap, aJx, aJy, (const T*)an, (T*)a, D, C);
    return cudaGetLastError();
}

}  // namespace

cudaError_t adjoint_step_dispatch(tf_lbm_handle* H, const void* f, const void* an, void* a, void* gk,
                                  cudaStream_t st)
{
    if (!H->adj) {
        cudaError_t e = cudaMalloc(&H->adj, 10ull * H->G.nx * H->G.ny * H->esize);
        if (e != cudaSuccess) return e;
    }
    return H->dbl ? adjoint_t<double>(H, f, an, a, gk, st) : adjoint_t<float>(H, f, an, a, gk, st);
}

namespace {

template <typename SM, typename T, int BX>
cudaError_t march_t(tf_lbm_handle* H, const void* fin, const void* an, void* a, void* gk, int rows,
                    cudaStream_t st)
{
    const Geom& G = H->G;
    const T* f0 = (const T*)fin;
    const SM* fm = (const SM*)((const char*)fin + G.plane * sizeof(T));
    int bands = (G.ny + rows - 1) / rows;
    if (bands > 65535) bands = 65535;
    const dim3 grid((G.nx + BX - 9) / (BX - 8), bands);
    k_adjoint_march<SM, T, BX><<<grid, BX, 0, st>>>(f0, fm, (const T*)an, (T*)a, (T*)gk, (const T*)H->kappa, G,
                                                    make_consts<T>(H));
    return cudaGetLastError();
}

template <typename SM, typename T, int BX>
int march_rows(const tf_lbm_handle* H)
{
    int occ = 0, sms = sm_count();
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_adjoint_march<SM, T, BX>, BX, 0) != cudaSuccess) {
        cudaGetLastError();
        occ = 1;
    }
    const int strips = (H->G.nx + BX - 9) / (BX - 8);
    const int bands = std::max(1, std::max(occ, 1) * sms / strips);
    return std::max(4, (H->G.ny + bands - 1) / bands);
}

}  // namespace

// Fused adjoint step from the raw buffer whose pull is f(t).
cudaError_t adjoint_march_dispatch(tf_lbm_handle* H, const void* fin, const void* an, void* a, void* gk,
                                   cudaStream_t st)
{
    switch (H->desc.store) {
        case kStoreF32: return march_t<float, float, 128>(H, fin, an, a, gk, march_rows<float, float, 128>(H), st);
        case kStoreF64: return march_t<double, double, 64>(H, fin, an, a, gk, march_rows<double, double, 64>(H), st);
        case kStoreF16: return march_t<__half, float, 128>(H, fin, an, a, gk, march_rows<__half, float, 128>(H), st);
        case kStoreBF16:
            return march_t<__nv_bfloat16, float, 128>(H, fin, an, a, gk, march_rows<__nv_bfloat16, float, 128>(H), st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace tflbm

// ---------------------------------------------------------------- the tape

struct tf_lbm_tape {
    tf_lbm_handle* H = nullptr;
    int64_t nsteps = 0;
    int every = 1;
    int nck = 0;                   // checkpoints: states at 0, K, 2K, ...
    size_t state_bytes = 0;        // one raw population buffer
    void* ck = nullptr;            // nck raw buffers, then the final state
    void* seg = nullptr;           // every raw population buffers: the states of one segment
    void* abuf = nullptr;          // 2 adjoint states
    void* gk = nullptr;            // dL/dkappa
    void* h0 = nullptr;            // copy of h0 (compute type)
    void* theta = nullptr;         // copy of theta or null (uniform)
    int64_t t0 = 0;                // handle time when the forward started
    bool forwarded = false;
    // CUDA graphs of one full segment: recompute and the adjoint chain (by
    // starting adjoint buffer)
    cudaGraphExec_t g_rec[2] = {nullptr, nullptr};  // only [0] is used
    cudaGraphExec_t g_adj[2] = {nullptr, nullptr};
    cudaStream_t cap = nullptr;
};

namespace {

int tape_fail(tf_lbm_tape* tp, int code, const char* msg) { return handle_fail(tp ? tp->H : nullptr, code, msg); }

#define TK(tp, call, what)                                                       \
    do {                                                                         \
        cudaError_t e_ = (call);                                                 \
        if (e_ != cudaSuccess) return handle_cuda_fail((tp)->H, e_, what);      \
    } while (0)

// Recompute the len states of a segment: seg slot 0 holds the checkpoint;
// each step writes the next slot, so no state is exported or copied.
cudaError_t recompute(tf_lbm_tape* tp, int64_t len, cudaStream_t st)
{
    char* seg = (char*)tp->seg;
    for (int64_t i = 0; i + 1 < len; ++i) {
        cudaError_t e = launch_step_between(tp->H, seg + i * tp->state_bytes, seg + (i + 1) * tp->state_bytes, st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Fused adjoint steps backwards through a segment of len states, starting
// from the adjoint state in abuf slot `from`.
cudaError_t adjoint_chain(tf_lbm_tape* tp, int from, int64_t len, cudaStream_t st)
{
    tf_lbm_handle* H = tp->H;
    const size_t abytes = 9ull * H->G.nx * H->G.ny * H->esize;
    char* seg = (char*)tp->seg;
    char* ab = (char*)tp->abuf;
    int cur = from;
    for (int64_t i = len - 1; i >= 0; --i) {
        cudaError_t e = adjoint_march_dispatch(H, seg + i * tp->state_bytes, ab + cur * abytes,
                                               ab + (cur ^ 1) * abytes, tp->gk, st);
        if (e != cudaSuccess) return e;
        cur ^= 1;
    }
    return cudaSuccess;
}

// Capture fn into an executable graph (on the tape's own capture stream).
template <typename Fn>
cudaError_t capture(tf_lbm_tape* tp, cudaGraphExec_t* out, Fn fn)
{
    cudaError_t e;
    if (!tp->cap && (e = cudaStreamCreateWithFlags(&tp->cap, cudaStreamNonBlocking)) != cudaSuccess) return e;
    if ((e = cudaStreamBeginCapture(tp->cap, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) return e;
    cudaError_t fe = fn(tp->cap);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(tp->cap, &g);
    if (fe != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return fe;
    }
    if (e != cudaSuccess) return e;
    e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    return e;
}

}  // namespace

extern "C" {

int tf_lbm_adjoint_step(tf_lbm_handle* H, const void* f_t, const void* a_next, void* a_t, void* grad_kappa,
                        void* stream)
{
    if (!H) return handle_fail(nullptr, TF_LBM_ERR_ARG, "handle is NULL");
    if (!f_t || !a_next || !a_t || !grad_kappa)
        return handle_fail(H, TF_LBM_ERR_ARG, "f_t, a_next, a_t and grad_kappa must not be NULL");
    if (a_t == a_next) return handle_fail(H, TF_LBM_ERR_ARG, "a_t must not alias a_next");
    if (H->p.forcing != 0)
        return handle_fail(H, TF_LBM_ERR_UNSUPPORTED, "the adjoint differentiates Eq. (LBE) as printed (forcing = 0)");
    cudaError_t e = adjoint_step_dispatch(H, f_t, a_next, a_t, grad_kappa, (cudaStream_t)stream);
    if (e != cudaSuccess) return handle_cuda_fail(H, e, "adjoint kernels");
    return TF_LBM_OK;
}

int tf_lbm_tape_create(tf_lbm_handle* H, const void* h0, const void* theta, int64_t nsteps, int32_t every,
                       tf_lbm_tape** out)
{
    if (!H) return handle_fail(nullptr, TF_LBM_ERR_ARG, "handle is NULL");
    if (!out) return handle_fail(H, TF_LBM_ERR_ARG, "out must not be NULL");
    *out = nullptr;
    if (!h0) return handle_fail(H, TF_LBM_ERR_ARG, "h0 must not be NULL");
    if (nsteps < 1) return handle_fail(H, TF_LBM_ERR_ARG, "nsteps must be >= 1");
    if (H->p.forcing != 0)
        return handle_fail(H, TF_LBM_ERR_UNSUPPORTED, "the adjoint differentiates Eq. (LBE) as printed (forcing = 0)");
    if (every <= 0) every = (int32_t)ceil(sqrt((double)nsteps));
    if (every > nsteps) every = (int32_t)nsteps;
    tf_lbm_tape* tp = new tf_lbm_tape();
    tp->H = H;
    tp->nsteps = nsteps;
    tp->every = every;
    tp->nck = (int)((nsteps + every - 1) / every);
    tp->state_bytes = (size_t)H->G.plane * (H->esize + 8 * H->msize);
    const long long n = (long long)H->G.nx * H->G.ny;
    cudaError_t e;
    auto bail = [&](cudaError_t err, const char* what) {
        int rc = handle_cuda_fail(H, err, what);
        tf_lbm_tape_destroy(tp);
        return rc;
    };
    if ((e = cudaMalloc(&tp->ck, tp->state_bytes * (tp->nck + 1))) != cudaSuccess) return bail(e, "cudaMalloc checkpoints");
    if ((e = cudaMalloc(&tp->seg, tp->state_bytes * every)) != cudaSuccess) return bail(e, "cudaMalloc segment");
    if ((e = cudaMalloc(&tp->abuf, 18ull * n * H->esize)) != cudaSuccess) return bail(e, "cudaMalloc adjoint");
    if ((e = cudaMalloc(&tp->gk, n * H->esize)) != cudaSuccess) return bail(e, "cudaMalloc grad kappa");
    if ((e = cudaMalloc(&tp->h0, n * H->esize)) != cudaSuccess) return bail(e, "cudaMalloc h0");
    if ((e = cudaMemcpy(tp->h0, h0, n * H->esize, cudaMemcpyDeviceToDevice)) != cudaSuccess) return bail(e, "copy h0");
    if (theta) {
        if ((e = cudaMalloc(&tp->theta, n * H->esize)) != cudaSuccess) return bail(e, "cudaMalloc theta");
        if ((e = cudaMemcpy(tp->theta, theta, n * H->esize, cudaMemcpyDeviceToDevice)) != cudaSuccess)
            return bail(e, "copy theta");
    }
    *out = tp;
    return TF_LBM_OK;
}

int tf_lbm_tape_forward(tf_lbm_tape* tp, void* stream)
{
    if (!tp) return handle_fail(nullptr, TF_LBM_ERR_ARG, "tape is NULL");
    tf_lbm_handle* H = tp->H;
    cudaStream_t st = (cudaStream_t)stream;
    tp->t0 = H->time;
    char* ck = (char*)tp->ck;
    for (int c = 0; c < tp->nck; ++c) {
        TK(tp, cudaMemcpyAsync(ck + c * tp->state_bytes, H->buf[H->cur], tp->state_bytes, cudaMemcpyDeviceToDevice, st),
           "checkpoint copy");
        const int64_t len = (c + 1 == tp->nck) ? tp->nsteps - (int64_t)c * tp->every : tp->every;
        const int rc = tf_lbm_step(H, len, stream);
        if (rc) return rc;
    }
    TK(tp, cudaMemcpyAsync(ck + tp->nck * tp->state_bytes, H->buf[H->cur], tp->state_bytes, cudaMemcpyDeviceToDevice, st),
       "final state copy");
    tp->forwarded = true;
    return TF_LBM_OK;
}

int tf_lbm_tape_backward(tf_lbm_tape* tp, const void* grad_h, void* grad_theta, void* grad_h0, void* stream)
{
    if (!tp) return handle_fail(nullptr, TF_LBM_ERR_ARG, "tape is NULL");
    tf_lbm_handle* H = tp->H;
    if (!tp->forwarded) return tape_fail(tp, TF_LBM_ERR_ARG, "tf_lbm_tape_forward must run first");
    if (!grad_h) return tape_fail(tp, TF_LBM_ERR_ARG, "grad_h must not be NULL");
    cudaStream_t st = (cudaStream_t)stream;
    const long long n = (long long)H->G.nx * H->G.ny;
    const size_t sbytes = 9ull * n * H->esize;
    char* seg = (char*)tp->seg;
    char* ab = (char*)tp->abuf;
    char* ck = (char*)tp->ck;
    Dims D{H->G.nx, H->G.ny, n};
    int cur = 0;  // adjoint state in ab + cur * sbytes
    if (H->dbl) k_seed<double><<<g1(D), 256, 0, st>>>((const double*)grad_h, (double*)ab, D);
    else k_seed<float><<<g1(D), 256, 0, st>>>((const float*)grad_h, (float*)ab, D);
    TK(tp, cudaGetLastError(), "seed kernel");
    TK(tp, cudaMemsetAsync(tp->gk, 0, n * H->esize, st), "cudaMemsetAsync");
    for (int c = tp->nck - 1; c >= 0; --c) {
        const int64_t len = (c + 1 == tp->nck) ? tp->nsteps - (int64_t)c * tp->every : tp->every;
        // the checkpoint starts the segment; recompute its states, then run
        // the adjoint back through them; full segments replay captured graphs
        TK(tp, cudaMemcpyAsync(seg, ck + c * tp->state_bytes, tp->state_bytes, cudaMemcpyDeviceToDevice, st),
           "checkpoint restore");
        if (len == tp->every && len > 1) {
            const int afrom = cur;
            if (!tp->g_rec[0])
                TK(tp, capture(tp, &tp->g_rec[0], [&](cudaStream_t cs) { return recompute(tp, len, cs); }),
                   "recompute graph");
            if (!tp->g_adj[afrom])
                TK(tp, capture(tp, &tp->g_adj[afrom], [&](cudaStream_t cs) { return adjoint_chain(tp, afrom, len, cs); }),
                   "adjoint graph");
            TK(tp, cudaGraphLaunch(tp->g_rec[0], st), "cudaGraphLaunch");
            TK(tp, cudaGraphLaunch(tp->g_adj[afrom], st), "cudaGraphLaunch");
        } else {
            TK(tp, recompute(tp, len, st), "recompute");
            TK(tp, adjoint_chain(tp, cur, len, st), "adjoint chain");
        }
        cur ^= (int)(len & 1);
    }
    if (grad_h0 || grad_theta) {
        const double kc = (double)(H->p.n_exp - 1) * (H->p.m_exp - 1) / ((double)(H->p.n_exp - H->p.m_exp) * H->p.hstar);
        if (H->dbl)
            k_adj_init<double><<<g1(D), 256, 0, st>>>((const double*)tp->h0, (const double*)(ab + cur * sbytes),
                                                      (double*)grad_h0, (const double*)tp->gk, (const double*)tp->theta,
                                                      (double*)grad_theta, D, make_consts<double>(H), kc,
                                                      H->p.theta_uniform);
        else
            k_adj_init<float><<<g1(D), 256, 0, st>>>((const float*)tp->h0, (const float*)(ab + cur * sbytes),
                                                     (float*)grad_h0, (const float*)tp->gk, (const float*)tp->theta,
                                                     (float*)grad_theta, D, make_consts<float>(H), (float)kc,
                                                     (float)H->p.theta_uniform);
        TK(tp, cudaGetLastError(), "init adjoint kernel");
    }
    return TF_LBM_OK;
}

void tf_lbm_tape_destroy(tf_lbm_tape* tp)
{
    if (!tp) return;
    cudaDeviceSynchronize();
    for (void* p : {tp->ck, tp->seg, tp->abuf, tp->gk, tp->h0, tp->theta})
        if (p) cudaFree(p);
    for (auto& g : tp->g_rec)
        if (g) cudaGraphExecDestroy(g);
    for (auto& g : tp->g_adj)
        if (g) cudaGraphExecDestroy(g);
    if (tp->cap) cudaStreamDestroy(tp->cap);
    delete tp;
}

}  // extern "C"
