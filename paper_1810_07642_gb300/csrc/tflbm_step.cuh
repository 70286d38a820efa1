// Fused thin-film D2Q9 step: pull-streaming, moments, 9-point Laplacian of h,
// film pressure with disjoining pressure, isotropic gradient of p, total force
// and forced BGK collision in one pass over the lattice (Section II of
// Zitz et al., arXiv:1810.07642; Eqs. LBE, equilibria, force, pfilm,
// disjoiningP, forcefric, alphafric, derivative, n_laplace).
//
// Design (HBM-bound stencil, no tensor cores):
//  * Populations live in SoA planes [9][ny][pitch].  The buffer read by a step
//    holds post-collision values of the previous step, so streaming is a pull:
//    f_l(x, y) = fin_l(x - c_l).  Each step reads 9 and writes 9 values per
//    node (+ kappa when theta varies); h, p and F never touch DRAM.
//  * A CTA of BX threads covers BX consecutive columns, one per thread, and
//    marches down a band of rows; neighbouring CTAs overlap by 4 columns, so
//    each CTA stores BX - 4 columns and needs no divergent halo work.
//    March step k: (A) h - href of row r(k) into a 4-row shared ring while
//    the loads of row r(k+1) are already in flight; one __syncthreads; (B)
//    the film pressure of row r(k-1) (columns 1 .. BX-2) into a second 4-row
//    ring, and force + collision + store of row r(k-3) (columns 2 .. BX-3),
//    whose momentum was kept in registers.  With 4-row rings every shared row is rewritten
//    only after the barrier that follows its last read, so one barrier per
//    row suffices.  The radius-2 dependence of grad p on h costs 5 extra rows
//    per band and 4 extra columns per strip, served from L1/L2.
//  * Bands are balanced (band b covers rows [b ny / nb, (b+1) ny / nb)) and
//    alternate their march direction so that shared edge rows hit in L2.
//  * Plane 0 stores f_0 - href (see tflbm_internal.h).  The rest population
//    is written as (h - href) - sum_{l>0} f*_l, and the exact rounding
//    residuals of that subtraction and of the pull sum (error-free TwoSum)
//    are returned to the opposite pair (1, 5), so in FP32 the collision
//    conserves local mass up to roundings of the small moving populations.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <type_traits>
#include <utility>

#include "tflbm_internal.h"

namespace tflbm {

__device__ __forceinline__ int wrap_index(int i, int n)
{
    i %= n;
    return i < 0 ? i + n : i;
}

// a / b: CUDA's fast single-precision division (within 2 ulp) in FP32, the
// IEEE division in FP64.
__device__ __forceinline__ float fdiv(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double fdiv(double a, double b) { return a / b; }

// r^n for 0 <= n < 64 by binary powering over a fixed number of bits (no
// data-dependent branches; n is uniform).
template <typename T>
__device__ __forceinline__ T ipow(T r, int n)
{
    T out = T(1), b = r;
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        if ((n >> i) & 1) out *= b;
        b *= b;
    }
    return out;
}

// (hstar/h)^n - (hstar/h)^m from r = hstar/h; (3, 2) without the loop.
template <typename T>
__device__ __forceinline__ T fdisj(T r, int n, int m)
{
    if (n == 3 && m == 2) return r * r * (r - T(1));
    return ipow(r, n) - ipow(r, m);
}

template <typename S> __device__ __forceinline__ S ldro(const S* p) { return __ldg(p); }

// Programmatic dependent launch.  A step kernel lets the next kernel of its
// stream be scheduled as soon as all of its own CTAs have started (the next
// step's CTAs then take SMs as this step's CTAs retire, instead of waiting
// for a full launch), and waits for the previous kernel of the stream to
// complete, with its writes visible, before it touches global memory.  Both
// are hardware dependencies (no polling); without the launch attribute the
// wait returns at once.
__device__ __forceinline__ void dependent_launch_entry()
{
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

// Launch `kern` with the programmatic-stream-serialization attribute (see
// dependent_launch_entry).
template <typename... KArgs, typename... Args>
cudaError_t launch_dependent(void (*kern)(KArgs...), dim3 grid, int block, size_t smem, cudaStream_t st,
                             Args&&... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

// Element conversions of the moving-population storage types.
__device__ __forceinline__ float to_f(float q) { return q; }
__device__ __forceinline__ double to_f(double q) { return q; }
__device__ __forceinline__ float to_f(__half q) { return __half2float(q); }
__device__ __forceinline__ float to_f(__nv_bfloat16 q) { return __bfloat162float(q); }
template <typename SM> __device__ __forceinline__ SM from_f(float v);
template <> __device__ __forceinline__ __half from_f<__half>(float v) { return __float2half_rn(v); }
template <> __device__ __forceinline__ __nv_bfloat16 from_f<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }

// A moving population l (1..8) is kept as is when its storage type is the
// compute type.  In 16-bit storage it is kept as q = (f_l - R_l) * scale,
// R_l = f_eq_l(href, u = 0) (gh^2/6 on the axes, gh^2/24 on the diagonals),
// and read back as q / scale + R_l: one fma with an exact product, so the
// writer can compute the bits every reader will see.
template <typename SM, typename T>
__device__ __forceinline__ T load_moving(SM q, int l, const Consts<T>& C)
{
    if constexpr (std::is_same<SM, T>::value) return q;
    else return fmaf(to_f(q), C.minv, (l & 1) ? C.r_axis : C.r_diag);
}

// Error-free sum (Knuth's TwoSum): a + b = s + e exactly.  The _rn
// intrinsics keep the compiler from contracting or reordering the steps.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void two_sum(double a, double b, double& s, double& e)
{
    s = __dadd_rn(a, b);
    const double bb = __dsub_rn(s, a);
    e = __dadd_rn(__dsub_rn(a, __dsub_rn(s, bb)), __dsub_rn(b, bb));
}

// Pull the nine populations arriving at column x of row y: i0 = y*pitch + x,
// im / ip the same row offset for the wrapped columns x-1 / x+1, dm / dp the
// row steps to rows y-1 / y+1 (wrapped, in elements).  Plane 0 (f_0 - href)
// is f0[i]; moving population l is fm[(l-1)*plane + i].  32-bit offsets: the
// host checks 9 * plane < 2^31.  Order of Eq. (speeds): 1 (1,0) 2 (1,1)
// 3 (0,1) 4 (-1,1) 5 (-1,0) 6 (-1,-1) 7 (0,-1) 8 (1,-1); population l at x
// comes from x - c_l.
template <typename SM, typename T>
__device__ __forceinline__ void pull9(const T* __restrict__ f0, const SM* __restrict__ fm,
                                      int plane, int i0, int im, int ip, int dm, int dp,
                                      const Consts<T>& C, T (&v)[9])
{
    const long long m8 = 8LL * plane;  // extent of the moving planes
    int* st = C.status;
    v[0] = ldro(f0 + TFLBM_IDX(i0, plane, st));
    v[1] = load_moving(ldro(fm + TFLBM_IDX(im, m8, st)), 1, C);
    v[2] = load_moving(ldro(fm + TFLBM_IDX(plane + im + dm, m8, st)), 2, C);
    v[3] = load_moving(ldro(fm + TFLBM_IDX(2 * plane + i0 + dm, m8, st)), 3, C);
    v[4] = load_moving(ldro(fm + TFLBM_IDX(3 * plane + ip + dm, m8, st)), 4, C);
    v[5] = load_moving(ldro(fm + TFLBM_IDX(4 * plane + ip, m8, st)), 5, C);
    v[6] = load_moving(ldro(fm + TFLBM_IDX(5 * plane + ip + dp, m8, st)), 6, C);
    v[7] = load_moving(ldro(fm + TFLBM_IDX(6 * plane + i0 + dp, m8, st)), 7, C);
    v[8] = load_moving(ldro(fm + TFLBM_IDX(7 * plane + im + dp, m8, st)), 8, C);
    (void)m8;
    (void)st;
}

// dh = sum_l v_l with v_0 = f_0 - href: the moving populations are summed
// first (they are small), the final addition is error-free, so the exact sum
// of the nine inputs is dh + err up to roundings of the small partial sums.
template <typename T>
__device__ __forceinline__ T sum9(const T (&v)[9], T& err)
{
    const T m = ((v[1] + v[2]) + (v[3] + v[4])) + ((v[5] + v[6]) + (v[7] + v[8]));
    T dh;
    two_sum(v[0], m, dh, err);
    return dh;
}

// Film pressure p = -gamma (lap h + pi_sign kappa f(h)) at one node from the
// 3x3 neighbourhood of dh = h - href in the shared ring (rows n = +y, c,
// s = -y); the Laplacian is taken on dh, in which the offset cancels exactly.
// ih = 1/h of the node.
template <typename T>
__device__ __forceinline__ T film_pressure(const T* hn, const T* hc, const T* hs_, int j, T kap,
                                           T ih, const Consts<T>& C, bool disj, int n)
{
    TFLBM_CHECK(j >= 1 && j + 1 < n, C.status);  // the ring rows hold n columns
    (void)n;
    const T axis = (hc[j - 1] + hc[j + 1]) + (hn[j] + hs_[j]);
    const T diag = (hn[j - 1] + hn[j + 1]) + (hs_[j - 1] + hs_[j + 1]);
    T lap = (T(4) * axis + diag - T(20) * hc[j]) * T(1.0 / 6.0);
    if (disj) lap += C.pi_sgn * kap * fdisj(C.hstar * ih, C.n_exp, C.m_exp);
    return -C.gamma * lap;
}

// ---------------------------------------------------------------------------
// Force, collision and store of one node (both kernels).  pn, pc, ps are the
// shared p rows at o+1, o, o-1 and t the node's slot in them; dh = h - href,
// ih = 1/h, (jx, jy) the momentum, er the pull-sum residual, f the pulled
// populations (used when omega != 1).  The node's storage offset is
// row + x.
template <typename SM, typename T, bool OMEGA1>
__device__ __forceinline__ void collide_store(const T* pn, const T* pc, const T* ps, int t, T dh,
                                              T ih, T jx, T jy, T er, const T (&f)[9],
                                              T* __restrict__ fout0, SM* __restrict__ foutm,
                                              int row, int x, int plane, const Consts<T>& C, int n)
{
    constexpr bool NARROW = !std::is_same<SM, T>::value;
    TFLBM_CHECK(t >= 1 && t + 1 < n, C.status);  // the p ring rows hold n columns
    (void)n;
    const T third = T(1.0 / 3.0), twelfth = T(1.0 / 12.0), sixth = T(1.0 / 6.0);
    // Eq. (derivative): grad p = 3 sum_l w_l c_l p(x + c_l)
    const T gpx = (pc[t + 1] - pc[t - 1]) * third
                + ((pn[t + 1] - pn[t - 1]) + (ps[t + 1] - ps[t - 1])) * twelfth;
    const T gpy = (pn[t] - ps[t]) * third
                + ((pn[t + 1] - ps[t + 1]) + (pn[t - 1] - ps[t - 1])) * twelfth;
    const T h = dh + C.href;
    // Eqs. (force), (forcefric), (alphafric):
    // nu alpha u = 6 nu j / (2h^2 + 6 delta h + 3 delta^2)
    const T fr = fdiv(C.nu6, h * (T(2) * h + T(6) * C.delta) + T(3) * C.delta * C.delta);
    // Eq. (LBE) as printed: u = j/h and F with the friction at that velocity.
    // Second-order forcing (C.forcing): u = (j + F/2)/h with the friction
    // taken at that velocity, u (h + nu alpha/2) = j + F'/2; the equilibria
    // then use h u in place of j.
    T Fx, Fy, ux, uy, ex, ey;
    if (C.forcing) {
        const T fpx = h * (C.gx - gpx), fpy = h * (C.gy - gpy);
        const T q = fdiv(ih, T(1) + T(0.5) * fr);  // 1 / (h + nu alpha / 2)
        ux = (jx + T(0.5) * fpx) * q;
        uy = (jy + T(0.5) * fpy) * q;
        ex = h * ux;
        ey = h * uy;
        Fx = fpx - fr * ex;
        Fy = fpy - fr * ey;
    } else {
        Fx = h * (C.gx - gpx) - fr * jx;
        Fy = h * (C.gy - gpy) - fr * jy;
        ux = jx * ih;
        uy = jy * ih;
        ex = jx;
        ey = jy;
    }
    // Eq. (equilibria) with e^2 = 1, written as S +- D per pair of opposite
    // directions; source 3 w_l c_l . F.
    const T A = h * (C.g * h - (ux * ux + uy * uy)) * sixth;
    T Sx = A + T(0.5) * ex * ux;
    T Sy = A + T(0.5) * ey * uy;
    const T a = ux + uy, b = uy - ux;
    T Sa = (A + T(0.5) * h * a * a) * T(0.25);
    T Sb = (A + T(0.5) * h * b * b) * T(0.25);
    // second-order source (1 - omega/2) w_l [3 (c_l - u) + 9 (c_l.u) c_l].F:
    // its odd part is the printed 3 w_l c_l.F scaled by (1 - omega/2), its
    // even part T per pair of opposite directions
    T Tx = T(0), Ty = T(0), Ta = T(0), Tb = T(0);
    if (C.forcing) {
        const T ks = T(1) - T(0.5) * C.omega;
        Fx *= ks;
        Fy *= ks;
        const T uF3 = (ux * Fx + uy * Fy) * third;
        Tx = ux * Fx - uF3;
        Ty = uy * Fy - uF3;
        Ta = (a * (Fx + Fy) - uF3) * T(0.25);
        Tb = (b * (Fy - Fx) - uF3) * T(0.25);
        if (OMEGA1) {
            Sx += Tx;
            Sy += Ty;
            Sa += Ta;
            Sb += Tb;
        }
    }
    T o1, o2, o3, o4, o5, o6, o7, o8;
    if (OMEGA1) {
        const T Dx = (ex + Fx) * third, Dy = (ey + Fy) * third;
        const T Da = ((ex + ey) + (Fx + Fy)) * twelfth;
        const T Db = ((ey - ex) + (Fy - Fx)) * twelfth;
        o1 = Sx + Dx; o5 = Sx - Dx;
        o3 = Sy + Dy; o7 = Sy - Dy;
        o2 = Sa + Da; o6 = Sa - Da;
        o4 = Sb + Db; o8 = Sb - Db;
    } else {
        const T w = C.omega, m = T(1) - C.omega;
        const T Dx = ex * third, Dy = ey * third;
        const T Da = (ex + ey) * twelfth, Db = (ey - ex) * twelfth;
        const T Qx = Fx * third, Qy = Fy * third;
        const T Qa = (Fx + Fy) * twelfth, Qb = (Fy - Fx) * twelfth;
        o1 = m * f[1] + w * (Sx + Dx) + (Tx + Qx);
        o5 = m * f[5] + w * (Sx - Dx) + (Tx - Qx);
        o3 = m * f[3] + w * (Sy + Dy) + (Ty + Qy);
        o7 = m * f[7] + w * (Sy - Dy) + (Ty - Qy);
        o2 = m * f[2] + w * (Sa + Da) + (Ta + Qa);
        o6 = m * f[6] + w * (Sa - Da) + (Ta - Qa);
        o4 = m * f[4] + w * (Sb + Db) + (Tb + Qb);
        o8 = m * f[8] + w * (Sb - Db) + (Tb - Qb);
    }
    // In 16-bit storage, round the moving populations to what the readers
    // will reconstruct before the rest population is formed (f_1 possibly
    // after it, see below).
    SM q1, q2, q3, q4, q5, q6, q7, q8;
    // (o - R) * mscale in one rounding: o * mscale - R * mscale is exact
    auto narrow = [&](T& o, SM& q, T R, T NR) {
        q = from_f<SM>(fmaf(o, C.mscale, NR));
        o = fmaf(to_f(q), C.minv, R);
    };
    bool f1_last = false;
    if constexpr (NARROW) {
        narrow(o3, q3, C.r_axis, C.nr_axis);
        narrow(o5, q5, C.r_axis, C.nr_axis); narrow(o7, q7, C.r_axis, C.nr_axis);
        narrow(o2, q2, C.r_diag, C.nr_diag); narrow(o4, q4, C.r_diag, C.nr_diag);
        narrow(o6, q6, C.r_diag, C.nr_diag); narrow(o8, q8, C.r_diag, C.nr_diag);
    }
    // stored rest population: f*_0 - href = (h - href) - sum_{l>0} f*_l.  The
    // error-free sums give the exact rounding residuals of the pull sum and
    // of this subtraction.  With full-width storage they go to the opposite
    // pair (1, 5), half each, so the stored populations sum to the pulled
    // ones (mass conserved to roundings of small values) and the momentum is
    // untouched.  With 16-bit storage they are added to the rest population,
    // and the residual of that addition is left to the finer of two
    // roundings: the 16-bit one of f_1 - R (half-ulp 2^-11 relative in FP16,
    // 2^-8 in BF16) or the FP32 one of f_0 - href (2^-24 relative).  Where
    // f_1 rounds finer (a thick film that barely moves, e.g. a resting drop)
    // the residual goes into f_1 before f_1 is rounded; elsewhere f_1 is
    // rounded first and its own residual becomes part of the rest population.
    T osum = ((o1 + o5) + (o3 + o7)) + ((o2 + o6) + (o4 + o8));
    if constexpr (NARROW) {
        constexpr float kRatio = std::is_same<SM, __half>::value ? 8192.0f : 65536.0f;
        f1_last = fabsf(o1 - C.r_axis) * kRatio < fabsf(dh - osum);
        if (!f1_last) {
            const T o1u = o1;
            narrow(o1, q1, C.r_axis, C.nr_axis);
            osum += o1 - o1u;
        }
    }
    T o0v, e2;
    two_sum(dh, -osum, o0v, e2);
    if constexpr (NARROW) {
        T o0n, e3;
        two_sum(o0v, er + e2, o0n, e3);
        o0v = o0n;
        if (f1_last) {
            o1 += e3;
            narrow(o1, q1, C.r_axis, C.nr_axis);
        }
    } else {
        const T half_r = (er + e2) * T(0.5);
        o1 += half_r;
        o5 += half_r;
        q1 = o1; q2 = o2; q3 = o3; q4 = o4; q5 = o5; q6 = o6; q7 = o7; q8 = o8;
    }
    const int i = row + x;
    const long long m8 = 8LL * plane;
    int* st = C.status;
    fout0[TFLBM_IDX(i, plane, st)] = o0v;
    foutm[TFLBM_IDX(i, m8, st)] = q1;
    foutm[TFLBM_IDX(plane + i, m8, st)] = q2;
    foutm[TFLBM_IDX(2 * plane + i, m8, st)] = q3;
    foutm[TFLBM_IDX(3 * plane + i, m8, st)] = q4;
    foutm[TFLBM_IDX(4 * plane + i, m8, st)] = q5;
    foutm[TFLBM_IDX(5 * plane + i, m8, st)] = q6;
    foutm[TFLBM_IDX(6 * plane + i, m8, st)] = q7;
    foutm[TFLBM_IDX(7 * plane + i, m8, st)] = q8;
    (void)m8;
    (void)st;
}

// ---------------------------------------------------------------------------
// Common geometry of one CTA: BX columns x0-2 .. x0+BX-3, one per thread
// (neighbouring CTAs overlap by 4 columns, so each stores BX-4 columns and
// needs no divergent halo work), marching down a band of rows.
struct Band {
    int x0, weff, ybeg, yend, R, dir, rstart;
    bool hcol, pcol, ocol;
};

template <int BX>
__device__ __forceinline__ Band make_band(const Geom& G, int t, int strip, int band, int nbands, int flip)
{
    Band b;
    constexpr int W = BX - 4;
    b.x0 = strip * W;                           // first output column
    b.weff = min(W, G.nx - b.x0);               // output columns of this CTA
    b.hcol = t < b.weff + 4;                    // forms h
    b.pcol = t >= 1 && t < b.weff + 3;          // forms p
    b.ocol = t >= 2 && t < b.weff + 2;          // collides and stores
    b.ybeg = (int)(((long long)band * G.ny) / nbands);
    b.yend = (int)(((long long)(band + 1) * G.ny) / nbands);
    // March direction: even bands go +y, odd bands -y, so two neighbouring
    // bands read the rows around their common edge at the same time (both at
    // the start or both at the end of the kernel) and the second read hits
    // L2.  March step k forms h of row r(k) = rstart + k dir, the pressure of
    // row r(k-1) and collides row r(k-3), for k = 0 .. R+4.
    // Every other step (flip) all bands reverse, so a band starts on the rows
    // it wrote last, which are still in L2.
    b.dir = ((band + flip) & 1) ? -1 : 1;
    b.R = b.yend - b.ybeg;
    b.rstart = b.dir > 0 ? b.ybeg - 2 : b.yend + 1;
    return b;
}

// Per-thread asynchronous global-to-shared copies (cp.async, 4 or 8 bytes).
__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
template <int BYTES>
__device__ __forceinline__ void cp_async(void* dst, const void* src)
{
    static_assert(BYTES == 4 || BYTES == 8, "4- or 8-byte elements");
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(smem_u32(dst)), "l"(src), "n"(BYTES)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// ---------------------------------------------------------------------------
// Kernel 1: every thread loads its own nine pulled populations from global
// memory ahead of use: one row ahead into registers, or (ASYNC, full-width
// storage only) kAsyncStages - 1 rows ahead into a private shared-memory
// ring by cp.async, which keeps more bytes in flight without registers.
constexpr int kAsyncStages = 3;
template <typename SM, typename T, int BX, bool OMEGA1, bool KFIELD, bool ASYNC = false>
__device__ __forceinline__ void step_band(const T* __restrict__ fin0, const SM* __restrict__ finm,
                                          T* __restrict__ fout0, SM* __restrict__ foutm,
                                          const T* __restrict__ kappa, const Geom& G, const Consts<T>& C,
                                          int strip, int band, int nbands)
{
    static_assert(!ASYNC || std::is_same<SM, T>::value, "async staging needs full-width storage");
    __shared__ T hsm[4][BX];  // h - href ring: slot t = column x0 - 2 + t
    __shared__ T psm[4][BX];  // p ring, same columns
    // async ring: stage j % kAsyncStages holds the nine pulled values of row r(j)
    __shared__ T stg[ASYNC ? kAsyncStages : 1][9][ASYNC ? BX : 1];
    const int t = threadIdx.x;
    const int nx = G.nx, ny = G.ny, pitch = G.pitch, plane = (int)G.plane;
    const Band B = make_band<BX>(G, t, strip, band, nbands, C.flip);
    const bool disj = KFIELD || C.kappa_u != T(0);
    const int dir = B.dir, R = B.R;

    const int x = wrap_index(B.x0 - 2 + t, nx);
    const int xm = wrap_index(x - 1, nx), xp = wrap_index(x + 1, nx);

    // wrapped indices of rows r(k-1), r(k), r(k+1), r(k+2), r(k+3)
    int wm1 = wrap_index(B.rstart - dir, ny), w0 = wrap_index(B.rstart, ny);
    int w1 = wrap_index(B.rstart + dir, ny), w2 = wrap_index(B.rstart + 2 * dir, ny);
    int w3 = ASYNC ? wrap_index(B.rstart + 3 * dir, ny) : 0;

    T v[9];
    T kap_n = C.kappa_u;
    // the pulled populations of the last four rows, needed by the relaxation
    // when omega != 1: a per-thread shared ring in FP32 (keeps the kernel at
    // 64 registers), registers in FP64
    constexpr bool FRING = !OMEGA1 && sizeof(T) == 4;
    __shared__ T fsm[FRING ? 4 : 1][9][FRING ? BX : 1];
    T fv[FRING || OMEGA1 ? 1 : 4][9];
    T jxv[4], jyv[4], ihv[4], erv[4];
#pragma unroll
    for (int s = 0; s < 4; ++s) { jxv[s] = jyv[s] = ihv[s] = erv[s] = T(0); }

    // pull row w whose neighbours in march order are wb (behind) and wa (ahead)
    auto pull_row = [&](int wb, int w, int wa) {
        const int r0 = w * pitch;
        const int below = (dir > 0 ? wb : wa) - w, above = (dir > 0 ? wa : wb) - w;
        pull9<SM, T>(fin0, finm, plane, r0 + x, r0 + xm, r0 + xp, below * pitch, above * pitch, C, v);
    };
    // the same nine elements, copied asynchronously into stage st of the ring
    // (one commit group per row, empty for threads that load nothing)
    auto issue_row = [&](int st, int wb, int w, int wa) {
        if (B.hcol) {
            const int r0 = w * pitch;
            const int dm = ((dir > 0 ? wb : wa) - w) * pitch, dp = ((dir > 0 ? wa : wb) - w) * pitch;
            const int i0 = r0 + x, im = r0 + xm, ip = r0 + xp;
            T(&d)[9][ASYNC ? BX : 1] = stg[st];
            constexpr int E = sizeof(T);
            const long long m8 = 8LL * plane;
            int* cs = C.status;
            cp_async<E>(&d[0][t], fin0 + TFLBM_IDX(i0, plane, cs));
            cp_async<E>(&d[1][t], finm + TFLBM_IDX(im, m8, cs));
            cp_async<E>(&d[2][t], finm + TFLBM_IDX(plane + im + dm, m8, cs));
            cp_async<E>(&d[3][t], finm + TFLBM_IDX(2 * plane + i0 + dm, m8, cs));
            cp_async<E>(&d[4][t], finm + TFLBM_IDX(3 * plane + ip + dm, m8, cs));
            cp_async<E>(&d[5][t], finm + TFLBM_IDX(4 * plane + ip, m8, cs));
            cp_async<E>(&d[6][t], finm + TFLBM_IDX(5 * plane + ip + dp, m8, cs));
            cp_async<E>(&d[7][t], finm + TFLBM_IDX(6 * plane + i0 + dp, m8, cs));
            cp_async<E>(&d[8][t], finm + TFLBM_IDX(7 * plane + im + dp, m8, cs));
            (void)m8;
            (void)cs;
        }
        cp_async_commit();
    };
    if constexpr (ASYNC) {
        issue_row(0, wm1, w0, w1);
        issue_row(1, w0, w1, w2);
    } else {
        if (B.hcol) pull_row(wm1, w0, w1);
    }
    const long long nkap = (long long)nx * ny;  // kappa field extent
    (void)nkap;
    if (KFIELD && B.pcol) kap_n = kappa[TFLBM_IDX((long long)wm1 * nx + x, nkap, C.status)];

    auto body = [&](auto stage_c, int k) {
        constexpr int s = decltype(stage_c)::value;  // slot of row r(k) (and r(k-4))
        constexpr int s1 = (s + 3) & 3;              // slot of row r(k-1)
        constexpr int s2 = (s + 2) & 3;              // slot of row r(k-2)
        constexpr int s3 = (s + 1) & 3;              // slot of row r(k-3)
        // ---- (A) h of row r(k); the loads of row r(k+1) go out before anything waits
        const T kap = kap_n;  // kappa of row r(k-1), loaded last step
        if constexpr (ASYNC) {
            // row r(k) has landed once at most one younger group is pending;
            // then the stage of row r(k-1) (read last step) takes row r(k+2)
            if (k <= R + 3) {
                cp_async_wait<kAsyncStages - 2>();
                if (B.hcol) {
                    const int st = k % kAsyncStages;
#pragma unroll
                    for (int l = 0; l < 9; ++l) v[l] = stg[st][l][t];
                }
                if (k + 2 <= R + 3) issue_row((k + 2) % kAsyncStages, w1, w2, w3);
                else cp_async_commit();
            }
        }
        if (B.hcol && k <= R + 3) {
            hsm[s][t] = sum9(v, erv[s]);
            jxv[s] = ((v[1] + v[2]) + v[8]) - ((v[4] + v[5]) + v[6]);
            jyv[s] = ((v[2] + v[3]) + v[4]) - ((v[6] + v[7]) + v[8]);
            if constexpr (FRING) {
#pragma unroll
                for (int l = 0; l < 9; ++l) fsm[s][l][t] = v[l];
            } else if constexpr (!OMEGA1) {
#pragma unroll
                for (int l = 0; l < 9; ++l) fv[s][l] = v[l];
            }
            if (!ASYNC && k + 1 <= R + 3) pull_row(w0, w1, w2);
            if (KFIELD && B.pcol) kap_n = kappa[TFLBM_IDX((long long)w0 * nx + x, nkap, C.status)];
        }
        __syncthreads();
        // ---- (B1) film pressure of row r(k-1) (needs h rows r(k-2) .. r(k))
        if (B.pcol && k >= 2 && k <= R + 3) {
            const T ih = fdiv(T(1), hsm[s1][t] + C.href);
            ihv[s1] = ih;
            psm[s1][t] = film_pressure(hsm[s], hsm[s1], hsm[s2], t, kap, ih, C, disj, BX);
        }
        // ---- (B2) force, collision and store of row r(k-3) (needs p rows r(k-4) .. r(k-2))
        if (B.ocol && k >= 5) {
            const int o = B.rstart + (k - 3) * dir;  // inside [ybeg, yend), no wrap
            T fl[9];
            if constexpr (FRING) {
#pragma unroll
                for (int l = 0; l < 9; ++l) fl[l] = fsm[s3][l][t];
            } else if constexpr (!OMEGA1) {
#pragma unroll
                for (int l = 0; l < 9; ++l) fl[l] = fv[s3][l];
            } else {
#pragma unroll
                for (int l = 0; l < 9; ++l) fl[l] = T(0);  // unused at omega == 1
            }
            collide_store<SM, T, OMEGA1>(dir > 0 ? psm[s2] : psm[s], psm[s3], dir > 0 ? psm[s] : psm[s2], t,
                                         hsm[s3][t], ihv[s3], jxv[s3], jyv[s3], erv[s3], fl,
                                         fout0, foutm, o * pitch, x, plane, C, BX);
        }
        wm1 = w0;
        w0 = w1;
        w1 = w2;
        if constexpr (ASYNC) {
            w2 = w3;
            w3 += dir;
            w3 = w3 == ny ? 0 : (w3 < 0 ? ny - 1 : w3);
        } else {
            w2 += dir;
            w2 = w2 == ny ? 0 : (w2 < 0 ? ny - 1 : w2);
        }
    };

    const int last = R + 4;
    for (int k = 0;;) {
        body(std::integral_constant<int, 0>{}, k);
        if (++k > last) break;
        body(std::integral_constant<int, 1>{}, k);
        if (++k > last) break;
        body(std::integral_constant<int, 2>{}, k);
        if (++k > last) break;
        body(std::integral_constant<int, 3>{}, k);
        if (++k > last) break;
    }
}

template <typename SM, typename T, int BX, bool OMEGA1, bool KFIELD, bool ASYNC = false>
__global__ void __launch_bounds__(BX, sizeof(T) == 4 ? 1024 / BX : 1)
k_step(const T* __restrict__ fin0, const SM* __restrict__ finm, T* __restrict__ fout0,
       SM* __restrict__ foutm, const T* __restrict__ kappa, const Geom G, const Consts<T> C)
{
    dependent_launch_entry();
    step_band<SM, T, BX, OMEGA1, KFIELD, ASYNC>(fin0, finm, fout0, foutm, kappa, G, C, blockIdx.x,
                                                blockIdx.y, gridDim.y);
}

// One batched step.  Each work item is one band of one strip of one domain;
// every domain reads its buffer `parity` and writes the other one.  Domains
// share the storage type, the omega == 1 property and the presence of a kappa
// field (a uniform kappa is passed as a filled field).  With queue == null,
// CTA i takes item i (the hardware block scheduler is the work queue); else
// the grid is persistent and each CTA takes items from the counter queue[0]
// until they run out, and the last CTA to finish resets queue[0..1] to zero
// for the next launch.  No CTA ever waits on another.
template <typename SM, typename T, int BX, bool OMEGA1, bool KFIELD>
__device__ __forceinline__ void batch_item(const BatchItem it, const BatchDomain<T>* __restrict__ doms,
                                           int parity)
{
    const BatchDomain<T>& D = doms[it.dom];
    const Geom G = D.G;
    Consts<T> C = D.C;
    C.flip = parity;
    const void* fin = D.buf[parity];
    void* fout = D.buf[parity ^ 1];
    const T* f0 = (const T*)fin;
    const SM* fm = (const SM*)((const char*)fin + G.plane * sizeof(T));
    T* g0 = (T*)fout;
    SM* gm = (SM*)((char*)fout + G.plane * sizeof(T));
    step_band<SM, T, BX, OMEGA1, KFIELD>(f0, fm, g0, gm, D.kappa, G, C, it.strip, it.band, it.nbands);
}

template <typename SM, typename T, int BX, bool OMEGA1, bool KFIELD>
__global__ void __launch_bounds__(BX, sizeof(T) == 4 ? 1024 / BX : 1)
k_step_batch(const BatchItem* __restrict__ items, int nitems, const BatchDomain<T>* __restrict__ doms,
             int parity, int* queue)
{
    dependent_launch_entry();
    if (!queue) {
        batch_item<SM, T, BX, OMEGA1, KFIELD>(items[blockIdx.x], doms, parity);
        return;
    }
    __shared__ int next;
    for (;;) {
        __syncthreads();  // the previous item is done with the shared rings and with `next`
        if (threadIdx.x == 0) next = atomicAdd(queue, 1);
        __syncthreads();
        const int i = next;
        if (i >= nitems) break;
        batch_item<SM, T, BX, OMEGA1, KFIELD>(items[i], doms, parity);
    }
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(queue + 1, 1) == (int)gridDim.x - 1) {  // every CTA has taken its last item
            queue[0] = 0;
            queue[1] = 0;
        }
    }
}

// ---------------------------------------------------------------------------
// Kernel 2: the nine row segments each march step needs are streamed into
// shared memory by the tensor memory accelerator (cp.async.bulk, one issuing
// thread, completion on an mbarrier), four steps ahead of use; threads read
// their shifted populations from shared memory.  Memory-level parallelism no
// longer depends on registers or on the number of resident warps.

__device__ __forceinline__ uint32_t smem_addr(const void* p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_tx(uint64_t* b, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(b)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_test(uint64_t* b, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(b)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* b)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(b))
        : "memory");
}

constexpr int kStages = 4;  // TMA pipeline depth, in march steps

// Shared-memory layout of one pipeline stage: plane 0 (compute type) then the
// 8 moving planes (storage type), LMAX elements each.  LMAX covers the
// segment [x0-3, x0+W+3) rounded out to 16-byte boundaries.
template <typename SM, typename T, int BX>
struct TmaLayout {
    static constexpr int A = 16 / (sizeof(SM) < sizeof(T) ? sizeof(SM) : sizeof(T));
    static constexpr int LMAX = BX + 16;
    static constexpr int B0 = LMAX * (int)sizeof(T);
    static constexpr int BM = LMAX * (int)sizeof(SM);
    static constexpr int STAGE = (B0 + 8 * BM + 127) / 128 * 128;
    static constexpr int BYTES = kStages * STAGE;
    static_assert(B0 % 16 == 0 && BM % 16 == 0, "stage planes must stay 16-byte aligned");
};

__device__ __forceinline__ int floor_div(int a, int b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }

// Bulk copies of one march step, issued by warp 0: lane 0 arms the stage's
// mbarrier with the byte count, then lane l (0..8) copies plane l from row
// y - c_ly, lattice columns [a0, a1), into its slot of the stage.  Columns
// outside [0, nx) come from the periodic images, so a segment is copied in up
// to three pieces (the host only selects this kernel when nx is a multiple of
// 8 elements, which keeps every piece 16-byte aligned).
template <typename SM, typename T>
__device__ __noinline__ void issue_step(unsigned char* stage, uint64_t* bar, const T* fin0,
                                        const SM* finm, int plane, int pitch, int nx, int ny, int row,
                                        int a0, int a1, int b0, int bm, uint32_t bytes, int* status)
{
    const int lane = threadIdx.x & 31;
    // the periodic images taken left and right of the row must lie in it
    TFLBM_CHECK(a0 >= -nx && a1 <= 2 * nx && a0 < a1, status);
    (void)status;
    if (lane == 0) mbar_arrive_tx(bar, bytes);
    __syncwarp();
    if (lane < 9) {
        // c_ly of population l: 0 0 1 1 1 0 -1 -1 -1
        const int cy = (lane >= 2 && lane <= 4) ? 1 : (lane >= 6 ? -1 : 0);
        int r = row - cy;
        r = r < 0 ? r + ny : (r >= ny ? r - ny : r);
        const char* src;
        int es;
        unsigned char* dst;
        if (lane == 0) {
            src = reinterpret_cast<const char*>(fin0 + (long long)r * pitch);
            es = (int)sizeof(T);
            dst = stage;
        } else {
            src = reinterpret_cast<const char*>(finm + ((long long)(lane - 1) * plane + (long long)r * pitch));
            es = (int)sizeof(SM);
            dst = stage + b0 + (lane - 1) * bm;
        }
        int c = a0;
        if (c < 0) {  // left periodic image
            bulk_g2s(dst, src + (long long)(c + nx) * es, (uint32_t)(-c * es), bar);
            dst += -c * es;
            c = 0;
        }
        const int e = a1 < nx ? a1 : nx;
        bulk_g2s(dst, src + (long long)c * es, (uint32_t)((e - c) * es), bar);
        dst += (e - c) * es;
        if (a1 > nx) bulk_g2s(dst, src, (uint32_t)((a1 - nx) * es), bar);  // right image
    }
}

template <typename SM, typename T, int BX, bool OMEGA1, bool KFIELD>
__global__ void __launch_bounds__(BX, (OMEGA1 && sizeof(T) == 4) ? 1024 / BX : 1)
k_step_tma(const T* __restrict__ fin0, const SM* __restrict__ finm, T* __restrict__ fout0,
           SM* __restrict__ foutm, const T* __restrict__ kappa, const Geom G, const Consts<T> C)
{
    dependent_launch_entry();
    using L = TmaLayout<SM, T, BX>;
    extern __shared__ __align__(128) unsigned char stage_mem[];
    __shared__ T hsm[4][BX];  // h - href ring: slot t = column x0 - 2 + t
    __shared__ T psm[4][BX];  // p ring, same columns
    __shared__ __align__(8) uint64_t bars[kStages];

    const int t = threadIdx.x;
    const int nx = G.nx, ny = G.ny, pitch = G.pitch, plane = (int)G.plane;
    const Band B = make_band<BX>(G, t, blockIdx.x, blockIdx.y, gridDim.y, C.flip);
    const bool disj = KFIELD || C.kappa_u != T(0);
    const int dir = B.dir, R = B.R;
    const int x = wrap_index(B.x0 - 2 + t, nx);

    // the row segment [a0, a1) copied per plane; column X sits at X - a0
    const int a0 = floor_div(B.x0 - 3, L::A) * L::A;
    const int a1 = (B.x0 + B.weff + 3 + L::A - 1) / L::A * L::A;
    const int col = t + B.x0 - 2 - a0;
    const uint32_t bytes_step = (uint32_t)(a1 - a0) * (uint32_t)(sizeof(T) + 8 * sizeof(SM));
    auto issue = [&](int j) {  // march step j (h row r(j)) into stage j % kStages
        const int st = j & (kStages - 1);
        issue_step<SM, T>(stage_mem + st * L::STAGE, &bars[st], fin0, finm, plane, pitch, nx, ny,
                          wrap_index(B.rstart + j * dir, ny), a0, a1, L::B0, L::BM, bytes_step, C.status);
    };
    bool gave_up = false;  // this thread stopped waiting for a stage

    if (t == 0) {
#pragma unroll
        for (int s = 0; s < kStages; ++s) mbar_init(&bars[s], 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (t < 32)
        for (int j = 0; j < kStages && j <= R + 3; ++j) issue(j);

    int wk = wrap_index(B.rstart, ny);  // wrapped index of row r(k)
    T kap_n = C.kappa_u;
    const long long nkap = (long long)nx * ny;  // kappa field extent
    (void)nkap;
    if (KFIELD && B.pcol) kap_n = kappa[TFLBM_IDX((long long)wrap_index(B.rstart - dir, ny) * nx + x, nkap, C.status)];
    T fv[4][9];
    T jxv[4], jyv[4], ihv[4], erv[4];
#pragma unroll
    for (int s = 0; s < 4; ++s) { jxv[s] = jyv[s] = ihv[s] = erv[s] = T(0); }

    // one march step; false when the CTA gave up waiting for a bulk copy
    auto body = [&](auto stage_c, int k) -> bool {
        constexpr int s = decltype(stage_c)::value;  // ring slot and pipeline stage of row r(k)
        constexpr int s1 = (s + 3) & 3;              // slot of row r(k-1)
        constexpr int s2 = (s + 2) & 3;              // slot of row r(k-2)
        constexpr int s3 = (s + 1) & 3;              // slot of row r(k-3)
        const T kap = kap_n;                         // kappa of row r(k-1)
        // ---- (A) h of row r(k) from the stage that holds its pulled rows
        if (k <= R + 3 && B.hcol) {
            const uint32_t parity = (uint32_t)(k / kStages) & 1u;
            if (C.wait_limit <= 0) {
                gave_up = true;
            } else {
                int it = 0;
                while (!mbar_test(&bars[s], parity)) {
                    if (++it >= C.wait_limit) {
                        gave_up = true;
                        break;
                    }
                }
            }
            if (!gave_up) {
                const unsigned char* base = stage_mem + s * L::STAGE;
                const T* p0 = reinterpret_cast<const T*>(base);
                const SM* pm = reinterpret_cast<const SM*>(base + L::B0);
                constexpr int M = L::LMAX;
                // population l at column X comes from X - c_lx
                T v[9];
                // the stage holds M columns per plane; col - 1 .. col + 1 are read
                TFLBM_CHECK(col >= 1 && col + 1 < M, C.status);
                const int cc = TFLBM_IDX(col, M, C.status);
                v[0] = p0[cc];
                v[1] = load_moving(pm[0 * M + cc - 1], 1, C);
                v[2] = load_moving(pm[1 * M + cc - 1], 2, C);
                v[3] = load_moving(pm[2 * M + cc], 3, C);
                v[4] = load_moving(pm[3 * M + cc + 1], 4, C);
                v[5] = load_moving(pm[4 * M + cc + 1], 5, C);
                v[6] = load_moving(pm[5 * M + cc + 1], 6, C);
                v[7] = load_moving(pm[6 * M + cc], 7, C);
                v[8] = load_moving(pm[7 * M + cc - 1], 8, C);
                hsm[s][t] = sum9(v, erv[s]);
                jxv[s] = ((v[1] + v[2]) + v[8]) - ((v[4] + v[5]) + v[6]);
                jyv[s] = ((v[2] + v[3]) + v[4]) - ((v[6] + v[7]) + v[8]);
                if (!OMEGA1) {
#pragma unroll
                    for (int l = 0; l < 9; ++l) fv[s][l] = v[l];
                }
                if (KFIELD && B.pcol)  // row r(k), used next step
                    kap_n = kappa[TFLBM_IDX((long long)wk * nx + x, nkap, C.status)];
            }
        }
        // every thread is done with this stage (or the CTA gives up): refill
        // it for step k + kStages
        if (__syncthreads_or(gave_up)) return false;
        if (t < 32 && k + kStages <= R + 3) issue(k + kStages);
        // ---- (B1) film pressure of row r(k-1) (needs h rows r(k-2) .. r(k))
        if (B.pcol && k >= 2 && k <= R + 3) {
            const T ih = fdiv(T(1), hsm[s1][t] + C.href);
            ihv[s1] = ih;
            psm[s1][t] = film_pressure(hsm[s], hsm[s1], hsm[s2], t, kap, ih, C, disj, BX);
        }
        // ---- (B2) force, collision and store of row r(k-3)
        if (B.ocol && k >= 5) {
            const int o = B.rstart + (k - 3) * dir;
            collide_store<SM, T, OMEGA1>(dir > 0 ? psm[s2] : psm[s], psm[s3], dir > 0 ? psm[s] : psm[s2], t,
                                         hsm[s3][t], ihv[s3], jxv[s3], jyv[s3], erv[s3], fv[s3],
                                         fout0, foutm, o * pitch, x, plane, C, BX);
        }
        wk += dir;
        wk = wk == ny ? 0 : (wk < 0 ? ny - 1 : wk);
        return true;
    };

    const int last = R + 4;
    int k = 0;
    bool ok = true;
    for (;;) {
        if (!(ok = body(std::integral_constant<int, 0>{}, k))) break;
        if (++k > last) break;
        if (!(ok = body(std::integral_constant<int, 1>{}, k))) break;
        if (++k > last) break;
        if (!(ok = body(std::integral_constant<int, 2>{}, k))) break;
        if (++k > last) break;
        if (!(ok = body(std::integral_constant<int, 3>{}, k))) break;
        if (++k > last) break;
    }

    if (!ok && t == 0) {
        // report, then wait (bounded) for the copies still in flight before
        // the CTA's shared memory is released.  The CTA stopped at step k
        // before issuing step k + kStages, so the last step issued is jmax;
        // no stage is refilled before all threads passed its previous phase,
        // so each stage has at most one unfinished phase: its last issued step.
        if (C.status) atomicOr(C.status, kStatusTimeout);
        const int jmax = min(k + kStages - 1, R + 3);
        for (int s = 0; s < kStages; ++s) {
            if (jmax < s) continue;
            const int jl = jmax - ((jmax - s) % kStages);
            int it = 0;
            while (!mbar_test(&bars[s], (uint32_t)(jl / kStages) & 1u) && ++it < kWaitLimit) {
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Launchers.

template <typename SM, typename T, int BX, bool OM1, bool KF>
cudaError_t launch_one(int pipeline, dim3 grid, const T* fin0, const SM* finm, T* fout0, SM* foutm,
                       const T* kappa, const Geom& G, const Consts<T>& C, cudaStream_t st)
{
    if (pipeline == kPipeTma) {
        using L = TmaLayout<SM, T, BX>;
        static bool attr = false;  // one attribute call per instantiation
        if (!attr) {
            cudaError_t e = cudaFuncSetAttribute(k_step_tma<SM, T, BX, OM1, KF>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, L::BYTES);
            if (e != cudaSuccess) return e;
            attr = true;
        }
        return launch_dependent(k_step_tma<SM, T, BX, OM1, KF>, grid, BX, L::BYTES, st, fin0, finm, fout0, foutm,
                                kappa, G, C);
    } else if constexpr (std::is_same<SM, T>::value) {
        if (pipeline == kPipeAsync)
            return launch_dependent(k_step<SM, T, BX, OM1, KF, true>, grid, BX, 0, st, fin0, finm, fout0, foutm,
                                    kappa, G, C);
        return launch_dependent(k_step<SM, T, BX, OM1, KF>, grid, BX, 0, st, fin0, finm, fout0, foutm, kappa, G, C);
    }
    return launch_dependent(k_step<SM, T, BX, OM1, KF>, grid, BX, 0, st, fin0, finm, fout0, foutm, kappa, G, C);
}

template <typename SM, typename T, int BX>
cudaError_t launch_step_bx(int pipeline, const T* fin0, const SM* finm, T* fout0, SM* foutm,
                           const T* kappa, const Geom& G, const Consts<T>& C, int bands, cudaStream_t st)
{
    dim3 grid((G.nx + BX - 5) / (BX - 4), bands);
    const bool om1 = (C.omega == T(1));
    if (kappa) {
        if (om1) return launch_one<SM, T, BX, true, true>(pipeline, grid, fin0, finm, fout0, foutm, kappa, G, C, st);
        return launch_one<SM, T, BX, false, true>(pipeline, grid, fin0, finm, fout0, foutm, kappa, G, C, st);
    }
    if (om1) return launch_one<SM, T, BX, true, false>(pipeline, grid, fin0, finm, fout0, foutm, kappa, G, C, st);
    return launch_one<SM, T, BX, false, false>(pipeline, grid, fin0, finm, fout0, foutm, kappa, G, C, st);
}

template <typename SM, typename T, int BX, bool OM1, bool KF>
cudaError_t batch_one(const BatchLaunch& L, cudaStream_t st)
{
    const BatchDomain<T>* d = (const BatchDomain<T>*)L.doms;
    if (L.query_occupancy) {
        int n = 0;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_step_batch<SM, T, BX, OM1, KF>, BX, 0);
        *L.query_occupancy = e == cudaSuccess ? n : 0;
        return e;
    }
    return launch_dependent(k_step_batch<SM, T, BX, OM1, KF>, dim3(L.grid), BX, 0, st, L.items, L.nitems, d, L.parity,
                            L.queue);
}

template <typename SM, typename T, int BX>
cudaError_t batch_bx(const BatchLaunch& L, cudaStream_t st)
{
    if (L.kfield) return L.omega1 ? batch_one<SM, T, BX, true, true>(L, st) : batch_one<SM, T, BX, false, true>(L, st);
    return L.omega1 ? batch_one<SM, T, BX, true, false>(L, st) : batch_one<SM, T, BX, false, false>(L, st);
}

template <typename SM, typename T>
cudaError_t launch_batch_typed(const BatchLaunch& L, cudaStream_t st)
{
    switch (L.block_x) {
        case 64: return batch_bx<SM, T, 64>(L, st);
        case 128: return batch_bx<SM, T, 128>(L, st);
        case 256: return batch_bx<SM, T, 256>(L, st);
        default: return cudaErrorInvalidValue;
    }
}

// Resident CTAs per SM of one instantiation (for sizing the grid).
template <typename SM, typename T, int BX, bool OM1, bool KF>
int bps_one(int pipeline)
{
    int n = 0;
    cudaError_t e;
    if (pipeline == kPipeTma) {
        using L = TmaLayout<SM, T, BX>;
        cudaFuncSetAttribute(k_step_tma<SM, T, BX, OM1, KF>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             L::BYTES);
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_step_tma<SM, T, BX, OM1, KF>, BX, L::BYTES);
    } else if constexpr (std::is_same<SM, T>::value) {
        if (pipeline == kPipeAsync)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_step<SM, T, BX, OM1, KF, true>, BX, 0);
        else
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_step<SM, T, BX, OM1, KF>, BX, 0);
    } else {
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_step<SM, T, BX, OM1, KF>, BX, 0);
    }
    return e == cudaSuccess ? n : 0;
}

template <typename SM, typename T, int BX>
int blocks_per_sm_bx(int pipeline, bool omega1, bool kfield)
{
    if (kfield) return omega1 ? bps_one<SM, T, BX, true, true>(pipeline) : bps_one<SM, T, BX, false, true>(pipeline);
    return omega1 ? bps_one<SM, T, BX, true, false>(pipeline) : bps_one<SM, T, BX, false, false>(pipeline);
}

}  // namespace tflbm
