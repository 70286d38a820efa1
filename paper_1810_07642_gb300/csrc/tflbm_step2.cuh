// Paired-column fused step: the same time step as step_band (Section II of
// Zitz et al., arXiv:1810.07642: Eqs. LBE, equilibria, force, pfilm,
// disjoiningP, forcefric, alphafric, derivative, n_laplace), arranged so that
// each thread owns two adjacent lattice columns.
//
// Why: the one-column kernel issues about ten warp instructions per node and
// is limited by instruction issue, not by HBM.  Two columns per thread halve
// the per-node cost of addressing, loop control and barriers, turn every
// population load and store into one aligned 8-byte (FP32) or 4-byte (16-bit
// pair) access, and let the node arithmetic run on Blackwell's paired FP32
// instructions (two lanes of float math per issued instruction).
//
// Storage units.  16-bit storage keeps v_l = (f_l - R_l) * scale for the
// moving populations (R_l the rest equilibrium at href, scale a power of 2).
// The kernel computes on v_l as decoded (one conversion, no arithmetic):
// sums of moving populations need the R_l only through their total 4 (R_axis
// + R_diag), momenta not at all (the R_l are symmetric), and the collision
// forms (f*_l - R_l) * scale directly, with scale and R_l folded into its
// constants.  FP32 storage is the case scale = 1, R_l = 0.
//
// Streaming without misaligned loads.  Thread t loads the nine planes at its
// own aligned column pair (c, c+1).  Populations with c_x = 0 arrive from the
// same columns.  Those with c_x = +1 (l = 1, 2, 8) arrive from the column to
// the left and those with c_x = -1 (l = 4, 5, 6) from the right, so only one
// value per direction crosses a pair boundary.  At tau = 1 the collision
// needs h and j alone, so each thread first sums the three c_x = +1 and the
// three c_x = -1 populations of its own columns; per row four warp shuffles
// then move those two sums and their y-momenta across the pair boundary
// (general tau: six shuffles of the single values, which the relaxation
// needs).  Lane 0 and lane 31 of every warp read the three elements of their
// outer neighbour column themselves (predicated loads that hit L1/L2).
//
// Stencils.  The h and p rows live in 4-row shared rings at their own
// columns; a thread reads its pair as one aligned 8-byte load and the two
// outer neighbours as single values.  (A second, column-shifted copy of each
// row, which would make the shifted pairs aligned loads too, measured slower:
// its extra stores and shared memory cost more than the register moves they
// save.)
//
// Rows, bands, march direction, the reference-height storage and the exact
// mass folding are those of step_band (tflbm_step.cuh).  Needs nx even
// (pairs never straddle the periodic seam); compute type FP32, storage FP32,
// FP16 or BF16.
#pragma once
#include "tflbm_step.cuh"

namespace tflbm {

// ---- paired FP32 arithmetic (one instruction for both columns) ------------
__device__ __forceinline__ float2 pk(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 padd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 psub(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
__device__ __forceinline__ float2 pmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 pfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// Error-free TwoSum on both lanes: a + b = s + e exactly.
__device__ __forceinline__ void ptwo_sum(float2 a, float2 b, float2& s, float2& e)
{
    s = padd(a, b);
    const float2 bb = psub(s, a);
    e = padd(psub(a, psub(s, bb)), psub(b, bb));
}

// ---- pair storage of the moving populations --------------------------------
// V is one aligned pair of stored values; dec gives them as floats in storage
// units (exact), enc rounds two floats to the storage type, dec1 converts one
// stored element.
template <typename SM> struct PairIO;
template <> struct PairIO<float> {
    using V = float2;
    static __device__ __forceinline__ float2 dec(float2 q) { return q; }
    static __device__ __forceinline__ float2 enc(float2 v) { return v; }
    static __device__ __forceinline__ float dec1(float q) { return q; }
};
template <> struct PairIO<__half> {
    using V = __half2;
    static __device__ __forceinline__ float2 dec(__half2 q) { return __half22float2(q); }
    static __device__ __forceinline__ __half2 enc(float2 v) { return __float22half2_rn(v); }
    static __device__ __forceinline__ float dec1(__half q) { return __half2float(q); }
};
template <> struct PairIO<__nv_bfloat16> {
    using V = __nv_bfloat162;
    static __device__ __forceinline__ float2 dec(__nv_bfloat162 q) { return __bfloat1622float2(q); }
    static __device__ __forceinline__ __nv_bfloat162 enc(float2 v) { return __float22bfloat162_rn(v); }
    static __device__ __forceinline__ float dec1(__nv_bfloat16 q) { return __bfloat162float(q); }
};

template <typename V> __device__ __forceinline__ V ldpair(const V* p) { return __ldg(p); }
template <typename V> __device__ __forceinline__ uint32_t bits(V v)
{
    static_assert(sizeof(V) == 4, "16-bit pairs only");
    uint32_t u;
    memcpy(&u, &v, 4);
    return u;
}
template <typename V> __device__ __forceinline__ V from_bits(uint32_t u)
{
    V v;
    memcpy(&v, &u, 4);
    return v;
}
__device__ __forceinline__ float2 lds2(const float* p) { return *reinterpret_cast<const float2*>(p); }

// acc += the two stored values of q, each added to its lane in FP32 by the
// mixed-precision add of sm_100 and later (16-bit operand, FP32 sum, one
// rounding)
template <typename SM> __device__ __forceinline__ void mixed_add(float2& acc, typename PairIO<SM>::V q);
template <> __device__ __forceinline__ void mixed_add<__half>(float2& acc, __half2 q)
{
    unsigned short lo, hi;
    asm("mov.b32 {%0, %1}, %2;" : "=h"(lo), "=h"(hi) : "r"(bits(q)));
    asm("add.rn.f32.f16 %0, %1, %0;" : "+f"(acc.x) : "h"(lo));
    asm("add.rn.f32.f16 %0, %1, %0;" : "+f"(acc.y) : "h"(hi));
}
template <> __device__ __forceinline__ void mixed_add<__nv_bfloat16>(float2& acc, __nv_bfloat162 q)
{
    unsigned short lo, hi;
    asm("mov.b32 {%0, %1}, %2;" : "=h"(lo), "=h"(hi) : "r"(bits(q)));
    asm("add.rn.f32.bf16 %0, %1, %0;" : "+f"(acc.x) : "h"(lo));
    asm("add.rn.f32.bf16 %0, %1, %0;" : "+f"(acc.y) : "h"(hi));
}

// The nine pairs of one 3 x 4 stencil window of a shared row triple: for
// each of the rows n (+y), c, s (-y) the pair at the thread's own columns
// (x, x+1) and the shifted pairs (x-1, x) and (x+1, x+2).
struct Win {
    float2 n0, nL, nR, c0, cL, cR, s0, sL, sR;
};
// rows n, c, s of a ring; j is the slot of the pair's first column
__device__ __forceinline__ Win load_win(const float* rn, const float* rc, const float* rs, int j)
{
    Win w;
    w.n0 = lds2(rn + j); w.nL = make_float2(rn[j - 1], w.n0.x); w.nR = make_float2(w.n0.y, rn[j + 2]);
    w.c0 = lds2(rc + j); w.cL = make_float2(rc[j - 1], w.c0.x); w.cR = make_float2(w.c0.y, rc[j + 2]);
    w.s0 = lds2(rs + j); w.sL = make_float2(rs[j - 1], w.s0.x); w.sR = make_float2(w.s0.y, rs[j + 2]);
    return w;
}

// ---------------------------------------------------------------------------
// Node arithmetic.

// Film pressure (Eq. pfilm with Eq. disjoiningP) of the two nodes from the h
// window; writes 1/h to ih.
__device__ __forceinline__ float2 pair_pressure(const Win& H, float2 kap, bool disj, const Consts<float>& C,
                                                float2& ih)
{
    // Eq. (n_laplace): axis neighbours left + right + up + down, diagonal the four corners
    const float2 axis = padd(padd(H.cL, H.cR), padd(H.n0, H.s0));
    const float2 diag = padd(padd(H.nL, H.nR), padd(H.sL, H.sR));
    float2 lap = pmul(pfma(pk(4.0f), axis, pfma(pk(-20.0f), H.c0, diag)), pk(1.0f / 6.0f));
    const float2 h = padd(H.c0, pk(C.href));
    ih = make_float2(__fdividef(1.0f, h.x), __fdividef(1.0f, h.y));
    if (disj) {
        const float2 r = pmul(pk(C.hstar), ih);
        float2 fd;
        if (C.n_exp == 3 && C.m_exp == 2) fd = pmul(pmul(r, r), psub(r, pk(1.0f)));
        else fd = make_float2(fdisj(r.x, C.n_exp, C.m_exp), fdisj(r.y, C.n_exp, C.m_exp));
        lap = pfma(pmul(pk(C.pi_sgn), kap), fd, lap);
    }
    return pmul(pk(-C.gamma), lap);
}

// Force, collision and store of the two nodes (the arithmetic of
// collide_store on both lanes, in storage units).  P: the p window around
// the pair (n = row o+1, s = row o-1); f: the pulled moving populations in
// storage units (omega != 1 only); i: the storage offset of the pair's first
// column.
template <typename SM, bool OMEGA1>
__device__ __forceinline__ void pair_collide_store(const Win& P, float2 dh, float2 ih, float2 jx, float2 jy,
                                                   float2 er, const float2* f, int fstride,
                                                   float* __restrict__ fout0, SM* __restrict__ foutm, int i,
                                                   int plane, const Consts<float>& C)
{
    using IO = PairIO<SM>;
    using V = typename IO::V;
    constexpr bool NARROW = !std::is_same<SM, float>::value;
    // storage scale (1 for FP32, a compile-time constant there)
    const float ms = NARROW ? C.mscale : 1.0f;
    // Eq. (derivative): grad p = 3 sum_l w_l c_l p(x + c_l)
    const float2 gpx = pfma(psub(P.cR, P.cL), pk(1.0f / 3.0f),
                            pmul(padd(psub(P.nR, P.nL), psub(P.sR, P.sL)), pk(1.0f / 12.0f)));
    const float2 gpy = pfma(psub(P.n0, P.s0), pk(1.0f / 3.0f),
                            pmul(padd(psub(P.nR, P.sR), psub(P.nL, P.sL)), pk(1.0f / 12.0f)));
    const float2 h = padd(dh, pk(C.href));
    // Eqs. (force), (forcefric), (alphafric): nu alpha u = 6 nu j / (2h^2 + 6 delta h + 3 delta^2)
    const float2 den = pfma(h, pfma(pk(2.0f), h, pk(6.0f * C.delta)), pk(3.0f * C.delta * C.delta));
    const float2 fr = pmul(pk(C.nu6), make_float2(__fdividef(1.0f, den.x), __fdividef(1.0f, den.y)));
    // Eq. (LBE) as printed: u = j/h.  Second-order forcing (C.forcing):
    // u (h + nu alpha/2) = j + F'/2 and the equilibria use h u for j (see
    // collide_store)
    float2 Fx, Fy, ux, uy, ex, ey;
    if (C.forcing) {
        const float2 fpx = pmul(h, psub(pk(C.gx), gpx)), fpy = pmul(h, psub(pk(C.gy), gpy));
        const float2 d = pfma(pk(0.5f), fr, pk(1.0f));
        const float2 q = make_float2(__fdividef(ih.x, d.x), __fdividef(ih.y, d.y));
        ux = pmul(pfma(pk(0.5f), fpx, jx), q);
        uy = pmul(pfma(pk(0.5f), fpy, jy), q);
        ex = pmul(h, ux);
        ey = pmul(h, uy);
        Fx = psub(fpx, pmul(fr, ex));
        Fy = psub(fpy, pmul(fr, ey));
    } else {
        Fx = psub(pmul(h, psub(pk(C.gx), gpx)), pmul(fr, jx));
        Fy = psub(pmul(h, psub(pk(C.gy), gpy)), pmul(fr, jy));
        ux = pmul(jx, ih);
        uy = pmul(jy, ih);
        ex = jx;
        ey = jy;
    }
    // Eq. (equilibria) with e^2 = 1 as S +- D per opposite pair, source
    // 3 w_l c_l . F; in storage units S' = (S - R_l) ms, D' = D ms.
    // A6 = 6 A = h (g h - u^2).
    const float2 A6 = pmul(h, psub(pmul(pk(C.g), h), pfma(ux, ux, pmul(uy, uy))));
    const float2 Aa = NARROW ? pfma(A6, pk(ms * (1.0f / 6.0f)), pk(C.nr_axis)) : pmul(A6, pk(1.0f / 6.0f));
    const float2 Ad = NARROW ? pfma(A6, pk(ms * (1.0f / 24.0f)), pk(C.nr_diag)) : pmul(A6, pk(1.0f / 24.0f));
    float2 Sx = pfma(pmul(ex, pk(0.5f * ms)), ux, Aa);
    float2 Sy = pfma(pmul(ey, pk(0.5f * ms)), uy, Aa);
    const float2 a = padd(ux, uy), b = psub(uy, ux);
    const float2 h8 = pmul(h, pk(0.125f * ms));
    float2 Sa = pfma(pmul(h8, a), a, Ad);
    float2 Sb = pfma(pmul(h8, b), b, Ad);
    // second-order source: odd part scaled by (1 - omega/2), even part T
    float2 Tx = pk(0.0f), Ty = pk(0.0f), Ta = pk(0.0f), Tb = pk(0.0f);
    if (C.forcing) {
        const float2 ks = pk(1.0f - 0.5f * C.omega);
        Fx = pmul(Fx, ks);
        Fy = pmul(Fy, ks);
        const float2 uF3 = pmul(pfma(ux, Fx, pmul(uy, Fy)), pk(ms * (1.0f / 3.0f)));
        Tx = pfma(pmul(ux, Fx), pk(ms), make_float2(-uF3.x, -uF3.y));
        Ty = pfma(pmul(uy, Fy), pk(ms), make_float2(-uF3.x, -uF3.y));
        Ta = pmul(pfma(pmul(a, padd(Fx, Fy)), pk(ms), make_float2(-uF3.x, -uF3.y)), pk(0.25f));
        Tb = pmul(pfma(pmul(b, psub(Fy, Fx)), pk(ms), make_float2(-uF3.x, -uF3.y)), pk(0.25f));
        if constexpr (OMEGA1) {
            Sx = padd(Sx, Tx);
            Sy = padd(Sy, Ty);
            Sa = padd(Sa, Ta);
            Sb = padd(Sb, Tb);
        }
    }
    const float2 m3 = pk(ms * (1.0f / 3.0f)), m12 = pk(ms * (1.0f / 12.0f));
    float2 o1, o2, o3, o4, o5, o6, o7, o8;
    if constexpr (OMEGA1) {
        const float2 Gx = padd(ex, Fx), Gy = padd(ey, Fy);
        const float2 Dx = pmul(Gx, m3), Dy = pmul(Gy, m3);
        const float2 Da = pmul(padd(Gx, Gy), m12), Db = pmul(psub(Gy, Gx), m12);
        o1 = padd(Sx, Dx); o5 = psub(Sx, Dx);
        o3 = padd(Sy, Dy); o7 = psub(Sy, Dy);
        o2 = padd(Sa, Da); o6 = psub(Sa, Da);
        o4 = padd(Sb, Db); o8 = psub(Sb, Db);
    } else {
        // (1 - omega)(f_l - R_l) + omega (f_eq_l - R_l) + source, in storage units
        const float2 w = pk(C.omega), m = pk(1.0f - C.omega);
        const float2 Dx = pmul(ex, m3), Dy = pmul(ey, m3);
        const float2 Da = pmul(padd(ex, ey), m12), Db = pmul(psub(ey, ex), m12);
        const float2 Qx = pmul(Fx, m3), Qy = pmul(Fy, m3);
        const float2 Qa = pmul(padd(Fx, Fy), m12), Qb = pmul(psub(Fy, Fx), m12);
        o1 = padd(pfma(m, f[0 * fstride], pmul(w, padd(Sx, Dx))), padd(Tx, Qx));
        o5 = padd(pfma(m, f[4 * fstride], pmul(w, psub(Sx, Dx))), psub(Tx, Qx));
        o3 = padd(pfma(m, f[2 * fstride], pmul(w, padd(Sy, Dy))), padd(Ty, Qy));
        o7 = padd(pfma(m, f[6 * fstride], pmul(w, psub(Sy, Dy))), psub(Ty, Qy));
        o2 = padd(pfma(m, f[1 * fstride], pmul(w, padd(Sa, Da))), padd(Ta, Qa));
        o6 = padd(pfma(m, f[5 * fstride], pmul(w, psub(Sa, Da))), psub(Ta, Qa));
        o4 = padd(pfma(m, f[3 * fstride], pmul(w, padd(Sb, Db))), padd(Tb, Qb));
        o8 = padd(pfma(m, f[7 * fstride], pmul(w, psub(Sb, Db))), psub(Tb, Qb));
    }
    // stored rest population f*_0 - href = (h - href) - sum_{l>0} f*_l, with
    // the exact residuals folded back as in collide_store
    const int hp = plane >> 1;  // pairs per plane
    // the pair (i, i+1) of plane 0 and of the eight moving planes
    TFLBM_CHECK(i >= 0 && (i & 1) == 0 && i + 1 < plane, C.status);
    const int ip = TFLBM_IDX(i >> 1, hp, C.status);
    V* om = reinterpret_cast<V*>(foutm) + ip;
    if constexpr (!NARROW) {
        const float2 osum = padd(padd(padd(o1, o5), padd(o3, o7)), padd(padd(o2, o6), padd(o4, o8)));
        float2 o0v, e2;
        ptwo_sum(dh, make_float2(-osum.x, -osum.y), o0v, e2);
        const float2 half_r = pmul(padd(er, e2), pk(0.5f));
        o1 = padd(o1, half_r);
        o5 = padd(o5, half_r);
        reinterpret_cast<float2*>(fout0)[ip] = o0v;
        om[0] = o1; om[hp] = o2; om[2 * hp] = o3; om[3 * hp] = o4;
        om[4 * hp] = o5; om[5 * hp] = o6; om[6 * hp] = o7; om[7 * hp] = o8;
    } else {
        const V q2 = IO::enc(o2), q3 = IO::enc(o3), q4 = IO::enc(o4), q5 = IO::enc(o5);
        const V q6 = IO::enc(o6), q7 = IO::enc(o7), q8 = IO::enc(o8), q1r = IO::enc(o1);
        // what the readers reconstruct of l = 2..8 (storage units; each
        // stored value enters the FP32 sum by a mixed-precision add, which
        // takes the 16-bit operand as it is: one instruction per value
        // instead of a conversion and half a paired add)
        float2 rest = IO::dec(q2);
        mixed_add<SM>(rest, q3);
        mixed_add<SM>(rest, q4);
        mixed_add<SM>(rest, q5);
        mixed_add<SM>(rest, q6);
        mixed_add<SM>(rest, q7);
        mixed_add<SM>(rest, q8);
        float2 rest1 = rest;
        mixed_add<SM>(rest1, q1r);
        // the moving populations' total with f_1 unrounded and rounded
        const float2 osum = pfma(padd(rest, o1), pk(C.minv), pk(C.r_sum));
        const float2 osr = pfma(rest1, pk(C.minv), pk(C.r_sum));
        // the last residual goes to the finer of the two roundings: the 16-bit
        // one of f_1 - R or the FP32 one of f_0 - href (see collide_store)
        constexpr float kRatio = std::is_same<SM, __half>::value ? 8192.0f : 65536.0f;
        const float kr = kRatio * C.minv;  // |f_1 - R| = |o1| / ms
        const bool lx = fabsf(o1.x) * kr < fabsf(dh.x - osum.x);
        const bool ly = fabsf(o1.y) * kr < fabsf(dh.y - osum.y);
        const float2 os = make_float2(lx ? osum.x : osr.x, ly ? osum.y : osr.y);
        float2 o0v, e2, o0n, e3;
        ptwo_sum(dh, make_float2(-os.x, -os.y), o0v, e2);
        ptwo_sum(o0v, padd(er, e2), o0n, e3);
        const V q1l = IO::enc(pfma(e3, pk(ms), o1));
        const uint32_t mask = (lx ? 0x0000ffffu : 0u) | (ly ? 0xffff0000u : 0u);
        const V q1 = from_bits<V>((bits(q1l) & mask) | (bits(q1r) & ~mask));
        reinterpret_cast<float2*>(fout0)[ip] = o0n;
        om[0] = q1; om[hp] = q2; om[2 * hp] = q3; om[3 * hp] = q4;
        om[4 * hp] = q5; om[5 * hp] = q6; om[6 * hp] = q7; om[7 * hp] = q8;
    }
}

// ---------------------------------------------------------------------------
// One CTA of BX threads covers NC = 2 BX consecutive columns x0-2 .. x0+NC-3
// (thread t: local columns j = 2t, 2t+1) and marches down a band of rows;
// neighbouring CTAs overlap by 4 columns and each stores NC - 4.  The march
// is step_band's: step k forms h of row r(k) into a 4-row shared ring, one
// barrier, then the pressure of row r(k-1) and force, collision and store of
// row r(k-3).  The pulled values of row r(k) come from registers loaded
// one or two rows ahead, plus warp shuffles for the values that cross a pair
// boundary.
template <typename SM, int BX, bool OMEGA1, bool KFIELD>
__device__ __forceinline__ void step_band2(const float* __restrict__ fin0, const SM* __restrict__ finm,
                                           float* __restrict__ fout0, SM* __restrict__ foutm,
                                           const float* __restrict__ kappa, const Geom& G,
                                           const Consts<float>& C, int strip, int band, int nbands)
{
    using IO = PairIO<SM>;
    using V = typename IO::V;
    constexpr bool NARROW = !std::is_same<SM, float>::value;
    constexpr int NC = 2 * BX;  // columns per CTA
    constexpr int W = NC - 4;   // output columns per CTA
    constexpr int OFF = 2;      // ring slot of local column j is OFF + j (keeps pairs 8-byte aligned)
    constexpr int RW = NC + 4;  // ring row width
    // h - href and the film pressure (slot OFF + j: local column j)
    __shared__ __align__(16) float hsm[4][RW];
    __shared__ __align__(16) float psm[4][RW];
    // general tau: the eight pulled moving populations of the last four rows
    __shared__ __align__(16) float2 fsm[OMEGA1 ? 1 : 4][8][OMEGA1 ? 1 : BX];
    // per-thread rings of (j_x, j_y), the pull-sum residual and 1/h of the
    // last four rows (each thread reads back only its own slots)
    __shared__ __align__(16) float4 rsj[4][BX];
    __shared__ __align__(16) float2 rse[4][BX], rsi[4][BX];

    const int t = threadIdx.x, lane = t & 31;
    const int nx = G.nx, ny = G.ny, pitch = G.pitch, plane = (int)G.plane;
    const int x0 = strip * W;
    const int weff = min(W, nx - x0);     // output columns of this CTA (even)
    const bool pcol = 2 * t <= weff + 2;  // p needed at local columns 1 .. weff+2
    const bool ocol = t >= 1 && 2 * t <= weff;
    const int ybeg = (int)(((long long)band * ny) / nbands);
    const int yend = (int)(((long long)(band + 1) * ny) / nbands);
    const int dir = ((band + C.flip) & 1) ? -1 : 1;  // reversed every other step (see make_band)
    const int R = yend - ybeg;
    const int rstart = dir > 0 ? ybeg - 2 : yend + 1;
    const bool disj = KFIELD || C.kappa_u != 0.0f;
    const int c = wrap_index(x0 - 2 + 2 * t, nx);  // own pair (even)
    const int j2 = OFF + 2 * t;                    // ring slot of the pair

    const bool edge = lane == 0 || lane == 31;
    // the outer neighbour column: c - 1 for lane 0, c + 2 for lane 31
    const int ce = lane == 0 ? (c == 0 ? nx - 1 : c - 1) : (c + 2 == nx ? 0 : c + 2);
    // moving planes (index l - 1) a warp-edge lane reads at that column, from
    // rows y, y-1, y+1: lane 0 needs l = 1, 2, 8 (arriving from the left),
    // lane 31 needs l = 5, 4, 6 (from the right)
    const int e0 = (lane == 0 ? 0 : 4) * plane + ce;
    const int e1 = (lane == 0 ? 1 : 3) * plane + ce;
    const int e2 = (lane == 0 ? 7 : 5) * plane + ce;
    const float2* __restrict__ f0p = reinterpret_cast<const float2*>(fin0);
    const V* __restrict__ fmp = reinterpret_cast<const V*>(finm);
    const int half = plane >> 1;  // pairs per plane (pitch is even)
    // PF rows of loads in flight: 16-bit storage keeps two (rows r(k+1) and
    // r(k+2) go out while step k runs), FP32 one (its registers would
    // otherwise cost resident warps)
    constexpr int PF = NARROW ? 2 : 1;
    float2 q0[PF];
    V qm[PF][8];
    SM qe[PF][3];

    // wrapped rows r(k-1) .. r(k+3)
    int wm1 = wrap_index(rstart - dir, ny), w0 = wrap_index(rstart, ny);
    int w1 = wrap_index(rstart + dir, ny), w2 = wrap_index(rstart + 2 * dir, ny);
    int w3 = wrap_index(rstart + 3 * dir, ny);
    // the nine planes (and the edge elements) pulled into row w, into register set b
    auto load_row = [&](auto b_c, int wb, int w, int wa) {
        constexpr int b = decltype(b_c)::value;
        const int ys = dir > 0 ? wb : wa, yn = dir > 0 ? wa : wb;  // rows y-1, y+1
        const int i0 = (w * pitch + c) >> 1, is = (ys * pitch + c) >> 1, in = (yn * pitch + c) >> 1;
        const long long m8 = 8LL * half;  // pairs of the eight moving planes
        int* st = C.status;
        q0[b] = ldpair(f0p + TFLBM_IDX(i0, half, st));
        qm[b][0] = ldpair(fmp + TFLBM_IDX(i0, m8, st));               // l = 1 from row y
        qm[b][1] = ldpair(fmp + TFLBM_IDX(half + is, m8, st));        // l = 2 from row y-1
        qm[b][2] = ldpair(fmp + TFLBM_IDX(2 * half + is, m8, st));    // l = 3
        qm[b][3] = ldpair(fmp + TFLBM_IDX(3 * half + is, m8, st));    // l = 4
        qm[b][4] = ldpair(fmp + TFLBM_IDX(4 * half + i0, m8, st));    // l = 5 from row y
        qm[b][5] = ldpair(fmp + TFLBM_IDX(5 * half + in, m8, st));    // l = 6 from row y+1
        qm[b][6] = ldpair(fmp + TFLBM_IDX(6 * half + in, m8, st));    // l = 7
        qm[b][7] = ldpair(fmp + TFLBM_IDX(7 * half + in, m8, st));    // l = 8
        if (edge) {
            const long long e8 = 8LL * plane;
            qe[b][0] = ldro(finm + TFLBM_IDX(e0 + w * pitch, e8, st));
            qe[b][1] = ldro(finm + TFLBM_IDX(e1 + ys * pitch, e8, st));
            qe[b][2] = ldro(finm + TFLBM_IDX(e2 + yn * pitch, e8, st));
            (void)e8;
        }
        (void)m8;
        (void)st;
    };

    float2 kap_n = pk(C.kappa_u);
    load_row(std::integral_constant<int, 0>{}, wm1, w0, w1);
    if constexpr (PF == 2) load_row(std::integral_constant<int, 1>{}, w0, w1, w2);
    const long long npair = (long long)nx * ny / 2;  // kappa field extent in pairs (nx even)
    (void)npair;
    if (KFIELD && pcol)
        kap_n = reinterpret_cast<const float2*>(kappa)[TFLBM_IDX(((long long)wm1 * nx + c) >> 1, npair, C.status)];

    // ring slots no thread writes: columns -1 and NC (outer halves of the
    // edge columns' stencils)
    if (t < 2) {
        const int j = t == 0 ? OFF - 1 : OFF + NC;
#pragma unroll
        for (int s = 0; s < 4; ++s) hsm[s][j] = psm[s][j] = 0.0f;
    }

    auto body = [&](auto stage_c, int k) {
        constexpr int s = decltype(stage_c)::value;  // ring slot of row r(k)
        constexpr int s1 = (s + 3) & 3;              // r(k-1)
        constexpr int s2 = (s + 2) & 3;              // r(k-2)
        constexpr int s3 = (s + 1) & 3;              // r(k-3)
        const float2 kap = kap_n;                    // kappa of row r(k-1)
        // ---- (A) h, j of row r(k)
        if (k <= R + 3) {
            constexpr int rb = s % PF;  // register set of row r(k)
            const float2 f0 = q0[rb];   // f_0 - href
            float2 v[8];                // moving populations at the own columns, storage units
#pragma unroll
            for (int l = 0; l < 8; ++l) v[l] = IO::dec(qm[rb][l]);
            // the three crossing populations at the outer column (warp-edge lanes)
            float ea = 0.f, eb = 0.f, ed = 0.f;
            if (edge) {
                ea = IO::dec1(qe[rb][0]);  // l = 1 or 5
                eb = IO::dec1(qe[rb][1]);  // l = 2 or 4
                ed = IO::dec1(qe[rb][2]);  // l = 8 or 6
            }
            // the loads of row r(k+PF) go out before this row's arithmetic;
            // at tau = 1 right after the partial sums, which free the
            // registers they land in (FP32 values are used as loaded), so the
            // loads neither wait for nor copy this row (one box, 2048^2 step:
            // FP32 56.0 -> 52.7 us, long-scoreboard stalls 5.3 -> 3.8 per
            // issue; FP16 46.5 -> 45.3 us, BF16 47.1 -> 45.4 us)
            auto issue_next = [&]() {
                if constexpr (PF == 2) {
                    if (k + 2 <= R + 3) load_row(std::integral_constant<int, rb>{}, w1, w2, w3);
                } else {
                    if (k + 1 <= R + 3) load_row(std::integral_constant<int, rb>{}, w0, w1, w2);
                }
            };
            constexpr bool EARLY = !OMEGA1;
            if constexpr (EARLY) issue_next();
            if (KFIELD && pcol)
                kap_n = reinterpret_cast<const float2*>(kappa)[TFLBM_IDX(((long long)w0 * nx + c) >> 1, npair,
                                                                          C.status)];
            // Rs, Ls: sums of the populations arriving from the left (l = 1,
            // 2, 8) and from the right (l = 4, 5, 6) at the two nodes; tot:
            // all eight; jyr: their y momentum (storage units)
            float2 Rs, Ls, tot, jyr;
            if constexpr (OMEGA1) {
                const float2 Pc = padd(padd(v[0], v[1]), v[7]), Py = psub(v[1], v[7]);
                const float2 Qc = padd(padd(v[4], v[3]), v[5]), Qy = psub(v[3], v[5]);
                const float2 s26 = padd(v[2], v[6]), d26 = psub(v[2], v[6]);
                const float es = (ea + eb) + ed, ey = eb - ed;
                if constexpr (!EARLY) issue_next();
                float pl = __shfl_up_sync(0xffffffffu, Pc.y, 1), pyl = __shfl_up_sync(0xffffffffu, Py.y, 1);
                float qr = __shfl_down_sync(0xffffffffu, Qc.x, 1), qyr = __shfl_down_sync(0xffffffffu, Qy.x, 1);
                if (lane == 0) { pl = es; pyl = ey; }
                if (lane == 31) { qr = es; qyr = ey; }
                Rs = make_float2(pl, Pc.x);
                Ls = make_float2(Qc.y, qr);
                jyr = padd(d26, padd(make_float2(pyl, Py.x), make_float2(Qy.y, qyr)));
                tot = padd(s26, padd(Rs, Ls));
            } else {
                // the single arriving values, kept for the relaxation
                float u1 = __shfl_up_sync(0xffffffffu, v[0].y, 1);
                float u2 = __shfl_up_sync(0xffffffffu, v[1].y, 1);
                float u8 = __shfl_up_sync(0xffffffffu, v[7].y, 1);
                float d5 = __shfl_down_sync(0xffffffffu, v[4].x, 1);
                float d4 = __shfl_down_sync(0xffffffffu, v[3].x, 1);
                float d6 = __shfl_down_sync(0xffffffffu, v[5].x, 1);
                if (lane == 0) { u1 = ea; u2 = eb; u8 = ed; }
                if (lane == 31) { d5 = ea; d4 = eb; d6 = ed; }
                float2 n[8];
                n[0] = make_float2(u1, v[0].x);
                n[1] = make_float2(u2, v[1].x);
                n[2] = v[2];
                n[3] = make_float2(v[3].y, d4);
                n[4] = make_float2(v[4].y, d5);
                n[5] = make_float2(v[5].y, d6);
                n[6] = v[6];
                n[7] = make_float2(u8, v[7].x);
                Rs = padd(padd(n[0], n[1]), n[7]);
                Ls = padd(padd(n[4], n[3]), n[5]);
                jyr = padd(padd(psub(n[2], n[6]), psub(n[1], n[7])), psub(n[3], n[5]));
                tot = padd(padd(n[2], n[6]), padd(Rs, Ls));
#pragma unroll
                for (int l = 0; l < 8; ++l) fsm[s][l][t] = n[l];
            }
            // h - href: the moving total is small, the last addition is
            // error-free (see sum9)
            float2 dh, er, jx, jy;
            if constexpr (NARROW) {
                ptwo_sum(f0, pfma(tot, pk(C.minv), pk(C.r_sum)), dh, er);
                jx = pmul(psub(Rs, Ls), pk(C.minv));
                jy = pmul(jyr, pk(C.minv));
            } else {
                ptwo_sum(f0, tot, dh, er);
                jx = psub(Rs, Ls);
                jy = jyr;
            }
            TFLBM_CHECK(j2 >= OFF && j2 + 1 < RW, C.status);
            *reinterpret_cast<float2*>(&hsm[s][j2]) = dh;
            rsj[s][t] = make_float4(jx.x, jx.y, jy.x, jy.y);
            rse[s][t] = er;
        }
        __syncthreads();
        // ---- (B1) film pressure of row r(k-1) (needs h rows r(k-2) .. r(k))
        if (pcol && k >= 2 && k <= R + 3) {
            // the window reads slots j2 - 1 .. j2 + 2 of rings of RW
            TFLBM_CHECK(j2 >= 1 && j2 + 2 < RW, C.status);
            float2 ih;
            const Win Hw = load_win(hsm[s], hsm[s1], hsm[s2], j2);
            const float2 p = pair_pressure(Hw, kap, disj, C, ih);
            rsi[s1][t] = ih;
            *reinterpret_cast<float2*>(&psm[s1][j2]) = p;
        }
        // ---- (B2) force, collision and store of row r(k-3)
        if (ocol && k >= 5) {
            const int o = rstart + (k - 3) * dir;  // inside [ybeg, yend), no wrap
            TFLBM_CHECK(j2 >= 1 && j2 + 2 < RW && o >= 0 && o < ny, C.status);
            // rows o+1 and o-1 of the p ring
            const int sn = dir > 0 ? s2 : s, ss = dir > 0 ? s : s2;
            const Win Pw = load_win(psm[sn], psm[s3], psm[ss], j2);
            const float2 dh = lds2(&hsm[s3][j2]);
            const float4 jj = rsj[s3][t];
            const float2* fp = nullptr;
            if constexpr (!OMEGA1) fp = &fsm[s3][0][t];
            pair_collide_store<SM, OMEGA1>(Pw, dh, rsi[s3][t], make_float2(jj.x, jj.y), make_float2(jj.z, jj.w),
                                           rse[s3][t], fp, BX, fout0, foutm, o * pitch + c, plane, C);
        }
        wm1 = w0;
        w0 = w1;
        w1 = w2;
        w2 = w3;
        w3 += dir;
        w3 = w3 == ny ? 0 : (w3 < 0 ? ny - 1 : w3);
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

// Register budget: 80 per thread (24 resident warps per SM), at which the
// kernel does not spill (measured faster than 128 registers and 16 warps).
template <typename SM, int BX, bool OMEGA1, bool KFIELD>
__global__ void __launch_bounds__(BX, 768 / BX)
k_step2(const float* __restrict__ fin0, const SM* __restrict__ finm, float* __restrict__ fout0,
        SM* __restrict__ foutm, const float* __restrict__ kappa, const Geom G, const Consts<float> C)
{
    dependent_launch_entry();
    step_band2<SM, BX, OMEGA1, KFIELD>(fin0, finm, fout0, foutm, kappa, G, C, blockIdx.x, blockIdx.y, gridDim.y);
}

// ---------------------------------------------------------------------------
// Batched form: the work items of k_step_batch (a band of a strip of one
// domain; block_x columns per strip in both kernels), each run as
// step_band2 with its domain's geometry and constants.  Every domain reads
// its buffer `parity` and writes the other one; queue as in k_step_batch (a
// persistent grid taking items from a counter, reset by the last CTA; no CTA
// waits on another).  Needs every domain's nx even and the FP32 compute type.
template <typename SM, int BX, bool OMEGA1, bool KFIELD>
__device__ __forceinline__ void batch_item2(const BatchItem it, const BatchDomain<float>* __restrict__ doms,
                                            int parity)
{
    const BatchDomain<float>& D = doms[it.dom];
    const Geom G = D.G;
    Consts<float> C = D.C;
    C.flip = parity;
    const void* fin = D.buf[parity];
    void* fout = D.buf[parity ^ 1];
    const float* f0 = (const float*)fin;
    const SM* fm = (const SM*)((const char*)fin + G.plane * sizeof(float));
    float* g0 = (float*)fout;
    SM* gm = (SM*)((char*)fout + G.plane * sizeof(float));
    step_band2<SM, BX, OMEGA1, KFIELD>(f0, fm, g0, gm, D.kappa, G, C, it.strip, it.band, it.nbands);
}

template <typename SM, int BX, bool OMEGA1, bool KFIELD>
__global__ void __launch_bounds__(BX, 768 / BX)
k_step2_batch(const BatchItem* __restrict__ items, int nitems, const BatchDomain<float>* __restrict__ doms,
              int parity, int* queue)
{
    dependent_launch_entry();
    if (!queue) {
        batch_item2<SM, BX, OMEGA1, KFIELD>(items[blockIdx.x], doms, parity);
        return;
    }
    __shared__ int next;
    for (;;) {
        __syncthreads();  // the previous item is done with the shared rings and with `next`
        if (threadIdx.x == 0) next = atomicAdd(queue, 1);
        __syncthreads();
        const int i = next;
        if (i >= nitems) break;
        batch_item2<SM, BX, OMEGA1, KFIELD>(items[i], doms, parity);
    }
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(queue + 1, 1) == (int)gridDim.x - 1) {  // every CTA has taken its last item
            queue[0] = 0;
            queue[1] = 0;
        }
    }
}

template <typename SM, int BX, bool OM1, bool KF>
cudaError_t batch2_one(const BatchLaunch& L, cudaStream_t st)
{
    const BatchDomain<float>* d = (const BatchDomain<float>*)L.doms;
    if (L.query_occupancy) {
        int n = 0;
        const cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_step2_batch<SM, BX, OM1, KF>, BX, 0);
        *L.query_occupancy = e == cudaSuccess ? n : 0;
        return e;
    }
    return launch_dependent(k_step2_batch<SM, BX, OM1, KF>, dim3(L.grid), BX, 0, st, L.items, L.nitems, d, L.parity,
                            L.queue);
}

// The batched paired step for one storage type (L.block_x columns per CTA).
template <typename SM>
cudaError_t pair_step_batch(const BatchLaunch& L, cudaStream_t st)
{
    auto pick = [&](auto bx_c) {
        constexpr int BX = decltype(bx_c)::value;
        if (L.kfield) return L.omega1 ? batch2_one<SM, BX, true, true>(L, st) : batch2_one<SM, BX, false, true>(L, st);
        return L.omega1 ? batch2_one<SM, BX, true, false>(L, st) : batch2_one<SM, BX, false, false>(L, st);
    };
    switch (L.block_x) {
        case 64: return pick(std::integral_constant<int, 32>{});
        case 128: return pick(std::integral_constant<int, 64>{});
        case 256: return pick(std::integral_constant<int, 128>{});
        default: return cudaErrorInvalidValue;
    }
}

// ---------------------------------------------------------------------------
// Launch of the paired kernel: block_x is the CTA width in columns (64, 128
// or 256), i.e. block_x / 2 threads.

template <typename SM, int BX>
cudaError_t launch_pair_bx(const float* fin0, const SM* finm, float* fout0, SM* foutm, const float* kappa,
                           const Geom& G, const Consts<float>& C, int bands, cudaStream_t st)
{
    constexpr int W = 2 * BX - 4;
    const dim3 grid((G.nx + W - 1) / W, bands);
    const bool om1 = C.omega == 1.0f;
    if (kappa) {
        if (om1) return launch_dependent(k_step2<SM, BX, true, true>, grid, BX, 0, st, fin0, finm, fout0, foutm, kappa, G, C);
        return launch_dependent(k_step2<SM, BX, false, true>, grid, BX, 0, st, fin0, finm, fout0, foutm, kappa, G, C);
    }
    if (om1) return launch_dependent(k_step2<SM, BX, true, false>, grid, BX, 0, st, fin0, finm, fout0, foutm, kappa, G, C);
    return launch_dependent(k_step2<SM, BX, false, false>, grid, BX, 0, st, fin0, finm, fout0, foutm, kappa, G, C);
}

template <typename SM, int BX, bool OM1, bool KF>
int bps_pair_one()
{
    int n = 0;
    const cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_step2<SM, BX, OM1, KF>, BX, 0);
    return e == cudaSuccess ? n : 0;
}

// The paired step for one storage type.
template <typename SM>
cudaError_t pair_step(int block_x, const void* fin, void* fout, const void* kappa, const Geom& G,
                      const Consts<float>& C, int bands, cudaStream_t st)
{
    const float* f0 = (const float*)fin;
    const SM* fm = (const SM*)((const char*)fin + G.plane * sizeof(float));
    float* g0 = (float*)fout;
    SM* gm = (SM*)((char*)fout + G.plane * sizeof(float));
    const float* k = (const float*)kappa;
    switch (block_x) {
        case 64: return launch_pair_bx<SM, 32>(f0, fm, g0, gm, k, G, C, bands, st);
        case 128: return launch_pair_bx<SM, 64>(f0, fm, g0, gm, k, G, C, bands, st);
        case 256: return launch_pair_bx<SM, 128>(f0, fm, g0, gm, k, G, C, bands, st);
        default: return cudaErrorInvalidValue;
    }
}

// Resident CTAs per SM of the paired step for a CTA width (0 if unknown).
template <typename SM>
int pair_blocks_per_sm(int block_x, bool omega1, bool kfield)
{
    auto pick = [&](auto bx_c) {
        constexpr int BX = decltype(bx_c)::value;
        if (kfield) return omega1 ? bps_pair_one<SM, BX, true, true>() : bps_pair_one<SM, BX, false, true>();
        return omega1 ? bps_pair_one<SM, BX, true, false>() : bps_pair_one<SM, BX, false, false>();
    };
    switch (block_x) {
        case 64: return pick(std::integral_constant<int, 32>{});
        case 128: return pick(std::integral_constant<int, 64>{});
        case 256: return pick(std::integral_constant<int, 128>{});
        default: return 0;
    }
}

}  // namespace tflbm
