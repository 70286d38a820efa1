// Paired-column fused step: the same time step as step_band (Section II of
// Zitz et al., arXiv:1810.07642: Eqs. LBE, equilibria, force, pfilm,
// disjoiningP, forcefric, alphafric, derivative, n_laplace), arranged so that
// each thread owns two adjacent lattice columns.
//
// Why: the one-column kernel issues about ten warp instructions per node and
// is limited by instruction issue, not by HBM.  Two columns per thread halve
// the per-node cost of addressing, loop control, shared-memory traffic and
// barriers, turn every population load and store into one aligned 8-byte
// (FP32) or 4-byte (16-bit pair) access, and let the node arithmetic run on
// Blackwell's paired FP32 instructions (two lanes of float math per issued
// instruction).
//
// Streaming without misaligned loads.  Thread t loads the nine planes at its
// own aligned column pair (c, c+1).  Populations with c_x = 0 arrive from the
// same columns.  Those with c_x = +1 (l = 1, 2, 8) arrive from the column to
// the left and those with c_x = -1 (l = 4, 5, 6) from the right, so only one
// value per direction crosses a pair boundary; it comes from the neighbouring
// lane by a warp shuffle.  At tau = 1 only their sums matter (the collision
// needs h and j alone), so per row four shuffles move the partial sums
// R = f1 + f2 + f8, L = f4 + f5 + f6 and their y-momenta.  Lane 0 and lane 31
// of every warp read the three planes of their outer neighbour column
// themselves (predicated loads that hit L1/L2).
//
// Rows, bands, shared rings, the reference-height storage and the exact mass
// folding are those of step_band (tflbm_step.cuh).  Needs nx even (pairs
// never straddle the periodic seam); compute type FP32, storage FP32, FP16 or
// BF16.
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
// V is one aligned pair of stored values; dec gives the two stored values as
// floats, enc rounds two floats to the storage type.
template <typename SM> struct PairIO;
template <> struct PairIO<float> {
    using V = float2;
    static __device__ __forceinline__ float2 dec(float2 q) { return q; }
    static __device__ __forceinline__ float2 enc(float2 v) { return v; }
};
template <> struct PairIO<__half> {
    using V = __half2;
    static __device__ __forceinline__ float2 dec(__half2 q) { return __half22float2(q); }
    static __device__ __forceinline__ __half2 enc(float2 v) { return __float22half2_rn(v); }
};
template <> struct PairIO<__nv_bfloat16> {
    using V = __nv_bfloat162;
    static __device__ __forceinline__ float2 dec(__nv_bfloat162 q) { return __bfloat1622float2(q); }
    static __device__ __forceinline__ __nv_bfloat162 enc(float2 v) { return __float22bfloat162_rn(v); }
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

// Stored pair -> population values (16-bit: q / scale + R_l, one fma each).
template <typename SM>
__device__ __forceinline__ float2 decode_pair(typename PairIO<SM>::V q, float R, const Consts<float>& C)
{
    if constexpr (std::is_same<SM, float>::value) return q;
    else return pfma(PairIO<SM>::dec(q), pk(C.minv), pk(R));
}

// Population values -> stored pair, and o replaced by what readers decode.
template <typename SM>
__device__ __forceinline__ typename PairIO<SM>::V narrow_pair(float2& o, float R, float NR, const Consts<float>& C)
{
    const typename PairIO<SM>::V q = PairIO<SM>::enc(pfma(o, pk(C.mscale), pk(NR)));
    o = pfma(PairIO<SM>::dec(q), pk(C.minv), pk(R));
    return q;
}


// ---------------------------------------------------------------------------
// Node arithmetic shared by both load paths.

// h - href, its pull-sum residual and j of the two nodes from their pulled
// populations n[l-1] (l = 1..8) and f_0 - href.  The moving populations are
// summed first (they are small), the last addition is error-free (see sum9).
__device__ __forceinline__ void pair_moments(const float2 (&n)[8], float2 f0, float2& dh, float2& er,
                                             float2& jx, float2& jy)
{
    const float2 rs = padd(padd(n[0], n[1]), n[7]);  // c_x = +1: l = 1, 2, 8
    const float2 ls = padd(padd(n[4], n[3]), n[5]);  // c_x = -1: l = 5, 4, 6
    ptwo_sum(f0, padd(padd(padd(n[2], n[6]), rs), ls), dh, er);
    jx = psub(rs, ls);
    jy = padd(padd(psub(n[2], n[6]), psub(n[1], n[7])), psub(n[3], n[5]));
}

// Film pressure (Eq. pfilm with Eq. disjoiningP) of the two nodes from the
// shared h rows n (+y), c, s (-y) at the pair's slot; writes 1/h to ih.
__device__ __forceinline__ float2 pair_pressure(const float* hn, const float* hc, const float* hs, float2 kap,
                                                bool disj, const Consts<float>& C, float2& ih)
{
    const float2 c0 = *reinterpret_cast<const float2*>(hc);
    const float2 n0 = *reinterpret_cast<const float2*>(hn);
    const float2 s0 = *reinterpret_cast<const float2*>(hs);
    const float cl = hc[-1], cr = hc[2], nl = hn[-1], nr = hn[2], sl = hs[-1], sr = hs[2];
    // Eq. (n_laplace): axis neighbours left + right + up + down, diagonal the four corners
    const float2 axis = padd(padd(make_float2(cl, c0.x), make_float2(c0.y, cr)), padd(n0, s0));
    const float2 diag = padd(padd(make_float2(nl, n0.x), make_float2(n0.y, nr)),
                             padd(make_float2(sl, s0.x), make_float2(s0.y, sr)));
    float2 lap = pmul(pfma(pk(4.0f), axis, pfma(pk(-20.0f), c0, diag)), pk(1.0f / 6.0f));
    const float2 h = padd(c0, pk(C.href));
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
// collide_store on both lanes).  pn, pc, ps: shared p rows o+1, o, o-1 at the
// pair's slot; f: the pulled moving populations (omega != 1 only); i: the
// storage offset of the pair's first column.
template <typename SM, bool OMEGA1>
__device__ __forceinline__ void pair_collide_store(const float* pn, const float* pc, const float* ps, float2 dh,
                                                   float2 ih, float2 jx, float2 jy, float2 er,
                                                   const float2* f, int fstride, float* __restrict__ fout0,
                                                   SM* __restrict__ foutm, int i, int plane,
                                                   const Consts<float>& C)
{
    using V = typename PairIO<SM>::V;
    constexpr bool NARROW = !std::is_same<SM, float>::value;
    const float2 n0 = *reinterpret_cast<const float2*>(pn);
    const float2 c0 = *reinterpret_cast<const float2*>(pc);
    const float2 s0 = *reinterpret_cast<const float2*>(ps);
    const float2 nL = make_float2(pn[-1], n0.x), nR = make_float2(n0.y, pn[2]);
    const float2 sL = make_float2(ps[-1], s0.x), sR = make_float2(s0.y, ps[2]);
    const float2 cL = make_float2(pc[-1], c0.x), cR = make_float2(c0.y, pc[2]);
    // Eq. (derivative): grad p = 3 sum_l w_l c_l p(x + c_l)
    const float2 gpx = pfma(psub(cR, cL), pk(1.0f / 3.0f), pmul(padd(psub(nR, nL), psub(sR, sL)), pk(1.0f / 12.0f)));
    const float2 gpy = pfma(psub(n0, s0), pk(1.0f / 3.0f), pmul(padd(psub(nR, sR), psub(nL, sL)), pk(1.0f / 12.0f)));
    const float2 h = padd(dh, pk(C.href));
    // Eqs. (force), (forcefric), (alphafric): nu alpha u = 6 nu j / (2h^2 + 6 delta h + 3 delta^2)
    const float2 den = pfma(h, pfma(pk(2.0f), h, pk(6.0f * C.delta)), pk(3.0f * C.delta * C.delta));
    const float2 fr = make_float2(__fdividef(C.nu6, den.x), __fdividef(C.nu6, den.y));
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
    // Eq. (equilibria) with e^2 = 1 as S +- D per opposite pair; source 3 w_l c_l . F
    const float2 A = pmul(pmul(h, psub(pmul(pk(C.g), h), pfma(ux, ux, pmul(uy, uy)))), pk(1.0f / 6.0f));
    float2 Sx = pfma(pk(0.5f), pmul(ex, ux), A);
    float2 Sy = pfma(pk(0.5f), pmul(ey, uy), A);
    const float2 a = padd(ux, uy), b = psub(uy, ux);
    float2 Sa = pmul(pfma(pk(0.5f), pmul(h, pmul(a, a)), A), pk(0.25f));
    float2 Sb = pmul(pfma(pk(0.5f), pmul(h, pmul(b, b)), A), pk(0.25f));
    // second-order source: odd part scaled by (1 - omega/2), even part T
    float2 Tx = pk(0.0f), Ty = pk(0.0f), Ta = pk(0.0f), Tb = pk(0.0f);
    if (C.forcing) {
        const float2 ks = pk(1.0f - 0.5f * C.omega);
        Fx = pmul(Fx, ks);
        Fy = pmul(Fy, ks);
        const float2 uF3 = pmul(pfma(ux, Fx, pmul(uy, Fy)), pk(1.0f / 3.0f));
        Tx = psub(pmul(ux, Fx), uF3);
        Ty = psub(pmul(uy, Fy), uF3);
        Ta = pmul(psub(pmul(a, padd(Fx, Fy)), uF3), pk(0.25f));
        Tb = pmul(psub(pmul(b, psub(Fy, Fx)), uF3), pk(0.25f));
        if constexpr (OMEGA1) {
            Sx = padd(Sx, Tx);
            Sy = padd(Sy, Ty);
            Sa = padd(Sa, Ta);
            Sb = padd(Sb, Tb);
        }
    }
    float2 o1, o2, o3, o4, o5, o6, o7, o8;
    if constexpr (OMEGA1) {
        const float2 Dx = pmul(padd(ex, Fx), pk(1.0f / 3.0f));
        const float2 Dy = pmul(padd(ey, Fy), pk(1.0f / 3.0f));
        const float2 Da = pmul(padd(padd(ex, ey), padd(Fx, Fy)), pk(1.0f / 12.0f));
        const float2 Db = pmul(padd(psub(ey, ex), psub(Fy, Fx)), pk(1.0f / 12.0f));
        o1 = padd(Sx, Dx); o5 = psub(Sx, Dx);
        o3 = padd(Sy, Dy); o7 = psub(Sy, Dy);
        o2 = padd(Sa, Da); o6 = psub(Sa, Da);
        o4 = padd(Sb, Db); o8 = psub(Sb, Db);
    } else {
        const float2 w = pk(C.omega), m = pk(1.0f - C.omega);
        const float2 Dx = pmul(ex, pk(1.0f / 3.0f)), Dy = pmul(ey, pk(1.0f / 3.0f));
        const float2 Da = pmul(padd(ex, ey), pk(1.0f / 12.0f)), Db = pmul(psub(ey, ex), pk(1.0f / 12.0f));
        const float2 Qx = pmul(Fx, pk(1.0f / 3.0f)), Qy = pmul(Fy, pk(1.0f / 3.0f));
        const float2 Qa = pmul(padd(Fx, Fy), pk(1.0f / 12.0f)), Qb = pmul(psub(Fy, Fx), pk(1.0f / 12.0f));
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
        const float Rax = C.r_axis, Rdg = C.r_diag, NRa = C.nr_axis, NRd = C.nr_diag;
        const V q3 = narrow_pair<SM>(o3, Rax, NRa, C);
        const V q5 = narrow_pair<SM>(o5, Rax, NRa, C);
        const V q7 = narrow_pair<SM>(o7, Rax, NRa, C);
        const V q2 = narrow_pair<SM>(o2, Rdg, NRd, C);
        const V q4 = narrow_pair<SM>(o4, Rdg, NRd, C);
        const V q6 = narrow_pair<SM>(o6, Rdg, NRd, C);
        const V q8 = narrow_pair<SM>(o8, Rdg, NRd, C);
        const float2 osum = padd(padd(padd(o1, o5), padd(o3, o7)), padd(padd(o2, o6), padd(o4, o8)));
        // the last residual goes to the finer of the two roundings: the 16-bit
        // one of f_1 - R or the FP32 one of f_0 - href (see collide_store)
        constexpr float kRatio = std::is_same<SM, __half>::value ? 8192.0f : 65536.0f;
        const bool lx = fabsf(o1.x - Rax) * kRatio < fabsf(dh.x - osum.x);
        const bool ly = fabsf(o1.y - Rax) * kRatio < fabsf(dh.y - osum.y);
        float2 o1r = o1;
        const V q1r = narrow_pair<SM>(o1r, Rax, NRa, C);
        const float2 adj = psub(o1r, o1);
        const float2 os = make_float2(lx ? osum.x : osum.x + adj.x, ly ? osum.y : osum.y + adj.y);
        float2 o0v, e2, o0n, e3;
        ptwo_sum(dh, make_float2(-os.x, -os.y), o0v, e2);
        ptwo_sum(o0v, padd(er, e2), o0n, e3);
        float2 o1l = padd(o1, e3);
        const V q1l = narrow_pair<SM>(o1l, Rax, NRa, C);
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
    __shared__ __align__(16) float hsm[4][NC + 4];  // h - href
    __shared__ __align__(16) float psm[4][NC + 4];  // film pressure
    // general tau: the eight pulled moving populations of the last four rows
    __shared__ __align__(16) float2 fsm[OMEGA1 ? 1 : 4][8][OMEGA1 ? 1 : BX];
    // per-thread ring of j_x, j_y, the pull-sum residual and 1/h of the last
    // four rows (each thread reads back only its own slots)
    __shared__ __align__(16) float2 rsm[4][4][BX];

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
    const float Rax = C.r_axis, Rdg = C.r_diag;
    const int c = wrap_index(x0 - 2 + 2 * t, nx);  // own pair (even)

    const bool edge = lane == 0 || lane == 31;
    const int ce = lane == 0 ? wrap_index(c - 2, nx) : (c + 2 == nx ? 0 : c + 2);
    // moving planes (index l - 1) a warp-edge lane reads at its outer
    // neighbour pair, from rows y, y-1, y+1: lane 0 needs l = 1, 2, 8
    // (arriving from the left), lane 31 needs l = 5, 4, 6 (from the right)
    const int e0 = (lane == 0 ? 0 : 4) * plane;
    const int e1 = (lane == 0 ? 1 : 3) * plane;
    const int e2 = (lane == 0 ? 7 : 5) * plane;
    const float2* __restrict__ f0p = reinterpret_cast<const float2*>(fin0);
    const V* __restrict__ fmp = reinterpret_cast<const V*>(finm);
    const int half = plane >> 1;  // pairs per plane (pitch is even)
    // PF rows of loads in flight: 16-bit storage keeps two (rows r(k+1) and
    // r(k+2) go out while step k runs), FP32 one (its registers would
    // otherwise cost resident warps)
    constexpr int PF = NARROW ? 2 : 1;
    float2 q0[PF];
    V qm[PF][8], qe[PF][3];

    // wrapped rows r(k-1), r(k), r(k+1), r(k+2)
    // wrapped rows r(k-1) .. r(k+3)
    int wm1 = wrap_index(rstart - dir, ny), w0 = wrap_index(rstart, ny);
    int w1 = wrap_index(rstart + dir, ny), w2 = wrap_index(rstart + 2 * dir, ny);
    int w3 = wrap_index(rstart + 3 * dir, ny);
    // the nine planes (and the edge planes) pulled into row w, into register set b
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
            qe[b][0] = ldpair(fmp + TFLBM_IDX((e0 + w * pitch + ce) >> 1, m8, st));
            qe[b][1] = ldpair(fmp + TFLBM_IDX((e1 + ys * pitch + ce) >> 1, m8, st));
            qe[b][2] = ldpair(fmp + TFLBM_IDX((e2 + yn * pitch + ce) >> 1, m8, st));
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

    // ring slots no thread writes (outer halves of the edge columns' stencils)
    if (t < 4) {
        const int j = t < 2 ? t : NC + t;
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
            float2 f0, n[8];  // f_0 - href and the moving populations arriving at the pair
            {
                constexpr int rb = s % PF;  // register set of row r(k)
                f0 = q0[rb];
                float2 v[8];
#pragma unroll
                for (int l = 0; l < 8; ++l) v[l] = decode_pair<SM>(qm[rb][l], (l & 1) ? Rdg : Rax, C);
                float ex = 0.f, ey = 0.f, ez = 0.f;  // left column of lane 0 / right column of lane 31
                if (edge) {
                    const float2 a = decode_pair<SM>(qe[rb][0], Rax, C);  // l = 1 or 5: axis
                    const float2 b = decode_pair<SM>(qe[rb][1], Rdg, C);  // l = 2 or 4: diagonal
                    const float2 d = decode_pair<SM>(qe[rb][2], Rdg, C);  // l = 8 or 6: diagonal
                    ex = lane == 0 ? a.y : a.x;
                    ey = lane == 0 ? b.y : b.x;
                    ez = lane == 0 ? d.y : d.x;
                }
                // the loads of row r(k+PF) go out before this row's arithmetic
                if constexpr (PF == 2) {
                    if (k + 2 <= R + 3) load_row(std::integral_constant<int, rb>{}, w1, w2, w3);
                } else {
                    if (k + 1 <= R + 3) load_row(std::integral_constant<int, rb>{}, w0, w1, w2);
                }
                if (KFIELD && pcol)
                    kap_n = reinterpret_cast<const float2*>(kappa)[TFLBM_IDX(((long long)w0 * nx + c) >> 1, npair,
                                                                              C.status)];
                // l = 1, 2, 8 arrive from the left, l = 4, 5, 6 from the right
                float u1 = __shfl_up_sync(0xffffffffu, v[0].y, 1);
                float u2 = __shfl_up_sync(0xffffffffu, v[1].y, 1);
                float u8 = __shfl_up_sync(0xffffffffu, v[7].y, 1);
                float d5 = __shfl_down_sync(0xffffffffu, v[4].x, 1);
                float d4 = __shfl_down_sync(0xffffffffu, v[3].x, 1);
                float d6 = __shfl_down_sync(0xffffffffu, v[5].x, 1);
                if (lane == 0) { u1 = ex; u2 = ey; u8 = ez; }
                if (lane == 31) { d5 = ex; d4 = ey; d6 = ez; }
                n[0] = make_float2(u1, v[0].x);
                n[1] = make_float2(u2, v[1].x);
                n[2] = v[2];
                n[3] = make_float2(v[3].y, d4);
                n[4] = make_float2(v[4].y, d5);
                n[5] = make_float2(v[5].y, d6);
                n[6] = v[6];
                n[7] = make_float2(u8, v[7].x);
            }
            float2 dh, er, jx, jy;
            pair_moments(n, f0, dh, er, jx, jy);
            *reinterpret_cast<float2*>(&hsm[s][OFF + 2 * t]) = dh;
            rsm[s][0][t] = jx;
            rsm[s][1][t] = jy;
            rsm[s][2][t] = er;
            if constexpr (!OMEGA1) {
#pragma unroll
                for (int l = 0; l < 8; ++l) fsm[s][l][t] = n[l];
            }
        }
        __syncthreads();
        // ---- (B1) film pressure of row r(k-1) (needs h rows r(k-2) .. r(k))
        if (pcol && k >= 2 && k <= R + 3) {
            // the stencil reads slots OFF + 2t - 1 .. OFF + 2t + 2 of rings of NC + 4
            TFLBM_CHECK(OFF + 2 * t - 1 >= 0 && OFF + 2 * t + 2 < NC + 4, C.status);
            float2 ih;
            const float2 p = pair_pressure(hsm[s] + OFF + 2 * t, hsm[s1] + OFF + 2 * t, hsm[s2] + OFF + 2 * t, kap,
                                           disj, C, ih);
            rsm[s1][3][t] = ih;
            *reinterpret_cast<float2*>(&psm[s1][OFF + 2 * t]) = p;
        }
        // ---- (B2) force, collision and store of row r(k-3)
        if (ocol && k >= 5) {
            const int o = rstart + (k - 3) * dir;  // inside [ybeg, yend), no wrap
            TFLBM_CHECK(OFF + 2 * t - 1 >= 0 && OFF + 2 * t + 2 < NC + 4 && o >= 0 && o < ny, C.status);
            const float* pn = (dir > 0 ? psm[s2] : psm[s]) + OFF + 2 * t;  // row o+1
            const float* pc = psm[s3] + OFF + 2 * t;
            const float* ps = (dir > 0 ? psm[s] : psm[s2]) + OFF + 2 * t;  // row o-1
            const float2 dh = *reinterpret_cast<const float2*>(&hsm[s3][OFF + 2 * t]);
            const float2* fp = nullptr;
            if constexpr (!OMEGA1) fp = &fsm[s3][0][t];
            pair_collide_store<SM, OMEGA1>(pn, pc, ps, dh, rsm[s3][3][t], rsm[s3][0][t], rsm[s3][1][t], rsm[s3][2][t], fp, BX, fout0,
                                           foutm, o * pitch + c, plane, C);
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
// Launch of the paired kernel: block_x is the CTA width in columns (64, 128
// or 256), i.e. block_x / 2 threads.

template <typename SM, int BX>
cudaError_t launch_pair_bx(const float* fin0, const SM* finm, float* fout0, SM* foutm, const float* kappa,
                           const Geom& G, const Consts<float>& C, int rows, cudaStream_t st)
{
    int bands = (G.ny + rows - 1) / rows;
    if (bands > 65535) bands = 65535;
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
                      const Consts<float>& C, int rows, cudaStream_t st)
{
    const float* f0 = (const float*)fin;
    const SM* fm = (const SM*)((const char*)fin + G.plane * sizeof(float));
    float* g0 = (float*)fout;
    SM* gm = (SM*)((char*)fout + G.plane * sizeof(float));
    const float* k = (const float*)kappa;
    switch (block_x) {
        case 64: return launch_pair_bx<SM, 32>(f0, fm, g0, gm, k, G, C, rows, st);
        case 128: return launch_pair_bx<SM, 64>(f0, fm, g0, gm, k, G, C, rows, st);
        case 256: return launch_pair_bx<SM, 128>(f0, fm, g0, gm, k, G, C, rows, st);
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
