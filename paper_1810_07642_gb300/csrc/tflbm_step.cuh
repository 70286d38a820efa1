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
//    node; h, p and F never touch DRAM.
//  * A CTA of BX threads owns BX consecutive columns and marches down a band of
//    `rows` rows.  Per row r it pulls the populations of row r, forms h on the
//    row plus a 2-column halo into a 3-row shared ring, then the film pressure
//    of row r-1 (plus a 1-column halo) into a second ring, then the force and
//    collision of row r-2, whose populations were kept in registers.  The
//    radius-2 dependence of grad p on h thus costs 4 extra rows per band and 4
//    extra columns per strip of recomputed h, all served from L1/L2.
//  * Loads use the read-only path; stores are aligned and coalesced.
//  * The rest population is written as h - sum_{l>0} f*_l, which keeps the
//    local mass of the collision exact up to the rounding of that sum.
#pragma once
#include <type_traits>

#include "tflbm_internal.h"

namespace tflbm {

__device__ __forceinline__ int wrap_index(int i, int n)
{
    i %= n;
    return i < 0 ? i + n : i;
}

template <typename T> __device__ __forceinline__ T rcp(T x);
template <> __device__ __forceinline__ float rcp<float>(float x) { return __frcp_rn(x); }
template <> __device__ __forceinline__ double rcp<double>(double x) { return __drcp_rn(x); }

// r^n for integer n >= 0 by binary powering (n is uniform across the CTA).
template <typename T>
__device__ __forceinline__ T ipow(T r, int n)
{
    T out = T(1), b = r;
    while (n) {
        if (n & 1) out *= b;
        b *= b;
        n >>= 1;
    }
    return out;
}

template <typename S> __device__ __forceinline__ S ldro(const S* p) { return __ldg(p); }

// Pull the nine populations arriving at column x of row `row0` (row offsets
// already multiplied by the pitch; rowm = row above in -y, rowp = row in +y).
// Order of Eq. (speeds): 1 (1,0) 2 (1,1) 3 (0,1) 4 (-1,1) 5 (-1,0) 6 (-1,-1)
// 7 (0,-1) 8 (1,-1); population l at x comes from x - c_l.
template <typename S, typename T>
__device__ __forceinline__ void pull9(const S* __restrict__ f, long long plane, long long rowm,
                                      long long row0, long long rowp, int x, int xm, int xp,
                                      T (&v)[9])
{
    v[0] = T(ldro(f + row0 + x));
    v[1] = T(ldro(f + plane + row0 + xm));
    v[2] = T(ldro(f + 2 * plane + rowm + xm));
    v[3] = T(ldro(f + 3 * plane + rowm + x));
    v[4] = T(ldro(f + 4 * plane + rowm + xp));
    v[5] = T(ldro(f + 5 * plane + row0 + xp));
    v[6] = T(ldro(f + 6 * plane + rowp + xp));
    v[7] = T(ldro(f + 7 * plane + rowp + x));
    v[8] = T(ldro(f + 8 * plane + rowp + xm));
}

template <typename T>
__device__ __forceinline__ T sum9(const T (&v)[9])
{
    return ((v[0] + v[1]) + (v[2] + v[3])) + ((v[4] + v[5]) + (v[6] + v[7])) + v[8];
}

// Film pressure p = -gamma (lap h + pi_sign kappa f(h)) at one node from the
// 3x3 neighbourhood of h in the shared ring (rows n = +y, c, s = -y).
template <typename T>
__device__ __forceinline__ T film_pressure(const T* hn, const T* hc, const T* hs_, int j, T kap,
                                           const Consts<T>& C, bool disj)
{
    const T axis = (hc[j - 1] + hc[j + 1]) + (hn[j] + hs_[j]);
    const T diag = (hn[j - 1] + hn[j + 1]) + (hs_[j - 1] + hs_[j + 1]);
    const T h = hc[j];
    T lap = (T(4) * axis + diag - T(20) * h) * T(1.0 / 6.0);
    if (disj) {
        const T r = C.hstar * rcp(h);
        lap += C.pi_sgn * kap * (ipow(r, C.n_exp) - ipow(r, C.m_exp));
    }
    return -C.gamma * lap;
}

template <typename S, typename T, int BX, bool OMEGA1, bool KFIELD>
__global__ void __launch_bounds__(BX)
k_step(const S* __restrict__ fin, S* __restrict__ fout, const T* __restrict__ kappa,
       const Geom G, const Consts<T> C, const int rows)
{
    constexpr int NW = BX / 32;
    __shared__ T hsm[3][BX + 4];  // h of rows r, r-1, r-2 (ring), columns x0-2 .. x0+W+1
    __shared__ T psm[3][BX + 2];  // p of rows r-1, r-2, r-3 (ring), columns x0-1 .. x0+W

    const int t = threadIdx.x;
    const int nx = G.nx, ny = G.ny;
    const long long plane = G.plane, pitch = G.pitch;
    const int x0 = blockIdx.x * BX;
    const int weff = min(BX, nx - x0);
    const bool own = t < weff;
    const int ybeg = blockIdx.y * rows;
    const int yend = min(ybeg + rows, ny);
    const bool disj = KFIELD || C.kappa_u != T(0);

    // Halo roles, spread over warps: 0..3 compute h at columns x0-2, x0-1,
    // x0+W, x0+W+1; 4..5 compute p at columns x0-1, x0+W.
    int role = -1;
#pragma unroll
    for (int q = 0; q < 6; ++q)
        if (t == (q % NW) * 32 + q / NW) role = q;
    int hcol = x0, hslot = 0;
    if (role == 0) { hcol = x0 - 2; hslot = 0; }
    else if (role == 1) { hcol = x0 - 1; hslot = 1; }
    else if (role == 2) { hcol = x0 + weff; hslot = weff + 2; }
    else if (role == 3) { hcol = x0 + weff + 1; hslot = weff + 3; }
    else if (role == 4) { hcol = x0 - 1; hslot = 1; }         // hs slot; p slot = hslot - 1
    else if (role == 5) { hcol = x0 + weff; hslot = weff + 2; }
    hcol = wrap_index(hcol, nx);
    const int hxm = wrap_index(hcol - 1, nx), hxp = wrap_index(hcol + 1, nx);

    const int x = own ? x0 + t : x0;
    const int xm = wrap_index(x - 1, nx), xp = wrap_index(x + 1, nx);

    // rolling wrapped row indices of rows r-1, r, r+1
    int rm = wrap_index(ybeg - 3, ny), r0 = wrap_index(ybeg - 2, ny), rp = wrap_index(ybeg - 1, ny);

    T fv[3][9];
    T jxv[3], jyv[3], ihv[3];
#pragma unroll
    for (int s = 0; s < 3; ++s) { jxv[s] = jyv[s] = ihv[s] = T(0); }

    const T third = T(1.0 / 3.0), twelfth = T(1.0 / 12.0), sixth = T(1.0 / 6.0);
    const T one_m_omega = T(1) - C.omega;
    const T d6 = T(6) * C.delta, d3sq = T(3) * C.delta * C.delta;

    auto body = [&](auto stage_c, int r) {
        constexpr int s = decltype(stage_c)::value;   // slot of row r
        constexpr int s1 = (s + 2) % 3;               // slot of row r-1
        constexpr int s2 = (s + 1) % 3;               // slot of row r-2 (and r+1)
        const long long om = (long long)rm * pitch, o0 = (long long)r0 * pitch,
                        op = (long long)rp * pitch;
        // (1) pull row r: h into the ring, momentum into registers
        if (own) {
            T v[9];
            pull9<S, T>(fin, plane, om, o0, op, x, xm, xp, v);
            hsm[s][t + 2] = sum9(v);
            jxv[s] = ((v[1] + v[2]) + v[8]) - ((v[4] + v[5]) + v[6]);
            jyv[s] = ((v[2] + v[3]) + v[4]) - ((v[6] + v[7]) + v[8]);
            if (!OMEGA1) {
#pragma unroll
                for (int l = 0; l < 9; ++l) fv[s][l] = v[l];
            }
        }
        if (role >= 0 && role < 4) {
            T v[9];
            pull9<S, T>(fin, plane, om, o0, op, hcol, hxm, hxp, v);
            hsm[s][hslot] = sum9(v);
        }
        __syncthreads();
        // (2) film pressure of row r-1 (needs h rows r-2 .. r)
        if (r >= ybeg) {
            const int q = rm;  // wrapped index of row r-1
            if (own) {
                const T kap = KFIELD ? kappa[(long long)q * nx + x] : C.kappa_u;
                psm[s1][t + 1] = film_pressure(hsm[s], hsm[s1], hsm[s2], t + 2, kap, C, disj);
                ihv[s1] = rcp(hsm[s1][t + 2]);
            }
            if (role >= 4) {
                const T kap = KFIELD ? kappa[(long long)q * nx + hcol] : C.kappa_u;
                psm[s1][hslot - 1] = film_pressure(hsm[s], hsm[s1], hsm[s2], hslot, kap, C, disj);
            }
        }
        __syncthreads();
        // (3) force and collision of row r-2 (needs p rows r-3 .. r-1)
        if (r >= ybeg + 2 && own) {
            const int o = r - 2;  // inside [ybeg, yend), no wrap
            const T* pn = psm[s1];
            const T* pc = psm[s2];
            const T* ps = psm[s];
            const int j = t + 1;
            // Eq. (derivative): grad p = 3 sum_l w_l c_l p(x + c_l)
            const T gpx = (pc[j + 1] - pc[j - 1]) * third
                        + ((pn[j + 1] - pn[j - 1]) + (ps[j + 1] - ps[j - 1])) * twelfth;
            const T gpy = (pn[j] - ps[j]) * third
                        + ((pn[j + 1] - ps[j + 1]) + (pn[j - 1] - ps[j - 1])) * twelfth;
            const T h = hsm[s2][t + 2];
            const T ih = ihv[s2];
            const T jx = jxv[s2], jy = jyv[s2];
            // Eqs. (force), (forcefric), (alphafric): nu alpha u = 6 nu j / (2h^2 + 6 delta h + 3 delta^2)
            const T fr = C.nu6 * rcp(h * (T(2) * h + d6) + d3sq);
            const T Fx = h * (C.gx - gpx) - fr * jx;
            const T Fy = h * (C.gy - gpy) - fr * jy;
            // Eq. (equilibria) with e^2 = 1, written as S +- D per pair of
            // opposite directions; source 3 w_l c_l . F.
            const T ux = jx * ih, uy = jy * ih;
            const T A = h * (C.g * h - (ux * ux + uy * uy)) * sixth;
            const T Sx = A + T(0.5) * jx * ux;
            const T Sy = A + T(0.5) * jy * uy;
            const T a = ux + uy, b = uy - ux;
            const T Sa = (A + T(0.5) * h * a * a) * T(0.25);
            const T Sb = (A + T(0.5) * h * b * b) * T(0.25);
            T o1, o2, o3, o4, o5, o6, o7, o8;
            if (OMEGA1) {
                const T Dx = (jx + Fx) * third, Dy = (jy + Fy) * third;
                const T Da = ((jx + jy) + (Fx + Fy)) * twelfth;
                const T Db = ((jy - jx) + (Fy - Fx)) * twelfth;
                o1 = Sx + Dx; o5 = Sx - Dx;
                o3 = Sy + Dy; o7 = Sy - Dy;
                o2 = Sa + Da; o6 = Sa - Da;
                o4 = Sb + Db; o8 = Sb - Db;
            } else {
                const T w = C.omega;
                const T Dx = jx * third, Dy = jy * third;
                const T Da = (jx + jy) * twelfth, Db = (jy - jx) * twelfth;
                const T Qx = Fx * third, Qy = Fy * third;
                const T Qa = (Fx + Fy) * twelfth, Qb = (Fy - Fx) * twelfth;
                const T(&f)[9] = fv[s2];
                o1 = one_m_omega * f[1] + w * (Sx + Dx) + Qx;
                o5 = one_m_omega * f[5] + w * (Sx - Dx) - Qx;
                o3 = one_m_omega * f[3] + w * (Sy + Dy) + Qy;
                o7 = one_m_omega * f[7] + w * (Sy - Dy) - Qy;
                o2 = one_m_omega * f[2] + w * (Sa + Da) + Qa;
                o6 = one_m_omega * f[6] + w * (Sa - Da) - Qa;
                o4 = one_m_omega * f[4] + w * (Sb + Db) + Qb;
                o8 = one_m_omega * f[8] + w * (Sb - Db) - Qb;
            }
            const T o0v = h - (((o1 + o5) + (o3 + o7)) + ((o2 + o6) + (o4 + o8)));
            S* out = fout + (long long)o * pitch + x;
            out[0] = S(o0v);
            out[plane] = S(o1);
            out[2 * plane] = S(o2);
            out[3 * plane] = S(o3);
            out[4 * plane] = S(o4);
            out[5 * plane] = S(o5);
            out[6 * plane] = S(o6);
            out[7 * plane] = S(o7);
            out[8 * plane] = S(o8);
        }
        // advance the wrapped row window
        rm = r0;
        r0 = rp;
        rp = (rp + 1 == ny) ? 0 : rp + 1;
    };

    const int last = yend + 1;
    for (int r = ybeg - 2;;) {
        body(std::integral_constant<int, 0>{}, r);
        if (++r > last) break;
        body(std::integral_constant<int, 1>{}, r);
        if (++r > last) break;
        body(std::integral_constant<int, 2>{}, r);
        if (++r > last) break;
    }
}

template <typename S, typename T, int BX>
cudaError_t launch_step_bx(const S* fin, S* fout, const T* kappa, const Geom& G,
                           const Consts<T>& C, int rows, cudaStream_t st)
{
    dim3 grid((G.nx + BX - 1) / BX, (G.ny + rows - 1) / rows);
    const bool om1 = (C.omega == T(1));
    if (kappa) {
        if (om1) k_step<S, T, BX, true, true><<<grid, BX, 0, st>>>(fin, fout, kappa, G, C, rows);
        else k_step<S, T, BX, false, true><<<grid, BX, 0, st>>>(fin, fout, kappa, G, C, rows);
    } else {
        if (om1) k_step<S, T, BX, true, false><<<grid, BX, 0, st>>>(fin, fout, kappa, G, C, rows);
        else k_step<S, T, BX, false, false><<<grid, BX, 0, st>>>(fin, fout, kappa, G, C, rows);
    }
    return cudaGetLastError();
}

}  // namespace tflbm
