// Fused adjoint of one thin-film step (the transpose of the phases listed in
// tflbm_adjoint.cu, evaluated in one pass over the lattice).
//
// Input: the raw population buffer whose pull is the state f(t) (exactly what
// the forward step reads), a(t+1) = dL/df(t+1) and dL/dkappa so far; output
// a(t) = dL/df(t), and dL/dkappa += the step's contribution.  Per node and
// step: 36 B of populations, 36 B of a(t+1) (gathered a second time, from
// L1/L2, only when omega != 1), kappa, the read-modify-write of dL/dkappa and
// 36 B of a(t) in FP32.
//
// A CTA of BX threads covers BX columns and marches down a band of rows like
// the forward step.  The adjoint has four nested radius-1 stencils (h -> p ->
// grad p and -h aF -> transposed gradient -> Laplacian), so CTAs overlap by
// 8 columns and a band needs 4 halo rows on each side.  March step k, for
// rows r(m) = rstart + m dir:
//   A  row r(k):    pull f, h, j                             -> rings
//   (one __syncthreads)
//   B  row r(k-1):  film pressure p (needs h of rows r(k-2) .. r(k))
//   C  row r(k-3):  with mu_l = a_l(x + c_l, t+1) (loads issued before the
//                   barrier), the equilibrium and source adjoints at the node (aF, dL/dh and dL/dj through
//                   f_eq); grad p (p rows r(k-4) .. r(k-2)); the force
//                   adjoint: dL/dh += aF.(G - grad p) - fr'(h) aF.j,
//                   dL/dj -= fr aF, ag = -h aF
//   D  row r(k-5):  transposed gradient of ag (rows r(k-6) .. r(k-4)):
//                   ap; the disjoining-pressure adjoint into dL/dh and
//                   dL/dkappa; alap = -gamma ap
//   E  row r(k-7):  dL/dh += Laplacian of alap (rows r(k-8) .. r(k-6));
//                   a_l(t) = dL/dh + c_l.dL/dj + (1 - omega) mu_l
// Every stage reads only rows written before the current step's barrier, and
// each shared ring is deep enough that a slot is rewritten only after the
// barrier that follows its last read.  Values a thread needs only at its own
// column later (j, the node adjoints) wait in per-thread shared rings.
#pragma once

#include "tflbm_step.cuh"

namespace tflbm {

template <typename SM, typename T, int BX>
__global__ void __launch_bounds__(BX, sizeof(T) == 4 ? 768 / BX : 1)
k_adjoint_march(const T* __restrict__ fin0, const SM* __restrict__ finm, const T* __restrict__ an,
                T* __restrict__ a, T* __restrict__ gk, const T* __restrict__ kappa, const Geom G,
                const Consts<T> C)
{
    constexpr int W = BX - 8;
    // shared rings (read across columns), by march index
    __shared__ T hsm[8][BX];   // h - href
    __shared__ T psm[4][BX];   // p
    __shared__ T agx[4][BX], agy[4][BX];
    __shared__ T als[4][BX];   // -gamma ap
    // per-thread rings (own column)
    __shared__ T rjx[4][BX], rjy[4][BX];
    __shared__ T rah[8][BX], rajx[8][BX], rajy[8][BX];

    const int t = threadIdx.x;
    const int nx = G.nx, ny = G.ny, pitch = G.pitch, plane = (int)G.plane;
    const long long n = (long long)nx * ny;
    const int x0 = blockIdx.x * W;
    const int weff = min(W, nx - x0);
    const bool cA = t < weff + 8, cB = t >= 1 && t < weff + 7, cC = t >= 2 && t < weff + 6;
    const bool cD = t >= 3 && t < weff + 5, cE = t >= 4 && t < weff + 4;
    const int band = blockIdx.y, nb = gridDim.y;
    const int ybeg = (int)(((long long)band * ny) / nb), yend = (int)(((long long)(band + 1) * ny) / nb);
    const int R = yend - ybeg;
    const int dir = (band & 1) ? -1 : 1;
    const int rstart = dir > 0 ? ybeg - 4 : yend + 3;
    const int x = wrap_index(x0 - 4 + t, nx);
    const int xm = wrap_index(x - 1, nx), xp = wrap_index(x + 1, nx);
    const bool disj = kappa != nullptr || C.kappa_u != T(0);
    const T third = T(1.0 / 3.0), twelfth = T(1.0 / 12.0);

    // wrapped rows: r(k-1), r(k), r(k+1) (stages A, B); r(k-5) (D);
    // r(k-8), r(k-7), r(k-6) (E)
    int am = wrap_index(rstart - dir, ny), a0 = wrap_index(rstart, ny), ap1 = wrap_index(rstart + dir, ny);
    int cm = wrap_index(rstart - 4 * dir, ny), c0 = wrap_index(rstart - 3 * dir, ny);
    int cp = wrap_index(rstart - 2 * dir, ny);
    int d0 = wrap_index(rstart - 5 * dir, ny);
    int em = wrap_index(rstart - 8 * dir, ny), e0 = wrap_index(rstart - 7 * dir, ny);
    int ep = wrap_index(rstart - 6 * dir, ny);
    auto adv = [&](int& w) {
        w += dir;
        w = w == ny ? 0 : (w < 0 ? ny - 1 : w);
    };
    // mu_l(x, y) = a_l(x + c_l, y + c_l) of a(t+1), lattice rows yU = y + 1, yD = y - 1
    auto gather = [&](int y, int yU, int yD, T (&mu)[9]) {
        const long long r0 = (long long)y * nx, rU = (long long)yU * nx, rD = (long long)yD * nx;
        mu[0] = ldro(an + (r0 + x));
        mu[1] = ldro(an + (n + r0 + xp));
        mu[2] = ldro(an + (2 * n + rU + xp));
        mu[3] = ldro(an + (3 * n + rU + x));
        mu[4] = ldro(an + (4 * n + rU + xm));
        mu[5] = ldro(an + (5 * n + r0 + xm));
        mu[6] = ldro(an + (6 * n + rD + xm));
        mu[7] = ldro(an + (7 * n + rD + x));
        mu[8] = ldro(an + (8 * n + rD + xp));
    };

    const int last = R + 10;
    for (int k = 0; k <= last; ++k) {
        // ---- A: row r(k)
        if (k <= R + 7 && cA) {
            const int y = a0, yU = dir > 0 ? ap1 : am, yD = dir > 0 ? am : ap1;
            const int r0 = y * pitch;
            T v[9];
            pull9<SM, T>(fin0, finm, plane, r0 + x, r0 + xm, r0 + xp, (yD - y) * pitch, (yU - y) * pitch, C, v);
            T er;
            const T dh = sum9(v, er);
            const T jx = ((v[1] + v[2]) + v[8]) - ((v[4] + v[5]) + v[6]);
            const T jy = ((v[2] + v[3]) + v[4]) - ((v[6] + v[7]) + v[8]);
            const int s4 = k & 3;
            hsm[k & 7][t] = dh;
            rjx[s4][t] = jx;
            rjy[s4][t] = jy;
        }
        // mu_l = a_l(x + c_l, t+1) for stage C's row r(k-3), requested before
        // the barrier so that the loads overlap it and stage B
        T mu[9];
        const bool runC = k >= 5 && k <= R + 8 && cC;
        if (runC) gather(c0, dir > 0 ? cp : cm, dir > 0 ? cm : cp, mu);
        __syncthreads();
        // ---- B: film pressure of row r(k-1)
        if (k >= 2 && k <= R + 7 && cB) {
            const int m = k - 1;
            const T* hn = hsm[(m + dir) & 7];
            const T* hc = hsm[m & 7];
            const T* hs = hsm[(m - dir) & 7];
            const T kap = kappa ? kappa[(long long)am * nx + x] : C.kappa_u;
            const T ih = fdiv(T(1), hc[t] + C.href);
            psm[m & 3][t] = film_pressure(hn, hc, hs, t, kap, ih, C, disj, BX);
        }
        // ---- C: force adjoint at row r(k-3)
        if (runC) {
            const int m = k - 3, s4 = m & 3, s8 = m & 7;
            const T* pn = psm[(m + dir) & 3];
            const T* pc = psm[s4];
            const T* ps = psm[(m - dir) & 3];
            const T gpx = (pc[t + 1] - pc[t - 1]) * third + ((pn[t + 1] - pn[t - 1]) + (ps[t + 1] - ps[t - 1])) * twelfth;
            const T gpy = (pn[t] - ps[t]) * third + ((pn[t + 1] - ps[t + 1]) + (pn[t - 1] - ps[t - 1])) * twelfth;
            const T h = hsm[s8][t] + C.href;
            const T Jx = rjx[s4][t], Jy = rjy[s4][t];
            // adjoints through the equilibria (Eq. equilibria, e = 1) and the
            // source 3 w_l c_l . F, summed over l in closed form
            const T ih = fdiv(T(1), h);
            const T ux = Jx * ih, uy = Jy * ih, q = ux * ux + uy * uy, gh = C.g * h;
            const T p15 = mu[1] + mu[5], p37 = mu[3] + mu[7], p26 = mu[2] + mu[6], p48 = mu[4] + mu[8];
            const T sax = p15 + p37, sdg = p26 + p48;
            const T aFx = (mu[1] - mu[5]) * third + ((mu[2] - mu[6]) + (mu[8] - mu[4])) * twelfth;
            const T aFy = (mu[3] - mu[7]) * third + ((mu[2] - mu[6]) + (mu[4] - mu[8])) * twelfth;
            const T ua = ux + uy, ub = ux - uy;
            const T ahe = mu[0] * (T(1) - T(5.0 / 3.0) * gh + T(2.0 / 3.0) * q)
                        + (gh * third + q * T(1.0 / 6.0)) * sax - T(0.5) * (ux * ux * p15 + uy * uy * p37)
                        + (gh * twelfth + q * T(1.0 / 24.0)) * sdg - T(0.125) * (ua * ua * p26 + ub * ub * p48);
            const T cross_x = T(0.25) * (ua * p26 + ub * p48), cross_y = T(0.25) * (ua * p26 - ub * p48);
            const T ajxe = -T(4.0 / 3.0) * ux * mu[0] + aFx + ux * p15 - ux * sax * third + cross_x - ux * sdg * twelfth;
            const T ajye = -T(4.0 / 3.0) * uy * mu[0] + aFy + uy * p37 - uy * sax * third + cross_y - uy * sdg * twelfth;
            // Eqs. (forcefric, alphafric): nu alpha u = fr j, fr = 6 nu / (2h^2 + 6 delta h + 3 delta^2)
            const T den = h * (T(2) * h + T(6) * C.delta) + T(3) * C.delta * C.delta;
            const T iden = fdiv(T(1), den);
            const T fr = C.nu6 * iden;
            const T dfr = -fr * (T(4) * h + T(6) * C.delta) * iden;
            rah[s8][t] = C.omega * ahe + aFx * (C.gx - gpx) + aFy * (C.gy - gpy) - dfr * (aFx * Jx + aFy * Jy);
            rajx[s8][t] = C.omega * ajxe - fr * aFx;
            rajy[s8][t] = C.omega * ajye - fr * aFy;
            agx[s4][t] = -h * aFx;
            agy[s4][t] = -h * aFy;
        }
        // ---- D: transposed gradient and disjoining-pressure adjoint at row r(k-5)
        if (k >= 8 && k <= R + 9 && cD) {
            const int m = k - 5, s8 = m & 7;
            const int gu = (m + dir) & 3, gc = m & 3, gd = (m - dir) & 3;
            // ap(x) = sum_l 3 w_l c_l . ag(x - c_l)
            const T apv = ((agx[gc][t - 1] - agx[gc][t + 1]) + (agy[gd][t] - agy[gu][t])) * third
                        + (((agx[gd][t - 1] + agy[gd][t - 1]) + (agy[gd][t + 1] - agx[gd][t + 1]))
                           + ((agx[gu][t - 1] - agy[gu][t - 1]) - (agx[gu][t + 1] + agy[gu][t + 1]))) * twelfth;
            als[gc][t] = -C.gamma * apv;
            // d/dkappa of Pi does not vanish where kappa does: always accumulate
            const T api = -C.gamma * C.pi_sgn * apv;
            const T h = hsm[s8][t] + C.href, ih = fdiv(T(1), h);
            const T r = C.hstar * ih;
            const T rn = ipow(r, C.n_exp), rm = ipow(r, C.m_exp);
            const long long i = (long long)d0 * nx + x;
            const T kap = kappa ? kappa[i] : C.kappa_u;
            rah[s8][t] += api * kap * (T(C.m_exp) * rm - T(C.n_exp) * rn) * ih;
            if (m >= 4 && m <= R + 3 && cE) gk[i] += api * (rn - rm);
        }
        // ---- E: Laplacian transpose and a(t) at row r(k-7)
        if (k >= 11 && cE) {
            const int m = k - 7, s8 = m & 7;
            const int lu = (m + dir) & 3, lc = m & 3, ld = (m - dir) & 3;
            const T axis = (als[lc][t - 1] + als[lc][t + 1]) + (als[lu][t] + als[ld][t]);
            const T diag = (als[lu][t - 1] + als[lu][t + 1]) + (als[ld][t - 1] + als[ld][t + 1]);
            const T ah = rah[s8][t] + (T(4) * axis + diag - T(20) * als[lc][t]) * T(1.0 / 6.0);
            const T ajx = rajx[s8][t], ajy = rajy[s8][t], om = T(1) - C.omega;
            const int y = e0, yU = dir > 0 ? ep : em, yD = dir > 0 ? em : ep;
            T mu[9];
            if (om != T(0)) {
                gather(y, yU, yD, mu);
            } else {  // (1 - omega) mu_l vanishes at tau = 1
#pragma unroll
                for (int l = 0; l < 9; ++l) mu[l] = T(0);
            }
            T* o = a + ((long long)y * nx + x);
            o[0] = ah + om * mu[0];
            o[n] = ah + ajx + om * mu[1];
            o[2 * n] = ah + (ajx + ajy) + om * mu[2];
            o[3 * n] = ah + ajy + om * mu[3];
            o[4 * n] = ah + (ajy - ajx) + om * mu[4];
            o[5 * n] = ah - ajx + om * mu[5];
            o[6 * n] = ah - (ajx + ajy) + om * mu[6];
            o[7 * n] = ah - ajy + om * mu[7];
            o[8 * n] = ah + (ajx - ajy) + om * mu[8];
        }
        adv(am);
        adv(a0);
        adv(ap1);
        adv(cm);
        adv(c0);
        adv(cp);
        adv(d0);
        adv(em);
        adv(e0);
        adv(ep);
    }
}

}  // namespace tflbm
