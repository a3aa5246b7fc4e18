// Device code shared by the DD-CCLB kernels (arXiv 2311.10314, Sec. 3).
//
// The per-node update is written once, against two small interfaces so the
// tile kernel and the row-sweep kernel feed it from their own shared-memory
// layouts:
//   accessor  C(j, dy, dx)  C_j (j < N-1) at the neighbour (x+dx, y+dy)
//             psi(dy, dx)   the characteristic function psi
//             mu(j, dy, dx) mu_j (j < N) of Eq. 2.14
//             a(dy, dx)     the lagged antisymmetric-flux field a
//             lag(k)        lagged plane k at the node
//             f(i, p), g(p) pre-collision populations at the node
//   sink      f_out(i, p, v), g_out(p, v)   post-collision populations that
//                                           leave the node in direction p
//             lag_out(k, v)                 lagged plane k of the next step
//             macro(C, rho, ux, uy, P, mu)  read-out mode only
#pragma once

#include "ddcc_internal.h"

namespace ddcc {
namespace dev {

// Periodic wrap, or reflection about the outer wall half a node outside
// the first and last node (mirror ghost nodes).
__device__ __forceinline__ int map_index(int g, int n, int periodic) {
    if (periodic) {
        g %= n;
        return g < 0 ? g + n : g;
    }
    const int n2 = 2 * n;
    int m = g % n2;
    if (m < 0) m += n2;
    return m >= n ? n2 - 1 - m : m;
}

// g(C) = C^2 (C - 1)^2  =>  g'(C) = 2 C (C - 1) (2 C - 1)  (Sec. 2.1).
template <typename T>
__device__ __forceinline__ T gprime(T c) {
    return T(2) * c * (c - T(1)) * (T(2) * c - T(1));
}

// Gradient stencil sum_p w_p c_p chi(x + c_p) / cs2 (isotropic, radius 1).
template <typename T, class A>
__device__ __forceinline__ void grad9(const KParams<T>& P, const A& chi, T& gx, T& gy) {
    const T e = chi(0, 1), w = chi(0, -1), n = chi(1, 0), s = chi(-1, 0);
    const T ne = chi(1, 1), nw = chi(1, -1), sw = chi(-1, -1), se = chi(-1, 1);
    gx = P.gw1 * (e - w) + P.gw2 * ((ne - nw) + (se - sw));
    gy = P.gw1 * (n - s) + P.gw2 * ((ne + nw) - (se + sw));
}

// mu_i = psi mu_i / psi with psi mu_i of Eq. 2.14: beta_ij = 3 sigma_ij / eps,
// gradient term (3 eps / 4) sigma_ij div(psi grad C_j), wetting term
// 3 sigma_ij sum_{q != j} cos(theta_jq) C_j C_q |grad psi| with cos(theta_jq)
// from the N-1 angles theta_iN by Eq. 2.9 (cth holds cos(theta_iN)).  With
// several solids (Sec. 4.5) cth holds e_j = sum_k cos(theta^k_jN) |grad psi_k|
// and |grad psi| is replaced by 1: Eq. 2.9 is linear in the cosines, so
// sum_k cos(theta^k_jq) |grad psi_k| = (sigma_jN e_j - sigma_qN e_q) / sigma_jq.
// Cx(j, dy, dx) gives C_j for j < NP-1; Ps(dy, dx) gives psi.
template <typename T, int NP, class CA, class PA>
__device__ __forceinline__ void chem_pot(const KParams<T>& P, const CA& Cx, const PA& Ps,
                                         const T* cth, T mu[NP]) {
    const T p0 = Ps(0, 0);
    const T pE = Ps(0, 1), pW = Ps(0, -1), pN = Ps(1, 0), pS = Ps(-1, 0);
    const T pNE = Ps(1, 1), pNW = Ps(1, -1), pSW = Ps(-1, -1), pSE = Ps(-1, 1);
    const T gpx = P.gw1 * (pE - pW) + P.gw2 * ((pNE - pNW) + (pSE - pSW));
    const T gpy = P.gw1 * (pN - pS) + P.gw2 * ((pNE + pNW) - (pSE + pSW));
    // with several solids the angle planes already carry |grad psi_k|
    const T agp = P.wet_field ? T(1) : sqrt(gpx * gpx + gpy * gpy);
    T Cv[NP], L[NP];
    T sumC = T(0), sumL = T(0);
#pragma unroll
    for (int j = 0; j < NP - 1; ++j) {
        const T c0 = Cx(j, 0, 0);
        // div(psi grad C) = sum_p w_p (psi + psi_p)(C_p - C) / cs2
        const T l = P.lw1 * ((p0 + pE) * (Cx(j, 0, 1) - c0) + (p0 + pW) * (Cx(j, 0, -1) - c0) +
                             (p0 + pN) * (Cx(j, 1, 0) - c0) + (p0 + pS) * (Cx(j, -1, 0) - c0)) +
                    P.lw2 * ((p0 + pNE) * (Cx(j, 1, 1) - c0) + (p0 + pNW) * (Cx(j, 1, -1) - c0) +
                             (p0 + pSW) * (Cx(j, -1, -1) - c0) + (p0 + pSE) * (Cx(j, -1, 1) - c0));
        Cv[j] = c0;
        L[j] = l;
        sumC += c0;
        sumL += l;
    }
    Cv[NP - 1] = T(1) - sumC;
    L[NP - 1] = -sumL;
    // a_j = sigma_jN cos(theta_jN) (zero for j = N, sigma_NN = 0), so that
    // cos(theta_jq) = (a_j - a_q) / sigma_jq, antisymmetric in (j, q)
    T aj[NP], gp[NP];
#pragma unroll
    for (int j = 0; j < NP; ++j) {
        aj[j] = j < NP - 1 ? P.sigN[j] * cth[j] : T(0);
        gp[j] = gprime(Cv[j]);
    }
    // symmetric g'(C_i + C_j) and antisymmetric cos(theta_ij), once per pair
    T gpair[NP][NP], cpair[NP][NP];
#pragma unroll
    for (int i = 0; i < NP; ++i) {
        cpair[i][i] = T(0);
        gpair[i][i] = T(0);
#pragma unroll
        for (int j = i + 1; j < NP; ++j) {
            gpair[i][j] = gpair[j][i] = gprime(Cv[i] + Cv[j]);
            const T c = (aj[i] - aj[j]) * P.invsig[i][j];
            cpair[i][j] = c;
            cpair[j][i] = -c;
        }
    }
    // W_j = C_j sum_{q != j} cos(theta_jq) C_q
    T Wj[NP];
#pragma unroll
    for (int j = 0; j < NP; ++j) {
        T acc = T(0);
#pragma unroll
        for (int q = 0; q < NP; ++q)
            if (q != j) acc += cpair[j][q] * Cv[q];
        Wj[j] = Cv[j] * acc;
    }
    const T inv_p0 = T(1) / p0;
#pragma unroll
    for (int i = 0; i < NP; ++i) {
        T bulk = T(0), grad = T(0), wet = T(0);
#pragma unroll
        for (int j = 0; j < NP; ++j) {
            if (j != i) bulk += P.beta2[i][j] * (gp[i] - gpair[i][j]);
            grad += P.kap[i][j] * L[j];
            wet += P.wet[i][j] * Wj[j];
        }
        const T psimu = p0 * bulk + grad + agp * wet;
        mu[i] = psimu * inv_p0;
    }
}

// Hermite moments m_ab = sum_p v_p h_a(cx_p) h_b(cy_p), h = (1, c, c^2 - cs2),
// in the order (00, 10, 01, 20, 02, 11, 21, 12, 22).
template <typename T>
__device__ __forceinline__ void hermite_moments(const T v[9], T cs2, T m[9]) {
    // pass over cx in each row cy = -1, 0, +1 (populations (cx, cy)):
    //   A0 = sum, A1 = v(+1) - v(-1), A2 = v(+1) + v(-1) - cs2 A0
    const T sm0 = v[7] + v[8], sz0 = v[3] + v[1], sp0 = v[6] + v[5];
    const T A0m = sm0 + v[4], A0z = sz0 + v[0], A0p = sp0 + v[2];
    const T A1m = v[8] - v[7], A1z = v[1] - v[3], A1p = v[5] - v[6];
    const T A2m = sm0 - cs2 * A0m, A2z = sz0 - cs2 * A0z, A2p = sp0 - cs2 * A0p;
    // pass over cy with h_b(cy)
    m[0] = A0m + A0z + A0p;
    m[2] = A0p - A0m;
    m[4] = (A0p + A0m) - cs2 * m[0];
    m[1] = A1m + A1z + A1p;
    m[5] = A1p - A1m;
    m[7] = (A1p + A1m) - cs2 * m[1];
    m[3] = A2m + A2z + A2p;
    m[6] = A2p - A2m;
    m[8] = (A2p + A2m) - cs2 * m[3];
}

// Rounded to nearest and never fused or reassociated by the compiler.
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }

// B_p = sum_ab h_a(cx_p) h_b(cy_p) k_ab; out_p = v_p - w_p B_p.
// kConserve (the phase populations, which carry the conserved psi C): the
// rest population holds nearly all of psi C, so v_0 - w_0 B_0 rounds at the
// ulp of psi C, and in a steady flow the same rounding repeats every step
// and drifts the phase mass.  Then w_0 B_0 and the subtraction are rounded
// explicitly, the exact error of the subtraction is recovered (TwoSum) and
// split evenly (halving is exact) between out_1 and out_3, the +x and -x
// populations, far smaller in magnitude: sum_p out_p keeps the exchange up
// to roundings at that smaller scale, and the recovered mass leaves the
// node in no preferred direction (a steady error put on one direction
// would carry phase mass along it every step).
template <typename T, bool kConserve = false>
__device__ __forceinline__ void hermite_relax_back(const T k[9], T cs2, const T w1d[3], const T v[9],
                                                   T out[9]) {
    // R_a(cy) = k_a0 + cy k_a1 + (cy^2 - cs2) k_a2 for a = 0, 1, 2
    const T ka0[3] = {k[0], k[1], k[3]};
    const T ka1[3] = {k[2], k[5], k[6]};
    const T ka2[3] = {k[4], k[7], k[8]};
    T Rm[3], R0[3], Rp[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const T base = ka0[a] + (T(1) - cs2) * ka2[a];
        R0[a] = ka0[a] - cs2 * ka2[a];
        Rp[a] = base + ka1[a];
        Rm[a] = base - ka1[a];
    }
    // B(cx, cy) = R_0 + cx R_1 + (cx^2 - cs2) R_2
    const T one_m = T(1) - cs2;
    const T wm = w1d[0], wz = w1d[1], wp = w1d[2];
    T err = T(0);
    if constexpr (kConserve) {
        const T t0 = mul_rn(wz * wz, R0[0] - cs2 * R0[2]);
        const T o0 = add_rn(v[0], -t0);
        const T bb = add_rn(o0, -v[0]);                 // TwoSum(v_0, -t_0)
        err = add_rn(add_rn(v[0], -add_rn(o0, -bb)), add_rn(-t0, -bb));
        out[0] = o0;
    } else {
        out[0] = v[0] - wz * wz * (R0[0] - cs2 * R0[2]);
    }
    out[1] = v[1] - wp * wz * (R0[0] + R0[1] + one_m * R0[2]);
    out[2] = v[2] - wz * wp * (Rp[0] - cs2 * Rp[2]);
    out[3] = v[3] - wm * wz * (R0[0] - R0[1] + one_m * R0[2]);
    if constexpr (kConserve) {
        const T half = T(0.5) * err;
        out[1] = add_rn(out[1], half);
        out[3] = add_rn(out[3], half);
    }
    out[4] = v[4] - wz * wm * (Rm[0] - cs2 * Rm[2]);
    out[5] = v[5] - wp * wp * (Rp[0] + Rp[1] + one_m * Rp[2]);
    out[6] = v[6] - wm * wp * (Rp[0] - Rp[1] + one_m * Rp[2]);
    out[7] = v[7] - wm * wm * (Rm[0] - Rm[1] + one_m * Rm[2]);
    out[8] = v[8] - wp * wm * (Rm[0] + Rm[1] + one_m * Rm[2]);
}

// One node of the step: order parameters and gradients (a1, a2), mobility
// flux and m^C (a4), force, the joint velocity / Eq. 19 pressure solve
// (a5, a6), then (MODE 0) both collisions in Hermite moment space (a7, a8)
// and the lagged fields (a10), or (MODE 1) the macroscopic read-out.
template <typename T, int NP, int MODE, class Acc, class Sink>
__device__ __forceinline__ void node_update(const KParams<T>& P, const Acc& A, Sink& out) {
    const T cs2 = P.cs2;
    const T psi = A.psi(0, 0);

    // ---- order parameters and their gradients -----------------------------
    T Cv[NP], gCx[NP], gCy[NP];
    {
        T sC = T(0), sx = T(0), sy = T(0);
#pragma unroll
        for (int j = 0; j < NP - 1; ++j) {
            Cv[j] = A.C(j, 0, 0);
            grad9(P, [&](int dy, int dx) { return A.C(j, dy, dx); }, gCx[j], gCy[j]);
            sC += Cv[j];
            sx += gCx[j];
            sy += gCy[j];
        }
        Cv[NP - 1] = T(1) - sC;
        gCx[NP - 1] = -sx;
        gCy[NP - 1] = -sy;
    }
    T rho = T(0), nu = T(0), grx = T(0), gry = T(0);
#pragma unroll
    for (int j = 0; j < NP; ++j) {
        rho += Cv[j] * P.rho[j];
        nu += Cv[j] * P.nu[j];
        grx += P.rho[j] * gCx[j];
        gry += P.rho[j] * gCy[j];
    }
    // s21 and s22 from nu by Eq. 16
    const T inv_s21 = nu * P.nu_to_s21 + T(0.5);
    const T s21 = T(1) / inv_s21;
    const T s22 = T(1) / (nu * P.nu_to_s22 + T(0.5));
    T gpx, gpy;
    grad9(P, [&](int dy, int dx) { return A.psi(dy, dx); }, gpx, gpy);
    // grad(psi rho): stencil on psi(x+c) rho(x+c), rho = rho_N + sum (rho_j - rho_N) C_j
    T gprx, gpry;
    grad9(
        P,
        [&](int dy, int dx) {
            T r = P.rho[NP - 1];
#pragma unroll
            for (int j = 0; j < NP - 1; ++j) r += (P.rho[j] - P.rho[NP - 1]) * A.C(j, dy, dx);
            return A.psi(dy, dx) * r;
        },
        gprx, gpry);

    // ---- chemical potentials, mobility flux, m^C --------------------------
    T mu[NP], gmx[NP], gmy[NP];
#pragma unroll
    for (int j = 0; j < NP; ++j) {
        mu[j] = A.mu(j, 0, 0);
        grad9(P, [&](int dy, int dx) { return A.mu(j, dy, dx); }, gmx[j], gmy[j]);
    }
    // Q_i = sum_j M_ij grad mu_j = m0 C_i (S_C grad mu_i - sum_j C_j grad mu_j)
    T SC = T(0), Gx = T(0), Gy = T(0);
#pragma unroll
    for (int j = 0; j < NP; ++j) {
        SC += Cv[j];
        Gx += Cv[j] * gmx[j];
        Gy += Cv[j] * gmy[j];
    }
    // q_i = Q_i / m0; m^C = -m0 sum_i rho_i q_i
    T Qx[NP], Qy[NP];
    T mCx = T(0), mCy = T(0);
#pragma unroll
    for (int i = 0; i < NP; ++i) {
        Qx[i] = Cv[i] * (SC * gmx[i] - Gx);
        Qy[i] = Cv[i] * (SC * gmy[i] - Gy);
        mCx -= P.rho[i] * Qx[i];
        mCy -= P.rho[i] * Qy[i];
    }
    mCx *= P.m0;
    mCy *= P.m0;

    // ---- lagged fields of the previous step --------------------------------
    T dax, day;
    grad9(P, [&](int dy, int dx) { return A.a(dy, dx); }, dax, day);
    const T psimu_prev = A.lag(2 * NP + 2);

    // ---- flow populations, velocity and pressure ---------------------------
    T g[9];
#pragma unroll
    for (int p = 0; p < 9; ++p) g[p] = A.g(p);
    const T Jx = (g[1] - g[3]) + (g[5] - g[6]) + (g[8] - g[7]);
    const T Jy = (g[2] - g[4]) + (g[5] + g[6]) - (g[7] + g[8]);
    T F0x = day + psi * rho * P.body[0];
    T F0y = -dax + psi * rho * P.body[1];
#pragma unroll
    for (int j = 0; j < NP; ++j) {
        const T pm = psi * mu[j];
        F0x += pm * gCx[j];
        F0y += pm * gCy[j];
    }
    const T dmp = P.damp * (T(1) - psi);
    const T inv_den = T(1) / (psi * rho + T(0.5) * dmp);
    const T u0x = (Jx + T(0.5) * F0x) * inv_den;
    const T u0y = (Jy + T(0.5) * F0y) * inv_den;
    const T ex = T(0.5) * gpx * inv_den;
    const T ey = T(0.5) * gpy * inv_den;
    const T Hs = P.Hfac * (s21 - T(2)) * inv_s21;     // H / s21
    const T bx = P.A_P * psi * grx + P.gam * psi * mCx + Hs * gprx;
    const T by = P.A_P * psi * gry + P.gam * psi * mCy + Hs * gpry;
    const T gq = P.gam * psi * rho;
    const T sum_g = ((g[1] + g[2]) + (g[3] + g[4])) + ((g[5] + g[6]) + (g[7] + g[8]));
    const T G0 = sum_g - P.Kh * psimu_prev;
    const T qa = P.cP * gq * (ex * ex + ey * ey);
    const T qb = P.cP * (bx * ex + by * ey + T(2) * gq * (u0x * ex + u0y * ey)) - psi;
    const T qc = P.cP * (G0 + bx * u0x + by * u0y + gq * (u0x * u0x + u0y * u0y));
    T disc = qb * qb - T(4) * qa * qc;
    disc = disc > T(0) ? disc : T(0);
    const T root = sqrt(disc);
    const T Pr = T(-2) * qc / (qb < T(0) ? qb - root : qb + root);
    const T ux = u0x + Pr * ex;
    const T uy = u0y + Pr * ey;
    const T Fx = F0x + Pr * gpx - dmp * ux;
    const T Fy = F0y + Pr * gpy - dmp * uy;
    const T psiP = psi * Pr;

    if (MODE == 1) {
        out.macro(Cv, rho, ux, uy, Pr, mu);
        return;
    }

    const T w1d[3] = {P.w1d[0], P.w1d[1], P.w1d[2]};

    // ---- phase LB, Eqs. 3.1, 3.5-3.7 ---------------------------------------
#pragma unroll
    for (int i = 0; i < NP - 1; ++i) {
        T v[9], m[9], k[9], o9[9];
#pragma unroll
        for (int p = 0; p < 9; ++p) v[p] = A.f(i, p);
        hermite_moments(v, cs2, m);
        const T psiC = m[0];
        const T pcux = psiC * ux, pcuy = psiC * uy;
        const T dtx = pcux - A.lag(1 + 2 * i);
        const T dty = pcuy - A.lag(2 + 2 * i);
        // S_i = (psi / m0) Q_i - psi grad mu_i, with Qx holding Q_i / m0
        const T Sx = psi * (Qx[i] - gmx[i]);
        const T Sy = psi * (Qy[i] - gmy[i]);
        const T ceta = cs2 * P.eta[i];
        const T Vx = dtx + ceta * (mu[i] * gpx - Sx);
        const T Vy = dty + ceta * (mu[i] * gpy - Sy);
        const T X = psiC - P.eta[i] * psi * mu[i];
        const T* lam = P.lamf[i];
        k[0] = T(0);
        k[1] = lam[1] * (m[1] - pcux + T(0.5) * Vx) - Vx * P.invN[1];
        k[2] = lam[2] * (m[2] - pcuy + T(0.5) * Vy) - Vy * P.invN[2];
        k[3] = lam[3] * (m[3] + cs2 * X);
        k[4] = lam[4] * (m[4] + cs2 * X);
        k[5] = lam[5] * m[5];
        k[6] = lam[6] * m[6];
        k[7] = lam[7] * m[7];
        k[8] = lam[8] * (m[8] - cs2 * cs2 * X);
        hermite_relax_back<T, true>(k, cs2, w1d, v, o9);
#pragma unroll
        for (int p = 0; p < 9; ++p) out.f_out(i, p, o9[p]);
        out.lag_out(1 + 2 * i, pcux);
        out.lag_out(2 + 2 * i, pcuy);
    }

    // ---- flow LB, Eqs. 3.2, 3.8, 3.10 --------------------------------------
    {
        T m[9], k[9], o9[9];
        hermite_moments(g, cs2, m);
        const T psirho = psi * rho;
        const T Axx = psirho * ux * ux + psi * mCx * ux;
        const T Ayy = psirho * uy * uy + psi * mCy * uy;
        const T Axy = psirho * ux * uy + T(0.5) * (psi * mCx * uy + psi * ux * mCy);
        const T Txx = psi * mCx * ux;
        const T Tyy = psi * mCy * uy;
        const T Txy = T(0.5) * (psi * mCx * uy + psi * ux * mCy);
        const T ugpr = ux * gprx + uy * gpry;
        const T Mxx = (Txx - A.lag(2 * NP - 1)) + T(2) * cs2 * ux * gprx + P.c2m3cs2 * ugpr;
        const T Myy = (Tyy - A.lag(2 * NP)) + T(2) * cs2 * uy * gpry + P.c2m3cs2 * ugpr;
        const T Mxy = (Txy - A.lag(2 * NP + 1)) + cs2 * (ux * gpry + gprx * uy);
        const T a0 = psi * (ux * grx + uy * gry);
        const T l20 = s21 * P.invN20, l11 = s22 * P.invN11;
        k[0] = P.lg00 * (m[0] + T(0.5) * a0) - a0;
        k[1] = P.lg1 * (m[1] - psirho * ux + T(0.5) * Fx) - Fx * P.invN[1];
        k[2] = P.lg1 * (m[2] - psirho * uy + T(0.5) * Fy) - Fy * P.invN[2];
        k[3] = l20 * (m[3] - psiP - Axx + T(0.5) * Mxx) - Mxx * P.invN20;
        k[4] = l20 * (m[4] - psiP - Ayy + T(0.5) * Myy) - Myy * P.invN20;
        k[5] = l11 * (m[5] - Axy + T(0.5) * Mxy) - Mxy * P.invN11;
        k[6] = P.lg3 * m[6];
        k[7] = P.lg3 * m[7];
        k[8] = P.lg4 * (m[8] + cs2 * psiP);
        hermite_relax_back(k, cs2, w1d, g, o9);
#pragma unroll
        for (int p = 0; p < 9; ++p) out.g_out(p, o9[p]);
        out.lag_out(0, T(0.5) * psi * (mCx * uy - ux * mCy));
        out.lag_out(2 * NP - 1, Txx);
        out.lag_out(2 * NP, Tyy);
        out.lag_out(2 * NP + 1, Txy);
        out.lag_out(2 * NP + 2, psi * (rho * (ux * ux + uy * uy) + mCx * ux + mCy * uy));
    }
}

}  // namespace dev
}  // namespace ddcc
