// sm_103a kernels of the DD-CCLB time step (arXiv 2311.10314, Sec. 3).
//
// One step is two launches:
//   k_order_param  psi C_i = sum_p f^i_p, C_i = psi C_i / psi  (recovery of
//                  the order parameters, Sec. 3) -> C scratch planes;
//   k_step         per 32 x 8 tile: C and psi with a 2-node halo and the
//                  lagged field a with a 1-node halo are staged in shared
//                  memory, mu_i (Eq. 2.14) is evaluated on the tile plus a
//                  1-node halo, then every node computes the mobility flux
//                  (Eq. 2.5, 3.7), m^C, the force, the joint velocity /
//                  pressure solve (Sec. 3, Eq. 19), both collisions in
//                  Hermite moment space and pushes its post-collision
//                  populations to its neighbours (Eqs. 3.1, 3.2).
// The collision Lambda = H^-1 S H is applied as moments -> relax -> back,
// using that the d0 weights factor as w(cx, cy) = w1(cx) w1(cy) with
// w1 = (d0/2, 1-d0, d0/2): the Hermite rows are then orthogonal with norms
// N_ab = n_a n_b (n = 1, d0, d0 (1-d0)) and H^-1 = W H^T N^-1, so each
// 9 x 9 transform is two passes of 3-point transforms.
#include "ddcc_internal.h"

namespace ddcc {
namespace {

constexpr int BX = kTileX;
constexpr int BY = kTileY;
constexpr int NT = BX * BY;
constexpr int H2W = BX + 4, H2H = BY + 4;   // tile + 2-node halo
constexpr int H1W = BX + 2, H1H = BY + 2;   // tile + 1-node halo

// D2Q9 velocities (Sec. 3): 0 rest, 1-4 axis, 5-8 diagonal.
__constant__ int kCx[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
__constant__ int kCy[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};

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

template <typename T, int NP>
struct Smem {
    T C[NP - 1][H2H][H2W];
    T psi[H2H][H2W];
    T mu[NP][H1H][H1W];
    T a[H1H][H1W];
    T cth[NP - 1][H1H][H1W];
};

// Stage C (N-1 planes) and psi with a 2-node halo, a and cos(theta_iN)
// with a 1-node halo.
template <typename T, int NP>
__device__ void load_tile(const KParams<T>& P, Smem<T, NP>& sm, const T* __restrict__ C,
                          const T* __restrict__ psi, const T* __restrict__ cosf,
                          const T* __restrict__ a_in, int x0, int y0, int tid) {
    for (int k = tid; k < H2H * H2W; k += NT) {
        const int ly = k / H2W, lx = k - ly * H2W;
        const int gx = map_index(x0 + lx - 2, P.nx, P.px);
        const int gy = map_index(y0 + ly - 2, P.ny, P.py);
        const long long o = (long long)gy * P.pitch + gx;
        sm.psi[ly][lx] = psi[o];
#pragma unroll
        for (int i = 0; i < NP - 1; ++i) sm.C[i][ly][lx] = C[i * P.plane + o];
    }
    for (int k = tid; k < H1H * H1W; k += NT) {
        const int ly = k / H1W, lx = k - ly * H1W;
        const int gx = map_index(x0 + lx - 1, P.nx, P.px);
        const int gy = map_index(y0 + ly - 1, P.ny, P.py);
        const long long o = (long long)gy * P.pitch + gx;
        sm.a[ly][lx] = a_in ? a_in[o] : T(0);
#pragma unroll
        for (int i = 0; i < NP - 1; ++i)
            sm.cth[i][ly][lx] = P.has_cos_field ? cosf[i * P.plane + o] : P.cos_uni[i];
    }
}

// mu_i = psi mu_i / psi with psi mu_i of Eq. 2.14 (beta_ij = 3 sigma_ij / eps,
// the wetting weights cos(theta_jq) of Eq. 2.9) on the tile + 1-node halo.
template <typename T, int NP>
__device__ void compute_mu_tile(const KParams<T>& P, Smem<T, NP>& sm, int tid) {
    for (int k = tid; k < H1H * H1W; k += NT) {
        const int ly = k / H1W, lx = k - ly * H1W;
        const int cy = ly + 1, cx = lx + 1;
        const T p0 = sm.psi[cy][cx];
        const T pE = sm.psi[cy][cx + 1], pW = sm.psi[cy][cx - 1];
        const T pN = sm.psi[cy + 1][cx], pS = sm.psi[cy - 1][cx];
        const T pNE = sm.psi[cy + 1][cx + 1], pNW = sm.psi[cy + 1][cx - 1];
        const T pSW = sm.psi[cy - 1][cx - 1], pSE = sm.psi[cy - 1][cx + 1];
        const T gpx = P.gw1 * (pE - pW) + P.gw2 * ((pNE - pNW) + (pSE - pSW));
        const T gpy = P.gw1 * (pN - pS) + P.gw2 * ((pNE + pNW) - (pSE + pSW));
        const T agp = sqrt(gpx * gpx + gpy * gpy);
        T Cv[NP], L[NP];
        T sumC = T(0), sumL = T(0);
#pragma unroll
        for (int j = 0; j < NP - 1; ++j) {
            const T c0 = sm.C[j][cy][cx];
            // div(psi grad C) = sum_p w_p (psi + psi_p)(C_p - C) / cs2
            const T l = P.lw1 * ((p0 + pE) * (sm.C[j][cy][cx + 1] - c0) +
                                 (p0 + pW) * (sm.C[j][cy][cx - 1] - c0) +
                                 (p0 + pN) * (sm.C[j][cy + 1][cx] - c0) +
                                 (p0 + pS) * (sm.C[j][cy - 1][cx] - c0)) +
                        P.lw2 * ((p0 + pNE) * (sm.C[j][cy + 1][cx + 1] - c0) +
                                 (p0 + pNW) * (sm.C[j][cy + 1][cx - 1] - c0) +
                                 (p0 + pSW) * (sm.C[j][cy - 1][cx - 1] - c0) +
                                 (p0 + pSE) * (sm.C[j][cy - 1][cx + 1] - c0));
            Cv[j] = c0;
            L[j] = l;
            sumC += c0;
            sumL += l;
        }
        Cv[NP - 1] = T(1) - sumC;
        L[NP - 1] = -sumL;
        T cN[NP];
#pragma unroll
        for (int i = 0; i < NP - 1; ++i) cN[i] = sm.cth[i][ly][lx];
        cN[NP - 1] = T(0);
        // W_j = C_j sum_{q != j} cos(theta_jq) C_q
        T Wj[NP], gp[NP];
#pragma unroll
        for (int j = 0; j < NP; ++j) {
            T acc = T(0);
#pragma unroll
            for (int q = 0; q < NP; ++q) {
                if (q == j) continue;
                const T cjq = (P.sigN[j] * cN[j] - P.sigN[q] * cN[q]) * P.invsig[j][q];
                acc += cjq * Cv[q];
            }
            Wj[j] = Cv[j] * acc;
            gp[j] = gprime(Cv[j]);
        }
#pragma unroll
        for (int i = 0; i < NP; ++i) {
            T bulk = T(0), grad = T(0), wet = T(0);
#pragma unroll
            for (int j = 0; j < NP; ++j) {
                if (j != i) bulk += P.beta2[i][j] * (gp[i] - gprime(Cv[i] + Cv[j]));
                grad += P.kap[i][j] * L[j];
                wet += P.wet[i][j] * Wj[j];
            }
            const T psimu = p0 * bulk + grad + agp * wet;
            sm.mu[i][ly][lx] = psimu / p0;
        }
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

// B_p = sum_ab h_a(cx_p) h_b(cy_p) k_ab; out_p = v_p - w_p B_p.
template <typename T>
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
    auto B = [&](const T R[3], int cx) -> T {
        const T c2 = (cx == 0) ? -cs2 : (T(1) - cs2);
        return R[0] + T(cx) * R[1] + c2 * R[2];
    };
    const T wm = w1d[0], wz = w1d[1], wp = w1d[2];
    out[0] = v[0] - wz * wz * B(R0, 0);
    out[1] = v[1] - wp * wz * B(R0, 1);
    out[2] = v[2] - wz * wp * B(Rp, 0);
    out[3] = v[3] - wm * wz * B(R0, -1);
    out[4] = v[4] - wz * wm * B(Rm, 0);
    out[5] = v[5] - wp * wp * B(Rp, 1);
    out[6] = v[6] - wm * wp * B(Rp, -1);
    out[7] = v[7] - wm * wm * B(Rm, -1);
    out[8] = v[8] - wp * wm * B(Rm, 1);
}

// Gradient stencil sum_p w_p c_p chi(x + c_p) / cs2 on a shared array.
#define DDCC_GRAD(arr, yy, xx, gx, gy)                                                   \
    do {                                                                                 \
        const T _e = arr[yy][xx + 1], _w = arr[yy][xx - 1];                              \
        const T _n = arr[yy + 1][xx], _s = arr[yy - 1][xx];                              \
        const T _ne = arr[yy + 1][xx + 1], _nw = arr[yy + 1][xx - 1];                    \
        const T _sw = arr[yy - 1][xx - 1], _se = arr[yy - 1][xx + 1];                    \
        gx = P.gw1 * (_e - _w) + P.gw2 * ((_ne - _nw) + (_se - _sw));                    \
        gy = P.gw1 * (_n - _s) + P.gw2 * ((_ne + _nw) - (_se + _sw));                    \
    } while (0)

// MODE 0: full step (collide + push-stream + lagged fields).
// MODE 1: macroscopic read-out of the current state (no state change).
template <typename T, int NP, int MODE>
__global__ void __launch_bounds__(NT) k_step(KParams<T> P, Fields<T> F, int cur) {
    __shared__ Smem<T, NP> sm;
    const int tid = threadIdx.x + BX * threadIdx.y;
    const int x0 = blockIdx.x * BX, y0 = blockIdx.y * BY;
    // select ping-pong copies without indexing the parameter struct at run
    // time (that would copy it to local memory)
    const T* __restrict__ lag_in = cur ? F.lag[1] : F.lag[0];
    T* __restrict__ lag_out = cur ? F.lag[0] : F.lag[1];
    const T* __restrict__ fin = cur ? F.f[1] : F.f[0];
    T* __restrict__ fout = cur ? F.f[0] : F.f[1];
    const T* __restrict__ gin = cur ? F.g[1] : F.g[0];
    T* __restrict__ gout = cur ? F.g[0] : F.g[1];
    load_tile<T, NP>(P, sm, F.C, F.psi, F.cosf, lag_in, x0, y0, tid);
    __syncthreads();
    compute_mu_tile<T, NP>(P, sm, tid);
    __syncthreads();

    const int x = x0 + threadIdx.x, y = y0 + threadIdx.y;
    if (x >= P.nx || y >= P.ny) return;
    const long long o = (long long)y * P.pitch + x;
    const int cx = threadIdx.x + 2, cy = threadIdx.y + 2;   // halo-2 coordinates
    const int hx = threadIdx.x + 1, hy = threadIdx.y + 1;   // halo-1 coordinates
    const T cs2 = P.cs2;
    const T psi = sm.psi[cy][cx];

    // ---- order parameters and their gradients (a1, a2) ------------------
    T Cv[NP], gCx[NP], gCy[NP];
    {
        T sC = T(0), sx = T(0), sy = T(0);
#pragma unroll
        for (int j = 0; j < NP - 1; ++j) {
            Cv[j] = sm.C[j][cy][cx];
            DDCC_GRAD(sm.C[j], cy, cx, gCx[j], gCy[j]);
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
    const T s21 = T(1) / (nu * P.nu_to_s21 + T(0.5));
    const T s22 = T(1) / (nu * P.nu_to_s22 + T(0.5));
    T gpx, gpy;
    DDCC_GRAD(sm.psi, cy, cx, gpx, gpy);
    // grad(psi rho): stencil on psi(x+c) rho(x+c)
    T gprx, gpry;
    {
        T pr[3][3];
#pragma unroll
        for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
            for (int dx = -1; dx <= 1; ++dx) {
                if (dx == 0 && dy == 0) continue;
                T r = P.rho[NP - 1];
#pragma unroll
                for (int j = 0; j < NP - 1; ++j)
                    r += (P.rho[j] - P.rho[NP - 1]) * sm.C[j][cy + dy][cx + dx];
                pr[dy + 1][dx + 1] = sm.psi[cy + dy][cx + dx] * r;
            }
        pr[1][1] = T(0);
        gprx = P.gw1 * (pr[1][2] - pr[1][0]) + P.gw2 * ((pr[2][2] - pr[2][0]) + (pr[0][2] - pr[0][0]));
        gpry = P.gw1 * (pr[2][1] - pr[0][1]) + P.gw2 * ((pr[2][2] + pr[2][0]) - (pr[0][2] + pr[0][0]));
    }

    // ---- chemical potentials, mobility flux, m^C (a3, a4) ---------------
    T mu[NP], gmx[NP], gmy[NP];
#pragma unroll
    for (int j = 0; j < NP; ++j) {
        mu[j] = sm.mu[j][hy][hx];
        DDCC_GRAD(sm.mu[j], hy, hx, gmx[j], gmy[j]);
    }
    // Q_i = sum_j M_ij grad mu_j = m0 C_i (S_C grad mu_i - sum_j C_j grad mu_j)
    T SC = T(0), Gx = T(0), Gy = T(0);
#pragma unroll
    for (int j = 0; j < NP; ++j) {
        SC += Cv[j];
        Gx += Cv[j] * gmx[j];
        Gy += Cv[j] * gmy[j];
    }
    T Qx[NP], Qy[NP];
    T mCx = T(0), mCy = T(0);
#pragma unroll
    for (int i = 0; i < NP; ++i) {
        Qx[i] = P.m0 * Cv[i] * (SC * gmx[i] - Gx);
        Qy[i] = P.m0 * Cv[i] * (SC * gmy[i] - Gy);
        mCx -= P.rho[i] * Qx[i];
        mCy -= P.rho[i] * Qy[i];
    }

    // ---- lagged fields of the previous step -------------------------------
    T dax, day;
    DDCC_GRAD(sm.a, hy, hx, dax, day);
    const T psimu_prev = lag_in[(2 * NP + 2) * P.plane + o];

    // ---- flow populations, velocity and pressure (a5, a6) ------------------
    T g[9];
#pragma unroll
    for (int p = 0; p < 9; ++p) g[p] = gin[p * P.plane + o];
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
    const T den = psi * rho + T(0.5) * dmp;
    const T u0x = (Jx + T(0.5) * F0x) / den;
    const T u0y = (Jy + T(0.5) * F0y) / den;
    const T ex = T(0.5) * gpx / den;
    const T ey = T(0.5) * gpy / den;
    const T Hc = P.Hfac * (s21 - T(2));
    const T bx = P.A_P * psi * grx + P.gam * psi * mCx + Hc / s21 * gprx;
    const T by = P.A_P * psi * gry + P.gam * psi * mCy + Hc / s21 * gpry;
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
        T* out = F.macro;
#pragma unroll
        for (int j = 0; j < NP; ++j) {
            out[j * P.plane + o] = Cv[j];
            out[(NP + 4 + j) * P.plane + o] = mu[j];
        }
        out[NP * P.plane + o] = rho;
        out[(NP + 1) * P.plane + o] = ux;
        out[(NP + 2) * P.plane + o] = uy;
        out[(NP + 3) * P.plane + o] = Pr;
        return;
    }

    // ---- streaming targets (push; halfway bounce-back at outer walls) ----
    long long tgt[9];
    int tdir[9];
#pragma unroll
    for (int p = 0; p < 9; ++p) {
        int tx = x + kCx[p], ty = y + kCy[p];
        bool bounce = false;
        if (tx < 0 || tx >= P.nx) {
            if (P.px) tx = tx < 0 ? tx + P.nx : tx - P.nx;
            else bounce = true;
        }
        if (ty < 0 || ty >= P.ny) {
            if (P.py) ty = ty < 0 ? ty + P.ny : ty - P.ny;
            else bounce = true;
        }
        if (bounce) {
            tgt[p] = o;
            tdir[p] = (p == 0) ? 0 : (p <= 4 ? ((p + 1) & 3) + 1 : ((p - 3) & 3) + 5);
        } else {
            tgt[p] = (long long)ty * P.pitch + tx;
            tdir[p] = p;
        }
    }

    const T w1d[3] = {P.w1d[0], P.w1d[1], P.w1d[2]};

    // ---- phase LB (a7), Eqs. 3.1, 3.5-3.7 ---------------------------------
#pragma unroll
    for (int i = 0; i < NP - 1; ++i) {
        T v[9], m[9], k[9], out[9];
#pragma unroll
        for (int p = 0; p < 9; ++p) v[p] = fin[(i * 9 + p) * P.plane + o];
        hermite_moments(v, cs2, m);
        const T psiC = m[0];
        const T pcux = psiC * ux, pcuy = psiC * uy;
        const T dtx = pcux - lag_in[(1 + 2 * i) * P.plane + o];
        const T dty = pcuy - lag_in[(2 + 2 * i) * P.plane + o];
        // S_i = (psi / m0) Q_i - psi grad mu_i
        const T Sx = psi * Qx[i] / P.m0 - psi * gmx[i];
        const T Sy = psi * Qy[i] / P.m0 - psi * gmy[i];
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
        hermite_relax_back(k, cs2, w1d, v, out);
#pragma unroll
        for (int p = 0; p < 9; ++p) fout[(i * 9 + tdir[p]) * P.plane + tgt[p]] = out[p];
        lag_out[(1 + 2 * i) * P.plane + o] = pcux;
        lag_out[(2 + 2 * i) * P.plane + o] = pcuy;
    }

    // ---- flow LB (a8), Eqs. 3.2, 3.8, 3.10 ---------------------------------
    {
        T m[9], k[9], out[9];
        hermite_moments(g, cs2, m);
        const T psirho = psi * rho;
        const T Axx = psirho * ux * ux + psi * mCx * ux;
        const T Ayy = psirho * uy * uy + psi * mCy * uy;
        const T Axy = psirho * ux * uy + T(0.5) * (psi * mCx * uy + psi * ux * mCy);
        const T Txx = psi * mCx * ux;
        const T Tyy = psi * mCy * uy;
        const T Txy = T(0.5) * (psi * mCx * uy + psi * ux * mCy);
        const T ugpr = ux * gprx + uy * gpry;
        const T Mxx = (Txx - lag_in[(2 * NP - 1) * P.plane + o]) + T(2) * cs2 * ux * gprx + P.c2m3cs2 * ugpr;
        const T Myy = (Tyy - lag_in[(2 * NP) * P.plane + o]) + T(2) * cs2 * uy * gpry + P.c2m3cs2 * ugpr;
        const T Mxy = (Txy - lag_in[(2 * NP + 1) * P.plane + o]) + cs2 * (ux * gpry + gprx * uy);
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
        hermite_relax_back(k, cs2, w1d, g, out);
#pragma unroll
        for (int p = 0; p < 9; ++p) gout[tdir[p] * P.plane + tgt[p]] = out[p];
        // lagged fields (a10)
        lag_out[o] = T(0.5) * psi * (mCx * uy - ux * mCy);
        lag_out[(2 * NP - 1) * P.plane + o] = Txx;
        lag_out[(2 * NP) * P.plane + o] = Tyy;
        lag_out[(2 * NP + 1) * P.plane + o] = Txy;
        lag_out[(2 * NP + 2) * P.plane + o] = psi * (rho * (ux * ux + uy * uy) + mCx * ux + mCy * uy);
    }
}

// Initial state (reading of the paper's set-ups): f = f^eq(C0, mu(C0), u = 0)
// by Eq. 3.5, g = g^eq(P = 0, u = 0) by Eq. 3.8 (g_0 - rho0 = 0), lagged
// fields zero.  F.C holds C0.
template <typename T, int NP>
__global__ void __launch_bounds__(NT) k_init(KParams<T> P, Fields<T> F, int cur) {
    __shared__ Smem<T, NP> sm;
    const int tid = threadIdx.x + BX * threadIdx.y;
    const int x0 = blockIdx.x * BX, y0 = blockIdx.y * BY;
    load_tile<T, NP>(P, sm, F.C, F.psi, F.cosf, nullptr, x0, y0, tid);
    __syncthreads();
    compute_mu_tile<T, NP>(P, sm, tid);
    __syncthreads();
    const int x = x0 + threadIdx.x, y = y0 + threadIdx.y;
    if (x >= P.nx || y >= P.ny) return;
    const long long o = (long long)y * P.pitch + x;
    const T psi = sm.psi[threadIdx.y + 2][threadIdx.x + 2];
    T* f = cur ? F.f[1] : F.f[0];
    const T w0 = P.w1d[1] * P.w1d[1];
#pragma unroll
    for (int i = 0; i < NP - 1; ++i) {
        const T psiC = psi * sm.C[i][threadIdx.y + 2][threadIdx.x + 2];
        const T emu = P.eta[i] * psi * sm.mu[i][threadIdx.y + 1][threadIdx.x + 1];
#pragma unroll
        for (int p = 0; p < 9; ++p) {
            const int cxp = p == 0 ? 0 : (p == 1 || p == 5 || p == 8 ? 1 : (p == 2 || p == 4 ? 0 : -1));
            const int cyp = p == 0 ? 0 : (p == 2 || p == 5 || p == 6 ? 1 : (p == 1 || p == 3 ? 0 : -1));
            const T wp = P.w1d[cxp + 1] * P.w1d[cyp + 1];
            f[(i * 9 + p) * P.plane + o] = p == 0 ? (w0 - T(1)) * emu + psiC : wp * emu;
        }
    }
    T* g = cur ? F.g[1] : F.g[0];
#pragma unroll
    for (int p = 0; p < 9; ++p) g[p * P.plane + o] = T(0);
    T* lag = cur ? F.lag[1] : F.lag[0];
    for (int q = 0; q < 2 * NP + 3; ++q) lag[q * P.plane + o] = T(0);
}

// psi C_i = sum_p f^i_p and C_i = psi C_i / psi (Sec. 3).
template <typename T, int NP>
__global__ void __launch_bounds__(256) k_order_param(KParams<T> P, const T* __restrict__ f,
                                                     const T* __restrict__ psi, T* __restrict__ C) {
    const long long n = (long long)P.nx * P.ny;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
         idx += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(idx / P.nx), x = (int)(idx - (long long)y * P.nx);
        const long long o = (long long)y * P.pitch + x;
        const T inv = T(1) / psi[o];
#pragma unroll
        for (int i = 0; i < NP - 1; ++i) {
            T s = T(0);
#pragma unroll
            for (int p = 0; p < 9; ++p) s += f[(i * 9 + p) * P.plane + o];
            C[i * P.plane + o] = s * inv;
        }
    }
}

// Per-phase sum over nodes of sum_p f^i_p in double, fixed order:
// pass 1 writes one partial per block, pass 2 sums them.
template <typename T, int NP>
__global__ void __launch_bounds__(256) k_mass_partial(KParams<T> P, const T* __restrict__ f,
                                                      double* __restrict__ partial) {
    __shared__ double red[NP - 1][256];
    const long long n = (long long)P.nx * P.ny;
    double acc[NP - 1];
#pragma unroll
    for (int i = 0; i < NP - 1; ++i) acc[i] = 0.0;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
         idx += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(idx / P.nx), x = (int)(idx - (long long)y * P.nx);
        const long long o = (long long)y * P.pitch + x;
#pragma unroll
        for (int i = 0; i < NP - 1; ++i) {
            double s = 0.0;
#pragma unroll
            for (int p = 0; p < 9; ++p) s += (double)f[(i * 9 + p) * P.plane + o];
            acc[i] += s;
        }
    }
#pragma unroll
    for (int i = 0; i < NP - 1; ++i) red[i][threadIdx.x] = acc[i];
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) {
#pragma unroll
            for (int i = 0; i < NP - 1; ++i) red[i][threadIdx.x] += red[i][threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
#pragma unroll
        for (int i = 0; i < NP - 1; ++i) partial[blockIdx.x * kMaxPhases + i] = red[i][0];
    }
}

__global__ void k_mass_final(const double* __restrict__ partial, int nblocks, int nph,
                             double* __restrict__ out) {
    if (threadIdx.x < nph) {
        double s = 0.0;
        for (int b = 0; b < nblocks; ++b) s += partial[b * kMaxPhases + threadIdx.x];
        out[threadIdx.x] = s;
    }
}

template <typename T>
__global__ void k_convert(const double* __restrict__ src, T* __restrict__ dst, int nx, int ny,
                          int pitch, long long plane, int planes) {
    const long long n = (long long)nx * ny;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n * planes;
         idx += (long long)gridDim.x * blockDim.x) {
        const long long q = idx / n, r = idx - q * n;
        const int y = (int)(r / nx), x = (int)(r - (long long)y * nx);
        dst[q * plane + (long long)y * pitch + x] = (T)src[idx];
    }
}

template <typename T>
__global__ void k_export(const T* __restrict__ src, double* __restrict__ dst, int nx, int ny,
                         int pitch) {
    const long long n = (long long)nx * ny;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
         idx += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(idx / nx), x = (int)(idx - (long long)y * nx);
        dst[idx] = (double)src[(long long)y * pitch + x];
    }
}

inline dim3 tile_grid(int nx, int ny) {
    return dim3((nx + BX - 1) / BX, (ny + BY - 1) / BY);
}

inline int flat_blocks(long long n) {
    long long b = (n + 255) / 256;
    return (int)(b < 152 * 16 ? (b < 1 ? 1 : b) : 152 * 16);
}

template <typename T, int NP>
cudaError_t order_param_n(const KParams<T>& kp, const Fields<T>& fd, int cur, cudaStream_t s) {
    k_order_param<T, NP><<<flat_blocks((long long)kp.nx * kp.ny), 256, 0, s>>>(kp, fd.f[cur], fd.psi, fd.C);
    return cudaGetLastError();
}

template <typename T, int NP>
cudaError_t collide_n(const KParams<T>& kp, const Fields<T>& fd, int cur, cudaStream_t s) {
    k_step<T, NP, 0><<<tile_grid(kp.nx, kp.ny), dim3(BX, BY), 0, s>>>(kp, fd, cur);
    return cudaGetLastError();
}

template <typename T, int NP>
cudaError_t macro_n(const KParams<T>& kp, const Fields<T>& fd, int cur, cudaStream_t s) {
    k_order_param<T, NP><<<flat_blocks((long long)kp.nx * kp.ny), 256, 0, s>>>(kp, fd.f[cur], fd.psi, fd.C);
    k_step<T, NP, 1><<<tile_grid(kp.nx, kp.ny), dim3(BX, BY), 0, s>>>(kp, fd, cur);
    return cudaGetLastError();
}

template <typename T, int NP>
cudaError_t init_n(const KParams<T>& kp, const Fields<T>& fd, int cur, cudaStream_t s) {
    k_init<T, NP><<<tile_grid(kp.nx, kp.ny), dim3(BX, BY), 0, s>>>(kp, fd, cur);
    return cudaGetLastError();
}

template <typename T, int NP>
cudaError_t mass_n(const KParams<T>& kp, const Fields<T>& fd, int cur, double* out, cudaStream_t s) {
    k_mass_partial<T, NP><<<kMassBlocks, 256, 0, s>>>(kp, fd.f[cur], fd.partial);
    k_mass_final<<<1, 32, 0, s>>>(fd.partial, kMassBlocks, NP - 1, out);
    return cudaGetLastError();
}

}  // namespace

#define DDCC_DISPATCH(fn, ...)                                \
    switch (kp.N) {                                           \
        case 2: return fn<T, 2>(__VA_ARGS__);                 \
        case 3: return fn<T, 3>(__VA_ARGS__);                 \
        case 4: return fn<T, 4>(__VA_ARGS__);                 \
        default: return cudaErrorInvalidValue;                \
    }

template <typename T>
cudaError_t launch_init(const KParams<T>& kp, const Fields<T>& fd, int cur, cudaStream_t s) {
    DDCC_DISPATCH(init_n, kp, fd, cur, s);
}
template <typename T>
cudaError_t launch_order_param(const KParams<T>& kp, const Fields<T>& fd, int cur, cudaStream_t s) {
    DDCC_DISPATCH(order_param_n, kp, fd, cur, s);
}
template <typename T>
cudaError_t launch_collide(const KParams<T>& kp, const Fields<T>& fd, int cur, cudaStream_t s) {
    DDCC_DISPATCH(collide_n, kp, fd, cur, s);
}
template <typename T>
cudaError_t launch_macro(const KParams<T>& kp, const Fields<T>& fd, int cur, cudaStream_t s) {
    DDCC_DISPATCH(macro_n, kp, fd, cur, s);
}
template <typename T>
cudaError_t launch_mass(const KParams<T>& kp, const Fields<T>& fd, int cur, double* out,
                        cudaStream_t s) {
    DDCC_DISPATCH(mass_n, kp, fd, cur, out, s);
}
template <typename T>
cudaError_t launch_convert(const double* src, T* dst, int nx, int ny, int pitch, long long plane,
                           int planes, cudaStream_t s) {
    k_convert<T><<<flat_blocks((long long)nx * ny * planes), 256, 0, s>>>(src, dst, nx, ny, pitch, plane,
                                                                          planes);
    return cudaGetLastError();
}
template <typename T>
cudaError_t launch_export(const T* src, double* dst, int nx, int ny, int pitch, cudaStream_t s) {
    k_export<T><<<flat_blocks((long long)nx * ny), 256, 0, s>>>(src, dst, nx, ny, pitch);
    return cudaGetLastError();
}

#define DDCC_INSTANTIATE(T)                                                                      \
    template cudaError_t launch_init<T>(const KParams<T>&, const Fields<T>&, int, cudaStream_t);  \
    template cudaError_t launch_order_param<T>(const KParams<T>&, const Fields<T>&, int,          \
                                               cudaStream_t);                                    \
    template cudaError_t launch_collide<T>(const KParams<T>&, const Fields<T>&, int, cudaStream_t); \
    template cudaError_t launch_macro<T>(const KParams<T>&, const Fields<T>&, int, cudaStream_t); \
    template cudaError_t launch_mass<T>(const KParams<T>&, const Fields<T>&, int, double*,        \
                                        cudaStream_t);                                           \
    template cudaError_t launch_convert<T>(const double*, T*, int, int, int, long long, int,       \
                                           cudaStream_t);                                        \
    template cudaError_t launch_export<T>(const T*, double*, int, int, int, cudaStream_t);

DDCC_INSTANTIATE(double)
DDCC_INSTANTIATE(float)

}  // namespace ddcc
