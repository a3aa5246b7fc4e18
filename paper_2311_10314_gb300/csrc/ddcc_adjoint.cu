// Discrete adjoint (reverse mode) of one DD-CCLB step and of the initial
// state (arXiv 2311.10314, Sec. 3): the transpose of the Jacobian of exactly
// the arithmetic the forward kernels perform, applied to an adjoint state.
//
// One reverse step n+1 -> n runs these kernels, each over every node (one
// thread per node, plain loads; the ghost frames hold periodic or mirror
// copies exactly as in the forward step):
//   k_adj_order / k_adj_mu   recompute C_i and mu_i of step n from the
//                            checkpointed state, on the domain and its
//                            1-node ghost ring
//   k_adj_node               the node update's VJP: adjoints of the node's
//                            own populations and lagged planes, and of every
//                            stencil output the update reads (grad C_j,
//                            grad psi, grad(psi rho), grad mu_j, grad a and
//                            the centre values); the streaming is transposed
//                            by pulling the adjoint from each push target
//   k_adj_gather3            transposed gradient stencils: adjoints of C_j,
//                            psi, mu_j and a at each node, summed over the
//                            node and its ghost-ring images (periodic wrap or
//                            wall mirror), followed in the same thread by
//                            the VJP of Eq. 2.14 per node (mu_node_at):
//                            adjoints of the centre C_j and psi, of
//                            div(psi grad C_j) and grad psi, and
//                            dJ/dcos(theta_iN) at the node
//   k_adj_gather2            transposed div(psi grad .) and grad psi stencils
//                            (folded the same way), then C_i = sum_p f^i_p /
//                            psi reversed, and dJ/dpsi
// The initial state (f = f^eq(psi C0, psi mu(C0), u = 0), g and the lagged
// planes zero) is reversed by k_adj_init_node followed by the same mu stage
// as a kernel of its own (k_adj_mu_node).
#include "ddcc_device.cuh"

namespace ddcc {
namespace {

using dev::map_index;

constexpr int AX = 32, AY = 8;   // thread block of the node kernels
constexpr double kKinkGradPsi = 1e-6;

// D2Q9 velocities (Sec. 3): 0 rest, 1-4 axis, 5-8 diagonal.
__constant__ int aCx[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
__constant__ int aCy[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};

__device__ __forceinline__ int opp(int p) { return p == 0 ? 0 : (p <= 4 ? ((p + 1) & 3) + 1 : ((p - 3) & 3) + 5); }

// B_p = sum_ab h_a(cx_p) h_b(cy_p) k_ab (the transpose of hermite_moments).
template <typename T>
__device__ __forceinline__ void hermite_B(const T k[9], T cs2, T B[9]) {
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
    const T one_m = T(1) - cs2;
    B[0] = R0[0] - cs2 * R0[2];
    B[1] = R0[0] + R0[1] + one_m * R0[2];
    B[2] = Rp[0] - cs2 * Rp[2];
    B[3] = R0[0] - R0[1] + one_m * R0[2];
    B[4] = Rm[0] - cs2 * Rm[2];
    B[5] = Rp[0] + Rp[1] + one_m * Rp[2];
    B[6] = Rp[0] - Rp[1] + one_m * Rp[2];
    B[7] = Rm[0] - Rm[1] + one_m * Rm[2];
    B[8] = Rm[0] + Rm[1] + one_m * Rm[2];
}

// g''(C) for g(C) = C^2 (C - 1)^2.
template <typename T>
__device__ __forceinline__ T gsecond(T c) {
    return T(12) * c * c - T(12) * c + T(2);
}

template <typename T>
__device__ __forceinline__ T wgt(const KParams<T>& P, int p) {
    return P.w1d[aCx[p] + 1] * P.w1d[aCy[p] + 1];
}
template <typename T>
__device__ __forceinline__ T gw(const KParams<T>& P, int p) { return p <= 4 ? P.gw1 : P.gw2; }
template <typename T>
__device__ __forceinline__ T lw(const KParams<T>& P, int p) { return p <= 4 ? P.lw1 : P.lw2; }

// ---------------------------------------------------------------------------
// recompute C_i and mu_i of step n
// ---------------------------------------------------------------------------

template <typename T, int NP>
__global__ void __launch_bounds__(256) k_adj_order(KParams<T> P, const T* __restrict__ f,
                                                   const T* __restrict__ psi, T* __restrict__ C) {
    // over the domain and its 1-node ghost ring: a ring cell gets the value
    // of the node it copies (periodic wrap or wall mirror), computed the same
    // way, so no ghost fill is needed
    const int x = blockIdx.x * AX + threadIdx.x - 1, y = blockIdx.y * AY + threadIdx.y - 1;
    if (x > P.nx || y > P.ny) return;
    const long long o = P.org + (long long)y * P.pitch + x;
    const long long os = P.org + (long long)map_index(y, P.ny, P.py) * P.pitch + map_index(x, P.nx, P.px);
    const T inv = T(1) / psi[os];
#pragma unroll
    for (int i = 0; i < NP - 1; ++i) {
        T s = T(0);
#pragma unroll
        for (int p = 0; p < 9; ++p) s += f[(i * 9 + p) * P.plane + os];
        C[i * P.plane + o] = s * inv;
    }
}

template <typename T>
struct PlaneAt {
    const T* base;
    long long plane, o;
    int pitch;
    __device__ T operator()(int j, int dy, int dx) const { return base[j * plane + o + (long long)dy * pitch + dx]; }
    __device__ T operator()(int dy, int dx) const { return base[o + (long long)dy * pitch + dx]; }
};

template <typename T, int NP>
__device__ __forceinline__ void node_cth(const KParams<T>& P, const T* cosf, long long o, T cth[NP]) {
#pragma unroll
    for (int i = 0; i < NP - 1; ++i) cth[i] = P.has_cos_field ? cosf[i * P.plane + o] : P.cos_uni[i];
    cth[NP - 1] = T(0);
}

template <typename T, int NP>
__global__ void __launch_bounds__(256) k_adj_mu(KParams<T> P, const T* __restrict__ C, const T* __restrict__ psi,
                                                const T* __restrict__ cosf, T* __restrict__ mu) {
    // over the domain and its 1-node ghost ring, as k_adj_order (C and psi
    // are read around the copied node, whose ring the C pass has written)
    const int x = blockIdx.x * AX + threadIdx.x - 1, y = blockIdx.y * AY + threadIdx.y - 1;
    if (x > P.nx || y > P.ny) return;
    const long long od = P.org + (long long)y * P.pitch + x;
    const long long o = P.org + (long long)map_index(y, P.ny, P.py) * P.pitch + map_index(x, P.nx, P.px);
    const PlaneAt<T> Ca{C, P.plane, o, P.pitch}, Pa{psi, P.plane, o, P.pitch};
    T cth[NP], m[NP];
    node_cth<T, NP>(P, cosf, o, cth);
    dev::chem_pot<T, NP>(P, [&](int j, int dy, int dx) { return Ca(j, dy, dx); },
                         [&](int dy, int dx) { return Pa(dy, dx); }, cth, m);
#pragma unroll
    for (int i = 0; i < NP; ++i) mu[i * P.plane + od] = m[i];
}

// ---------------------------------------------------------------------------
// scratch planes (each a padded plane of T)
// ---------------------------------------------------------------------------

template <typename T, int NP>
struct AdjPlanes {
    T* C;     // N-1   C_i of step n
    T* mu;    // N     mu_i of step n
    T* lC;    // N-1   node VJP: centre C_j
    T* lgC;   // 2(N-1)          grad C_j (x, y)
    T* lpsi;  // 1               centre psi
    T* lgp;   // 2               grad psi
    T* lgpr;  // 2               grad(psi rho)
    T* lmu;   // N               centre mu_j
    T* lgm;   // 2N              grad mu_j
    T* lga;   // 2               grad a
    T* LC;    // N-1   gathered adjoint of C_j (padded frame)
    T* Lpsi;  // 1                         psi
    T* Lmu;   // N                         mu_j
    T* mC;    // N-1   mu VJP: centre C_j
    T* mL;    // N-1           div(psi grad C_j)
    T* mpsi;  // 1             centre psi
    T* mgp;   // 2             grad psi
    const T* a;   // lagged plane a of step n (the state's own plane, ghost frame filled)
    __host__ __device__ static constexpr int planes() { return 12 * NP + 4; }
    __host__ static AdjPlanes carve(T* base, long long plane) {
        AdjPlanes A;
        T* q = base;
        auto take = [&](int n) { T* r = q; q += (long long)n * plane; return r; };
        A.C = take(NP - 1);
        A.mu = take(NP);
        A.lC = take(NP - 1);
        A.lpsi = take(1);
        A.lmu = take(NP);
        // the 2N+2 vector pairs the first gather reads, consecutive
        A.lgC = take(2 * (NP - 1));
        A.lgp = take(2);
        A.lgpr = take(2);
        A.lgm = take(2 * NP);
        A.lga = take(2);
        A.LC = take(NP - 1);
        A.Lpsi = take(1);
        A.Lmu = take(NP);
        A.mC = take(NP - 1);
        A.mpsi = take(1);
        // mL_j and the grad psi pair the second gather reads, consecutive
        A.mL = take(NP - 1);
        A.mgp = take(2);
        A.a = nullptr;
        return A;
    }
};

// ---------------------------------------------------------------------------
// VJP of the node update (a1-a10 at one node)
// ---------------------------------------------------------------------------

template <typename T, int NP>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 2 : 1) k_adj_node(KParams<T> P, const T* __restrict__ psi_pl,
                                                  const T* __restrict__ st_pop, const T* __restrict__ st_lag,
                                                  const T* __restrict__ ad_pop_in,
                                                  const T* __restrict__ ad_lag_in, T* __restrict__ ad_pop_out,
                                                  T* __restrict__ ad_lag_out, AdjPlanes<T, NP> W) {
    const int x = blockIdx.x * AX + threadIdx.x, y = blockIdx.y * AY + threadIdx.y;
    if (x >= P.nx || y >= P.ny) return;
    const long long pl = P.plane;
    const long long o = P.org + (long long)y * P.pitch + x;
    const PlaneAt<T> Ca{W.C, pl, o, P.pitch}, Pa{psi_pl, pl, o, P.pitch}, Ma{W.mu, pl, o, P.pitch},
        Aa{W.a, pl, o, P.pitch};
    auto grad = [&](auto chi, T& gx, T& gy) { dev::grad9(P, chi, gx, gy); };
    const T cs2 = P.cs2;
    const T* st_g = st_pop + (long long)9 * (NP - 1) * pl;

    // ---- forward recomputation (the arithmetic of dev::node_update) -------
    const T psi = Pa(0, 0);
    T Cv[NP], gCx[NP], gCy[NP];
    {
        T sC = T(0), sx = T(0), sy = T(0);
#pragma unroll
        for (int j = 0; j < NP - 1; ++j) {
            Cv[j] = Ca(j, 0, 0);
            grad([&](int dy, int dx) { return Ca(j, dy, dx); }, gCx[j], gCy[j]);
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
    const T inv_s21 = nu * P.nu_to_s21 + T(0.5);
    const T s21 = T(1) / inv_s21;
    const T s22 = T(1) / (nu * P.nu_to_s22 + T(0.5));
    T gpx, gpy;
    grad([&](int dy, int dx) { return Pa(dy, dx); }, gpx, gpy);
    T gprx, gpry;
    grad(
        [&](int dy, int dx) {
            T r = P.rho[NP - 1];
#pragma unroll
            for (int j = 0; j < NP - 1; ++j) r += (P.rho[j] - P.rho[NP - 1]) * Ca(j, dy, dx);
            return Pa(dy, dx) * r;
        },
        gprx, gpry);
    T mu[NP], gmx[NP], gmy[NP];
#pragma unroll
    for (int j = 0; j < NP; ++j) {
        mu[j] = Ma(j, 0, 0);
        grad([&](int dy, int dx) { return Ma(j, dy, dx); }, gmx[j], gmy[j]);
    }
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
        Qx[i] = Cv[i] * (SC * gmx[i] - Gx);
        Qy[i] = Cv[i] * (SC * gmy[i] - Gy);
        mCx -= P.rho[i] * Qx[i];
        mCy -= P.rho[i] * Qy[i];
    }
    mCx *= P.m0;
    mCy *= P.m0;
    T dax, day;
    grad([&](int dy, int dx) { return Aa(dy, dx); }, dax, day);
    T lag[2 * NP + 3];
#pragma unroll
    for (int k = 0; k < 2 * NP + 3; ++k) lag[k] = st_lag[k * pl + o];
    const T psimu_prev = lag[2 * NP + 2];
    T g[9];
#pragma unroll
    for (int p = 0; p < 9; ++p) g[p] = st_g[p * pl + o];
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
    const T Hs = P.Hfac * (s21 - T(2)) * inv_s21;
    const T bx = P.A_P * psi * grx + P.gam * psi * mCx + Hs * gprx;
    const T by = P.A_P * psi * gry + P.gam * psi * mCy + Hs * gpry;
    const T gq = P.gam * psi * rho;
    const T qa = P.cP * gq * (ex * ex + ey * ey);
    const T qb = P.cP * (bx * ex + by * ey + T(2) * gq * (u0x * ex + u0y * ey)) - psi;
    const T sum_g = ((g[1] + g[2]) + (g[3] + g[4])) + ((g[5] + g[6]) + (g[7] + g[8]));
    const T G0 = sum_g - P.Kh * psimu_prev;
    const T qc = P.cP * (G0 + bx * u0x + by * u0y + gq * (u0x * u0x + u0y * u0y));
    const T disc_raw = qb * qb - T(4) * qa * qc;
    const T disc = disc_raw > T(0) ? disc_raw : T(0);
    const T root = sqrt(disc);
    const T sgn = qb < T(0) ? T(-1) : T(1);
    const T D = qb + sgn * root;
    const T Pr = T(-2) * qc / D;
    const T ux = u0x + Pr * ex;
    const T uy = u0y + Pr * ey;
    const T psiP = psi * Pr;

    // ---- adjoints of the outputs: transposed push streaming -------------
    // (the forward sends population p of this node to tgt in direction tdir)
    long long tgt[9];
    int tdir[9];
#pragma unroll
    for (int p = 0; p < 9; ++p) {
        int tx = x + aCx[p], ty = y + aCy[p];
        bool bounce = false;
        if (tx < 0 || tx >= P.nx) {
            if (P.px) tx = tx < 0 ? tx + P.nx : tx - P.nx;
            else bounce = true;
        }
        if (ty < 0 || ty >= P.ny) {
            if (P.py) ty = ty < 0 ? ty + P.ny : ty - P.ny;
            else bounce = true;
        }
        tgt[p] = bounce ? o : P.org + (long long)ty * P.pitch + tx;
        tdir[p] = bounce ? opp(p) : p;
    }
    T lo_lag[2 * NP + 3];
#pragma unroll
    for (int k = 0; k < 2 * NP + 3; ++k) lo_lag[k] = ad_lag_in[k * pl + o];
    T li_lag[2 * NP + 3];   // adjoint of the lagged inputs (k >= 1)
#pragma unroll
    for (int k = 0; k < 2 * NP + 3; ++k) li_lag[k] = T(0);

    // accumulators of the intermediate adjoints
    T l_psi = T(0), l_rho = T(0), l_nu = T(0), l_grx = T(0), l_gry = T(0);
    T l_gpx = T(0), l_gpy = T(0), l_gprx = T(0), l_gpry = T(0);
    T l_mCx = T(0), l_mCy = T(0), l_dax = T(0), l_day = T(0);
    T l_ux = T(0), l_uy = T(0), l_Fx = T(0), l_Fy = T(0), l_psiP = T(0);
    T l_s21 = T(0), l_s22 = T(0);
    T l_Cv[NP], l_gCx[NP], l_gCy[NP], l_mu[NP], l_gmx[NP], l_gmy[NP], l_Qx[NP], l_Qy[NP];
#pragma unroll
    for (int j = 0; j < NP; ++j) {
        l_Cv[j] = l_gCx[j] = l_gCy[j] = l_mu[j] = l_gmx[j] = l_gmy[j] = l_Qx[j] = l_Qy[j] = T(0);
    }
    T l_g[9];

    // ---- flow LB (Eqs. 3.2, 3.8, 3.10) reversed ---------------------------
    {
        const T Fx = F0x + Pr * gpx - dmp * ux;
        const T Fy = F0y + Pr * gpy - dmp * uy;
        T mg[9];
        dev::hermite_moments(g, cs2, mg);
        const T psirho = psi * rho;
        const T Txx = psi * mCx * ux;
        const T Tyy = psi * mCy * uy;
        const T Txy = T(0.5) * (psi * mCx * uy + psi * ux * mCy);
        const T Axx = psirho * ux * ux + Txx;
        const T Ayy = psirho * uy * uy + Tyy;
        const T Axy = psirho * ux * uy + Txy;
        const T ugpr = ux * gprx + uy * gpry;
        const T Mxx = (Txx - lag[2 * NP - 1]) + T(2) * cs2 * ux * gprx + P.c2m3cs2 * ugpr;
        const T Myy = (Tyy - lag[2 * NP]) + T(2) * cs2 * uy * gpry + P.c2m3cs2 * ugpr;
        const T Mxy = (Txy - lag[2 * NP + 1]) + cs2 * (ux * gpry + gprx * uy);
        const T l20 = s21 * P.invN20, l11 = s22 * P.invN11;
        const T R3 = mg[3] - psiP - Axx + T(0.5) * Mxx;
        const T R4 = mg[4] - psiP - Ayy + T(0.5) * Myy;
        const T R5 = mg[5] - Axy + T(0.5) * Mxy;
        T lout[9], wl[9], lk[9], lm[9];
#pragma unroll
        for (int p = 0; p < 9; ++p) {
            lout[p] = ad_pop_in[((long long)9 * (NP - 1) + tdir[p]) * pl + tgt[p]];
            wl[p] = wgt(P, p) * lout[p];
        }
        dev::hermite_moments(wl, cs2, lk);
#pragma unroll
        for (int a = 0; a < 9; ++a) {
            lk[a] = -lk[a];
            lm[a] = T(0);
        }
        lm[0] += P.lg00 * lk[0];
        const T l_a0 = (T(0.5) * P.lg00 - T(1)) * lk[0];
        lm[1] += P.lg1 * lk[1];
        T l_psirho = -P.lg1 * (ux * lk[1] + uy * lk[2]);
        l_ux += -P.lg1 * psirho * lk[1];
        l_Fx += (T(0.5) * P.lg1 - P.invN[1]) * lk[1];
        lm[2] += P.lg1 * lk[2];
        l_uy += -P.lg1 * psirho * lk[2];
        l_Fy += (T(0.5) * P.lg1 - P.invN[2]) * lk[2];
        const T l_l20 = R3 * lk[3] + R4 * lk[4];
        lm[3] += l20 * lk[3];
        lm[4] += l20 * lk[4];
        l_psiP += -l20 * (lk[3] + lk[4]);
        T l_Axx = -l20 * lk[3], l_Ayy = -l20 * lk[4];
        T l_Mxx = (T(0.5) * l20 - P.invN20) * lk[3];
        T l_Myy = (T(0.5) * l20 - P.invN20) * lk[4];
        const T l_l11 = R5 * lk[5];
        lm[5] += l11 * lk[5];
        T l_Axy = -l11 * lk[5];
        T l_Mxy = (T(0.5) * l11 - P.invN11) * lk[5];
        lm[6] += P.lg3 * lk[6];
        lm[7] += P.lg3 * lk[7];
        lm[8] += P.lg4 * lk[8];
        l_psiP += cs2 * P.lg4 * lk[8];
        l_s21 += P.invN20 * l_l20;
        l_s22 += P.invN11 * l_l11;
        // a0 = psi (u . grad rho)
        l_psi += (ux * grx + uy * gry) * l_a0;
        l_ux += psi * grx * l_a0;
        l_uy += psi * gry * l_a0;
        l_grx += psi * ux * l_a0;
        l_gry += psi * uy * l_a0;
        // M^2G
        T l_Txx = l_Mxx, l_Tyy = l_Myy, l_Txy = l_Mxy;
        li_lag[2 * NP - 1] -= l_Mxx;
        li_lag[2 * NP] -= l_Myy;
        li_lag[2 * NP + 1] -= l_Mxy;
        const T l_ugpr = P.c2m3cs2 * (l_Mxx + l_Myy);
        l_ux += T(2) * cs2 * gprx * l_Mxx + cs2 * gpry * l_Mxy + gprx * l_ugpr;
        l_uy += T(2) * cs2 * gpry * l_Myy + cs2 * gprx * l_Mxy + gpry * l_ugpr;
        l_gprx += T(2) * cs2 * ux * l_Mxx + cs2 * uy * l_Mxy + ux * l_ugpr;
        l_gpry += T(2) * cs2 * uy * l_Myy + cs2 * ux * l_Mxy + uy * l_ugpr;
        // A = psi rho u u + T
        l_psirho += ux * ux * l_Axx + uy * uy * l_Ayy + ux * uy * l_Axy;
        l_ux += T(2) * psirho * ux * l_Axx + psirho * uy * l_Axy;
        l_uy += T(2) * psirho * uy * l_Ayy + psirho * ux * l_Axy;
        l_Txx += l_Axx + lo_lag[2 * NP - 1];
        l_Tyy += l_Ayy + lo_lag[2 * NP];
        l_Txy += l_Axy + lo_lag[2 * NP + 1];
        // a_new = psi (mCx uy - ux mCy) / 2
        {
            const T lo = lo_lag[0];
            l_psi += T(0.5) * (mCx * uy - ux * mCy) * lo;
            l_mCx += T(0.5) * psi * uy * lo;
            l_uy += T(0.5) * psi * mCx * lo;
            l_ux -= T(0.5) * psi * mCy * lo;
            l_mCy -= T(0.5) * psi * ux * lo;
        }
        // (psi m . u)_new = psi (rho |u|^2 + mC . u)
        {
            const T lo = lo_lag[2 * NP + 2];
            l_psi += (rho * (ux * ux + uy * uy) + mCx * ux + mCy * uy) * lo;
            l_rho += psi * (ux * ux + uy * uy) * lo;
            l_ux += psi * (T(2) * rho * ux + mCx) * lo;
            l_uy += psi * (T(2) * rho * uy + mCy) * lo;
            l_mCx += psi * ux * lo;
            l_mCy += psi * uy * lo;
        }
        // T = psi (mC u + u mC) / 2
        l_psi += mCx * ux * l_Txx + mCy * uy * l_Tyy + T(0.5) * (mCx * uy + ux * mCy) * l_Txy;
        l_mCx += psi * ux * l_Txx + T(0.5) * psi * uy * l_Txy;
        l_mCy += psi * uy * l_Tyy + T(0.5) * psi * ux * l_Txy;
        l_ux += psi * mCx * l_Txx + T(0.5) * psi * mCy * l_Txy;
        l_uy += psi * mCy * l_Tyy + T(0.5) * psi * mCx * l_Txy;
        l_psi += rho * l_psirho;
        l_rho += psi * l_psirho;
        T Bm[9];
        hermite_B(lm, cs2, Bm);
#pragma unroll
        for (int p = 0; p < 9; ++p) l_g[p] = lout[p] + Bm[p];
        (void)Fx;
        (void)Fy;
    }

    // ---- phase LB (Eqs. 3.1, 3.5-3.7) reversed, one phase at a time ------
#pragma unroll
    for (int i = 0; i < NP - 1; ++i) {
        T v[9], m[9];
#pragma unroll
        for (int p = 0; p < 9; ++p) v[p] = st_pop[(9 * i + p) * pl + o];
        dev::hermite_moments(v, cs2, m);
        const T psiC = m[0];
        const T ceta = cs2 * P.eta[i];
        const T* lam = P.lamf[i];
        T lout[9], wl[9], lk[9], lm[9];
#pragma unroll
        for (int p = 0; p < 9; ++p) {
            lout[p] = ad_pop_in[(9 * i + tdir[p]) * pl + tgt[p]];
            wl[p] = wgt(P, p) * lout[p];
        }
        dev::hermite_moments(wl, cs2, lk);
#pragma unroll
        for (int a = 0; a < 9; ++a) {
            lk[a] = -lk[a];
            lm[a] = T(0);
        }
        lm[1] += lam[1] * lk[1];
        T l_pcux = -lam[1] * lk[1];
        const T l_Vx = (T(0.5) * lam[1] - P.invN[1]) * lk[1];
        lm[2] += lam[2] * lk[2];
        T l_pcuy = -lam[2] * lk[2];
        const T l_Vy = (T(0.5) * lam[2] - P.invN[2]) * lk[2];
        lm[3] += lam[3] * lk[3];
        lm[4] += lam[4] * lk[4];
        lm[5] += lam[5] * lk[5];
        lm[6] += lam[6] * lk[6];
        lm[7] += lam[7] * lk[7];
        lm[8] += lam[8] * lk[8];
        const T l_X = cs2 * (lam[3] * lk[3] + lam[4] * lk[4]) - cs2 * cs2 * lam[8] * lk[8];
        // X = psi C - eta psi mu_i
        T l_psiC = l_X;
        l_psi += -P.eta[i] * mu[i] * l_X;
        l_mu[i] += -P.eta[i] * psi * l_X;
        // V = dt(psi C u) + cs2 eta (mu grad psi - S), S = psi (Q - grad mu)
        l_mu[i] += ceta * (gpx * l_Vx + gpy * l_Vy);
        l_gpx += ceta * mu[i] * l_Vx;
        l_gpy += ceta * mu[i] * l_Vy;
        const T l_Sx = -ceta * l_Vx, l_Sy = -ceta * l_Vy;
        l_psi += (Qx[i] - gmx[i]) * l_Sx + (Qy[i] - gmy[i]) * l_Sy;
        l_Qx[i] += psi * l_Sx;
        l_Qy[i] += psi * l_Sy;
        l_gmx[i] -= psi * l_Sx;
        l_gmy[i] -= psi * l_Sy;
        l_pcux += l_Vx + lo_lag[1 + 2 * i];
        l_pcuy += l_Vy + lo_lag[2 + 2 * i];
        li_lag[1 + 2 * i] -= l_Vx;
        li_lag[2 + 2 * i] -= l_Vy;
        l_psiC += ux * l_pcux + uy * l_pcuy;
        l_ux += psiC * l_pcux;
        l_uy += psiC * l_pcuy;
        lm[0] += l_psiC;
        T Bm[9];
        hermite_B(lm, cs2, Bm);
#pragma unroll
        for (int p = 0; p < 9; ++p) ad_pop_out[(9 * i + p) * pl + o] = lout[p] + Bm[p];
    }

    // ---- velocity, force and the Eq. 19 pressure reversed ---------------
    l_psi += Pr * l_psiP;
    T l_Pr = psi * l_psiP;
    // F = F0 + P grad psi - dmp u
    T l_F0x = l_Fx, l_F0y = l_Fy;
    l_Pr += gpx * l_Fx + gpy * l_Fy;
    l_gpx += Pr * l_Fx;
    l_gpy += Pr * l_Fy;
    T l_dmp = -(ux * l_Fx + uy * l_Fy);
    l_ux += -dmp * l_Fx;
    l_uy += -dmp * l_Fy;
    // u = u0 + P e
    T l_u0x = l_ux, l_u0y = l_uy;
    l_Pr += ex * l_ux + ey * l_uy;
    T l_ex = Pr * l_ux, l_ey = Pr * l_uy;
    // P = -2 qc / (qb + sgn sqrt(qb^2 - 4 qa qc))
    T l_qc = T(-2) / D * l_Pr;
    const T l_D = T(2) * qc / (D * D) * l_Pr;
    T l_qb = l_D;
    const T l_root = sgn * l_D;
    const T l_disc = disc_raw > T(0) ? l_root / (T(2) * root) : T(0);
    l_qb += T(2) * qb * l_disc;
    const T l_qa = T(-4) * qc * l_disc;
    l_qc += T(-4) * qa * l_disc;
    T l_gq = P.cP * (ex * ex + ey * ey) * l_qa;
    l_ex += T(2) * P.cP * gq * ex * l_qa;
    l_ey += T(2) * P.cP * gq * ey * l_qa;
    T l_bx = P.cP * ex * l_qb, l_by = P.cP * ey * l_qb;
    l_ex += P.cP * (bx + T(2) * gq * u0x) * l_qb;
    l_ey += P.cP * (by + T(2) * gq * u0y) * l_qb;
    l_gq += T(2) * P.cP * (u0x * ex + u0y * ey) * l_qb;
    l_u0x += T(2) * P.cP * gq * ex * l_qb;
    l_u0y += T(2) * P.cP * gq * ey * l_qb;
    l_psi -= l_qb;
    const T l_G0 = P.cP * l_qc;
    l_bx += P.cP * u0x * l_qc;
    l_by += P.cP * u0y * l_qc;
    l_u0x += P.cP * (bx + T(2) * gq * u0x) * l_qc;
    l_u0y += P.cP * (by + T(2) * gq * u0y) * l_qc;
    l_gq += P.cP * (u0x * u0x + u0y * u0y) * l_qc;
    // G0 = sum_{p>0} g_p - K/2 (psi m.u)_prev
#pragma unroll
    for (int p = 1; p < 9; ++p) l_g[p] += l_G0;
    li_lag[2 * NP + 2] += -P.Kh * l_G0;
    // gq = gamma psi rho
    l_psi += P.gam * rho * l_gq;
    l_rho += P.gam * psi * l_gq;
    // b = A_P psi grad rho + gamma psi mC + (H / s21) grad(psi rho)
    l_psi += (P.A_P * grx + P.gam * mCx) * l_bx + (P.A_P * gry + P.gam * mCy) * l_by;
    l_grx += P.A_P * psi * l_bx;
    l_gry += P.A_P * psi * l_by;
    l_mCx += P.gam * psi * l_bx;
    l_mCy += P.gam * psi * l_by;
    const T l_Hs = gprx * l_bx + gpry * l_by;
    l_gprx += Hs * l_bx;
    l_gpry += Hs * l_by;
    // Hs = Hfac (1 - 2 inv_s21)
    T l_inv_s21 = T(-2) * P.Hfac * l_Hs;
    // e = grad psi / (2 den)
    l_gpx += T(0.5) * inv_den * l_ex;
    l_gpy += T(0.5) * inv_den * l_ey;
    T l_inv_den = T(0.5) * (gpx * l_ex + gpy * l_ey);
    // u0 = (J + F0 / 2) / den
    const T l_Jx = inv_den * l_u0x, l_Jy = inv_den * l_u0y;
    l_F0x += T(0.5) * inv_den * l_u0x;
    l_F0y += T(0.5) * inv_den * l_u0y;
    l_inv_den += (Jx + T(0.5) * F0x) * l_u0x + (Jy + T(0.5) * F0y) * l_u0y;
    // den = psi rho + dmp / 2
    const T l_den = -inv_den * inv_den * l_inv_den;
    l_psi += rho * l_den;
    l_rho += psi * l_den;
    l_dmp += T(0.5) * l_den;
    l_psi += -P.damp * l_dmp;
    // F0 = (d_y a, -d_x a) + psi rho b + sum_j psi mu_j grad C_j
    l_day += l_F0x;
    l_dax -= l_F0y;
    l_psi += rho * (P.body[0] * l_F0x + P.body[1] * l_F0y);
    l_rho += psi * (P.body[0] * l_F0x + P.body[1] * l_F0y);
#pragma unroll
    for (int j = 0; j < NP; ++j) {
        l_psi += mu[j] * (gCx[j] * l_F0x + gCy[j] * l_F0y);
        l_mu[j] += psi * (gCx[j] * l_F0x + gCy[j] * l_F0y);
        l_gCx[j] += psi * mu[j] * l_F0x;
        l_gCy[j] += psi * mu[j] * l_F0y;
    }
    // J = sum_p c_p g_p
#pragma unroll
    for (int p = 1; p < 9; ++p) l_g[p] += T(aCx[p]) * l_Jx + T(aCy[p]) * l_Jy;
    // mC = -m0 sum_i rho_i Q_i
#pragma unroll
    for (int i = 0; i < NP; ++i) {
        l_Qx[i] += -P.m0 * P.rho[i] * l_mCx;
        l_Qy[i] += -P.m0 * P.rho[i] * l_mCy;
    }
    // Q_i = C_i (S_C grad mu_i - sum_j C_j grad mu_j)
    T l_SC = T(0), l_Gx = T(0), l_Gy = T(0);
#pragma unroll
    for (int i = 0; i < NP; ++i) {
        l_Cv[i] += (SC * gmx[i] - Gx) * l_Qx[i] + (SC * gmy[i] - Gy) * l_Qy[i];
        l_SC += Cv[i] * (gmx[i] * l_Qx[i] + gmy[i] * l_Qy[i]);
        l_gmx[i] += Cv[i] * SC * l_Qx[i];
        l_gmy[i] += Cv[i] * SC * l_Qy[i];
        l_Gx -= Cv[i] * l_Qx[i];
        l_Gy -= Cv[i] * l_Qy[i];
    }
#pragma unroll
    for (int j = 0; j < NP; ++j) {
        l_Cv[j] += gmx[j] * l_Gx + gmy[j] * l_Gy + l_SC;
        l_gmx[j] += Cv[j] * l_Gx;
        l_gmy[j] += Cv[j] * l_Gy;
    }
    // s21 = 1 / inv_s21, s22 = 1 / (nu nu_to_s22 + 1/2)
    l_inv_s21 += -s21 * s21 * l_s21;
    l_nu += P.nu_to_s21 * l_inv_s21 + P.nu_to_s22 * (-s22 * s22 * l_s22);
#pragma unroll
    for (int j = 0; j < NP; ++j) {
        l_Cv[j] += P.rho[j] * l_rho + P.nu[j] * l_nu;
        l_gCx[j] += P.rho[j] * l_grx;
        l_gCy[j] += P.rho[j] * l_gry;
    }
    // C_N = 1 - sum_j C_j
#pragma unroll
    for (int j = 0; j < NP - 1; ++j) {
        l_Cv[j] -= l_Cv[NP - 1];
        l_gCx[j] -= l_gCx[NP - 1];
        l_gCy[j] -= l_gCy[NP - 1];
    }

    // ---- write the local adjoints and the stencil-output adjoints --------
    T* ad_g = ad_pop_out + (long long)9 * (NP - 1) * pl;
#pragma unroll
    for (int p = 0; p < 9; ++p) ad_g[p * pl + o] = l_g[p];
    ad_lag_out[o] = T(0);   // lagged plane a: added from the gathered adjoint
#pragma unroll
    for (int k = 1; k < 2 * NP + 3; ++k) ad_lag_out[k * pl + o] = li_lag[k];
#pragma unroll
    for (int j = 0; j < NP - 1; ++j) {
        W.lC[j * pl + o] = l_Cv[j];
        W.lgC[(2 * j) * pl + o] = l_gCx[j];
        W.lgC[(2 * j + 1) * pl + o] = l_gCy[j];
    }
    W.lpsi[o] = l_psi;
    W.lgp[o] = l_gpx;
    W.lgp[pl + o] = l_gpy;
    W.lgpr[o] = l_gprx;
    W.lgpr[pl + o] = l_gpry;
#pragma unroll
    for (int j = 0; j < NP; ++j) {
        W.lmu[j * pl + o] = l_mu[j];
        W.lgm[(2 * j) * pl + o] = l_gmx[j];
        W.lgm[(2 * j + 1) * pl + o] = l_gmy[j];
    }
    W.lga[o] = l_dax;
    W.lga[pl + o] = l_day;
}

// sum_p gw_p (c_p . (vx, vy))(q - c_p) over interior source nodes q - c_p
template <typename T>
__device__ __forceinline__ T grad_T(const KParams<T>& P, const T* vx, const T* vy, int X, int Y) {
    T s = T(0);
#pragma unroll
    for (int p = 1; p < 9; ++p) {
        const int sx = X - aCx[p], sy = Y - aCy[p];
        if (sx < 0 || sx >= P.nx || sy < 0 || sy >= P.ny) continue;
        const long long so = P.org + (long long)sy * P.pitch + sx;
        s += gw(P, p) * (T(aCx[p]) * vx[so] + T(aCy[p]) * vy[so]);
    }
    return s;
}

// The positions whose values are copies of node (x, y): the node itself and,
// at the domain edge, its images in the 1-node ghost ring (periodic wrap or
// wall mirror; an axis of length 1 or 2 may give two images on one side).
// A transposed stencil gathered at each of them and summed is the node's
// adjoint, so no ghost-ring pass is needed.
struct Images {
    int xi[2], yi[2];   // ghost-ring coordinates that copy x (resp. y); nx / ny unused
    int nxi, nyi;
};
template <typename T>
__device__ __forceinline__ void images_of(const KParams<T>& P, int x, int y, Images& im) {
    im.nxi = im.nyi = 0;
    if (x == map_index(-1, P.nx, P.px)) im.xi[im.nxi++] = -1;
    if (x == map_index(P.nx, P.nx, P.px)) im.xi[im.nxi++] = P.nx;
    if (y == map_index(-1, P.ny, P.py)) im.yi[im.nyi++] = -1;
    if (y == map_index(P.ny, P.ny, P.py)) im.yi[im.nyi++] = P.ny;
}
// f(X, Y) for every image of (x, y) other than the node itself
template <typename T, class F>
__device__ __forceinline__ void for_images(const KParams<T>& P, int x, int y, F f) {
    Images im;
    images_of(P, x, y, im);
#pragma unroll
    for (int a = 0; a < 2; ++a)
        if (a < im.nxi) f(im.xi[a], y);
#pragma unroll
    for (int b = 0; b < 2; ++b)
        if (b < im.nyi) f(x, im.yi[b]);
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b)
            if (a < im.nxi && b < im.nyi) f(im.xi[a], im.yi[b]);
}

// Shared-memory copy of planes over a tile plus a 1-node ring: entry
// (k, ly, lx) holds plane k at node (x0 - 1 + lx, y0 - 1 + ly), zero where
// that position is outside the domain (not a source node).
constexpr int RW = AX + 2, RH = AY + 2, RN = RW * RH;
// The planes are read through the read-only path (no kernel that loads a
// ring writes those planes), so the loads need not wait for the earlier
// shared-memory stores and are all in flight at once.
template <typename T, int NPL>
__device__ __forceinline__ void load_ring(const KParams<T>& P, T* sm, const T* __restrict__ base, int x0, int y0) {
    // thread (tx, ty) copies rows ty and ty + 8, columns tx and tx + 32
#pragma unroll
    for (int rr = 0; rr < 2; ++rr) {
        const int ly = threadIdx.y + rr * AY;
        if (ly >= RH) continue;
        const int Y = y0 - 1 + ly;
        const bool yok = Y >= 0 && Y < P.ny;
#pragma unroll
        for (int cc = 0; cc < 2; ++cc) {
            const int lx = threadIdx.x + cc * AX;
            if (lx >= RW) continue;
            const int X = x0 - 1 + lx;
            const bool ok = yok && X >= 0 && X < P.nx;
            const long long g = P.org + (long long)Y * P.pitch + X;
#pragma unroll
            for (int q = 0; q < NPL; ++q) sm[q * RN + ly * RW + lx] = ok ? __ldg(base + q * P.plane + g) : T(0);
        }
    }
}
// sum_p gw_p (c_p . (vx, vy))(q - c_p) from the ring copy, q = thread's node
template <typename T>
__device__ __forceinline__ T grad_T_sm(const KParams<T>& P, const T* vx, const T* vy, int lx, int ly) {
    T s = T(0);
#pragma unroll
    for (int p = 1; p < 9; ++p) {
        const int r = (ly + 1 - aCy[p]) * RW + lx + 1 - aCx[p];
        s += gw(P, p) * (T(aCx[p]) * vx[r] + T(aCy[p]) * vy[r]);
    }
    return s;
}

// ---- transposed stencils of the node update, folded -----------------------
// LC_j, Lpsi, Lmu_j at every node (sum over the node and its ghost images),
// and the adjoint of the lagged plane a straight into the output state.
// Ring copies (shared memory) of the 2N+2 vector pairs: grad C_j (N-1),
// grad psi, grad(psi rho), grad mu_j (N), grad a.
template <typename T, int NP>
__device__ __forceinline__ void mu_node_at(const KParams<T>& P, const T* __restrict__ psi_pl,
                                           const T* __restrict__ cosf, const AdjPlanes<T, NP>& W,
                                           double* __restrict__ dJ_dcos, int x, int y, const T (&Lmu)[NP]);

// kMu: the chemical-potential VJP (mu_node_at) of the node follows in the
// same thread from the gathered adjoint of mu, which then never reaches
// memory (the initial state's reverse runs k_adj_mu_node on its own).
template <typename T, int NP, bool kMu>
__global__ void __launch_bounds__(256) k_adj_gather3(KParams<T> P, const T* __restrict__ psi_pl,
                                                     AdjPlanes<T, NP> W, T* __restrict__ ad_lag_out,
                                                     const T* __restrict__ cosf, double* __restrict__ dJ_dcos) {
    constexpr int NV = 2 * (2 * NP + 2);
    extern __shared__ __align__(16) unsigned char g3_raw[];
    T* sm = reinterpret_cast<T*>(g3_raw);
    const long long pl = P.plane;
    const int x0 = blockIdx.x * AX, y0 = blockIdx.y * AY;
    load_ring<T, NV>(P, sm, W.lgC, x0, y0);
    __syncthreads();
    const int x = x0 + threadIdx.x, y = y0 + threadIdx.y;
    if (x >= P.nx || y >= P.ny) return;
    const int lx = threadIdx.x, ly = threadIdx.y;
    const long long o = P.org + (long long)y * P.pitch + x;
    auto V = [&](int k) { return sm + k * RN; };
    const int kC = 0, kP = 2 * (NP - 1), kR = kP + 2, kM = kR + 2, kA = kM + 2 * NP;
    T LC[NP], Lmu[NP];
    T Lpsi = W.lpsi[o];
    T rq = P.rho[NP - 1];
#pragma unroll
    for (int j = 0; j < NP - 1; ++j) rq += (P.rho[j] - P.rho[NP - 1]) * W.C[j * pl + o];
    const T psiq = psi_pl[o];
    // the node's own position, from the ring copy
    {
        const T lchi = grad_T_sm(P, V(kR), V(kR + 1), lx, ly);
#pragma unroll
        for (int j = 0; j < NP - 1; ++j)
            LC[j] = W.lC[j * pl + o] + grad_T_sm(P, V(kC + 2 * j), V(kC + 2 * j + 1), lx, ly) +
                    psiq * (P.rho[j] - P.rho[NP - 1]) * lchi;
        Lpsi += grad_T_sm(P, V(kP), V(kP + 1), lx, ly) + rq * lchi;
#pragma unroll
        for (int j = 0; j < NP; ++j)
            Lmu[j] = W.lmu[j * pl + o] + grad_T_sm(P, V(kM + 2 * j), V(kM + 2 * j + 1), lx, ly);
        ad_lag_out[o] = grad_T_sm(P, V(kA), V(kA + 1), lx, ly);
    }
    // ghost-ring images of edge nodes, from global memory
    if (x == 0 || y == 0 || x == P.nx - 1 || y == P.ny - 1) {
        T La = T(0);
        for_images<T>(P, x, y, [&](int X, int Y) {
            const long long q = P.org + (long long)Y * P.pitch + X;
            const T lchi = grad_T(P, W.lgpr, W.lgpr + pl, X, Y);
            T rg = P.rho[NP - 1];
#pragma unroll
            for (int j = 0; j < NP - 1; ++j) rg += (P.rho[j] - P.rho[NP - 1]) * W.C[j * pl + q];
            const T psig = psi_pl[q];
#pragma unroll
            for (int j = 0; j < NP - 1; ++j)
                LC[j] += grad_T(P, W.lgC + (2 * j) * pl, W.lgC + (2 * j + 1) * pl, X, Y) +
                         psig * (P.rho[j] - P.rho[NP - 1]) * lchi;
            Lpsi += grad_T(P, W.lgp, W.lgp + pl, X, Y) + rg * lchi;
#pragma unroll
            for (int j = 0; j < NP; ++j) Lmu[j] += grad_T(P, W.lgm + (2 * j) * pl, W.lgm + (2 * j + 1) * pl, X, Y);
            La += grad_T(P, W.lga, W.lga + pl, X, Y);
        });
        ad_lag_out[o] += La;
    }
#pragma unroll
    for (int j = 0; j < NP - 1; ++j) W.LC[j * pl + o] = LC[j];
    W.Lpsi[o] = Lpsi;
    if constexpr (kMu) {
        mu_node_at<T, NP>(P, psi_pl, cosf, W, dJ_dcos, x, y, Lmu);
    } else {
#pragma unroll
        for (int j = 0; j < NP; ++j) W.Lmu[j * pl + o] = Lmu[j];
    }
}

// ---- VJP of the chemical potential (Eq. 2.14) per node ---------------------
template <typename T, int NP>
__device__ __forceinline__ void mu_node_at(const KParams<T>& P, const T* __restrict__ psi_pl,
                                           const T* __restrict__ cosf, const AdjPlanes<T, NP>& W,
                                           double* __restrict__ dJ_dcos, int x, int y, const T (&Lmu)[NP]) {
    const long long pl = P.plane;
    const long long o = P.org + (long long)y * P.pitch + x;
    const PlaneAt<T> Ca{W.C, pl, o, P.pitch}, Ps{psi_pl, pl, o, P.pitch};
    T cth[NP];
    node_cth<T, NP>(P, cosf, o, cth);
    // forward (dev::chem_pot)
    const T p0 = Ps(0, 0);
    T gpx, gpy;
    dev::grad9(P, [&](int dy, int dx) { return Ps(dy, dx); }, gpx, gpy);
    const T agp = sqrt(gpx * gpx + gpy * gpy);
    T Cv[NP], L[NP];
    {
        T sC = T(0), sL = T(0);
#pragma unroll
        for (int j = 0; j < NP - 1; ++j) {
            const T c0 = Ca(j, 0, 0);
            T l = T(0);
#pragma unroll
            for (int p = 1; p < 9; ++p)
                l += lw(P, p) * (p0 + Ps(aCy[p], aCx[p])) * (Ca(j, aCy[p], aCx[p]) - c0);
            Cv[j] = c0;
            L[j] = l;
            sC += c0;
            sL += l;
        }
        Cv[NP - 1] = T(1) - sC;
        L[NP - 1] = -sL;
    }
    T aj[NP], gpv[NP];
#pragma unroll
    for (int j = 0; j < NP; ++j) {
        aj[j] = j < NP - 1 ? P.sigN[j] * cth[j] : T(0);
        gpv[j] = dev::gprime(Cv[j]);
    }
    T gpair[NP][NP], cpair[NP][NP];
#pragma unroll
    for (int i = 0; i < NP; ++i) {
        gpair[i][i] = cpair[i][i] = T(0);
#pragma unroll
        for (int j = i + 1; j < NP; ++j) {
            gpair[i][j] = gpair[j][i] = dev::gprime(Cv[i] + Cv[j]);
            const T c = (aj[i] - aj[j]) * P.invsig[i][j];
            cpair[i][j] = c;
            cpair[j][i] = -c;
        }
    }
    T Wj[NP], accj[NP];
#pragma unroll
    for (int j = 0; j < NP; ++j) {
        T acc = T(0);
#pragma unroll
        for (int q = 0; q < NP; ++q)
            if (q != j) acc += cpair[j][q] * Cv[q];
        accj[j] = acc;
        Wj[j] = Cv[j] * acc;
    }
    const T inv_p0 = T(1) / p0;
    T bulk[NP], wet[NP], psimu[NP];
#pragma unroll
    for (int i = 0; i < NP; ++i) {
        T b = T(0), gr = T(0), w = T(0);
#pragma unroll
        for (int j = 0; j < NP; ++j) {
            if (j != i) b += P.beta2[i][j] * (gpv[i] - gpair[i][j]);
            gr += P.kap[i][j] * L[j];
            w += P.wet[i][j] * Wj[j];
        }
        bulk[i] = b;
        wet[i] = w;
        psimu[i] = p0 * b + gr + agp * w;
    }
    // reverse
    T lpm[NP];
    T l_inv = T(0);
#pragma unroll
    for (int i = 0; i < NP; ++i) {
        const T lmu = Lmu[i];
        lpm[i] = lmu * inv_p0;
        l_inv += psimu[i] * lmu;
    }
    T l_p0 = -inv_p0 * inv_p0 * l_inv;
    T l_agp = T(0), l_L[NP], l_W[NP], l_gp[NP], l_Cv[NP];
#pragma unroll
    for (int j = 0; j < NP; ++j) {
        T sL = T(0), sW = T(0);
#pragma unroll
        for (int i = 0; i < NP; ++i) {
            sL += P.kap[i][j] * lpm[i];
            sW += P.wet[i][j] * lpm[i];
        }
        l_L[j] = sL;
        l_W[j] = agp * sW;
        l_gp[j] = T(0);
        l_Cv[j] = T(0);
    }
#pragma unroll
    for (int i = 0; i < NP; ++i) {
        l_p0 += bulk[i] * lpm[i];
        l_agp += wet[i] * lpm[i];
    }
    // bulk_i = sum_{j != i} 2 beta_ij (g'(C_i) - g'(C_i + C_j))
#pragma unroll
    for (int i = 0; i < NP; ++i) {
        const T lb = p0 * lpm[i];
#pragma unroll
        for (int j = 0; j < NP; ++j)
            if (j != i) l_gp[i] += P.beta2[i][j] * lb;
    }
#pragma unroll
    for (int i = 0; i < NP; ++i) {
#pragma unroll
        for (int j = i + 1; j < NP; ++j) {
            const T t = -(P.beta2[i][j] * p0 * lpm[i] + P.beta2[j][i] * p0 * lpm[j]);
            const T gs = gsecond(Cv[i] + Cv[j]) * t;
            l_Cv[i] += gs;
            l_Cv[j] += gs;
        }
        l_Cv[i] += gsecond(Cv[i]) * l_gp[i];
    }
    // W_j = C_j sum_{q != j} cos_jq C_q, cos_jq = (a_j - a_q) / sigma_jq
    T l_aj[NP];
#pragma unroll
    for (int j = 0; j < NP; ++j) l_aj[j] = T(0);
#pragma unroll
    for (int j = 0; j < NP; ++j) {
        l_Cv[j] += accj[j] * l_W[j];
#pragma unroll
        for (int q = 0; q < NP; ++q) {
            if (q == j) continue;
            l_Cv[q] += Cv[j] * cpair[j][q] * l_W[j];
            // cpair[j][q] = (a_j - a_q) invsig_jq
            const T lc = Cv[j] * Cv[q] * l_W[j] * P.invsig[j][q];
            l_aj[j] += lc;
            l_aj[q] -= lc;
        }
    }
    const long long node = (long long)y * P.nx + x;
    const long long nn = (long long)P.nx * P.ny;
#pragma unroll
    for (int j = 0; j < NP - 1; ++j) dJ_dcos[j * nn + node] += (double)(P.sigN[j] * l_aj[j]);
    // |grad psi| has a kink at grad psi = 0.  In the fluid bulk psi is 1 up
    // to rounding, and the direction of a rounding-level gradient would
    // carry the wetting term's full weight into dJ/dpsi there; below
    // kKinkGradPsi the derivative is taken as zero, the value central
    // differences give at the kink.
    T l_gpx = T(0), l_gpy = T(0);
    if (agp > T(kKinkGradPsi)) {
        l_gpx = gpx / agp * l_agp;
        l_gpy = gpy / agp * l_agp;
    }
#pragma unroll
    for (int j = 0; j < NP - 1; ++j) {
        l_Cv[j] -= l_Cv[NP - 1];
        l_L[j] -= l_L[NP - 1];
        W.mC[j * pl + o] = l_Cv[j];
        W.mL[j * pl + o] = l_L[j];
    }
    W.mpsi[o] = l_p0;
    W.mgp[o] = l_gpx;
    W.mgp[pl + o] = l_gpy;
}

template <typename T, int NP>
__global__ void __launch_bounds__(256) k_adj_mu_node(KParams<T> P, const T* __restrict__ psi_pl,
                                                     const T* __restrict__ cosf, AdjPlanes<T, NP> W,
                                                     double* __restrict__ dJ_dcos) {
    const int x = blockIdx.x * AX + threadIdx.x, y = blockIdx.y * AY + threadIdx.y;
    if (x >= P.nx || y >= P.ny) return;
    const long long o = P.org + (long long)y * P.pitch + x;
    T Lmu[NP];
#pragma unroll
    for (int i = 0; i < NP; ++i) Lmu[i] = W.Lmu[i * P.plane + o];
    mu_node_at<T, NP>(P, psi_pl, cosf, W, dJ_dcos, x, y, Lmu);
}

// ---- transposed div(psi grad C_j) and grad psi stencils, folded, then
//      C_i = sum_p f^i_p / psi reversed and dJ/dpsi ------------------------------
// Ring copies: mL_j (N-1), grad psi pair, psi, C_j (N-1).
template <typename T, int NP>
__device__ __forceinline__ void gather2_at(const KParams<T>& P, const T* psi_pl, const AdjPlanes<T, NP>& W, int X,
                                           int Y, T lC[NP], T& lpsi) {
    const long long pl = P.plane;
    const long long q = P.org + (long long)Y * P.pitch + X;
    const T psiq = psi_pl[q];
    lpsi += grad_T(P, W.mgp, W.mgp + pl, X, Y);
#pragma unroll
    for (int p = 1; p < 9; ++p) {
        const int sx = X - aCx[p], sy = Y - aCy[p];
        if (sx < 0 || sx >= P.nx || sy < 0 || sy >= P.ny) continue;
        const long long so = P.org + (long long)sy * P.pitch + sx;
        const T w = lw(P, p);
        const T psis = psi_pl[so];
#pragma unroll
        for (int j = 0; j < NP - 1; ++j) {
            const T mL = W.mL[j * pl + so];
            lC[j] += w * (psis + psiq) * mL;
            lpsi += w * (W.C[j * pl + q] - W.C[j * pl + so]) * mL;
        }
    }
}

template <typename T, int NP>
__global__ void __launch_bounds__(256) k_adj_gather2(KParams<T> P, const T* __restrict__ psi_pl,
                                                     AdjPlanes<T, NP> W, T* __restrict__ ad_pop_out,
                                                     double* __restrict__ dJ_dpsi, int initial) {
    extern __shared__ __align__(16) unsigned char g2_raw[];
    T* sm = reinterpret_cast<T*>(g2_raw);
    const long long pl = P.plane;
    const int x0 = blockIdx.x * AX, y0 = blockIdx.y * AY;
    load_ring<T, NP + 1>(P, sm, W.mL, x0, y0);                  // mL_j, grad psi pair
    load_ring<T, 1>(P, sm + (NP + 1) * RN, psi_pl, x0, y0);
    load_ring<T, NP - 1>(P, sm + (NP + 2) * RN, W.C, x0, y0);
    __syncthreads();
    const int x = x0 + threadIdx.x, y = y0 + threadIdx.y;
    if (x >= P.nx || y >= P.ny) return;
    const int lx = threadIdx.x, ly = threadIdx.y;
    const long long o = P.org + (long long)y * P.pitch + x;
    const T* sL = sm;
    const T* sG = sm + (NP - 1) * RN;
    const T* sP = sG + 2 * RN;
    const T* sC = sP + RN;
    const int rc = (ly + 1) * RW + lx + 1;
    const T psio = sP[rc];
    T lC[NP];
    T lpsi = W.Lpsi[o] + W.mpsi[o] + grad_T_sm(P, sG, sG + RN, lx, ly);
#pragma unroll
    for (int j = 0; j < NP - 1; ++j) lC[j] = W.LC[j * pl + o] + W.mC[j * pl + o];
    // the node as the neighbour o = s + c_p of a node s (ring entries outside
    // the domain hold mL = 0)
#pragma unroll
    for (int p = 1; p < 9; ++p) {
        const int r = rc - aCy[p] * RW - aCx[p];
        const T w = lw(P, p);
        const T psis = sP[r];
#pragma unroll
        for (int j = 0; j < NP - 1; ++j) {
            const T mL = sL[j * RN + r];
            lC[j] += w * (psis + psio) * mL;
            lpsi += w * (sC[j * RN + rc] - sC[j * RN + r]) * mL;
        }
    }
    // the node as the centre of its own stencil: neighbours from the ring
    // copy, or at the domain edge from the padded planes, whose ghost frames
    // hold the copies the forward step read
    const bool edge = x == 0 || y == 0 || x == P.nx - 1 || y == P.ny - 1;
#pragma unroll
    for (int j = 0; j < NP - 1; ++j) {
        const T mL = sL[j * RN + rc];
        const T co = sC[j * RN + rc];
        T sps = T(0), scs = T(0);
        if (!edge) {
#pragma unroll
            for (int p = 1; p < 9; ++p) {
                const int r = rc + aCy[p] * RW + aCx[p];
                sps += lw(P, p) * (psio + sP[r]);
                scs += lw(P, p) * (sC[j * RN + r] - co);
            }
        } else {
#pragma unroll
            for (int p = 1; p < 9; ++p) {
                const long long nb = o + (long long)aCy[p] * P.pitch + aCx[p];
                sps += lw(P, p) * (psio + psi_pl[nb]);
                scs += lw(P, p) * (W.C[j * pl + nb] - co);
            }
        }
        lC[j] -= mL * sps;
        lpsi += mL * scs;
    }
    if (edge)
        for_images<T>(P, x, y, [&](int X, int Y) { gather2_at<T, NP>(P, psi_pl, W, X, Y, lC, lpsi); });
    if (!initial) {
        // C_i = sum_p f^i_p / psi
        const T inv = T(1) / psio;
#pragma unroll
        for (int i = 0; i < NP - 1; ++i) {
            const T d = lC[i] * inv;
            // all nine loads before any store (the compiler cannot tell the
            // planes apart, so interleaved read-modify-writes would serialise)
            T v[9];
#pragma unroll
            for (int p = 0; p < 9; ++p) v[p] = ad_pop_out[(9 * i + p) * pl + o];
#pragma unroll
            for (int p = 0; p < 9; ++p) ad_pop_out[(9 * i + p) * pl + o] = v[p] + d;
            lpsi -= d * sC[i * RN + rc];
        }
    }
    dJ_dpsi[(long long)y * P.nx + x] += (double)lpsi;
}

// ---- initial state reversed: f^i_p = w_p eta_i psi mu_i (p > 0),
//      f^i_0 = (w_0 - 1) eta_i psi mu_i + psi C0_i ------------------------------
template <typename T, int NP>
__global__ void __launch_bounds__(256) k_adj_init_node(KParams<T> P, const T* __restrict__ psi_pl,
                                                       const T* __restrict__ ad_pop0, AdjPlanes<T, NP> W) {
    const int x = blockIdx.x * AX + threadIdx.x, y = blockIdx.y * AY + threadIdx.y;
    if (x >= P.nx || y >= P.ny) return;
    const long long pl = P.plane;
    const long long o = P.org + (long long)y * P.pitch + x;
    const T psi = psi_pl[o];
    T lpsi = T(0);
#pragma unroll
    for (int i = 0; i < NP - 1; ++i) {
        T lemu = T(0);
#pragma unroll
        for (int p = 0; p < 9; ++p) lemu += wgt(P, p) * ad_pop0[(9 * i + p) * pl + o];
        const T l0 = ad_pop0[(9 * i) * pl + o];
        lemu -= l0;
        lpsi += W.C[i * pl + o] * l0 + P.eta[i] * W.mu[i * pl + o] * lemu;
        W.Lmu[i * pl + o] = P.eta[i] * psi * lemu;
    }
    W.Lmu[(NP - 1) * pl + o] = T(0);
    W.Lpsi[o] = lpsi;
}

// ---- objective: phase centroid J = sum_x x m(x) / sum_x m(x), m = sum_p f^i_p
template <typename T>
__global__ void __launch_bounds__(256) k_centroid_partial(KParams<T> P, const T* __restrict__ f,
                                                          double* __restrict__ part) {
    double s0 = 0.0, s1 = 0.0;
    const long long n = (long long)P.nx * P.ny;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
         idx += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(idx / P.nx), x = (int)(idx - (long long)y * P.nx);
        const long long o = P.org + (long long)y * P.pitch + x;
        double m = 0.0;
        for (int p = 0; p < 9; ++p) m += (double)f[p * P.plane + o];
        s0 += m;
        s1 += (double)x * m;
    }
    __shared__ double r0[256], r1[256];
    r0[threadIdx.x] = s0;
    r1[threadIdx.x] = s1;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            r0[threadIdx.x] += r0[threadIdx.x + w];
            r1[threadIdx.x] += r1[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = r0[0];
        part[2 * blockIdx.x + 1] = r1[0];
    }
}

__global__ void k_centroid_final(const double* __restrict__ part, int nblocks, double* __restrict__ out) {
    if (threadIdx.x != 0) return;
    double s0 = 0.0, s1 = 0.0;
    for (int b = 0; b < nblocks; ++b) {
        s0 += part[2 * b];
        s1 += part[2 * b + 1];
    }
    out[0] = s1 / s0;   // J
    out[1] = s0;        // M
}

template <typename T>
__global__ void __launch_bounds__(256) k_centroid_seed(KParams<T> P, const double* __restrict__ JM,
                                                       T* __restrict__ lf) {
    const int x = blockIdx.x * AX + threadIdx.x, y = blockIdx.y * AY + threadIdx.y;
    if (x >= P.nx || y >= P.ny) return;
    const long long o = P.org + (long long)y * P.pitch + x;
    const T v = (T)(((double)x - JM[0]) / JM[1]);
#pragma unroll
    for (int p = 0; p < 9; ++p) lf[p * P.plane + o] = v;
}

inline dim3 node_grid(int nx, int ny) { return dim3((nx + AX - 1) / AX, (ny + AY - 1) / AY); }

template <typename T, int NP>
cudaError_t recompute_fields(const AdjStepArgs<T>& a, const AdjPlanes<T, NP>& W, bool from_state,
                             cudaStream_t s) {
    const KParams<T>& k = *a.kp;
    // every adjoint kernel reads C and mu at most one node outside the
    // domain: both passes run over the domain and its 1-node ring
    const dim3 blk(AX, AY), grd = node_grid(k.nx + 2, k.ny + 2);
    cudaError_t e;
    if (from_state) {
        k_adj_order<T, NP><<<grd, blk, 0, s>>>(k, a.st_pop, a.psi, W.C);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    } else if ((e = launch_fill_ghosts<T>(W.C, NP - 1, k, s, 1, 1)) != cudaSuccess) {
        return e;   // C0 was put into W.C by the caller
    }
    k_adj_mu<T, NP><<<grd, blk, 0, s>>>(k, W.C, a.psi, a.cosf, W.mu);
    return cudaGetLastError();
}

template <typename T, int NP>
cudaError_t gather_smem_attrs() {
    cudaError_t e = cudaFuncSetAttribute(k_adj_gather3<T, NP, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(sizeof(T) * RN * 2 * (2 * NP + 2)));
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_adj_gather2<T, NP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(sizeof(T) * RN * (2 * (NP - 1) + 3)));
}

template <typename T, int NP>
cudaError_t adjoint_step_n(const AdjStepArgs<T>& a, cudaStream_t s) {
    const KParams<T>& k = *a.kp;
    // the shared-memory limit is a per-device attribute: set it on every call
    const cudaError_t attrs = gather_smem_attrs<T, NP>();
    if (attrs != cudaSuccess) return attrs;
    AdjPlanes<T, NP> W = AdjPlanes<T, NP>::carve(a.scratch, k.plane);
    W.a = a.st_lag;   // lagged plane 0
    const dim3 blk(AX, AY), grd = node_grid(k.nx, k.ny);
    cudaError_t e;
    if ((e = recompute_fields<T, NP>(a, W, true, s)) != cudaSuccess) return e;
    k_adj_node<T, NP><<<grd, blk, 0, s>>>(k, a.psi, a.st_pop, a.st_lag, a.ad_pop_in, a.ad_lag_in,
                                          a.ad_pop_out, a.ad_lag_out, W);
    k_adj_gather3<T, NP, true><<<grd, blk, sizeof(T) * RN * 2 * (2 * NP + 2), s>>>(k, a.psi, W, a.ad_lag_out,
                                                                                   a.cosf, a.dJ_dcos);
    k_adj_gather2<T, NP><<<grd, blk, sizeof(T) * RN * (2 * (NP - 1) + 3), s>>>(k, a.psi, W, a.ad_pop_out,
                                                                              a.dJ_dpsi, 0);
    return cudaGetLastError();
}

template <typename T, int NP>
cudaError_t adjoint_initial_n(const AdjStepArgs<T>& a, cudaStream_t s) {
    const KParams<T>& k = *a.kp;
    // the shared-memory limit is a per-device attribute: set it on every call
    const cudaError_t attrs = gather_smem_attrs<T, NP>();
    if (attrs != cudaSuccess) return attrs;
    const AdjPlanes<T, NP> W = AdjPlanes<T, NP>::carve(a.scratch, k.plane);
    const dim3 blk(AX, AY), grd = node_grid(k.nx, k.ny);
    cudaError_t e;
    // the caller has put C0 into W.C
    if ((e = recompute_fields<T, NP>(a, W, false, s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(W.LC, 0, sizeof(T) * k.plane * (NP - 1), s)) != cudaSuccess) return e;
    k_adj_init_node<T, NP><<<grd, blk, 0, s>>>(k, a.psi, a.ad_pop_in, W);
    k_adj_mu_node<T, NP><<<grd, blk, 0, s>>>(k, a.psi, a.cosf, W, a.dJ_dcos);
    k_adj_gather2<T, NP><<<grd, blk, sizeof(T) * RN * (2 * (NP - 1) + 3), s>>>(k, a.psi, W, nullptr,
                                                                              a.dJ_dpsi, 1);
    return cudaGetLastError();
}

}  // namespace

template <typename T>
size_t adjoint_scratch_planes(int N) {
    return (size_t)(12 * N + 4);
}

template <typename T>
T* adjoint_c_planes(T* scratch) {
    return scratch;   // W.C is the first block of the scratch
}

#define DDCC_ADJ_DISPATCH(fn, ...)                            \
    switch (a.kp->N) {                                        \
        case 2: return fn<T, 2>(__VA_ARGS__);                 \
        case 3: return fn<T, 3>(__VA_ARGS__);                 \
        case 4: return fn<T, 4>(__VA_ARGS__);                 \
        default: return cudaErrorInvalidValue;                \
    }

template <typename T>
cudaError_t launch_adjoint_step(const AdjStepArgs<T>& a, cudaStream_t s) {
    DDCC_ADJ_DISPATCH(adjoint_step_n, a, s);
}

template <typename T>
cudaError_t launch_adjoint_initial(const AdjStepArgs<T>& a, cudaStream_t s) {
    DDCC_ADJ_DISPATCH(adjoint_initial_n, a, s);
}

template <typename T>
cudaError_t launch_centroid(const KParams<T>& kp, const T* f_phase, double* part, double* JM,
                            T* seed_f_phase, cudaStream_t s) {
    k_centroid_partial<T><<<kMassBlocks, 256, 0, s>>>(kp, f_phase, part);
    k_centroid_final<<<1, 32, 0, s>>>(part, kMassBlocks, JM);
    if (seed_f_phase)
        k_centroid_seed<T><<<node_grid(kp.nx, kp.ny), dim3(AX, AY), 0, s>>>(kp, JM, seed_f_phase);
    return cudaGetLastError();
}

#define DDCC_ADJ_INSTANTIATE(T)                                                                      \
    template size_t adjoint_scratch_planes<T>(int);                                                  \
    template T* adjoint_c_planes<T>(T*);                                                             \
    template cudaError_t launch_adjoint_step<T>(const AdjStepArgs<T>&, cudaStream_t);                \
    template cudaError_t launch_adjoint_initial<T>(const AdjStepArgs<T>&, cudaStream_t);             \
    template cudaError_t launch_centroid<T>(const KParams<T>&, const T*, double*, double*, T*,       \
                                            cudaStream_t);

DDCC_ADJ_INSTANTIATE(float)
DDCC_ADJ_INSTANTIATE(double)

}  // namespace ddcc
