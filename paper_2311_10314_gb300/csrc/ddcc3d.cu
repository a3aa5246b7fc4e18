// Three-dimensional DD-CCLB stepper (C ABI in include/ddcc3d.h): phase
// populations on D3Q7, flow populations on D3Q15 (Sec. 3), periodic box.
//
// One step is three kernels over a 32 x 4 x 2 thread block per 256 nodes:
//   k3_order   C_i = sum_p f^i_p / psi                      (Sec. 3)
//   k3_mu      mu_i of Eq. 2.14 from C and psi on the 15-point stencil
//   k3_update  gradients (D3Q15-weighted isotropic stencils), mobility
//              (Eq. 2.5), S_i (Eq. 3.7), m^C, force, the joint velocity /
//              Eq. 19 pressure solve, both collisions (Eqs. 3.1, 3.2 with
//              Eqs. 3.5-3.10), push streaming and the lagged fields.
// The rest population of each phase carries nearly all of psi C, so its
// update rounds at the ulp of psi C, with the same error every step once the
// flow is steady; the exact rounding error is recovered (TwoSum) and split
// evenly between the +x and -x populations, which keeps sum_p f to
// roundings at that smaller scale (in FP32 a steady drop otherwise loses
// mass every step) and sends the recovered mass in no preferred direction.
// Populations, lagged fields and the per-step C and mu are SoA planes of
// nx*ny*nz elements (x fastest), each plane 256-byte aligned; neighbours
// wrap periodically by index arithmetic.  g_0 is stored as g_0 - rho0 (the
// constant cancels in every moment difference).
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include <cuda_runtime.h>

#include "ddcc3d.h"

namespace {

constexpr int kMaxN = DDCC_MAX_PHASES;
constexpr int kBX = 32, kBY = 4, kBZ = 2;
constexpr int kBX4 = kBX / 4;        // threads along x of the four-nodes-per-thread kernel
constexpr int kThreads = kBX * kBY * kBZ;
constexpr int kMassBlocks = 304;     // 2 x 152 SMs
constexpr int kKinds = 4;            // order, mu, update, fused step
constexpr int kFusedTY = 8;          // rows of the fused step's column

// Velocities of Sec. 3: p = 0 rest; 1..6 = +x, -x, +y, -y, +z, -z; 7..14 the
// corners (+-1, +-1, +-1) with bit 0, 1, 2 of p - 7 giving a minus sign in
// x, y, z.  D3Q7 is p = 0..6 of the same list.
__host__ __device__ constexpr int cx(int p) { return p == 1 ? 1 : p == 2 ? -1 : p >= 7 ? (((p - 7) & 1) ? -1 : 1) : 0; }
__host__ __device__ constexpr int cy(int p) { return p == 3 ? 1 : p == 4 ? -1 : p >= 7 ? (((p - 7) & 2) ? -1 : 1) : 0; }
__host__ __device__ constexpr int cz(int p) { return p == 5 ? 1 : p == 6 ? -1 : p >= 7 ? (((p - 7) & 4) ? -1 : 1) : 0; }
__host__ __device__ constexpr int cc(int p, int a) { return a == 0 ? cx(p) : a == 1 ? cy(p) : cz(p); }
// the seven pairs of opposite velocities: p = pair_rep(q), c_pair_opp(q) = -c_p
__host__ __device__ constexpr int pair_rep(int q) { return q < 3 ? 2 * q + 1 : 7 + (q - 3); }
__host__ __device__ constexpr int pair_opp(int q) { return q < 3 ? 2 * q + 2 : 14 - (q - 3); }

// Kernel constants, derived on the host (make_params) from ddcc3d_params.
template <typename T>
struct P3 {
    int nx, ny, nz, N;
    long long nxy, plane;
    int has_cos_field;
    T cs2, inv_cs2;
    T ga, gc;                  // w_axis / cs2, w_corner / cs2 (D3Q15 weights)
    T w7_0, w7_1;              // D3Q7 weights
    T w15[3];                  // D3Q15 weights: rest, axis, corner
    T rho[kMaxN], nu[kMaxN];
    T beta2[kMaxN][kMaxN];     // 2 beta_ij = 6 sigma_ij / eps
    T kap[kMaxN][kMaxN];       // 3 eps sigma_ij / 4
    T wet[kMaxN][kMaxN];       // 3 sigma_ij
    T sigN[kMaxN];             // sigma_iN
    T invsig[kMaxN][kMaxN];
    T cos_uni[kMaxN];
    T eta[kMaxN];
    T m0, inv_m0;
    T s0f, s21f, s1f[kMaxN];   // D3Q7 rates
    T lg0, lg1, lg3, lg3c, lg4; // D3Q15 constant rates over the row norms
    T inv_n2d, inv_n2o;        // 1 / norm of the s21 and s22 rows
    T nu_to_s21, inv_cs2_nu;   // 2 / (1 - cs2), 1 / cs2 (Eq. 16)
    T damp;                    // 1 / eps0^3
    T K, Hfac;                 // K = 1 - 2 d0; H = Hfac (s21 - 2)
    T A_P, cP, kk, c2m3;       // Eq. 19 coefficients; 1 - 3 cs2
    T diag_den, off_den;       // 1 / (cs2 (1 - cs2)), 1 / cs2^2
    T body[3];
};

template <typename T>
struct F3 {
    T* f[2];        // 7 (N-1) planes: the D3Q7 populations, plane 7 (i-1) + p
    T* g[2];        // 15 planes
    T* lag[2];      // 3N + 7 planes
    T* psi;
    T* cosf;        // N-1 planes or null
    T* C;           // N-1 planes
    T* mu;          // N planes
    double* stage;  // 1 double plane (host staging, read-out)
    double* partial;
    int* flag;
};

// lagged plane indices
__host__ __device__ constexpr int lag_a(int k) { return k; }                   // xy, yz, zx
__host__ __device__ constexpr int lag_cu(int i, int a) { return 3 + 3 * i + a; }
template <int NP> __host__ __device__ constexpr int lag_T(int k) { return 3 + 3 * NP + k; }
template <int NP> __host__ __device__ constexpr int lag_pm() { return 9 + 3 * NP; }
__host__ __device__ constexpr int n_lag(int N) { return 3 * N + 7; }

struct Site {
    int x, y, z;
    long long zo[3];
    int yo[3], xo[3];
    __device__ long long at(int dx, int dy, int dz) const { return zo[dz + 1] + yo[dy + 1] + xo[dx + 1]; }
    __device__ long long self() const { return zo[1] + yo[1] + xo[1]; }
};

template <typename T>
__device__ __forceinline__ bool site(const P3<T>& P, Site& s) {
    s.x = blockIdx.x * kBX + threadIdx.x;
    s.y = blockIdx.y * kBY + threadIdx.y;
    s.z = blockIdx.z * kBZ + threadIdx.z;
    if (s.x >= P.nx || s.y >= P.ny || s.z >= P.nz) return false;
    s.xo[0] = s.x == 0 ? P.nx - 1 : s.x - 1;
    s.xo[1] = s.x;
    s.xo[2] = s.x == P.nx - 1 ? 0 : s.x + 1;
    s.yo[0] = (s.y == 0 ? P.ny - 1 : s.y - 1) * P.nx;
    s.yo[1] = s.y * P.nx;
    s.yo[2] = (s.y == P.ny - 1 ? 0 : s.y + 1) * P.nx;
    s.zo[0] = (long long)(s.z == 0 ? P.nz - 1 : s.z - 1) * P.nxy;
    s.zo[1] = (long long)s.z * P.nxy;
    s.zo[2] = (long long)(s.z == P.nz - 1 ? 0 : s.z + 1) * P.nxy;
    return true;
}

// Ping-pong buffer c of a pair without a dynamically indexed parameter array
// (which would be copied to local memory).
template <typename X>
__device__ __forceinline__ X* pick(X* const (&a)[2], int c) { return c ? a[1] : a[0]; }

// Rounded to nearest and never fused or reassociated by the compiler.
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }

template <typename T>
__device__ __forceinline__ T gprime(T C) {
    const T Cm = C - T(1);
    return T(2) * C * Cm * Cm + T(2) * C * C * Cm;
}

// ---------------------------------------------------------------------------
// volume fractions
// ---------------------------------------------------------------------------
template <typename T, int NP>
__global__ void __launch_bounds__(kThreads) k3_order(P3<T> P, F3<T> F, int cur) {
    Site s;
    if (!site(P, s)) return;
    const long long i0 = s.self();
    const T psi = F.psi[i0];
    const T* f = pick(F.f, cur);
#pragma unroll
    for (int i = 0; i < NP; ++i) {
        T acc = T(0);
#pragma unroll
        for (int p = 0; p < 7; ++p) acc += f[(7 * i + p) * P.plane + i0];
        F.C[i * P.plane + i0] = acc / psi;
    }
}

// ---------------------------------------------------------------------------
// chemical potentials, Eq. 2.14 (beta_ij = 3 sigma_ij / eps)
// ---------------------------------------------------------------------------
// mu_i of one node from its stencil sums: L_j = div(psi grad C_j) and
// grad psi, with the angles cos(theta_jN) (cN[N-1] = 0).
template <typename T, int NP>
__device__ __forceinline__ void mu_from_stencil(const P3<T>& P, T psi, const T C[NP + 1], const T L[NP + 1],
                                                T gpx, T gpy, T gpz, const T cN[NP + 1], T mu[NP + 1]) {
    constexpr int N = NP + 1;
    const T agp = sqrt(gpx * gpx + gpy * gpy + gpz * gpz);
    T wetj[N];    // sum_{q != j} cos(theta_jq) C_j C_q, cos(theta_jq) by Eq. 2.9 (sigma_NN = 0)
#pragma unroll
    for (int j = 0; j < N; ++j) {
        T acc = T(0);
#pragma unroll
        for (int q = 0; q < N; ++q)
            if (q != j) acc += (P.sigN[j] * cN[j] - P.sigN[q] * cN[q]) * P.invsig[j][q] * C[j] * C[q];
        wetj[j] = acc;
    }
    const T inv_psi = T(1) / psi;
#pragma unroll
    for (int i = 0; i < N; ++i) {
        const T gi = gprime(C[i]);
        T acc = T(0);
#pragma unroll
        for (int j = 0; j < N; ++j) {
            if (j == i) continue;
            acc += P.beta2[i][j] * psi * (gi - gprime(C[i] + C[j]));
            acc += P.kap[i][j] * L[j];
            acc += P.wet[i][j] * wetj[j] * agp;
        }
        mu[i] = acc * inv_psi;
    }
}

template <typename T, int NP>
__global__ void __launch_bounds__(kThreads) k3_mu(P3<T> P, F3<T> F) {
    constexpr int N = NP + 1;
    Site s;
    if (!site(P, s)) return;
    const long long i0 = s.self();
    const T psi = F.psi[i0];
    T C[N];
    {
        T sum = T(0);
#pragma unroll
        for (int j = 0; j < NP; ++j) {
            C[j] = F.C[j * P.plane + i0];
            sum += C[j];
        }
        C[NP] = T(1) - sum;
    }
    T L[N];
#pragma unroll
    for (int j = 0; j < N; ++j) L[j] = T(0);
    T gpx = T(0), gpy = T(0), gpz = T(0);
#pragma unroll
    for (int p = 1; p < 15; ++p) {
        const long long ip = s.at(cx(p), cy(p), cz(p));
        const T w = p < 7 ? P.ga : P.gc;
        const T psp = F.psi[ip];
        const T wp = w * psp;
        if (cx(p)) gpx += T(cx(p)) * wp;
        if (cy(p)) gpy += T(cy(p)) * wp;
        if (cz(p)) gpz += T(cz(p)) * wp;
        const T wpsi = w * (psi + psp);
        T sum = T(0);
#pragma unroll
        for (int j = 0; j < NP; ++j) {
            const T Cp = F.C[j * P.plane + ip];
            sum += Cp;
            L[j] += wpsi * (Cp - C[j]);
        }
        L[NP] += wpsi * ((T(1) - sum) - C[NP]);
    }
    T cN[N];
#pragma unroll
    for (int j = 0; j < NP; ++j) cN[j] = P.has_cos_field ? F.cosf[j * P.plane + i0] : P.cos_uni[j];
    cN[NP] = T(0);
    T m[N];
    mu_from_stencil<T, NP>(P, psi, C, L, gpx, gpy, gpz, cN, m);
#pragma unroll
    for (int i = 0; i < N; ++i) F.mu[i * P.plane + i0] = m[i];
}

// The same chemical potentials for four consecutive x nodes per thread
// (FP32, nx a multiple of 4; 8 x 4 x 2 threads cover 32 x 4 x 2 nodes):
// each stencil row of psi and C_j is one aligned float4 load, and the values
// one node to the left and right of the quad come from the neighbouring
// lanes by warp shuffle (scalar loads at the block's x edges and at the
// periodic seam).  Lanes beyond the box load clamped rows and store nothing.
template <int NP>
__global__ void __launch_bounds__(kThreads, NP <= 2 ? 3 : 2) k3_mu4(P3<float> P, F3<float> F) {
    constexpr int N = NP + 1;
    constexpr int NF = NP + 1;                 // fields: psi, C_1..C_{N-1}
    const int tx = threadIdx.x;
    const int x0 = 4 * (blockIdx.x * kBX4 + tx);
    const int y = blockIdx.y * kBY + threadIdx.y, z = blockIdx.z * kBZ + threadIdx.z;
    const bool live = x0 < P.nx && y < P.ny && z < P.nz;
    const int xa = x0 < P.nx ? x0 : P.nx - 4;
    const int ya = y < P.ny ? y : P.ny - 1, za = z < P.nz ? z : P.nz - 1;
    const int xm = xa == 0 ? P.nx - 1 : xa - 1;
    const int xp = xa + 4 == P.nx ? 0 : xa + 4;
    const float* fld[NF];
    fld[0] = F.psi;
#pragma unroll
    for (int j = 0; j < NP; ++j) fld[1 + j] = F.C + j * P.plane;
    auto rowbase = [&](int dy, int dz) {
        int yy = ya + dy, zz = za + dz;
        yy = yy < 0 ? yy + P.ny : (yy >= P.ny ? yy - P.ny : yy);
        zz = zz < 0 ? zz + P.nz : (zz >= P.nz ? zz - P.nz : zz);
        return (long long)zz * P.nxy + (long long)yy * P.nx;
    };
    // one row: v[f][0..3] at x0..x0+3, lf / rt[f] at x0 - 1 and x0 + 4
    float v[NF][4], lf[NF], rt[NF];
    auto load_row = [&](int dy, int dz, bool sides) {
        const long long b = rowbase(dy, dz);
#pragma unroll
        for (int f = 0; f < NF; ++f) {
            const float4 q = *reinterpret_cast<const float4*>(fld[f] + b + xa);
            v[f][0] = q.x; v[f][1] = q.y; v[f][2] = q.z; v[f][3] = q.w;
            if (sides) {
                const float l = __shfl_up_sync(0xffffffffu, q.w, 1);
                const float r = __shfl_down_sync(0xffffffffu, q.x, 1);
                lf[f] = tx > 0 ? l : fld[f][b + xm];
                rt[f] = (tx < kBX4 - 1 && xa + 4 < P.nx) ? r : fld[f][b + xp];
            }
        }
    };
    auto at = [&](int f, int k, int dx) {
        return dx == 0 ? v[f][k] : (dx < 0 ? (k == 0 ? lf[f] : v[f][k - 1]) : (k == 3 ? rt[f] : v[f][k + 1]));
    };
    float psi[4], C[N][4], L[N][4], g[3][4];
    load_row(0, 0, true);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        psi[k] = v[0][k];
        float sum = 0.f;
#pragma unroll
        for (int j = 0; j < NP; ++j) {
            C[j][k] = v[1 + j][k];
            sum += C[j][k];
        }
        C[NP][k] = 1.f - sum;
#pragma unroll
        for (int j = 0; j < N; ++j) L[j][k] = 0.f;
        g[0][k] = g[1][k] = g[2][k] = 0.f;
    }
    // neighbour (dx, dy, dz) of node k, stencil weight w, from the loaded row
    auto accumulate = [&](int dx, int dy, int dz, float w) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float psp = at(0, k, dx);
            const float wp = w * psp;
            if (dx) g[0][k] += float(dx) * wp;
            if (dy) g[1][k] += float(dy) * wp;
            if (dz) g[2][k] += float(dz) * wp;
            const float wpsi = w * (psi[k] + psp);
            float sum = 0.f;
#pragma unroll
            for (int j = 0; j < NP; ++j) {
                const float Cp = at(1 + j, k, dx);
                sum += Cp;
                L[j][k] += wpsi * (Cp - C[j][k]);
            }
            L[NP][k] += wpsi * ((1.f - sum) - C[NP][k]);
        }
    };
    accumulate(1, 0, 0, P.ga);
    accumulate(-1, 0, 0, P.ga);
#pragma unroll
    for (int a = 0; a < 4; ++a) {                 // the four axis rows: +-y, +-z
        const int dy = a < 2 ? (a == 0 ? 1 : -1) : 0, dz = a < 2 ? 0 : (a == 2 ? 1 : -1);
        load_row(dy, dz, false);
        accumulate(0, dy, dz, P.ga);
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) {                 // the four corner rows
        const int dy = (c & 1) ? -1 : 1, dz = (c & 2) ? -1 : 1;
        load_row(dy, dz, true);
        accumulate(1, dy, dz, P.gc);
        accumulate(-1, dy, dz, P.gc);
    }
    if (!live) return;
    const long long i0 = (long long)za * P.nxy + (long long)ya * P.nx + xa;
    float cN[NP][4];
#pragma unroll
    for (int j = 0; j < NP; ++j) {
        if (P.has_cos_field) {
            const float4 q = *reinterpret_cast<const float4*>(F.cosf + j * P.plane + i0);
            cN[j][0] = q.x; cN[j][1] = q.y; cN[j][2] = q.z; cN[j][3] = q.w;
        } else {
            cN[j][0] = cN[j][1] = cN[j][2] = cN[j][3] = P.cos_uni[j];
        }
    }
    float out[N][4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        float Ck[N], Lk[N], ck[N], m[N];
#pragma unroll
        for (int j = 0; j < N; ++j) {
            Ck[j] = C[j][k];
            Lk[j] = L[j][k];
            ck[j] = j < NP ? cN[j < NP ? j : 0][k] : 0.f;
        }
        mu_from_stencil<float, NP>(P, psi[k], Ck, Lk, g[0][k], g[1][k], g[2][k], ck, m);
#pragma unroll
        for (int i = 0; i < N; ++i) out[i][k] = m[i];
    }
#pragma unroll
    for (int i = 0; i < N; ++i)
        *reinterpret_cast<float4*>(F.mu + i * P.plane + i0) = make_float4(out[i][0], out[i][1], out[i][2], out[i][3]);
}

// ---------------------------------------------------------------------------
// node update (kMacro = false) or read-out of rho, u, P (kMacro = true)
// ---------------------------------------------------------------------------
// sum_p w_p c_p v(p) / cs2 on the 15-point stencil (p = 1..14), from the
// pairs of opposite neighbours: an axis pair gives its difference to its
// own component; the corner pairs (7, 14), (8, 13), (9, 12), (10, 11) give
// their differences d, signed by the first member's velocity.
template <typename T, class V>
__device__ __forceinline__ void grad15(const P3<T>& P, const V& v, T g[3]) {
    const T d0 = v(7) - v(14), d1 = v(8) - v(13), d2 = v(9) - v(12), d3 = v(10) - v(11);
    const T s01 = d0 + d1, s23 = d2 + d3;
    g[0] = P.ga * (v(1) - v(2)) + P.gc * ((d0 - d1) + (d2 - d3));
    g[1] = P.ga * (v(3) - v(4)) + P.gc * (s01 - s23);
    g[2] = P.ga * (v(5) - v(6)) + P.gc * (s01 + s23);
}

// Where the node update reads psi, C and mu: neighbour p of the velocity
// list (p = 0 the node itself) and the global index of that neighbour (the
// lagged field a is read there, populations are pushed there).
template <typename T>
struct GlobalSrc {     // the per-step C and mu planes in global memory
    Site s;
    const T* psi_;
    const T* C_;
    const T* mu_;
    const T* g_;       // flow populations and lagged planes of the input copy
    const T* lag_;
    long long plane;
    __device__ long long at(int p) const { return s.at(cx(p), cy(p), cz(p)); }
    __device__ T g(int p) const { return g_[p * plane + s.self()]; }
    __device__ T lag(int k) const { return lag_[k * plane + s.self()]; }
    __device__ T psi(int p) const { return psi_[at(p)]; }
    __device__ T C(int j, int p) const { return C_[j * plane + at(p)]; }
    __device__ T mu(int j, int p) const { return mu_[j * plane + at(p)]; }
};

template <typename T, int NP, bool kMacro, class S>
__device__ __forceinline__ void update_node(const P3<T>& P, const F3<T>& F, int cur, int field, double* out,
                                            const S& src) {
    constexpr int N = NP + 1;
    const long long i0 = src.at(0);
    const int nxt = cur ^ 1;
    const T psi = src.psi(0);
    const T cs2 = P.cs2;
    T C[N], mu[N];
    {
        T sum = T(0);
#pragma unroll
        for (int j = 0; j < NP; ++j) {
            C[j] = src.C(j, 0);
            sum += C[j];
        }
        C[NP] = T(1) - sum;
    }
#pragma unroll
    for (int j = 0; j < N; ++j) mu[j] = src.mu(j, 0);

    // gradients on the 15-point stencil: psi, C_j (j < N-1), mu_j, psi rho,
    // and the derivatives of a_xy, a_yz, a_zx the divergence needs.  FP64
    // (bound by its FP64 pipe) takes them field by field from the pairs of
    // opposite neighbours (grad15, fewer operations); FP32 (bound by the
    // fused kernel's registers) in one pass over the neighbours.
    const T* lagc = pick(F.lag, cur);
    T gps[3], gpr[3], gC[NP][3], gmu[N][3];
    T dxy_y, dxy_x, dyz_z, dyz_y, dzx_x, dzx_z;
    if constexpr (sizeof(T) == 8) {
        grad15(P, [&](int p) { return src.psi(p); }, gps);
#pragma unroll
        for (int j = 0; j < NP; ++j) grad15(P, [&](int p) { return src.C(j, p); }, gC[j]);
#pragma unroll
        for (int j = 0; j < N; ++j) grad15(P, [&](int p) { return src.mu(j, p); }, gmu[j]);
        grad15(P, [&](int p) {
            T rhop = T(0), sum = T(0);
#pragma unroll
            for (int j = 0; j < NP; ++j) {
                const T Cp = src.C(j, p);
                sum += Cp;
                rhop += P.rho[j] * Cp;
            }
            rhop += P.rho[NP] * (T(1) - sum);
            return src.psi(p) * rhop;
        }, gpr);
        T gaxy[3], gayz[3], gazx[3];
        grad15(P, [&](int p) { return lagc[lag_a(0) * P.plane + src.at(p)]; }, gaxy);
        grad15(P, [&](int p) { return lagc[lag_a(1) * P.plane + src.at(p)]; }, gayz);
        grad15(P, [&](int p) { return lagc[lag_a(2) * P.plane + src.at(p)]; }, gazx);
        dxy_x = gaxy[0];
        dxy_y = gaxy[1];
        dyz_y = gayz[1];
        dyz_z = gayz[2];
        dzx_z = gazx[2];
        dzx_x = gazx[0];
    } else {
        gps[0] = gps[1] = gps[2] = T(0);
        gpr[0] = gpr[1] = gpr[2] = T(0);
#pragma unroll
        for (int j = 0; j < NP; ++j) gC[j][0] = gC[j][1] = gC[j][2] = T(0);
#pragma unroll
        for (int j = 0; j < N; ++j) gmu[j][0] = gmu[j][1] = gmu[j][2] = T(0);
        dxy_y = dxy_x = dyz_z = dyz_y = dzx_x = dzx_z = T(0);
#pragma unroll
        for (int p = 1; p < 15; ++p) {
            const long long ip = src.at(p);
            const T w = p < 7 ? P.ga : P.gc;
            const T psp = src.psi(p);
            T rhop = T(0), sum = T(0);
#pragma unroll
            for (int j = 0; j < NP; ++j) {
                const T Cp = src.C(j, p);
                sum += Cp;
                rhop += P.rho[j] * Cp;
                const T wc = w * Cp;
#pragma unroll
                for (int a = 0; a < 3; ++a)
                    if (cc(p, a)) gC[j][a] += T(cc(p, a)) * wc;
            }
            rhop += P.rho[NP] * (T(1) - sum);
#pragma unroll
            for (int j = 0; j < N; ++j) {
                const T wm = w * src.mu(j, p);
#pragma unroll
                for (int a = 0; a < 3; ++a)
                    if (cc(p, a)) gmu[j][a] += T(cc(p, a)) * wm;
            }
            const T wp = w * psp, wpr = w * psp * rhop;
#pragma unroll
            for (int a = 0; a < 3; ++a)
                if (cc(p, a)) {
                    gps[a] += T(cc(p, a)) * wp;
                    gpr[a] += T(cc(p, a)) * wpr;
                }
            const T axy = w * lagc[lag_a(0) * P.plane + ip];
            const T ayz = w * lagc[lag_a(1) * P.plane + ip];
            const T azx = w * lagc[lag_a(2) * P.plane + ip];
            if (cx(p)) { dxy_x += T(cx(p)) * axy; dzx_x += T(cx(p)) * azx; }
            if (cy(p)) { dxy_y += T(cy(p)) * axy; dyz_y += T(cy(p)) * ayz; }
            if (cz(p)) { dyz_z += T(cz(p)) * ayz; dzx_z += T(cz(p)) * azx; }
        }
    }
    T grho[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        T gN = T(0), acc = T(0);
#pragma unroll
        for (int j = 0; j < NP; ++j) {
            gN -= gC[j][a];
            acc += P.rho[j] * gC[j][a];
        }
        grho[a] = acc + P.rho[NP] * gN;
    }

    T rho = T(0), nu = T(0);
#pragma unroll
    for (int j = 0; j < N; ++j) {
        rho += C[j] * P.rho[j];
        nu += C[j] * P.nu[j];
    }
    const T t21 = nu * P.nu_to_s21 + T(0.5);   // 1 / s21
    const T s21 = T(1) / t21;
    const T s22 = T(1) / (nu * P.inv_cs2_nu + T(0.5));

    // mobility (Eq. 2.5): M_ij = -m0 C_i C_j, M_ii = m0 C_i sum_{j != i} C_j;
    // m^C = -sum_ij rho_i M_ij grad mu_j
    T mC[3] = {T(0), T(0), T(0)};
#pragma unroll
    for (int i = 0; i < N; ++i)
#pragma unroll
        for (int j = 0; j < N; ++j) {
            T Mij;
            if (i == j) {
                T o = T(0);
#pragma unroll
                for (int q = 0; q < N; ++q)
                    if (q != i) o += C[q];
                Mij = P.m0 * C[i] * o;
            } else {
                Mij = -P.m0 * C[i] * C[j];
            }
#pragma unroll
            for (int a = 0; a < 3; ++a) mC[a] -= P.rho[i] * Mij * gmu[j][a];
        }

    // force without P grad psi and the damping: sum_i psi mu_i grad C_i,
    // -div A (A_jk = psi (m^C_j u_k - u_j m^C_k)/2, lagged), psi rho b
    T Fv[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        T acc = T(0), gN = T(0);
#pragma unroll
        for (int j = 0; j < NP; ++j) {
            acc += psi * mu[j] * gC[j][a];
            gN -= gC[j][a];
        }
        acc += psi * mu[NP] * gN;
        Fv[a] = acc;
    }
    Fv[0] += dxy_y - dzx_z;
    Fv[1] += dyz_z - dxy_x;
    Fv[2] += dzx_x - dyz_y;
#pragma unroll
    for (int a = 0; a < 3; ++a) Fv[a] += psi * rho * P.body[a];

    T g[15];
#pragma unroll
    for (int p = 0; p < 15; ++p) g[p] = src.g(p);
    T sum_g = T(0), J[3] = {T(0), T(0), T(0)};
#pragma unroll
    for (int p = 1; p < 15; ++p) {
        sum_g += g[p];
#pragma unroll
        for (int a = 0; a < 3; ++a)
            if (cc(p, a)) J[a] += T(cc(p, a)) * g[p];
    }
    const T damp = (T(1) - psi) * P.damp;
    const T den = psi * rho + T(0.5) * damp;
    const T Hc = P.Hfac * (s21 - T(2));
    const T inv_den = T(1) / den;
    T u0[3], e[3], bv[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        u0[a] = (J[a] + T(0.5) * Fv[a]) * inv_den;
        e[a] = T(0.5) * gps[a] * inv_den;
        bv[a] = P.A_P * psi * grho[a] + P.kk * psi * mC[a] + Hc * t21 * gpr[a];
    }
    const T gam = P.kk * psi * rho;
    const T G0 = sum_g - T(0.5) * P.K * src.lag(lag_pm<NP>());
    const T ee = e[0] * e[0] + e[1] * e[1] + e[2] * e[2];
    const T be = bv[0] * e[0] + bv[1] * e[1] + bv[2] * e[2];
    const T ue = u0[0] * e[0] + u0[1] * e[1] + u0[2] * e[2];
    const T bu = bv[0] * u0[0] + bv[1] * u0[1] + bv[2] * u0[2];
    const T uu = u0[0] * u0[0] + u0[1] * u0[1] + u0[2] * u0[2];
    const T qa = P.cP * gam * ee;
    const T qb = P.cP * (be + T(2) * gam * ue) - psi;
    const T qc = P.cP * (G0 + bu + gam * uu);
    const T disc = fmax(qb * qb - T(4) * qa * qc, T(0));
    const T root = sqrt(disc);
    const T Pp = T(-2) * qc / (qb < T(0) ? qb - root : qb + root);
    T u[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        u[a] = u0[a] + Pp * e[a];
        Fv[a] += Pp * gps[a] - damp * u[a];
    }
    if constexpr (kMacro) {
        double v = 0.0;
        if (field == DDCC_FIELD_RHO) v = (double)rho;
        else if (field == DDCC_FIELD_UX) v = (double)u[0];
        else if (field == DDCC_FIELD_UY) v = (double)u[1];
        else if (field == DDCC_FIELD_UZ) v = (double)u[2];
        else if (field == DDCC_FIELD_P) v = (double)Pp;
        out[i0] = v;
        return;
    } else {
        T* lagn = pick(F.lag, nxt);
        // ---- phase LB (Eqs. 3.1, 3.5-3.7), D3Q7 ----
        const T* fcur = pick(F.f, cur);
        T* fnew = pick(F.f, nxt);
#pragma unroll
        for (int i = 0; i < NP; ++i) {
            T f[7];
            T psiC = T(0);
#pragma unroll
            for (int p = 0; p < 7; ++p) {
                f[p] = fcur[(7 * i + p) * P.plane + i0];
                psiC += f[p];
            }
            // S_i = psi [(C_i sum_{j != i} C_j - 1) grad mu_i - sum_{j != i} C_i C_j grad mu_j]
            T V[3];
            T o = T(0);
#pragma unroll
            for (int q = 0; q < N; ++q)
                if (q != i) o += C[q];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                T S = (C[i] * o - T(1)) * gmu[i][a];
#pragma unroll
                for (int j = 0; j < N; ++j)
                    if (j != i) S -= C[i] * C[j] * gmu[j][a];
                S *= psi;
                const T cu = psiC * u[a];
                V[a] = (cu - src.lag(lag_cu(i, a)))
                       + cs2 * P.eta[i] * (mu[i] * gps[a] - S);
                lagn[lag_cu(i, a) * P.plane + i0] = cu;
            }
            const T epm = P.eta[i] * psi * mu[i];
            // Lambda v, v = f - f^eq + F/2, on the D3Q7 rows 1, c_a,
            // c_a^2 - cs2 (S = s0, s1, s21) from the moments of v: the zeroth
            // vanishes (sum f^eq = psi C = sum f, sum F = 0); the first is
            // j_a(f) - psi C u_a + V_a / 2; the raw second, sum_{+-a} v, is
            // e_a(f) - d0 eta psi mu (Eqs. 3.5, 3.6, B.5b, B.5c)
            T Es = T(0), wv[7];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const T fp = f[1 + 2 * a], fm = f[2 + 2 * a];
                const T Ja = P.s1f[i] * ((fp - fm) - psiC * u[a] + T(0.5) * V[a]);
                const T Ea = P.s21f * ((fp + fm) - cs2 * epm);
                wv[1 + 2 * a] = T(0.5) * (Ea + Ja);
                wv[2 + 2 * a] = T(0.5) * (Ea - Ja);
                Es += Ea;
            }
            wv[0] = -Es;
            // F_p = w_p c_p . V / cs2 (Eq. 3.6): zero at rest, +-w1 V_a / cs2.
            // The rest population's new value f_0 - wv_0 is rounded
            // explicitly and its exact rounding error (TwoSum) is split
            // evenly between the populations p = 1 and 2 (+x and -x), so
            // sum_p f keeps the exchange and no direction is preferred.
            const T o0 = add_rn(f[0], -wv[0]);
            const T bb = add_rn(o0, -f[0]);
            const T err = T(0.5) * add_rn(add_rn(f[0], -add_rn(o0, -bb)), add_rn(-wv[0], -bb));
            fnew[(7 * i) * P.plane + i0] = o0;
#pragma unroll
            for (int p = 1; p < 7; ++p) {
                const int a = (p - 1) >> 1;
                const T Fp = T(cc(p, a)) * P.w7_1 * V[a] * P.inv_cs2;
                T out = f[p] - wv[p] + Fp;
                if (p <= 2) out = add_rn(out, err);
                fnew[(7 * i + p) * P.plane + src.at(p)] = out;
            }
        }

        // ---- flow LB (Eqs. 3.2, 3.8, 3.10), D3Q15 ----
        T diag[3], off[3], Tn[6];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            diag[a] = psi * rho * u[a] * u[a] + psi * mC[a] * u[a];
            Tn[a] = psi * mC[a] * u[a];
        }
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const int a = k, b = (k + 1) % 3;
            off[k] = psi * rho * u[a] * u[b] + T(0.5) * (psi * mC[a] * u[b] + psi * u[a] * mC[b]);
            Tn[3 + k] = T(0.5) * (psi * mC[a] * u[b] + psi * u[a] * mC[b]);
        }
        const T ugpr = u[0] * gpr[0] + u[1] * gpr[1] + u[2] * gpr[2];
        T M2[6];
#pragma unroll
        for (int a = 0; a < 3; ++a)
            M2[a] = (Tn[a] - src.lag(lag_T<NP>(a))) + T(2) * cs2 * u[a] * gpr[a] + P.c2m3 * ugpr;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const int a = k, b = (k + 1) % 3;
            M2[3 + k] = (Tn[3 + k] - src.lag(lag_T<NP>(3 + k)))
                        + cs2 * (u[a] * gpr[b] + gpr[a] * u[b]);
        }
        const T a0 = psi * (u[0] * grho[0] + u[1] * grho[1] + u[2] * grho[2]);
        const T psiP = psi * Pp;
        // The collision runs in moment space on the orthogonal D3Q15 rows
        // h_k: with v = g - g^eq + G/2 and G = w (sum_k h_k <h_k, G> / |h_k|^2)
        // (G is w times a polynomial of degree <= 2),
        //   g* = g - Lambda v + G = g - w sum_k h_k mu_k,
        //   mu_k = (s_k / |h_k|^2) <h_k, v> - <h_k, G> / |h_k|^2.
        // <h_k, g^eq> (Eq. 3.8, g_0 stored as g_0 - rho0) = 0, psi rho u_a,
        // diag_a + psi P, off_k, 0 (third order), -2 cs2 psi P (the rest
        // population's -psi P / cs2 on the last row); <h_k, G> (Eq. 3.10) =
        // a0, F_a, M_aa, M_ab, 0 (Eqs. B.5d, B.5e).
        // Opposite velocities come in seven pairs (p, pb), c_pb = -c_p: an even
        // polynomial of c takes the pair's sum g_p + g_pb, an odd one its
        // difference, and the collided pair is g - w (E +- O) with E, O the
        // even and odd parts of sum_k h_k(c_p) m_k.
        T gs[7], gd[7];
#pragma unroll
        for (int q = 0; q < 7; ++q) {
            gs[q] = g[pair_rep(q)] + g[pair_opp(q)];
            gd[q] = g[pair_rep(q)] - g[pair_opp(q)];
        }
        T m[15];
        {
            T mm = g[0], j[3] = {T(0), T(0), T(0)}, e2[3] = {T(0), T(0), T(0)};
            T o2[3] = {T(0), T(0), T(0)}, t3[3] = {T(0), T(0), T(0)}, xyz = T(0), corner = T(0);
#pragma unroll
            for (int q = 0; q < 7; ++q) {
                const int p = pair_rep(q);
                mm += gs[q];
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    if (cc(p, a)) {
                        j[a] = cc(p, a) > 0 ? j[a] + gd[q] : j[a] - gd[q];
                        e2[a] += gs[q];
                    }
                }
                if (p >= 7) {
                    corner += gs[q];
                    xyz = cx(p) * cy(p) * cz(p) > 0 ? xyz + gd[q] : xyz - gd[q];
#pragma unroll
                    for (int k = 0; k < 3; ++k) {
                        o2[k] = cc(p, k) * cc(p, (k + 1) % 3) > 0 ? o2[k] + gs[q] : o2[k] - gs[q];
                        t3[k] = cc(p, k) > 0 ? t3[k] + gd[q] : t3[k] - gd[q];
                    }
                }
            }
            m[0] = P.lg0 * (mm + T(0.5) * a0) - a0;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                m[1 + a] = P.lg1 * (j[a] - psi * rho * u[a] + T(0.5) * Fv[a]) - Fv[a] * P.inv_cs2;
                m[4 + a] = P.inv_n2d * (s21 * ((e2[a] - cs2 * mm) - (diag[a] + psiP) + T(0.5) * M2[a]) - M2[a]);
                m[7 + a] = P.inv_n2o * (s22 * (o2[a] - off[a] + T(0.5) * M2[3 + a]) - M2[3 + a]);
                m[10 + a] = P.lg3 * (t3[a] - cs2 * j[a]);
            }
            m[13] = P.lg3c * xyz;
            m[14] = P.lg4 * (corner - cs2 * (e2[0] + e2[1] + e2[2]) + T(2) * cs2 * cs2 * mm + T(2) * cs2 * psiP);
        }
        T* gnew = pick(F.g, nxt);
        const T c4 = T(2) * cs2 * cs2;
        gnew[src.at(0)] = g[0] - P.w15[0] * (m[0] - cs2 * (m[4] + m[5] + m[6]) + c4 * m[14]);
#pragma unroll
        for (int q = 0; q < 7; ++q) {
            const int p = pair_rep(q), pb = pair_opp(q);
            const int x = cx(p), y = cy(p), z = cz(p);
            T E = m[0] + (T(x * x) - cs2) * m[4] + (T(y * y) - cs2) * m[5] + (T(z * z) - cs2) * m[6];
            if (x * y) E += T(x * y) * m[7];
            if (y * z) E += T(y * z) * m[8];
            if (z * x) E += T(z * x) * m[9];
            E += (T(x * x * y * y * z * z) - cs2 * T(x * x + y * y + z * z) + c4) * m[14];
            T O = T(0);
            if (x) O += T(x) * m[1];
            if (y) O += T(y) * m[2];
            if (z) O += T(z) * m[3];
            if (x) O += T(x) * (T(y * y) - cs2) * m[10];
            if (y) O += T(y) * (T(z * z) - cs2) * m[11];
            if (z) O += T(z) * (T(x * x) - cs2) * m[12];
            if (x * y * z) O += T(x * y * z) * m[13];
            const T wp = P.w15[p < 7 ? 1 : 2];
            gnew[p * P.plane + src.at(p)] = g[p] - wp * (E + O);
            gnew[pb * P.plane + src.at(pb)] = g[pb] - wp * (E - O);
        }
        // lagged: a (three components), T, psi m.u
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const int a = k, b = (k + 1) % 3;
            lagn[lag_a(k) * P.plane + i0] = T(0.5) * psi * (mC[a] * u[b] - u[a] * mC[b]);
        }
#pragma unroll
        for (int k = 0; k < 6; ++k) lagn[lag_T<NP>(k) * P.plane + i0] = Tn[k];
        lagn[lag_pm<NP>() * P.plane + i0] =
            psi * (rho * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]) + mC[0] * u[0] + mC[1] * u[1] + mC[2] * u[2]);
    }
}

template <typename T, int NP, bool kMacro>
__global__ void __launch_bounds__(kThreads, sizeof(T) == 4 ? 2 : 1) k3_update(P3<T> P, F3<T> F, int cur, int field,
                                                      double* out) {
    Site s;
    if (!site(P, s)) return;
    update_node<T, NP, kMacro>(P, F, cur, field, out,
                               GlobalSrc<T>{s, F.psi, F.C, F.mu, pick(F.g, cur), pick(F.lag, cur), P.plane});
}

// ---------------------------------------------------------------------------
// the fused step: one kernel per step, each CTA marching along z
// ---------------------------------------------------------------------------
// A CTA owns a column of 32 x TY nodes and the planes [zb, ze) of it.  The
// update of plane z reads C, psi and mu at planes z-1..z+1 on the column
// plus one node a side; mu at plane z+1 reads C and psi at planes z..z+2 on
// the column plus two nodes a side.  So for each output plane z the CTA
// forms C and psi at plane z+2 on the region x0-4 .. x0+35 (40 columns, so
// that rows are whole aligned quads) by y0-2 .. y0+TY+1, then mu at plane
// z+1 on the (32+2) x (TY+2) region, then updates plane z, with two
// barriers.  C and psi sit in a ring of five planes in shared memory and
// mu in a ring of three:
//   * the C pass for plane z+2 may overlap the slower threads' update of
//     plane z-1, which reads C at z-2..z: five slots keep them apart;
//   * the mu pass for plane z+1 starts after the barrier that follows the
//     C pass, when every thread has finished the update of plane z-1, so
//     the slot of mu at z-2 is free.
// With kVec (FP32, nx a multiple of 4, so that a periodic wrap maps aligned
// quads to aligned quads) the phase populations and psi of the C region
// arrive by 16-byte cp.async copies issued one plane ahead: the thread that
// forms C for a quad of 4 nodes copies that quad's 7(N-1) + 1 values and
// nothing else, so it waits for its own copies only and needs no barrier.
// The copies of plane z+3 fly during the mu pass and the update of plane z.
// With kStage (kVec and N <= 3, where the staging still leaves room for two
// CTAs per SM) each thread also copies its own node's 15 flow populations
// and 3N + 4 lagged values of plane z+1 (4-byte cp.async) as soon as its
// update of plane z has read those of plane z; they fly during the C pass,
// the mu pass and both barriers.  Copy groups are committed in the same
// order by every thread (empty groups where a thread has nothing to copy):
// raw(z+2), stage(z), raw(z+3), stage(z+1), ..., so "all but the newest
// group" is the data each wait needs.
// The per-step C and mu planes of global memory are neither read nor
// written; the update arithmetic is update_node's, the same as the
// three-kernel step's.
template <typename T, int NP, int TY, bool kVec, bool kStage = false>
struct FusedGeom {
    static constexpr int N = NP + 1;
    static constexpr int CW = kBX + 8, CH = TY + 4, CN = CW * CH;   // C, psi region
    static constexpr int MW = kBX + 2, MH = TY + 2, MN = MW * MH;   // mu region
    static constexpr int NT = kBX * TY;
    static constexpr int KC = (CN + NT - 1) / NT;                   // C-region nodes per thread
    static constexpr int KM = (MN + NT - 1) / NT;                   // mu-region nodes per thread
    static constexpr int NQ = CN / 4;                               // quads of the C region
    static constexpr int RAW = kVec ? (7 * NP + 1) * CN : 0;        // staged populations and psi
    static constexpr int NSTG = 15 + 3 * N + 4;                     // own-node g and lagged values
    static constexpr int STG = kStage ? NSTG * NT : 0;
    static constexpr size_t smem = sizeof(T) * (5 * (NP + 1) * CN + 3 * N * MN + RAW + STG);
    static_assert(!kVec || (sizeof(T) == 4 && NQ <= NT), "one quad per thread, FP32");
    static_assert(!kStage || kVec, "staging needs the cp.async path");
};

template <typename T, int NP, int TY, bool kVec, bool kStage>
struct SmemSrc {     // C, psi and mu from the shared-memory rings
    using G = FusedGeom<T, NP, TY, kVec, kStage>;
    const T* sC;     // C ring: slot k holds NP x CN values
    const T* sPs;    // psi ring: slot k holds CN values
    const T* sMu;    // mu ring: slot k holds N x MN values
    const T* stg;    // (kStage) own-node g (15) and lagged planes 3.. (NT apart)
    const T* g_;     // else the flow populations and lagged planes in global memory
    const T* lag_;
    long long plane;
    int c5[3], m3[3];  // ring slots of planes z-1, z, z+1
    int ci, mi;        // the node in the C and mu regions
    int tid;
    int xo[3], yo[3], zo[3];  // wrapped x, y nx, z nx ny of the node and its neighbours
    __device__ int at(int p) const { return zo[cz(p) + 1] + yo[cy(p) + 1] + xo[cx(p) + 1]; }
    __device__ T g(int p) const {
        if constexpr (kStage) return stg[p * G::NT + tid];
        else return g_[p * plane + at(0)];
    }
    __device__ T lag(int k) const {   // k >= 3: the own node's lagged planes past a
        if constexpr (kStage) return stg[(12 + k) * G::NT + tid];
        else return lag_[k * plane + at(0)];
    }
    __device__ T psi(int p) const { return sPs[c5[cz(p) + 1] * G::CN + ci + cy(p) * G::CW + cx(p)]; }
    __device__ T C(int j, int p) const {
        return sC[(c5[cz(p) + 1] * NP + j) * G::CN + ci + cy(p) * G::CW + cx(p)];
    }
    __device__ T mu(int j, int p) const {
        return sMu[(m3[cz(p) + 1] * G::N + j) * G::MN + mi + cy(p) * G::MW + cx(p)];
    }
};

__device__ __forceinline__ int wrap_index(int v, int n) {
    v %= n;
    return v < 0 ? v + n : v;
}

__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gmem_src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async4(void* smem_dst, const void* gmem_src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

template <typename T, int NP, int TY, bool kVec, bool kStage>
__global__ void __launch_bounds__(kBX * TY, (sizeof(T) == 4 && TY <= 8) ? 2 : 1)
    k3_fused(P3<T> P, F3<T> F, int cur, int nchunk) {
    using G = FusedGeom<T, NP, TY, kVec, kStage>;
    constexpr int N = NP + 1, CW = G::CW, CN = G::CN, MW = G::MW, MN = G::MN, NT = G::NT;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sC = reinterpret_cast<T*>(smem_raw);    // 5 slots x NP x CN
    T* sPs = sC + 5 * NP * CN;                  // 5 slots x CN
    T* sMu = sPs + 5 * CN;                      // 3 slots x N x MN
    T* sRaw = sMu + 3 * N * MN;                 // (kVec) 7 NP + 1 planes x CN
    T* sStg = sRaw + G::RAW;                    // (kStage) NSTG x NT
    const int tid = threadIdx.x;
    const int x0 = blockIdx.x * kBX, y0 = blockIdx.y * TY;
    const int zb = (int)((long long)blockIdx.z * P.nz / nchunk);
    const int ze = (int)((long long)(blockIdx.z + 1) * P.nz / nchunk);
    const T* fcur = pick(F.f, cur);
    // ring slots: C and psi of plane z >= zb - 2, mu of plane z >= zb - 1
    auto slot5 = [&](int z) { return (z - zb + 2) % 5; };
    auto slot3 = [&](int z) { return (z - zb + 1) % 3; };
    auto zoff = [&](int z) { return (long long)wrap_index(z, P.nz) * P.nxy; };

    // wrapped x and y nx of the C region's columns (x0-4+k) and rows (y0-2+k)
    __shared__ int xs[CW], ys[G::CH];
    for (int k = tid; k < CW; k += NT) xs[k] = wrap_index(x0 + k - 4, P.nx);
    for (int k = tid; k < G::CH; k += NT) ys[k] = wrap_index(y0 + k - 2, P.ny) * P.nx;
    __syncthreads();

    // (kVec) copy the populations and psi of this thread's quad at plane z
    auto issue = [&](int z, bool any) {
        if constexpr (kVec) {
            if (any && tid < G::NQ) {
                const int o = 4 * tid;   // quad tid: row o / CW, columns o % CW .. + 3
                const long long g = zoff(z) + ys[o / CW] + xs[o % CW];
#pragma unroll
                for (int q = 0; q < 7 * NP; ++q) cp_async16(sRaw + q * CN + o, fcur + q * P.plane + g);
                cp_async16(sRaw + 7 * NP * CN + o, F.psi + g);
            }
            cp_async_commit();
        }
    };
    // C_i = sum_p f^i_p / psi and psi at plane z on the C region (as k3_order)
    auto c_pass = [&](int z, bool steady) {
        T* c = sC + slot5(z) * NP * CN;
        T* ps = sPs + slot5(z) * CN;
        if constexpr (kVec) {
            if (tid < G::NQ) {
                const int o = 4 * tid;
                if (steady) cp_async_wait<1>();   // stage(z - 2) may still fly
                else cp_async_wait<0>();
                const float4 psi = *reinterpret_cast<const float4*>(sRaw + 7 * NP * CN + o);
                *reinterpret_cast<float4*>(ps + o) = psi;
#pragma unroll
                for (int j = 0; j < NP; ++j) {
                    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                    for (int p = 0; p < 7; ++p) {
                        const float4 v = *reinterpret_cast<const float4*>(sRaw + (7 * j + p) * CN + o);
                        acc.x += v.x;
                        acc.y += v.y;
                        acc.z += v.z;
                        acc.w += v.w;
                    }
                    *reinterpret_cast<float4*>(c + j * CN + o) =
                        make_float4(acc.x / psi.x, acc.y / psi.y, acc.z / psi.z, acc.w / psi.w);
                }
            }
        } else {
            const long long zo = zoff(z);
#pragma unroll
            for (int r = 0; r < G::KC; ++r) {
                const int k = tid + r * NT;
                if (k < CN) {
                    const long long i = zo + ys[k / CW] + xs[k % CW];
                    const T psi = F.psi[i];
                    ps[k] = psi;
#pragma unroll
                    for (int j = 0; j < NP; ++j) {
                        T acc = T(0);
#pragma unroll
                        for (int p = 0; p < 7; ++p) acc += fcur[(7 * j + p) * P.plane + i];
                        c[j * CN + k] = acc / psi;
                    }
                }
            }
        }
    };

    // mu at plane z on the mu region (as k3_mu, same summation order)
    auto mu_pass = [&](int z) {
        const T* cpl[3];
        const T* ppl[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            cpl[d] = sC + slot5(z - 1 + d) * NP * CN;
            ppl[d] = sPs + slot5(z - 1 + d) * CN;
        }
        T* m = sMu + slot3(z) * N * MN;
        const long long zo = zoff(z);
#pragma unroll
        for (int r = 0; r < G::KM; ++r) {
            const int k = tid + r * NT;
            if (k < MN) {
                const int c0 = (k / MW + 1) * CW + k % MW + 3;
                const T psi = ppl[1][c0];
                T C[N];
                {
                    T sum = T(0);
#pragma unroll
                    for (int j = 0; j < NP; ++j) {
                        C[j] = cpl[1][j * CN + c0];
                        sum += C[j];
                    }
                    C[NP] = T(1) - sum;
                }
                T L[N];
#pragma unroll
                for (int j = 0; j < N; ++j) L[j] = T(0);
                T gpx = T(0), gpy = T(0), gpz = T(0);
#pragma unroll
                for (int p = 1; p < 15; ++p) {
                    const int o = c0 + cy(p) * CW + cx(p);
                    const T w = p < 7 ? P.ga : P.gc;
                    const T psp = ppl[cz(p) + 1][o];
                    const T wp = w * psp;
                    if (cx(p)) gpx += T(cx(p)) * wp;
                    if (cy(p)) gpy += T(cy(p)) * wp;
                    if (cz(p)) gpz += T(cz(p)) * wp;
                    const T wpsi = w * (psi + psp);
                    T sum = T(0);
#pragma unroll
                    for (int j = 0; j < NP; ++j) {
                        const T Cp = cpl[cz(p) + 1][j * CN + o];
                        sum += Cp;
                        L[j] += wpsi * (Cp - C[j]);
                    }
                    L[NP] += wpsi * ((T(1) - sum) - C[NP]);
                }
                T cN[N];
#pragma unroll
                for (int j = 0; j < NP; ++j)
                    cN[j] = P.has_cos_field ? F.cosf[j * P.plane + zo + ys[k / MW + 1] + xs[k % MW + 3]]
                                            : P.cos_uni[j];
                cN[NP] = T(0);
                T mv[N];
                mu_from_stencil<T, NP>(P, psi, C, L, gpx, gpy, gpz, cN, mv);
#pragma unroll
                for (int i = 0; i < N; ++i) m[i * MN + k] = mv[i];
            }
        }
    };

    // this thread's node of the column
    const int tx = tid % kBX, ty = tid / kBX;
    const int x = x0 + tx, y = y0 + ty;
    const bool live = x < P.nx && y < P.ny;
    SmemSrc<T, NP, TY, kVec, kStage> src;
    src.sC = sC;
    src.sPs = sPs;
    src.sMu = sMu;
    src.stg = sStg;
    src.g_ = pick(F.g, cur);
    src.lag_ = pick(F.lag, cur);
    src.plane = P.plane;
    src.tid = tid;
    src.ci = (ty + 2) * CW + tx + 4;
    src.mi = (ty + 1) * MW + tx + 1;
    src.xo[0] = wrap_index(x - 1, P.nx);
    src.xo[1] = x;
    src.xo[2] = wrap_index(x + 1, P.nx);
    src.yo[0] = wrap_index(y - 1, P.ny) * P.nx;
    src.yo[1] = y * P.nx;
    src.yo[2] = wrap_index(y + 1, P.ny) * P.nx;
    const int nxy = (int)P.nxy;   // nx ny nz < 2^31
    // (kStage) copy this node's g and lagged values of plane z
    auto stage = [&](int z, bool any) {
        if constexpr (kStage) {
            if (any && live) {
                const int i = wrap_index(z, P.nz) * nxy + src.yo[1] + src.xo[1];
#pragma unroll
                for (int p = 0; p < 15; ++p) cp_async4(sStg + p * NT + tid, src.g_ + p * P.plane + i);
#pragma unroll
                for (int k = 3; k < n_lag(N); ++k) cp_async4(sStg + (12 + k) * NT + tid, src.lag_ + k * P.plane + i);
            }
        }
        if constexpr (kVec) cp_async_commit();
    };

    for (int z = zb - 2; z <= zb + 1; ++z) {
        issue(z, true);
        c_pass(z, false);
    }
    issue(zb + 2, true);
    stage(zb, true);
    __syncthreads();
    mu_pass(zb - 1);
    mu_pass(zb);
    for (int z = zb; z < ze; ++z) {
        c_pass(z + 2, true);
        issue(z + 3, z + 1 < ze);
        __syncthreads();
        mu_pass(z + 1);
        __syncthreads();
        if (live) {
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                src.zo[d] = wrap_index(z - 1 + d, P.nz) * nxy;
                src.c5[d] = slot5(z - 1 + d);
                src.m3[d] = slot3(z - 1 + d);
            }
            if constexpr (kStage) cp_async_wait<1>();   // raw(z + 3) may still fly
            update_node<T, NP, false>(P, F, cur, 0, nullptr, src);
        }
        stage(z + 1, z + 1 < ze);
    }
}

// ---------------------------------------------------------------------------
// initial state, staging, read-out, reduction
// ---------------------------------------------------------------------------
template <typename T, int NP>
__global__ void __launch_bounds__(kThreads) k3_init(P3<T> P, F3<T> F) {
    Site s;
    if (!site(P, s)) return;
    const long long i0 = s.self();
    const T psi = F.psi[i0];
    T* f = F.f[0];
#pragma unroll
    for (int i = 0; i < NP; ++i) {
        const T epm = P.eta[i] * psi * F.mu[i * P.plane + i0];
        const T psiC = psi * F.C[i * P.plane + i0];
        f[(7 * i) * P.plane + i0] = (P.w7_0 - T(1)) * epm + psiC;
#pragma unroll
        for (int p = 1; p < 7; ++p) f[(7 * i + p) * P.plane + i0] = P.w7_1 * epm;
    }
    // g = g^eq(P = 0, u = 0): zero with g_0 stored as g_0 - rho0
#pragma unroll
    for (int p = 0; p < 15; ++p) F.g[0][p * P.plane + i0] = T(0);
}

template <typename T>
__global__ void k3_from_double(const double* __restrict__ src, T* __restrict__ dst, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        dst[i] = (T)src[i];
}

template <typename T>
__global__ void k3_to_double(const T* __restrict__ src, double* __restrict__ dst, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        dst[i] = (double)src[i];
}

template <typename T, int NP>
__global__ void k3_derived_C(P3<T> P, F3<T> F, double* out) {
    const long long n = P.nxy * P.nz;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        T sum = T(0);
#pragma unroll
        for (int j = 0; j < NP; ++j) sum += F.C[j * P.plane + i];
        out[i] = (double)(T(1) - sum);
    }
}

template <typename T, int NP>
__global__ void __launch_bounds__(256) k3_mass_partial(P3<T> P, F3<T> F, int cur) {
    __shared__ double red[256][NP];
    const long long n = P.nxy * P.nz;
    const long long chunk = (n + kMassBlocks - 1) / kMassBlocks;
    const long long lo = blockIdx.x * chunk;
    const long long hi = lo + chunk < n ? lo + chunk : n;
    double acc[NP];
#pragma unroll
    for (int i = 0; i < NP; ++i) acc[i] = 0.0;
    const T* f = pick(F.f, cur);
    for (long long k = lo + threadIdx.x; k < hi; k += 256) {
#pragma unroll
        for (int i = 0; i < NP; ++i) {
            double s = 0.0;
#pragma unroll
            for (int p = 0; p < 7; ++p) s += (double)f[(7 * i + p) * P.plane + k];
            acc[i] += s;
        }
    }
#pragma unroll
    for (int i = 0; i < NP; ++i) red[threadIdx.x][i] = acc[i];
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
#pragma unroll
            for (int i = 0; i < NP; ++i) red[threadIdx.x][i] += red[threadIdx.x + w][i];
        __syncthreads();
    }
    if (threadIdx.x == 0)
#pragma unroll
        for (int i = 0; i < NP; ++i) F.partial[blockIdx.x * kMaxN + i] = red[0][i];
}

__global__ void k3_mass_final(const double* partial, int np, double* out, int* flag) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int bad = 0;
    for (int i = 0; i < np; ++i) {
        double s = 0.0;
        for (int b = 0; b < kMassBlocks; ++b) s += partial[b * kMaxN + i];
        out[i] = s;
        if (!isfinite(s)) bad = 1;
    }
    *flag = bad;
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
size_t round256(size_t b) { return (b + 255) & ~size_t(255); }

// Every value in (0, 1] (NaN fails).  Branch-free within blocks so that the
// compiler can vectorise the scan of a whole box.
bool all_in_unit(const double* v, long long n) {
    constexpr long long kB = 4096;
    for (long long i0 = 0; i0 < n; i0 += kB) {
        const long long i1 = i0 + kB < n ? i0 + kB : n;
        int bad = 0;
        for (long long i = i0; i < i1; ++i) bad |= (int)!(v[i] > 0.0) | (int)!(v[i] <= 1.0);
        if (bad) return false;
    }
    return true;
}

bool valid(const ddcc3d_params* p) {
    if (!p) return false;
    if (p->nx < 3 || p->ny < 3 || p->nz < 3) return false;
    if ((long long)p->nx * p->ny * p->nz > (1LL << 31) - 1) return false;
    // launch grid (nx/32, ny/4, nz/2): y and z block counts are limited to 65535
    if ((long long)p->ny > 65535LL * kBY || (long long)p->nz > 65535LL * kBZ) return false;
    if (p->nphase < 2 || p->nphase > kMaxN) return false;
    if (p->precision != DDCC_FP64 && p->precision != DDCC_FP32) return false;
    if (p->reserved != 0 || (p->flags & ~(uint32_t)(DDCC3D_FLAG_SPLIT | DDCC3D_FLAG_FUSED)) != 0) return false;
    if ((p->flags & DDCC3D_FLAG_SPLIT) && (p->flags & DDCC3D_FLAG_FUSED)) return false;
    if (!(p->d0 > 0.0 && p->d0 < 0.5)) return false;     // D3Q15 rest weight (1-d0)(1-2d0) > 0
    if (!(p->width > 0.0) || !(p->eps0 > 0.0) || !(p->m0 > 0.0)) return false;
    const int N = p->nphase;
    for (int i = 0; i < N; ++i) {
        if (!(p->rho[i] > 0.0) || !(p->nu[i] > 0.0)) return false;
        for (int j = 0; j < N; ++j) {
            if (p->sigma[i][j] != p->sigma[j][i]) return false;
            if (i == j ? p->sigma[i][j] != 0.0 : !(p->sigma[i][j] > 0.0)) return false;
        }
    }
    for (int i = 0; i < N - 1; ++i)
        if (!(p->eta[i] > 0.0)) return false;
    for (double s : p->s_f)
        if (!(s > 0.0 && s < 2.0)) return false;
    for (double s : p->s_g)
        if (!(s > 0.0 && s < 2.0)) return false;
    return true;
}

struct Layout {
    size_t plane_bytes, planes, stage, partial, flag, total;
};

Layout layout(const ddcc3d_params* p) {
    Layout L{};
    const size_t e = p->precision == DDCC_FP64 ? 8 : 4;
    const size_t n = (size_t)p->nx * p->ny * p->nz;
    const int N = p->nphase;
    L.plane_bytes = round256(n * e);
    L.planes = 2 * (7 * (N - 1) + 15) + 2 * n_lag(N) + 1 + (N - 1) + (N - 1) + N;
    L.stage = round256(n * 8);
    L.partial = round256((kMassBlocks + 1) * kMaxN * 8);   // + the N-1 totals
    L.flag = 256;
    L.total = L.planes * L.plane_bytes + L.stage + L.partial + L.flag;
    return L;
}

template <typename T>
void make_params(const ddcc3d_params* p, P3<T>& K) {
    std::memset(&K, 0, sizeof(K));
    const double d0 = p->d0, cs2 = d0;
    K.nx = p->nx;
    K.ny = p->ny;
    K.nz = p->nz;
    K.N = p->nphase;
    K.nxy = (long long)p->nx * p->ny;
    const size_t e = sizeof(T);
    K.plane = (long long)(round256((size_t)K.nxy * p->nz * e) / e);
    K.cs2 = (T)cs2;
    K.inv_cs2 = (T)(1.0 / cs2);
    const double wa = (d0 - d0 * d0) / 2.0, wc = d0 * d0 / 8.0, w0 = 1.0 - 3.0 * d0 + 2.0 * d0 * d0;
    K.ga = (T)(wa / cs2);
    K.gc = (T)(wc / cs2);
    K.w7_0 = (T)(1.0 - 3.0 * d0);
    K.w7_1 = (T)(d0 / 2.0);
    K.w15[0] = (T)w0;
    K.w15[1] = (T)wa;
    K.w15[2] = (T)wc;
    const int N = p->nphase;
    for (int i = 0; i < N; ++i) {
        K.rho[i] = (T)p->rho[i];
        K.nu[i] = (T)p->nu[i];
        K.sigN[i] = (T)p->sigma[i][N - 1];
        for (int j = 0; j < N; ++j) {
            const double s = p->sigma[i][j];
            K.beta2[i][j] = (T)(6.0 * s / p->width);
            K.kap[i][j] = (T)(0.75 * p->width * s);
            K.wet[i][j] = (T)(3.0 * s);
            K.invsig[i][j] = (T)(i == j ? 0.0 : 1.0 / s);
        }
    }
    for (int i = 0; i < N - 1; ++i) {
        K.eta[i] = (T)p->eta[i];
        // Eq. 17: m0 = (1/s1 - 1/2) eta_i cs2
        K.s1f[i] = (T)(1.0 / (p->m0 / (p->eta[i] * cs2) + 0.5));
    }
    K.m0 = (T)p->m0;
    K.inv_m0 = (T)(1.0 / p->m0);
    K.s0f = (T)p->s_f[0];
    K.s21f = (T)p->s_f[1];
    // D3Q15 row norms under the weights: 1, d0, d0(1-d0), d0^2,
    // d0^2(1-d0), d0^2 (cx cy cz), d0^2 w0 (last row)
    const double n2d = d0 * (1.0 - d0), n2o = d0 * d0, n3 = d0 * d0 * (1.0 - d0), n4 = d0 * d0 * w0;
    K.lg0 = (T)p->s_g[0];
    K.lg1 = (T)(p->s_g[1] / d0);
    K.lg3 = (T)(p->s_g[2] / n3);
    K.lg3c = (T)(p->s_g[2] / (d0 * d0));
    K.lg4 = (T)(p->s_g[3] / n4);
    K.inv_n2d = (T)(1.0 / n2d);
    K.inv_n2o = (T)(1.0 / n2o);
    // Eq. 16: nu = (1/s21 - 1/2)(1 - cs2)/2 = (1/s22 - 1/2) cs2
    K.nu_to_s21 = (T)(2.0 / (1.0 - cs2));
    K.inv_cs2_nu = (T)(1.0 / cs2);
    K.damp = (T)(1.0 / (p->eps0 * p->eps0 * p->eps0));
    // Eq. 19 with the 3D constants K = 1 - 2 d0, H = K (3 - 7 d0)(s21 - 2)/2
    const double Kc = 1.0 - 2.0 * d0;
    K.K = (T)Kc;
    K.Hfac = (T)(Kc * (3.0 - 7.0 * d0) / 2.0);
    const double sg0 = p->s_g[0];
    K.A_P = (T)(0.5 + Kc * (1.0 - d0) * (2.0 - sg0) / (2.0 * sg0));
    K.cP = (T)(cs2 / (1.0 - w0));
    K.kk = (T)(Kc / 2.0 - w0 / (1.0 - cs2));
    K.c2m3 = (T)(1.0 - 3.0 * cs2);
    K.diag_den = (T)(1.0 / (cs2 * (1.0 - cs2)));
    K.off_den = (T)(1.0 / (cs2 * cs2));
    for (int a = 0; a < 3; ++a) K.body[a] = (T)p->body_force[a];
}

template <typename T>
void carve(const ddcc3d_params* p, char* ws, F3<T>& F) {
    const Layout L = layout(p);
    const int N = p->nphase;
    char* c = ws;
    auto take = [&](size_t planes) { T* r = (T*)c; c += planes * L.plane_bytes; return r; };
    for (int b = 0; b < 2; ++b) F.f[b] = take(7 * (N - 1));
    for (int b = 0; b < 2; ++b) F.g[b] = take(15);
    for (int b = 0; b < 2; ++b) F.lag[b] = take(n_lag(N));
    F.psi = take(1);
    F.cosf = take(N - 1);
    F.C = take(N - 1);
    F.mu = take(N);
    F.stage = (double*)c;
    c += L.stage;
    F.partial = (double*)c;
    c += L.partial;
    F.flag = (int*)c;
}

}  // namespace

struct ddcc3d_handle {
    ddcc3d_params prm;
    cudaStream_t stream;
    char* ws;
    int cur;
    int64_t steps;
    int has_cos_field;
    P3<double> kd;
    P3<float> kf;
    F3<double> fd;
    F3<float> ff;
    double* dev_mass;
    int fused;        // one k3_fused launch per step (else the three kernels)
    int cmu_valid;    // F.C and F.mu hold the current state's C and mu (cleared by a step)
    int nchunk;       // z chunks of the fused step's grid
    int profiling;
    std::vector<cudaEvent_t> events;
    std::vector<int> rec_kind;
};

namespace {

int prof_begin(ddcc3d_handle* h, int kind) {
    if (!h->profiling) return DDCC_OK;
    const size_t i = h->rec_kind.size();
    while (h->events.size() < 2 * (i + 1)) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return DDCC_ERR_CUDA;
        h->events.push_back(e);
    }
    h->rec_kind.push_back(kind);
    return cudaEventRecord(h->events[2 * i], h->stream) == cudaSuccess ? DDCC_OK : DDCC_ERR_CUDA;
}

int prof_end(ddcc3d_handle* h) {
    if (!h->profiling) return DDCC_OK;
    const size_t i = h->rec_kind.size() - 1;
    return cudaEventRecord(h->events[2 * i + 1], h->stream) == cudaSuccess ? DDCC_OK : DDCC_ERR_CUDA;
}

dim3 grid3(const ddcc3d_params& p) {
    return dim3((p.nx + kBX - 1) / kBX, (p.ny + kBY - 1) / kBY, (p.nz + kBZ - 1) / kBZ);
}

int launched() { return cudaGetLastError() == cudaSuccess ? DDCC_OK : DDCC_ERR_CUDA; }

template <typename T, int NP>
int order_mu(ddcc3d_handle* h, const P3<T>& K, const F3<T>& F, bool order) {
    const dim3 grid = grid3(h->prm), block(kBX, kBY, kBZ);
    int rc;
    if (order) {
        if ((rc = prof_begin(h, 0))) return rc;
        k3_order<T, NP><<<grid, block, 0, h->stream>>>(K, F, h->cur);
        if ((rc = launched()) || (rc = prof_end(h))) return rc;
    }
    if ((rc = prof_begin(h, 1))) return rc;
    if constexpr (sizeof(T) == 4) {
        if (K.nx % 4 == 0) {
            const dim3 grid4((K.nx / 4 + kBX4 - 1) / kBX4, grid.y, grid.z), block4(kBX4, kBY, kBZ);
            k3_mu4<NP><<<grid4, block4, 0, h->stream>>>(K, F);
        } else {
            k3_mu<T, NP><<<grid, block, 0, h->stream>>>(K, F);
        }
    } else {
        k3_mu<T, NP><<<grid, block, 0, h->stream>>>(K, F);
    }
    if ((rc = launched()) || (rc = prof_end(h))) return rc;
    return DDCC_OK;
}

// Shared memory of the fused step and its z chunks: the count of chunks n
// minimises (waves of CTAs) x (planes a CTA forms C for), i.e.
// ceil(columns n / resident CTAs) x (ceil(nz / n) + 3).
template <int NP, bool kVec>
constexpr bool fused_stage() { return kVec && NP <= 2; }

template <typename T, int NP, bool kVec>
int fused_setup_v(ddcc3d_handle* h) {
    constexpr bool kS = fused_stage<NP, kVec>();
    using G = FusedGeom<T, NP, kFusedTY, kVec, kS>;
    if (cudaFuncSetAttribute(k3_fused<T, NP, kFusedTY, kVec, kS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)G::smem) != cudaSuccess)
        return DDCC_ERR_CUDA;
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k3_fused<T, NP, kFusedTY, kVec, kS>, G::NT, G::smem) !=
            cudaSuccess)
        return DDCC_ERR_CUDA;
    if (per_sm < 1) return DDCC_ERR_CUDA;
    const long long cols = (long long)((h->prm.nx + kBX - 1) / kBX) * ((h->prm.ny + kFusedTY - 1) / kFusedTY);
    const long long resident = (long long)sms * per_sm;
    const int nz = h->prm.nz;
    long long best = -1;
    for (int n = 1; n <= nz && n <= 65535; ++n) {
        const long long cost = ((cols * n + resident - 1) / resident) * ((nz + n - 1) / n + 3);
        if (best < 0 || cost < best) {
            best = cost;
            h->nchunk = n;
        }
    }
    return DDCC_OK;
}

// The staged (cp.async) C pass runs in FP32 when nx is a multiple of 4.
template <typename T>
bool fused_vec(const ddcc3d_handle* h) { return sizeof(T) == 4 && h->prm.nx % 4 == 0; }

template <typename T, int NP>
int fused_setup(ddcc3d_handle* h) {
    if constexpr (sizeof(T) == 4) {
        if (fused_vec<T>(h)) return fused_setup_v<T, NP, true>(h);
    }
    return fused_setup_v<T, NP, false>(h);
}

template <typename T, int NP, bool kVec>
int fused_launch(ddcc3d_handle* h, const P3<T>& K, const F3<T>& F) {
    constexpr bool kS = fused_stage<NP, kVec>();
    using G = FusedGeom<T, NP, kFusedTY, kVec, kS>;
    const dim3 gf((h->prm.nx + kBX - 1) / kBX, (h->prm.ny + kFusedTY - 1) / kFusedTY, h->nchunk);
    k3_fused<T, NP, kFusedTY, kVec, kS><<<gf, G::NT, G::smem, h->stream>>>(K, F, h->cur, h->nchunk);
    return launched();
}

template <typename T, int NP>
int step_n(ddcc3d_handle* h, const P3<T>& K, const F3<T>& F, int64_t n) {
    const dim3 grid = grid3(h->prm), block(kBX, kBY, kBZ);
    if (h->fused) {
        for (int64_t s = 0; s < n; ++s) {
            int rc;
            if ((rc = prof_begin(h, 3))) return rc;
            if constexpr (sizeof(T) == 4) {
                rc = fused_vec<T>(h) ? fused_launch<T, NP, true>(h, K, F) : fused_launch<T, NP, false>(h, K, F);
            } else {
                rc = fused_launch<T, NP, false>(h, K, F);
            }
            if (rc || (rc = prof_end(h))) return rc;
            h->cur ^= 1;
            ++h->steps;
        }
        return DDCC_OK;
    }
    for (int64_t s = 0; s < n; ++s) {
        int rc = order_mu<T, NP>(h, K, F, true);
        if (rc) return rc;
        if ((rc = prof_begin(h, 2))) return rc;
        k3_update<T, NP, false><<<grid, block, 0, h->stream>>>(K, F, h->cur, 0, nullptr);
        if ((rc = launched()) || (rc = prof_end(h))) return rc;
        h->cur ^= 1;
        ++h->steps;
    }
    return DDCC_OK;
}

template <typename T, int NP>
int init_n(ddcc3d_handle* h, const P3<T>& K, const F3<T>& F) {
    const dim3 grid = grid3(h->prm), block(kBX, kBY, kBZ);
    int rc = order_mu<T, NP>(h, K, F, false);
    if (rc) return rc;
    k3_init<T, NP><<<grid, block, 0, h->stream>>>(K, F);
    return launched();
}

template <typename T, int NP>
int read_n(ddcc3d_handle* h, const P3<T>& K, const F3<T>& F, int field, double* host_out) {
    const dim3 grid = grid3(h->prm), block(kBX, kBY, kBZ);
    const int N = NP + 1;
    const long long n = K.nxy * K.nz;
    int rc;
    if (!h->cmu_valid) {
        if ((rc = order_mu<T, NP>(h, K, F, true))) return rc;
        h->cmu_valid = 1;
    }
    const int cb = 2 * 152 * 4, ct = 256;
    if (field >= DDCC_FIELD_C && field < DDCC_FIELD_C + N) {
        const int i = field - DDCC_FIELD_C;
        if (i < NP) k3_to_double<T><<<cb, ct, 0, h->stream>>>(F.C + i * K.plane, F.stage, n);
        else k3_derived_C<T, NP><<<cb, ct, 0, h->stream>>>(K, F, F.stage);
    } else if (field >= DDCC_FIELD_MU && field < DDCC_FIELD_MU + N) {
        k3_to_double<T><<<cb, ct, 0, h->stream>>>(F.mu + (field - DDCC_FIELD_MU) * K.plane, F.stage, n);
    } else if (field == DDCC_FIELD_PSI) {
        k3_to_double<T><<<cb, ct, 0, h->stream>>>(F.psi, F.stage, n);
    } else if (field == DDCC_FIELD_RHO || field == DDCC_FIELD_UX || field == DDCC_FIELD_UY ||
               field == DDCC_FIELD_UZ || field == DDCC_FIELD_P) {
        k3_update<T, NP, true><<<grid, block, 0, h->stream>>>(K, F, h->cur, field, F.stage);
    } else {
        return DDCC_ERR_PARAM;
    }
    if ((rc = launched())) return rc;
    if (cudaMemcpyAsync(host_out, F.stage, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream) != cudaSuccess)
        return DDCC_ERR_CUDA;
    return cudaStreamSynchronize(h->stream) == cudaSuccess ? DDCC_OK : DDCC_ERR_CUDA;
}

template <typename T, int NP>
int mass_n(ddcc3d_handle* h, const P3<T>& K, const F3<T>& F, double* host_out) {
    k3_mass_partial<T, NP><<<kMassBlocks, 256, 0, h->stream>>>(K, F, h->cur);
    k3_mass_final<<<1, 32, 0, h->stream>>>(F.partial, NP, h->dev_mass, F.flag);
    if (launched()) return DDCC_ERR_CUDA;
    double out[kMaxN + 1];
    int flag = 0;
    if (cudaMemcpyAsync(out, h->dev_mass, NP * sizeof(double), cudaMemcpyDeviceToHost, h->stream) != cudaSuccess ||
        cudaMemcpyAsync(&flag, F.flag, sizeof(int), cudaMemcpyDeviceToHost, h->stream) != cudaSuccess ||
        cudaStreamSynchronize(h->stream) != cudaSuccess)
        return DDCC_ERR_CUDA;
    std::memcpy(host_out, out, NP * sizeof(double));
    return flag ? DDCC_ERR_NONFINITE : DDCC_OK;
}

// Host double array -> device plane of T through the double staging plane.
template <typename T>
int upload_plane(ddcc3d_handle* h, double* stage, const double* src, T* dst, long long n) {
    if (cudaMemcpyAsync(stage, src, n * sizeof(double), cudaMemcpyHostToDevice, h->stream) != cudaSuccess)
        return DDCC_ERR_CUDA;
    k3_from_double<T><<<2 * 152 * 4, 256, 0, h->stream>>>(stage, dst, n);
    if (launched()) return DDCC_ERR_CUDA;
    // the staging plane is reused by the next upload: order the copies
    return cudaStreamSynchronize(h->stream) == cudaSuccess ? DDCC_OK : DDCC_ERR_CUDA;
}

template <typename T>
int create_t(ddcc3d_handle* h, const P3<T>& K, const F3<T>& F, const double* psi, const double* cosf,
             const double* C0) {
    const long long n = K.nxy * K.nz;
    const int N = h->prm.nphase;
    int rc = upload_plane<T>(h, F.stage, psi, F.psi, n);
    if (rc) return rc;
    if (cosf)
        for (int i = 0; i < N - 1; ++i)
            if ((rc = upload_plane<T>(h, F.stage, cosf + i * n, F.cosf + i * K.plane, n))) return rc;
    for (int i = 0; i < N - 1; ++i)
        if ((rc = upload_plane<T>(h, F.stage, C0 + i * n, F.C + i * K.plane, n))) return rc;
    const Layout L = layout(&h->prm);
    for (int b = 0; b < 2; ++b)
        if (cudaMemsetAsync(F.lag[b], 0, n_lag(N) * L.plane_bytes, h->stream) != cudaSuccess) return DDCC_ERR_CUDA;
    switch (N - 1) {
        case 1: rc = init_n<T, 1>(h, K, F); break;
        case 2: rc = init_n<T, 2>(h, K, F); break;
        default: rc = init_n<T, 3>(h, K, F); break;
    }
    if (rc) return rc;
    if (h->fused) {
        switch (N - 1) {
            case 1: rc = fused_setup<T, 1>(h); break;
            case 2: rc = fused_setup<T, 2>(h); break;
            default: rc = fused_setup<T, 3>(h); break;
        }
        if (rc) return rc;
    }
    return cudaStreamSynchronize(h->stream) == cudaSuccess ? DDCC_OK : DDCC_ERR_CUDA;
}

}  // namespace

extern "C" {

size_t ddcc3d_workspace_bytes(const ddcc3d_params* params) {
    if (!valid(params)) return 0;
    return layout(params).total;
}

int ddcc3d_create(const ddcc3d_params* params, void* dev_workspace, size_t bytes, void* cuda_stream,
                  const double* psi, const double* cos_theta_field, const double* cos_theta_uniform,
                  const double* C0, ddcc3d_handle** out) {
    if (!out) return DDCC_ERR_PARAM;
    *out = nullptr;
    if (!valid(params) || !psi || !C0 || (!cos_theta_field && !cos_theta_uniform)) return DDCC_ERR_PARAM;
    const long long n = (long long)params->nx * params->ny * params->nz;
    if (!all_in_unit(psi, n)) return DDCC_ERR_PARAM;
    if (!dev_workspace || ((uintptr_t)dev_workspace & 255) || bytes < layout(params).total) return DDCC_ERR_WORKSPACE;
    ddcc3d_handle* h = new (std::nothrow) ddcc3d_handle();
    if (!h) return DDCC_ERR_NOMEM;
    h->prm = *params;
    h->stream = (cudaStream_t)cuda_stream;
    h->ws = (char*)dev_workspace;
    h->cur = 0;
    h->steps = 0;
    h->has_cos_field = cos_theta_field != nullptr;
    h->profiling = 0;
    // FP32 steps fused by default; FP64 with the three kernels (its fused
    // kernel recomputes mu on the column halos and is bound by the FP64 pipe)
    h->fused = (params->flags & DDCC3D_FLAG_FUSED) ||
               (!(params->flags & DDCC3D_FLAG_SPLIT) && params->precision == DDCC_FP32);
    h->nchunk = 1;
    int rc;
    if (params->precision == DDCC_FP64) {
        make_params(params, h->kd);
        carve(params, h->ws, h->fd);
        h->kd.has_cos_field = h->has_cos_field;
        if (!h->has_cos_field)
            for (int i = 0; i < params->nphase - 1; ++i) h->kd.cos_uni[i] = cos_theta_uniform[i];
        h->dev_mass = h->fd.partial + kMassBlocks * kMaxN;
        rc = create_t<double>(h, h->kd, h->fd, psi, cos_theta_field, C0);
    } else {
        make_params(params, h->kf);
        carve(params, h->ws, h->ff);
        h->kf.has_cos_field = h->has_cos_field;
        if (!h->has_cos_field)
            for (int i = 0; i < params->nphase - 1; ++i) h->kf.cos_uni[i] = (float)cos_theta_uniform[i];
        h->dev_mass = h->ff.partial + kMassBlocks * kMaxN;
        rc = create_t<float>(h, h->kf, h->ff, psi, cos_theta_field, C0);
    }
    if (rc) {
        delete h;
        return rc;
    }
    *out = h;
    return DDCC_OK;
}

int ddcc3d_step(ddcc3d_handle* h, int64_t nsteps) {
    if (!h || nsteps < 0) return DDCC_ERR_PARAM;
    h->cmu_valid = 0;
    const int np = h->prm.nphase - 1;
    if (h->prm.precision == DDCC_FP64) {
        if (np == 1) return step_n<double, 1>(h, h->kd, h->fd, nsteps);
        if (np == 2) return step_n<double, 2>(h, h->kd, h->fd, nsteps);
        return step_n<double, 3>(h, h->kd, h->fd, nsteps);
    }
    if (np == 1) return step_n<float, 1>(h, h->kf, h->ff, nsteps);
    if (np == 2) return step_n<float, 2>(h, h->kf, h->ff, nsteps);
    return step_n<float, 3>(h, h->kf, h->ff, nsteps);
}

int ddcc3d_read(ddcc3d_handle* h, int field, double* host_out) {
    if (!h || !host_out) return DDCC_ERR_PARAM;
    const int np = h->prm.nphase - 1;
    if (h->prm.precision == DDCC_FP64) {
        if (np == 1) return read_n<double, 1>(h, h->kd, h->fd, field, host_out);
        if (np == 2) return read_n<double, 2>(h, h->kd, h->fd, field, host_out);
        return read_n<double, 3>(h, h->kd, h->fd, field, host_out);
    }
    if (np == 1) return read_n<float, 1>(h, h->kf, h->ff, field, host_out);
    if (np == 2) return read_n<float, 2>(h, h->kf, h->ff, field, host_out);
    return read_n<float, 3>(h, h->kf, h->ff, field, host_out);
}

int ddcc3d_mass(ddcc3d_handle* h, double* host_out) {
    if (!h || !host_out) return DDCC_ERR_PARAM;
    const int np = h->prm.nphase - 1;
    if (h->prm.precision == DDCC_FP64) {
        if (np == 1) return mass_n<double, 1>(h, h->kd, h->fd, host_out);
        if (np == 2) return mass_n<double, 2>(h, h->kd, h->fd, host_out);
        return mass_n<double, 3>(h, h->kd, h->fd, host_out);
    }
    if (np == 1) return mass_n<float, 1>(h, h->kf, h->ff, host_out);
    if (np == 2) return mass_n<float, 2>(h, h->kf, h->ff, host_out);
    return mass_n<float, 3>(h, h->kf, h->ff, host_out);
}

int64_t ddcc3d_step_count(const ddcc3d_handle* h) { return h ? h->steps : -1; }

int ddcc3d_profile(ddcc3d_handle* h, int enable) {
    if (!h) return DDCC_ERR_PARAM;
    h->profiling = enable != 0;
    return DDCC_OK;
}

int ddcc3d_kernel_times(ddcc3d_handle* h, double* ms_out, int64_t* launches_out, int max_kinds) {
    if (!h || max_kinds < 0) return DDCC_ERR_PARAM;
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return DDCC_ERR_CUDA;
    double ms[kKinds] = {0.0, 0.0, 0.0, 0.0};
    int64_t cnt[kKinds] = {0, 0, 0, 0};
    for (size_t i = 0; i < h->rec_kind.size(); ++i) {
        float t = 0.f;
        if (cudaEventElapsedTime(&t, h->events[2 * i], h->events[2 * i + 1]) != cudaSuccess) return DDCC_ERR_CUDA;
        ms[h->rec_kind[i]] += t;
        ++cnt[h->rec_kind[i]];
    }
    h->rec_kind.clear();
    for (int k = 0; k < kKinds && k < max_kinds; ++k) {
        if (ms_out) ms_out[k] = ms[k];
        if (launches_out) launches_out[k] = cnt[k];
    }
    return kKinds;
}

void ddcc3d_destroy(ddcc3d_handle* h) {
    if (!h) return;
    cudaStreamSynchronize(h->stream);
    for (cudaEvent_t e : h->events) cudaEventDestroy(e);
    delete h;
}

}  // extern "C"
