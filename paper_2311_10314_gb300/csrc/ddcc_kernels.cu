// Tile kernels of the DD-CCLB step (arXiv 2311.10314, Sec. 3) and the
// small utility kernels (initial state, read-out, reductions, uploads).
//
// Tile step (two launches):
//   k_order_param  psi C_i = sum_p f^i_p, C_i = psi C_i / psi -> C scratch;
//   k_step         per 32 x 8 tile: C and psi with a 2-node halo and the
//                  lagged field a with a 1-node halo are staged in shared
//                  memory, mu_i (Eq. 2.14) is evaluated on the tile plus a
//                  1-node halo, then every node runs dev::node_update and
//                  pushes its post-collision populations to its neighbours.
// k_step_tma is the same tile step with every input staged by TMA tensor
// copies (halo boxes of C, psi, cos(theta) and a first, then the tile's
// populations and lagged planes, which land while mu is evaluated); it is
// the collide kernel of the tile path whenever the planes are wide enough
// for its boxes.  k_step with plain loads covers tiny grids, the read-out
// and the initial state.
#include <algorithm>
#include "ddcc_device.cuh"
#include "ddcc_tma.cuh"

namespace ddcc {
namespace {

using dev::map_index;

constexpr int BX = kTileX;
constexpr int BY = kTileY;
constexpr int NT = BX * BY;
constexpr int H2W = BX + 4, H2H = BY + 4;   // tile + 2-node halo
constexpr int H1W = BX + 2, H1H = BY + 2;   // tile + 1-node halo

// D2Q9 velocities (Sec. 3): 0 rest, 1-4 axis, 5-8 diagonal.
__constant__ int kCx[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
__constant__ int kCy[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};

template <typename T, int NP>
struct Smem {
    T C[NP - 1][H2H][H2W];
    T psi[H2H][H2W];
    T mu[NP][H1H][H1W];
    T a[H1H][H1W];
    T cth[NP - 1][H1H][H1W];
};

// Stage C (N-1 planes) and psi with a 2-node halo, a and cos(theta_iN)
// with a 1-node halo (periodic wrap or mirror ghosts).
template <typename T, int NP>
__device__ void load_tile(const KParams<T>& P, Smem<T, NP>& sm, const T* __restrict__ C,
                          const T* __restrict__ psi, const T* __restrict__ cosf,
                          const T* __restrict__ a_in, int x0, int y0, int tid) {
    for (int k = tid; k < H2H * H2W; k += NT) {
        const int ly = k / H2W, lx = k - ly * H2W;
        const int gx = map_index(x0 + lx - 2, P.nx, P.px);
        const int gy = map_index(y0 + ly - 2, P.ny, P.py);
        const long long o = P.org + (long long)gy * P.pitch + gx;
        sm.psi[ly][lx] = psi[o];
#pragma unroll
        for (int i = 0; i < NP - 1; ++i) sm.C[i][ly][lx] = C[i * P.plane + o];
    }
    for (int k = tid; k < H1H * H1W; k += NT) {
        const int ly = k / H1W, lx = k - ly * H1W;
        const int gx = map_index(x0 + lx - 1, P.nx, P.px);
        const int gy = map_index(y0 + ly - 1, P.ny, P.py);
        const long long o = P.org + (long long)gy * P.pitch + gx;
        sm.a[ly][lx] = a_in ? a_in[o] : T(0);
#pragma unroll
        for (int i = 0; i < NP - 1; ++i)
            sm.cth[i][ly][lx] = P.has_cos_field ? cosf[i * P.plane + o] : P.cos_uni[i];
    }
}

// mu on the tile + 1-node halo.
template <typename T, int NP>
__device__ void compute_mu_tile(const KParams<T>& P, Smem<T, NP>& sm, int tid) {
    for (int k = tid; k < H1H * H1W; k += NT) {
        const int ly = k / H1W, lx = k - ly * H1W;
        const int cy = ly + 1, cx = lx + 1;
        T cth[NP];
#pragma unroll
        for (int i = 0; i < NP - 1; ++i) cth[i] = sm.cth[i][ly][lx];
        T mu[NP];
        dev::chem_pot<T, NP>(
            P, [&](int j, int dy, int dx) { return sm.C[j][cy + dy][cx + dx]; },
            [&](int dy, int dx) { return sm.psi[cy + dy][cx + dx]; }, cth, mu);
#pragma unroll
        for (int i = 0; i < NP; ++i) sm.mu[i][ly][lx] = mu[i];
    }
}

template <typename T, int NP>
struct TileAcc {
    const Smem<T, NP>& sm;
    int cy, cx, hy, hx;
    long long o, plane;
    const T* __restrict__ lag_in;
    const T* __restrict__ fin;
    const T* __restrict__ gin;
    __device__ T C(int j, int dy, int dx) const { return sm.C[j][cy + dy][cx + dx]; }
    __device__ T psi(int dy, int dx) const { return sm.psi[cy + dy][cx + dx]; }
    __device__ T mu(int j, int dy, int dx) const { return sm.mu[j][hy + dy][hx + dx]; }
    __device__ T a(int dy, int dx) const { return sm.a[hy + dy][hx + dx]; }
    __device__ T lag(int k) const { return lag_in[k * plane + o]; }
    __device__ T f(int i, int p) const { return fin[(i * 9 + p) * plane + o]; }
    __device__ T g(int p) const { return gin[p * plane + o]; }
};

// Push to x + c_p (periodic wrap), or back into the node's opposite
// direction where x + c_p lies beyond an outer wall (halfway bounce-back).
template <typename T, int NP>
struct TileSink {
    long long tgt[9];
    int tdir[9];
    long long o, plane;
    T* __restrict__ fout;
    T* __restrict__ gout;
    T* __restrict__ lout;
    T* __restrict__ macro_out;
    __device__ void f_out(int i, int p, T v) { fout[(i * 9 + tdir[p]) * plane + tgt[p]] = v; }
    __device__ void g_out(int p, T v) { gout[tdir[p] * plane + tgt[p]] = v; }
    __device__ void lag_out(int k, T v) { lout[k * plane + o] = v; }
    __device__ void macro(const T* Cv, T rho, T ux, T uy, T Pr, const T* mu) {
#pragma unroll
        for (int j = 0; j < NP; ++j) {
            macro_out[j * plane + o] = Cv[j];
            macro_out[(NP + 4 + j) * plane + o] = mu[j];
        }
        macro_out[NP * plane + o] = rho;
        macro_out[(NP + 1) * plane + o] = ux;
        macro_out[(NP + 2) * plane + o] = uy;
        macro_out[(NP + 3) * plane + o] = Pr;
    }
};

// D2Q9 velocity components as compile-time functions of p (after unrolling
// they fold into the addresses).
__host__ __device__ constexpr int cxp(int p) { return (p == 1 || p == 5 || p == 8) ? 1 : (p == 3 || p == 6 || p == 7) ? -1 : 0; }
__host__ __device__ constexpr int cyp(int p) { return (p == 2 || p == 5 || p == 6) ? 1 : (p == 4 || p == 7 || p == 8) ? -1 : 0; }

// Push sink of a tile whose pushes all land inside the domain (no periodic
// wrap, no wall): every target is the node's own address plus a fixed
// offset, taken in 32-bit element offsets from the node (the launcher checks
// that the population and lagged buffers fit them).
template <typename T, int NP>
struct InnerSink {
    T* __restrict__ pop;   // output populations at this node
    T* __restrict__ lag;   // output lagged planes at this node
    int plane, pitch;
    __device__ void f_out(int i, int p, T v) { pop[(9 * i + p) * plane + cyp(p) * pitch + cxp(p)] = v; }
    __device__ void g_out(int p, T v) { pop[(9 * (NP - 1) + p) * plane + cyp(p) * pitch + cxp(p)] = v; }
    __device__ void lag_out(int k, T v) { lag[k * plane] = v; }
    __device__ void macro(const T*, T, T, T, T, const T*) {}
};

__device__ __forceinline__ int opposite(int p) {
    return p == 0 ? 0 : (p <= 4 ? ((p + 1) & 3) + 1 : ((p - 3) & 3) + 5);
}

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
    const long long o = P.org + (long long)y * P.pitch + x;
    TileAcc<T, NP> acc{sm, (int)threadIdx.y + 2, (int)threadIdx.x + 2, (int)threadIdx.y + 1,
                       (int)threadIdx.x + 1, o, P.plane, lag_in, fin, gin};
    TileSink<T, NP> sink;
    sink.o = o;
    sink.plane = P.plane;
    sink.fout = fout;
    sink.gout = gout;
    sink.lout = lag_out;
    sink.macro_out = F.macro;
    if (MODE == 0) {
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
            sink.tgt[p] = bounce ? o : P.org + (long long)ty * P.pitch + tx;
            sink.tdir[p] = bounce ? opposite(p) : p;
        }
    }
    dev::node_update<T, NP, MODE>(P, acc, sink);
}

// ---- TMA-staged tile step -------------------------------------------------

template <typename T, int NP, bool TF>
struct TLay {
    static constexpr int NPOP = 9 * NP;
    static constexpr int NLAG = 2 * NP + 3;
    static constexpr int NST = TF ? NP : 1;
    static constexpr int HX = kTileHaloW;                  // halo box columns x0-4 .. x0+35
    static constexpr int pad(int e) { return (e * (int)sizeof(T) + 127) / 128 * 128 / (int)sizeof(T); }
    static constexpr int POP_BOX = NPOP * BY * BX;
    static constexpr int LAG_BOX = NLAG * BY * BX;
    static constexpr int C_BOX = (NP - 1) * (BY + 4) * HX;   // rows y0-2 .. y0+9
    static constexpr int ST_BOX = NST * (BY + 4) * HX;
    static constexpr int A_BOX = (BY + 2) * HX;               // rows y0-1 .. y0+8
    static constexpr int MU = NP * (BY + 2) * (BX + 2);
    static constexpr size_t pop_off = 0;
    static constexpr size_t lag_off = pop_off + pad(POP_BOX);
    static constexpr size_t c_off = lag_off + pad(LAG_BOX);
    static constexpr size_t st_off = c_off + pad(C_BOX);
    static constexpr size_t a_off = st_off + pad(ST_BOX);
    static constexpr size_t mu_off = a_off + pad(A_BOX);
    static constexpr size_t end = mu_off + MU;
    static constexpr size_t bar_byte_off = (end * sizeof(T) + 127) / 128 * 128;
    static constexpr size_t bytes = bar_byte_off + 64;
    static constexpr unsigned tx_halo = (unsigned)((C_BOX + ST_BOX + A_BOX) * sizeof(T));
    static constexpr unsigned tx_tile = (unsigned)((POP_BOX + LAG_BOX) * sizeof(T));
};

template <typename T, int NP, bool TF>
struct TmaAcc {
    using L = TLay<T, NP, TF>;
    const T* sm;
    int tx, ty;
    __device__ T C(int j, int dy, int dx) const {
        return sm[L::c_off + ((size_t)j * (BY + 4) + ty + 2 + dy) * L::HX + tx + 4 + dx];
    }
    __device__ T psi(int dy, int dx) const { return sm[L::st_off + (size_t)(ty + 2 + dy) * L::HX + tx + 4 + dx]; }
    __device__ T mu(int j, int dy, int dx) const {
        return sm[L::mu_off + ((size_t)j * (BY + 2) + ty + 1 + dy) * (BX + 2) + tx + 1 + dx];
    }
    __device__ T a(int dy, int dx) const { return sm[L::a_off + (size_t)(ty + 1 + dy) * L::HX + tx + 4 + dx]; }
    __device__ T lag(int k) const { return sm[L::lag_off + ((size_t)k * BY + ty) * BX + tx]; }
    __device__ T f(int i, int p) const { return sm[L::pop_off + ((size_t)(9 * i + p) * BY + ty) * BX + tx]; }
    __device__ T g(int p) const { return sm[L::pop_off + ((size_t)(9 * (NP - 1) + p) * BY + ty) * BX + tx]; }
};

// Two CTAs per SM in FP32 (128 registers, ~69 KB of shared memory each);
// FP64 tiles need twice the shared memory, so one.
template <typename T, int NP, bool TF>
__global__ void __launch_bounds__(NT, sizeof(T) == 4 ? 2 : 1)
    k_step_tma(const __grid_constant__ CUtensorMap tm_pop, const __grid_constant__ CUtensorMap tm_lag,
               const __grid_constant__ CUtensorMap tm_c, const __grid_constant__ CUtensorMap tm_st,
               const __grid_constant__ CUtensorMap tm_a, KParams<T> P, T* __restrict__ pop_out,
               T* __restrict__ lag_out, int* __restrict__ err) {
    using L = TLay<T, NP, TF>;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    T* sm = reinterpret_cast<T*>(smem_raw);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw + L::bar_byte_off);
    const int tid = threadIdx.x + BX * threadIdx.y;
    const int x0 = blockIdx.x * BX, y0 = blockIdx.y * BY;
    if (tid == 0) {
        tma::mbar_init(&bars[0], 1);
        tma::mbar_init(&bars[1], 1);
        tma::mbar_init_fence();
    }
    __syncthreads();
    // padded coordinates: column x0 - 4 is x0 (kGX = 4), row y is y + kGY
    if (tid == 0) {
        tma::mbar_expect_tx(&bars[0], L::tx_halo);
        tma::load_3d(sm + L::c_off, &tm_c, x0, y0 - 2 + kGY, 0, &bars[0]);
        tma::load_3d(sm + L::st_off, &tm_st, x0, y0 - 2 + kGY, 0, &bars[0]);
        tma::load_3d(sm + L::a_off, &tm_a, x0, y0 - 1 + kGY, 0, &bars[0]);
        tma::mbar_expect_tx(&bars[1], L::tx_tile);
        tma::load_3d(sm + L::pop_off, &tm_pop, x0 + kGX, y0 + kGY, 0, &bars[1]);
        tma::load_3d(sm + L::lag_off, &tm_lag, x0 + kGX, y0 + kGY, 0, &bars[1]);
    }
    bool ok = tma::mbar_wait_bounded(&bars[0], 0);
    if (!__syncthreads_and(ok)) {
        // a copy has not landed within the bounded wait: record it, and give
        // every copy still in flight a second bounded wait before the CTA and
        // its shared memory go
        if (tid == 0) {
            atomicOr(err, 1);
            tma::mbar_wait_bounded(&bars[0], 0);
            tma::mbar_wait_bounded(&bars[1], 0);
        }
        return;
    }
    // mu on the tile + 1-node halo while the tile's populations land
    for (int k = tid; k < (BY + 2) * (BX + 2); k += NT) {
        const int ly = k / (BX + 2), lx = k - ly * (BX + 2);
        const T* cb = sm + L::c_off + (size_t)(ly + 1) * L::HX + lx + 3;
        const T* sb = sm + L::st_off + (size_t)(ly + 1) * L::HX + lx + 3;
        T cth[NP];
#pragma unroll
        for (int i = 0; i < NP - 1; ++i)
            cth[i] = TF ? sb[(size_t)(1 + i) * (BY + 4) * L::HX] : P.cos_uni[i];
        T mu[NP];
        dev::chem_pot<T, NP>(
            P, [&](int j, int dy, int dx) { return cb[((size_t)j * (BY + 4) + dy) * L::HX + dx]; },
            [&](int dy, int dx) { return sb[dy * L::HX + dx]; }, cth, mu);
#pragma unroll
        for (int i = 0; i < NP; ++i) sm[L::mu_off + ((size_t)i * (BY + 2) + ly) * (BX + 2) + lx] = mu[i];
    }
    ok = tma::mbar_wait_bounded(&bars[1], 0);
    if (!__syncthreads_and(ok)) {
        if (tid == 0) {
            atomicOr(err, 1);
            tma::mbar_wait_bounded(&bars[1], 0);
        }
        return;
    }
    const int x = x0 + threadIdx.x, y = y0 + threadIdx.y;
    if (x >= P.nx || y >= P.ny) return;
    const long long o = P.org + (long long)y * P.pitch + x;
    TmaAcc<T, NP, TF> acc{sm, (int)threadIdx.x, (int)threadIdx.y};
    TileSink<T, NP> sink;
    sink.o = o;
    sink.plane = P.plane;
    sink.fout = pop_out;
    sink.gout = pop_out + (long long)9 * (NP - 1) * P.plane;
    sink.lout = lag_out;
    sink.macro_out = nullptr;
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
        sink.tgt[p] = bounce ? o : P.org + (long long)ty * P.pitch + tx;
        sink.tdir[p] = bounce ? opposite(p) : p;
    }
    dev::node_update<T, NP, 0>(P, acc, sink);
}

// ---- TMA-staged tile step that also forms the order parameters -------------
//
// The phase populations arrive with a 2-node halo (40 x 12 box), so C_i =
// sum_p f^i_p / psi is formed in shared memory for the tile and its halo and
// never goes through HBM; the flow populations and lagged planes arrive for
// the tile only.  At outer walls the f ghost nodes hold mirror copies, so
// the C they give is the mirror image the stencils expect.

// L2 prefetch distance of the fused tile kernel, in quarter waves of
// resident CTAs.
constexpr int kPrefetchQuarterWaves = 3;

template <typename T, int NP, bool TF>
struct FLay {
    static constexpr int NF = 9 * (NP - 1);
    static constexpr int NLAG = 2 * NP + 3;
    static constexpr int NST = TF ? NP : 1;
    static constexpr int HX = kTileHaloW;
    static constexpr int HY = BY + 4;
    static constexpr int pad(int e) { return (e * (int)sizeof(T) + 127) / 128 * 128 / (int)sizeof(T); }
    static constexpr int FH_BOX = NF * HY * HX;              // rows y0-2 .. y0+9, columns x0-4 .. x0+35
    static constexpr int G_BOX = 9 * BY * BX;
    static constexpr int LAG_BOX = NLAG * BY * BX;
    static constexpr int ST_BOX = NST * HY * HX;
    static constexpr int A_BOX = (BY + 2) * HX;
    static constexpr int C_ARR = (NP - 1) * HY * HX;
    static constexpr int MU = NP * (BY + 2) * (BX + 2);
    static constexpr size_t fh_off = 0;
    static constexpr size_t g_off = fh_off + pad(FH_BOX);
    static constexpr size_t lag_off = g_off + pad(G_BOX);
    static constexpr size_t st_off = lag_off + pad(LAG_BOX);
    static constexpr size_t a_off = st_off + pad(ST_BOX);
    static constexpr size_t c_off = a_off + pad(A_BOX);
    static constexpr size_t mu_off = c_off + C_ARR;
    static constexpr size_t end = mu_off + MU;
    static constexpr size_t bar_byte_off = (end * sizeof(T) + 127) / 128 * 128;
    static constexpr size_t bytes = bar_byte_off + 64;
    static constexpr unsigned tx_halo = (unsigned)((FH_BOX + ST_BOX + A_BOX) * sizeof(T));
    static constexpr unsigned tx_tile = (unsigned)((G_BOX + LAG_BOX) * sizeof(T));
};

template <typename T, int NP, bool TF>
struct FusedAcc {
    using L = FLay<T, NP, TF>;
    const T* sm;
    int tx, ty;
    __device__ T C(int j, int dy, int dx) const {
        return sm[L::c_off + ((size_t)j * L::HY + ty + 2 + dy) * L::HX + tx + 4 + dx];
    }
    __device__ T psi(int dy, int dx) const { return sm[L::st_off + (size_t)(ty + 2 + dy) * L::HX + tx + 4 + dx]; }
    __device__ T mu(int j, int dy, int dx) const {
        return sm[L::mu_off + ((size_t)j * (BY + 2) + ty + 1 + dy) * (BX + 2) + tx + 1 + dx];
    }
    __device__ T a(int dy, int dx) const { return sm[L::a_off + (size_t)(ty + 1 + dy) * L::HX + tx + 4 + dx]; }
    __device__ T lag(int k) const { return sm[L::lag_off + ((size_t)k * BY + ty) * BX + tx]; }
    __device__ T f(int i, int p) const {
        return sm[L::fh_off + ((size_t)(9 * i + p) * L::HY + ty + 2) * L::HX + tx + 4];
    }
    __device__ T g(int p) const { return sm[L::g_off + ((size_t)p * BY + ty) * BX + tx]; }
};

template <typename T, int NP, bool TF>
__global__ void __launch_bounds__(NT, sizeof(T) == 4 ? 2 : 1)
    k_step_fused(const __grid_constant__ CUtensorMap tm_fh, const __grid_constant__ CUtensorMap tm_g,
                 const __grid_constant__ CUtensorMap tm_lag, const __grid_constant__ CUtensorMap tm_st,
                 const __grid_constant__ CUtensorMap tm_a, KParams<T> P, T* __restrict__ pop_out,
                 T* __restrict__ lag_out, int* __restrict__ err, int pf_dist, int off32) {
    using L = FLay<T, NP, TF>;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    T* sm = reinterpret_cast<T*>(smem_raw);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw + L::bar_byte_off);
    const int tid = threadIdx.x + BX * threadIdx.y;
    const int x0 = blockIdx.x * BX, y0 = blockIdx.y * BY;
    if (tid == 0) {
        tma::mbar_init(&bars[0], 1);
        tma::mbar_init(&bars[1], 1);
        tma::mbar_init_fence();
    }
    __syncthreads();
    // padded coordinates: column x0 - 4 is x0 (kGX = 4), row y is y + kGY
    if (tid == 0) {
        tma::mbar_expect_tx(&bars[0], L::tx_halo);
        tma::load_3d(sm + L::fh_off, &tm_fh, x0, y0 - 2 + kGY, 0, &bars[0]);
        tma::load_3d(sm + L::st_off, &tm_st, x0, y0 - 2 + kGY, 0, &bars[0]);
        tma::load_3d(sm + L::a_off, &tm_a, x0, y0 - 1 + kGY, 0, &bars[0]);
        tma::mbar_expect_tx(&bars[1], L::tx_tile);
        tma::load_3d(sm + L::g_off, &tm_g, x0 + kGX, y0 + kGY, 0, &bars[1]);
        tma::load_3d(sm + L::lag_off, &tm_lag, x0 + kGX, y0 + kGY, 0, &bars[1]);
        // the tile pf_dist blocks later in launch order (roughly the CTA that
        // starts a wave of resident CTAs from now) is pulled into L2, so DRAM
        // keeps streaming while the resident CTAs compute
        const int nb = gridDim.x * gridDim.y, b = blockIdx.y * gridDim.x + blockIdx.x + pf_dist;
        if (pf_dist > 0 && b < nb) {
            const int px0 = (b % gridDim.x) * BX, py0 = (b / gridDim.x) * BY;
            tma::prefetch_3d(&tm_fh, px0, py0 - 2 + kGY, 0);
            tma::prefetch_3d(&tm_st, px0, py0 - 2 + kGY, 0);
            tma::prefetch_3d(&tm_g, px0 + kGX, py0 + kGY, 0);
            tma::prefetch_3d(&tm_lag, px0 + kGX, py0 + kGY, 0);
        }
    }
    bool ok = tma::mbar_wait_bounded(&bars[0], 0);
    if (!__syncthreads_and(ok)) {
        // a copy has not landed within the bounded wait: record it, and give
        // every copy still in flight a second bounded wait before the CTA and
        // its shared memory go
        if (tid == 0) {
            atomicOr(err, 1);
            tma::mbar_wait_bounded(&bars[0], 0);
            tma::mbar_wait_bounded(&bars[1], 0);
        }
        return;
    }
    // C_i = sum_p f^i_p / psi on the tile + 2-node halo (12 x 36 nodes)
    for (int k = tid; k < L::HY * (BX + 4); k += NT) {
        const int cy = k / (BX + 4), cx = k - cy * (BX + 4) + 2;   // box column of node x0-2+..
        const T inv = T(1) / sm[L::st_off + (size_t)cy * L::HX + cx];
        const T* fb = sm + L::fh_off + (size_t)cy * L::HX + cx;
#pragma unroll
        for (int i = 0; i < NP - 1; ++i) {
            T s = T(0);
#pragma unroll
            for (int p = 0; p < 9; ++p) s += fb[(size_t)(9 * i + p) * L::HY * L::HX];
            sm[L::c_off + ((size_t)i * L::HY + cy) * L::HX + cx] = s * inv;
        }
    }
    __syncthreads();
    // mu on the tile + 1-node halo
    for (int k = tid; k < (BY + 2) * (BX + 2); k += NT) {
        const int ly = k / (BX + 2), lx = k - ly * (BX + 2);
        const T* cb = sm + L::c_off + (size_t)(ly + 1) * L::HX + lx + 3;
        const T* sb = sm + L::st_off + (size_t)(ly + 1) * L::HX + lx + 3;
        T cth[NP];
#pragma unroll
        for (int i = 0; i < NP - 1; ++i)
            cth[i] = TF ? sb[(size_t)(1 + i) * L::HY * L::HX] : P.cos_uni[i];
        T mu[NP];
        dev::chem_pot<T, NP>(
            P, [&](int j, int dy, int dx) { return cb[((size_t)j * L::HY + dy) * L::HX + dx]; },
            [&](int dy, int dx) { return sb[dy * L::HX + dx]; }, cth, mu);
#pragma unroll
        for (int i = 0; i < NP; ++i) sm[L::mu_off + ((size_t)i * (BY + 2) + ly) * (BX + 2) + lx] = mu[i];
    }
    ok = tma::mbar_wait_bounded(&bars[1], 0);
    if (!__syncthreads_and(ok)) {
        if (tid == 0) {
            atomicOr(err, 1);
            tma::mbar_wait_bounded(&bars[1], 0);
        }
        return;
    }
    const int x = x0 + threadIdx.x, y = y0 + threadIdx.y;
    if (x >= P.nx || y >= P.ny) return;
    const long long o = P.org + (long long)y * P.pitch + x;
    FusedAcc<T, NP, TF> acc{sm, (int)threadIdx.x, (int)threadIdx.y};
    // most tiles push only into the domain's interior: fixed neighbour
    // offsets, no wrap or bounce-back, 32-bit offsets (a block-uniform branch)
    if (off32 && x0 >= 1 && y0 >= 1 && x0 + BX < P.nx && y0 + BY < P.ny) {
        InnerSink<T, NP> in{pop_out + o, lag_out + o, (int)P.plane, P.pitch};
        dev::node_update<T, NP, 0>(P, acc, in);
        return;
    }
    TileSink<T, NP> sink;
    sink.o = o;
    sink.plane = P.plane;
    sink.fout = pop_out;
    sink.gout = pop_out + (long long)9 * (NP - 1) * P.plane;
    sink.lout = lag_out;
    sink.macro_out = nullptr;
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
        sink.tgt[p] = bounce ? o : P.org + (long long)ty * P.pitch + tx;
        sink.tdir[p] = bounce ? opposite(p) : p;
    }
    dev::node_update<T, NP, 0>(P, acc, sink);
}

template <typename T, int NP, bool TF>
cudaError_t collide_fused_n(const TileTmaArgs<T>& a, cudaStream_t s) {
    using L = FLay<T, NP, TF>;
    const cudaError_t e = cudaFuncSetAttribute(k_step_fused<T, NP, TF>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::bytes);
    if (e != cudaSuccess) return e;
    const KParams<T>& kp = *a.kp;
    int sms = 0, dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        sms = 0;   // no prefetch
    // a wave of resident CTAs (two per SM in FP32, one in FP64) ahead
    const int pf_dist = kPrefetchQuarterWaves * sms * (sizeof(T) == 4 ? 2 : 1) / 4;
    // the inner tiles' 32-bit offsets reach every population and lagged plane
    const int off32 = (long long)(9 * NP) * kp.plane < (1LL << 31) ? 1 : 0;
    k_step_fused<T, NP, TF><<<dim3((kp.nx + BX - 1) / BX, (kp.ny + BY - 1) / BY), dim3(BX, BY), L::bytes, s>>>(
        *a.tm_pop, *a.tm_g, *a.tm_lag, *a.tm_st, *a.tm_a, kp, a.pop_out, a.lag_out, a.err, pf_dist, off32);
    return cudaGetLastError();
}

template <typename T, int NP, bool TF>
cudaError_t collide_tma_n(const TileTmaArgs<T>& a, cudaStream_t s) {
    using L = TLay<T, NP, TF>;
    const cudaError_t e = cudaFuncSetAttribute(k_step_tma<T, NP, TF>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::bytes);
    if (e != cudaSuccess) return e;
    const KParams<T>& kp = *a.kp;
    k_step_tma<T, NP, TF><<<dim3((kp.nx + BX - 1) / BX, (kp.ny + BY - 1) / BY), dim3(BX, BY), L::bytes, s>>>(
        *a.tm_pop, *a.tm_lag, *a.tm_c, *a.tm_st, *a.tm_a, kp, a.pop_out, a.lag_out, a.err);
    return cudaGetLastError();
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
    const long long o = P.org + (long long)y * P.pitch + x;
    const T psi = sm.psi[threadIdx.y + 2][threadIdx.x + 2];
    T* f = cur ? F.f[1] : F.f[0];
    const T w0 = P.w1d[1] * P.w1d[1];
#pragma unroll
    for (int i = 0; i < NP - 1; ++i) {
        const T psiC = psi * sm.C[i][threadIdx.y + 2][threadIdx.x + 2];
        const T emu = P.eta[i] * psi * sm.mu[i][threadIdx.y + 1][threadIdx.x + 1];
#pragma unroll
        for (int p = 0; p < 9; ++p) {
            const T wp = P.w1d[kCx[p] + 1] * P.w1d[kCy[p] + 1];
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
        const long long o = P.org + (long long)y * P.pitch + x;
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
        const long long o = P.org + (long long)y * P.pitch + x;
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
__global__ void k_convert(const double* __restrict__ src, T* __restrict__ dst, KParams<T> P,
                          int planes) {
    const long long n = (long long)P.nx * P.ny;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n * planes;
         idx += (long long)gridDim.x * blockDim.x) {
        const long long q = idx / n, r = idx - q * n;
        const int y = (int)(r / P.nx), x = (int)(r - (long long)y * P.nx);
        dst[q * P.plane + P.org + (long long)y * P.pitch + x] = (T)src[idx];
    }
}

template <typename T>
__global__ void k_export(const T* __restrict__ src, double* __restrict__ dst, KParams<T> P) {
    const long long n = (long long)P.nx * P.ny;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
         idx += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(idx / P.nx), x = (int)(idx - (long long)y * P.nx);
        dst[idx] = (double)src[P.org + (long long)y * P.pitch + x];
    }
}

// Ghost frame: every cell of [-kGX, nx + kGX) x [-kGY, ny + kGY) outside
// the domain takes the value of its periodic image or wall mirror.  The
// cells are enumerated as 2 kGY full-width ghost rows, then 2 kGX ghost
// columns of the ny domain rows.
template <typename T>
__global__ void k_fill_ghosts(GhostRing<T> g0, GhostRing<T> g1, KParams<T> P) {
    // one ghost cell per thread, plane blockIdx.y of ring g0 and then of
    // ring g1: first the 2 gy full rows (corners included), then the 2 gx
    // side columns of the ny interior rows, grouped by row so that a row's
    // side cells are neighbours in a warp.  Every source is an interior
    // node, so the cells are independent.
    const bool second = (int)blockIdx.y >= g0.planes;
    const int gx = second ? g1.gx : g0.gx, gy = second ? g1.gy : g0.gy;
    const int W = P.nx + 2 * gx;
    const int nrow = 2 * gy * W, ncol = 2 * gx * P.ny;
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nrow + ncol) return;
    int X, Y;
    if (r < nrow) {
        const int k = r / W;
        X = r - k * W - gx;
        Y = k < gy ? k - gy : P.ny + (k - gy);
    } else {
        const int c = r - nrow;
        Y = c / (2 * gx);
        const int k = c - Y * (2 * gx);
        X = k < gx ? k - gx : P.nx + (k - gx);
    }
    const int sx = map_index(X, P.nx, P.px), sy = map_index(Y, P.ny, P.py);
    T* pl = second ? g1.base + (long long)((int)blockIdx.y - g0.planes) * P.plane
                   : g0.base + (long long)blockIdx.y * P.plane;
    pl[P.org + (long long)Y * P.pitch + X] = pl[P.org + (long long)sy * P.pitch + sx];
}

// Open x ends: equilibrium at (u_in(y), 0) with mu = 0 and m^C = 0 (Eqs. 3.5,
// 3.8); C = C_in at the inlet, the neighbour column's at the outlet; psi P
// from the neighbour column by Eq. 19 without its velocity terms.
template <typename T, int NP>
__global__ void k_open_bc(KParams<T> P, T* __restrict__ pop, T* __restrict__ lag, const T* __restrict__ psi,
                          const T* __restrict__ inflow) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= 2 * P.ny) return;
    const int side = idx / P.ny, y = idx - side * P.ny;
    const int xb = side ? P.nx - 1 : 0, xn = side ? P.nx - 2 : 1;
    const long long pl = P.plane;
    const long long ob = P.org + (long long)y * P.pitch + xb, on = P.org + (long long)y * P.pitch + xn;
    const T psib = psi[ob], psin = psi[on];
    const T u = inflow[y];
    const T cs2 = P.cs2;
    T Cb[NP];
    T rho = T(0), sC = T(0);
#pragma unroll
    for (int j = 0; j < NP - 1; ++j) {
        T c;
        if (side == 0) {
            c = inflow[(1 + j) * P.ny + y];
        } else {
            T sf = T(0);
#pragma unroll
            for (int p = 0; p < 9; ++p) sf += pop[(9 * j + p) * pl + on];
            c = sf / psin;
        }
        Cb[j] = c;
        sC += c;
        rho += c * P.rho[j];
    }
    rho += (T(1) - sC) * P.rho[NP - 1];
    T* g = pop + (long long)9 * (NP - 1) * pl;
    T sum_g = T(0);
#pragma unroll
    for (int p = 1; p < 9; ++p) sum_g += g[p * pl + on];
    const T psiP = psib * (P.cP * (sum_g - P.Kh * lag[(2 * NP + 2) * pl + on]) / psin);
    // phases: f_0 = psi C, f_p = w_p psi C c_p.u / cs2
#pragma unroll
    for (int j = 0; j < NP - 1; ++j) {
        const T psiC = psib * Cb[j];
#pragma unroll
        for (int p = 0; p < 9; ++p) {
            const T wp = P.w1d[kCx[p] + 1] * P.w1d[kCy[p] + 1];
            pop[(9 * j + p) * pl + ob] = p == 0 ? psiC : wp * psiC * (T(kCx[p]) * u) / cs2;
        }
    }
    // flow: g_p = w_p psi P / cs2 + s_p (g_0 stored less rho0), s_p of the
    // resting-solid-free equilibrium with m^C = 0
    const T Axx = psib * rho * u * u;
#pragma unroll
    for (int p = 0; p < 9; ++p) {
        const T wp = P.w1d[kCx[p] + 1] * P.w1d[kCy[p] + 1];
        const T cx = T(kCx[p]), cy = T(kCy[p]);
        const T sp = wp * (cx * psib * rho * u / cs2 + Axx * (cx * cx - cs2) / (cs2 - cs2 * cs2));
        (void)cy;
        g[p * pl + ob] = (p == 0 ? (wp - T(1)) : wp) * psiP / cs2 + sp;
    }
    lag[ob] = T(0);
#pragma unroll
    for (int j = 0; j < NP - 1; ++j) {
        lag[(1 + 2 * j) * pl + ob] = psib * Cb[j] * u;
        lag[(2 + 2 * j) * pl + ob] = T(0);
    }
    lag[(2 * NP - 1) * pl + ob] = T(0);
    lag[(2 * NP) * pl + ob] = T(0);
    lag[(2 * NP + 1) * pl + ob] = T(0);
    lag[(2 * NP + 2) * pl + ob] = psib * rho * u * u;
}

template <typename T>
__global__ void k_walls_init(KParams<T> P, T* __restrict__ psi, T* __restrict__ e) {
    const long long n = (long long)P.nx * P.ny;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
         idx += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(idx / P.nx), x = (int)(idx - (long long)y * P.nx);
        const long long o = P.org + (long long)y * P.pitch + x;
        psi[o] = T(1);
        for (int j = 0; j < P.N - 1; ++j) e[j * P.plane + o] = T(0);
    }
}

// psi *= psi_k; e_j += cos(theta^k_jN) |grad psi_k| (the gradient stencil of
// the step, on psi_k with its ghost frame).
template <typename T>
__global__ void k_wall_accumulate(KParams<T> P, const T* __restrict__ stage, T* __restrict__ psi,
                                  T* __restrict__ e) {
    const long long n = (long long)P.nx * P.ny;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
         idx += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(idx / P.nx), x = (int)(idx - (long long)y * P.nx);
        const long long o = P.org + (long long)y * P.pitch + x;
        T gx, gy;
        dev::grad9(P, [&](int dy, int dx) { return stage[o + (long long)dy * P.pitch + dx]; }, gx, gy);
        const T ag = sqrt(gx * gx + gy * gy);
        psi[o] = psi[o] * stage[o];
        for (int j = 0; j < P.N - 1; ++j) e[j * P.plane + o] += stage[(1 + j) * P.plane + o] * ag;
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
size_t tile_tma_smem_bytes(int N, bool tf) {
    switch (N * 2 + (tf ? 1 : 0)) {
        case 4: return TLay<T, 2, false>::bytes;
        case 5: return TLay<T, 2, true>::bytes;
        case 6: return TLay<T, 3, false>::bytes;
        case 7: return TLay<T, 3, true>::bytes;
        case 8: return TLay<T, 4, false>::bytes;
        case 9: return TLay<T, 4, true>::bytes;
        default: return 0;
    }
}
template <typename T>
size_t tile_fused_smem_bytes(int N, bool tf) {
    switch (N * 2 + (tf ? 1 : 0)) {
        case 4: return FLay<T, 2, false>::bytes;
        case 5: return FLay<T, 2, true>::bytes;
        case 6: return FLay<T, 3, false>::bytes;
        case 7: return FLay<T, 3, true>::bytes;
        case 8: return FLay<T, 4, false>::bytes;
        case 9: return FLay<T, 4, true>::bytes;
        default: return 0;
    }
}
template <typename T>
cudaError_t launch_collide_fused(const TileTmaArgs<T>& a, cudaStream_t s) {
    const bool tf = a.kp->has_cos_field != 0;
    switch (a.kp->N * 2 + (tf ? 1 : 0)) {
        case 4: return collide_fused_n<T, 2, false>(a, s);
        case 5: return collide_fused_n<T, 2, true>(a, s);
        case 6: return collide_fused_n<T, 3, false>(a, s);
        case 7: return collide_fused_n<T, 3, true>(a, s);
        case 8: return collide_fused_n<T, 4, false>(a, s);
        case 9: return collide_fused_n<T, 4, true>(a, s);
        default: return cudaErrorInvalidValue;
    }
}
template <typename T>
cudaError_t launch_collide_tma(const TileTmaArgs<T>& a, cudaStream_t s) {
    const bool tf = a.kp->has_cos_field != 0;
    switch (a.kp->N * 2 + (tf ? 1 : 0)) {
        case 4: return collide_tma_n<T, 2, false>(a, s);
        case 5: return collide_tma_n<T, 2, true>(a, s);
        case 6: return collide_tma_n<T, 3, false>(a, s);
        case 7: return collide_tma_n<T, 3, true>(a, s);
        case 8: return collide_tma_n<T, 4, false>(a, s);
        case 9: return collide_tma_n<T, 4, true>(a, s);
        default: return cudaErrorInvalidValue;
    }
}
template <typename T>
cudaError_t launch_convert(const double* src, T* dst, const KParams<T>& kp, int planes,
                           cudaStream_t s) {
    k_convert<T><<<flat_blocks((long long)kp.nx * kp.ny * planes), 256, 0, s>>>(src, dst, kp, planes);
    return cudaGetLastError();
}
template <typename T>
cudaError_t launch_export(const T* src, double* dst, const KParams<T>& kp, cudaStream_t s) {
    k_export<T><<<flat_blocks((long long)kp.nx * kp.ny), 256, 0, s>>>(src, dst, kp);
    return cudaGetLastError();
}
template <typename T>
cudaError_t launch_fill_ghosts2(const GhostRing<T>& g0, const GhostRing<T>& g1, const KParams<T>& kp,
                                cudaStream_t s) {
    long long n = 0;   // cells per plane of the larger ring
    for (const GhostRing<T>* g : {&g0, &g1}) {
        if (g->planes < 0 || g->gx < 0 || g->gx > kGX || g->gy < 0 || g->gy > kGY) return cudaErrorInvalidValue;
        if (g->planes > 0) {
            if (!g->base) return cudaErrorInvalidValue;
            n = std::max(n, 2LL * g->gy * (kp.nx + 2 * g->gx) + 2LL * g->gx * kp.ny);
        }
    }
    const long long planes = (long long)g0.planes + g1.planes;
    if (n == 0 || planes == 0) return cudaSuccess;
    if (planes > 65535 || n > (1LL << 31) - 256) return cudaErrorInvalidValue;
    k_fill_ghosts<T><<<dim3((unsigned)((n + 255) / 256), (unsigned)planes), 256, 0, s>>>(g0, g1, kp);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_fill_ghosts(T* base, int planes, const KParams<T>& kp, cudaStream_t s, int gx, int gy) {
    return launch_fill_ghosts2<T>(GhostRing<T>{base, planes, gx, gy}, GhostRing<T>{nullptr, 0, 0, 0}, kp, s);
}

template <typename T, int NP>
cudaError_t open_bc_n(const KParams<T>& kp, T* pop, T* lag, const T* psi, const T* inflow, cudaStream_t s) {
    k_open_bc<T, NP><<<(2 * kp.ny + 127) / 128, 128, 0, s>>>(kp, pop, lag, psi, inflow);
    return cudaGetLastError();
}
template <typename T>
cudaError_t launch_open_bc(const KParams<T>& kp, T* pop, T* lag, const T* psi, const T* inflow,
                           cudaStream_t s) {
    DDCC_DISPATCH(open_bc_n, kp, pop, lag, psi, inflow, s);
}

template <typename T>
cudaError_t launch_walls_init(const KParams<T>& kp, T* psi, T* e, cudaStream_t s) {
    k_walls_init<T><<<flat_blocks((long long)kp.nx * kp.ny), 256, 0, s>>>(kp, psi, e);
    return cudaGetLastError();
}
template <typename T>
cudaError_t launch_wall_accumulate(const KParams<T>& kp, const T* stage, T* psi, T* e, cudaStream_t s) {
    k_wall_accumulate<T><<<flat_blocks((long long)kp.nx * kp.ny), 256, 0, s>>>(kp, stage, psi, e);
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
    template cudaError_t launch_convert<T>(const double*, T*, const KParams<T>&, int, cudaStream_t); \
    template cudaError_t launch_export<T>(const T*, double*, const KParams<T>&, cudaStream_t);    \
    template cudaError_t launch_fill_ghosts<T>(T*, int, const KParams<T>&, cudaStream_t, int, int);         \
    template cudaError_t launch_fill_ghosts2<T>(const GhostRing<T>&, const GhostRing<T>&, const KParams<T>&,    \
                                                cudaStream_t);                                            \
    template size_t tile_tma_smem_bytes<T>(int, bool);                                           \
    template size_t tile_fused_smem_bytes<T>(int, bool);                                         \
    template cudaError_t launch_walls_init<T>(const KParams<T>&, T*, T*, cudaStream_t);          \
    template cudaError_t launch_open_bc<T>(const KParams<T>&, T*, T*, const T*, const T*, cudaStream_t); \
    template cudaError_t launch_wall_accumulate<T>(const KParams<T>&, const T*, T*, T*, cudaStream_t); \
    template cudaError_t launch_collide_fused<T>(const TileTmaArgs<T>&, cudaStream_t);           \
    template cudaError_t launch_collide_tma<T>(const TileTmaArgs<T>&, cudaStream_t);

DDCC_INSTANTIATE(double)
DDCC_INSTANTIATE(float)

}  // namespace ddcc
