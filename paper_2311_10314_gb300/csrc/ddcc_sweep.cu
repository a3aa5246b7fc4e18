// Row-sweep kernel of the DD-CCLB step (arXiv 2311.10314, Sec. 3) for sm_103a.
//
// Each CTA owns a strip of W columns and a band of rows [ya, yb) and sweeps
// down it RY = 4 rows at a time.  Row blocks of every plane it reads -- the
// 9N populations (f then g), the 2N+3 lagged planes and the static planes
// (psi and the per-node cos(theta_iN)) -- arrive by TMA tensor copies
// (cp.async.bulk.tensor, completion on an mbarrier) into a ring of three
// slots, two blocks ahead of use, so HBM latency is covered by the pipeline
// rather than by occupancy.  The order parameters C_i and the chemical
// potentials mu_i (Eq. 2.14) live only in shared-memory row rings: each
// iteration computes C for rows r+2..r+5 (strip + 2 halo columns), mu for
// rows r+1..r+4 (strip + 1), then collides rows r..r+3 through
// dev::node_update and pushes the post-collision populations to their
// neighbours with plain coalesced stores.  HBM sees every population, the
// lagged planes and psi once per step; the strip halo columns are re-read
// by the neighbour strip (from L2).
//
// The planes carry a ghost frame (kGX columns, kGY rows) holding periodic
// copies (mirror copies of a at outer walls), kept current by the writers,
// so row blocks never wrap.  At outer walls the order parameters of ghost
// nodes are mirror images, filled in shared memory.
//
// Every wait on an mbarrier is bounded; a wait that runs out sets the error
// word, waits (bounded) for the CTA's copies in flight and returns.
#include <cuda.h>

#include "ddcc_device.cuh"
#include "ddcc_tma.cuh"

namespace ddcc {
namespace {

using dev::map_index;

constexpr int RY = 4;        // rows per iteration and per ring block
constexpr int NSLOT = 3;     // ring slots (two blocks in use, one in flight)
constexpr int CRING = 8;     // rows kept in the C and mu rings

__constant__ int kSCx[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
__constant__ int kSCy[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};

template <typename T, int NP, bool TF>
struct Lay {
    static constexpr int W = SweepWidth<T>::value;
    static_assert(RY == kSweepRows, "rows per iteration");
    static constexpr int NT = SweepWidth<T>::threads;
    static constexpr int TW = NT / RY;             // threads per row in the collision pass
    static_assert(TW >= W && TW >= W + 2 && (W + 4) * RY <= 2 * NT, "thread mapping");
    static constexpr int BW = W + 8;               // box width: strip + 4 halo columns a side
    static constexpr int NPOP = 9 * NP;
    static constexpr int NLAG = 2 * NP + 3;
    static constexpr int NST = TF ? NP : 1;
    static constexpr int PLANE = RY * BW;          // elements of one plane in a block
    static constexpr int pad(int e) { return (e * (int)sizeof(T) + 127) / 128 * 128 / (int)sizeof(T); }
    static constexpr int POP_BOX = NPOP * PLANE;
    static constexpr int LAG_BOX = NLAG * PLANE;
    static constexpr int ST_BOX = NST * PLANE;
    static constexpr int POP_SLOT = pad(POP_BOX);  // slot strides keep 128-byte alignment
    static constexpr int LAG_SLOT = pad(LAG_BOX);
    static constexpr int ST_SLOT = pad(ST_BOX);
    static constexpr int CW = W + 4;               // C ring row width (2 halo columns a side)
    static constexpr int MW = W + 2;               // mu ring row width
    static constexpr size_t pop_off = 0;
    static constexpr size_t lag_off = pop_off + (size_t)NSLOT * POP_SLOT;
    static constexpr size_t st_off = lag_off + (size_t)NSLOT * LAG_SLOT;
    static constexpr size_t c_off = st_off + (size_t)NSLOT * ST_SLOT;
    static constexpr size_t m_off = c_off + (size_t)CRING * (NP - 1) * CW;
    static constexpr size_t end = m_off + (size_t)CRING * NP * MW;
    static constexpr size_t bar_byte_off = (end * sizeof(T) + 127) / 128 * 128;
    static constexpr size_t bytes = bar_byte_off + 64;
    // bytes one block's three copies deliver (the boxes, not the padding)
    static constexpr unsigned tx_bytes = (unsigned)((POP_BOX + LAG_BOX + ST_BOX) * sizeof(T));
};

using tma::mbar_expect_tx;
using tma::mbar_init;
using tma::mbar_wait_bounded;
using tma::load_3d;

__device__ __forceinline__ int opposite(int p) {
    return p == 0 ? 0 : (p <= 4 ? ((p + 1) & 3) + 1 : ((p - 3) & 3) + 5);
}

// Addressing of the rings for a CTA sweeping rows from ya.  *_row(row)
// returns the row's base in its slot; plane k of that row is k * PLANE
// further.
template <typename T, int NP, bool TF>
struct Rings {
    using L = Lay<T, NP, TF>;
    T* pop;
    T* lag;
    T* st;
    T* C;
    T* M;
    int ya;
    // population block b covers rows [ya + b RY, ya + (b + 1) RY)
    __device__ const T* pop_row(int row) const {
        const int d = row - ya + RY;            // >= 0 for rows >= ya - RY
        const int b = d / RY;                   // block index + 1
        return pop + (size_t)((b + NSLOT - 1) % NSLOT) * L::POP_SLOT + (size_t)(d - b * RY) * L::BW;
    }
    // lagged and static blocks cover rows [ya - 1 + b RY, ya - 1 + (b + 1) RY)
    __device__ const T* lag_row(int row) const {
        const int d = row - ya + 1 + RY;
        const int b = d / RY;
        return lag + (size_t)((b + NSLOT - 1) % NSLOT) * L::LAG_SLOT + (size_t)(d - b * RY) * L::BW;
    }
    __device__ const T* st_row(int row) const {
        const int d = row - ya + 1 + RY;
        const int b = d / RY;
        return st + (size_t)((b + NSLOT - 1) % NSLOT) * L::ST_SLOT + (size_t)(d - b * RY) * L::BW;
    }
    __device__ T* C_row(int row, int j) const { return C + ((size_t)(row & (CRING - 1)) * (NP - 1) + j) * L::CW; }
    __device__ T* M_row(int row, int j) const { return M + ((size_t)(row & (CRING - 1)) * NP + j) * L::MW; }
};

// Accessor of dev::node_update for node (tx, y) of the strip; the row
// bases of rows y-1, y, y+1 are resolved once.
template <typename T, int NP, bool TF>
struct SweepAcc {
    using L = Lay<T, NP, TF>;
    const T* st_r[3];
    const T* lag_r[3];
    const T* pop_r;
    const T* C_r[3];
    const T* M_r[3];
    __device__ T C(int j, int dy, int dx) const { return C_r[dy + 1][j * L::CW + 2 + dx]; }
    __device__ T psi(int dy, int dx) const { return st_r[dy + 1][4 + dx]; }
    __device__ T mu(int j, int dy, int dx) const { return M_r[dy + 1][j * L::MW + 1 + dx]; }
    __device__ T a(int dy, int dx) const { return lag_r[dy + 1][4 + dx]; }
    __device__ T lag(int k) const { return lag_r[1][k * L::PLANE + 4]; }
    __device__ T f(int i, int p) const { return pop_r[(9 * i + p) * L::PLANE + 4]; }
    __device__ T g(int p) const { return pop_r[(9 * (NP - 1) + p) * L::PLANE + 4]; }
};

// Sink: push with periodic ghost copies (distance 2) or halfway bounce-back;
// lagged planes at the node, with a ghost copy of a (distance 1).
template <typename T, int NP>
struct SweepSink {
    long long tgt[9];
    unsigned char gfl[9];   // bit 0/1: x ghost at +nx/-nx, bit 2/3: y ghost at +ny/-ny
    long long o, plane, gx_step, gy_step;
    unsigned char afl;      // ghost copies of a: same bits, offsets in a_dx / a_dy
    long long a_dx, a_dy;
    T* __restrict__ pop;
    T* __restrict__ lout;
    __device__ void put(long long base, long long t, unsigned char fl, T v) {
        T* q = pop + base;
        q[t] = v;
        if (fl) {
            const long long dx = (fl & 1) ? gx_step : ((fl & 2) ? -gx_step : 0);
            const long long dy = (fl & 4) ? gy_step : ((fl & 8) ? -gy_step : 0);
            if (dx) q[t + dx] = v;
            if (dy) q[t + dy] = v;
            if (dx && dy) q[t + dx + dy] = v;
        }
    }
    __device__ void f_out(int i, int p, T v) {
        put((long long)(9 * i + dirs(p)) * plane, tgt[p], gfl[p], v);
    }
    __device__ void g_out(int p, T v) { put((long long)(9 * (NP - 1) + dirs(p)) * plane, tgt[p], gfl[p], v); }
    __device__ void lag_out(int k, T v) {
        T* q = lout + (long long)k * plane;
        q[o] = v;
        if (k == 0 && afl) {
            if (a_dx) q[o + a_dx] = v;
            if (a_dy) q[o + a_dy] = v;
            if (a_dx && a_dy) q[o + a_dx + a_dy] = v;
        }
    }
    __device__ void macro(const T*, T, T, T, T, const T*) {}
    int dir[9];
    __device__ int dirs(int p) const { return dir[p]; }
};

template <typename T, int NP, bool TF>
__global__ void __launch_bounds__(Lay<T, NP, TF>::NT, 1)
    k_sweep(const __grid_constant__ CUtensorMap tm_pop, const __grid_constant__ CUtensorMap tm_lag,
            const __grid_constant__ CUtensorMap tm_st, KParams<T> P, T* __restrict__ pop_out,
            T* __restrict__ lag_out, int* __restrict__ err, SweepPlan plan) {
    using L = Lay<T, NP, TF>;
    constexpr int W = L::W;
    constexpr int NT = L::NT;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    T* sm = reinterpret_cast<T*>(smem_raw);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw + L::bar_byte_off);

    const int tid = threadIdx.x;
    const int strip = blockIdx.x % plan.strips, seg = blockIdx.x / plan.strips;
    const int x0 = strip * W;
    const int ya = seg * plan.seg_base + min(seg, plan.seg_rem);
    const int yb = ya + plan.seg_base + (seg < plan.seg_rem ? 1 : 0);
    const int niter = (yb - ya + RY - 1) / RY;
    Rings<T, NP, TF> R{sm + L::pop_off, sm + L::lag_off, sm + L::st_off, sm + L::c_off, sm + L::m_off, ya};

    if (tid == 0) {
        for (int s = 0; s < NSLOT; ++s) mbar_init(&bars[s], 1);
        tma::mbar_init_fence();
    }
    __syncthreads();

    unsigned parity = 0;    // bit s: parity of the next phase of slot s
    unsigned pending = 0;   // bit s: copies issued into slot s and not yet waited
    // row block b (b >= -1) into slot (b + 3) % 3: populations from row
    // ya + b RY, lagged and static planes from row ya - 1 + b RY; the
    // padded column of x0 - 4 is x0 (kGX = 4), the padded row is row + kGY.
    auto issue = [&](int b) {
        const int s = (b + NSLOT) % NSLOT;
        pending |= 1u << s;
        if (tid == 0) {
            mbar_expect_tx(&bars[s], L::tx_bytes);
            load_3d(R.pop + (size_t)s * L::POP_SLOT, &tm_pop, x0, ya + b * RY + kGY, 0, &bars[s]);
            load_3d(R.lag + (size_t)s * L::LAG_SLOT, &tm_lag, x0, ya - 1 + b * RY + kGY, 0, &bars[s]);
            load_3d(R.st + (size_t)s * L::ST_SLOT, &tm_st, x0, ya - 1 + b * RY + kGY, 0, &bars[s]);
        }
    };
    auto wait_block = [&](int b) -> bool {
        const int s = (b + NSLOT) % NSLOT;
        const bool ok = mbar_wait_bounded(&bars[s], (parity >> s) & 1u);
        if (ok) {   // a slot whose wait ran out stays pending for bail()
            parity ^= 1u << s;
            pending &= ~(1u << s);
        }
        return ok;
    };
    auto bail = [&]() {
        if (tid == 0) atomicOr(err, 1);
        for (int s = 0; s < NSLOT; ++s)
            if (pending & (1u << s)) mbar_wait_bounded(&bars[s], (parity >> s) & 1u);
    };

    // C for rows [y0, y0 + nrows), columns x0 - 2 .. x0 + W + 1
    auto compute_C = [&](int y0r, int nrows) {
        for (int k = tid; k < nrows * L::CW; k += NT) {
            const int row = y0r + k / L::CW, c = k % L::CW;
            const T inv = T(1) / R.st_row(row)[c + 2];
            const T* pr = R.pop_row(row) + c + 2;
#pragma unroll
            for (int i = 0; i < NP - 1; ++i) {
                T s = T(0);
#pragma unroll
                for (int p = 0; p < 9; ++p) s += pr[(9 * i + p) * L::PLANE];
                R.C_row(row, i)[c] = s * inv;
            }
        }
    };
    // at outer walls the order parameters of ghost nodes are mirror images
    auto mirror_C = [&](int y0r, int nrows) {
        for (int k = tid; k < nrows * L::CW; k += NT) {
            const int row = y0r + k / L::CW, c = k % L::CW;
            const int x = x0 - 2 + c;
            const bool gy = !P.py && (row < 0 || row >= P.ny) && row >= -2 && row <= P.ny + 1;
            const bool gx = !P.px && (x < 0 || x >= P.nx) && x >= -2 && x <= P.nx + 1;
            if (!(gx || gy)) continue;
            // mirror only across a wall; a periodic axis keeps the window's
            // own (ghost) column or row, whose C came from periodic copies
            const int sy = gy ? map_index(row, P.ny, 0) : row;
            const int sx = gx ? map_index(x, P.nx, 0) : x;
#pragma unroll
            for (int i = 0; i < NP - 1; ++i) R.C_row(row, i)[c] = R.C_row(sy, i)[sx - x0 + 2];
        }
    };
    // mu for rows [y0, y0 + nrows), columns x0 - 1 .. x0 + W
    auto compute_mu = [&](int y0r, int nrows) {
        for (int k = tid; k < nrows * L::MW; k += NT) {
            const int row = y0r + k / L::MW, c = k % L::MW;
            const T* s_m = R.st_row(row - 1) + c + 3;
            const T* s_0 = R.st_row(row) + c + 3;
            const T* s_p = R.st_row(row + 1) + c + 3;
            const T* c_m = R.C_row(row - 1, 0) + c + 1;
            const T* c_0 = R.C_row(row, 0) + c + 1;
            const T* c_p = R.C_row(row + 1, 0) + c + 1;
            T cth[NP];
#pragma unroll
            for (int i = 0; i < NP - 1; ++i) cth[i] = TF ? s_0[(1 + i) * L::PLANE] : P.cos_uni[i];
            T mu[NP];
            dev::chem_pot<T, NP>(
                P,
                [&](int j, int dy, int dx) {
                    return (dy < 0 ? c_m : (dy > 0 ? c_p : c_0))[j * L::CW + dx];
                },
                [&](int dy, int dx) { return (dy < 0 ? s_m : (dy > 0 ? s_p : s_0))[dx]; }, cth, mu);
#pragma unroll
            for (int i = 0; i < NP; ++i) R.M_row(row, i)[c] = mu[i];
        }
    };

    // ---- prologue: blocks -1, 0, 1; C rows ya-2..ya+1; mu rows ya-1, ya ----
    issue(-1);
    issue(0);
    issue(1);
    bool ok = wait_block(-1);
    ok = wait_block(0) && ok;
    if (!__syncthreads_and(ok)) {
        bail();
        return;
    }
    const bool walls = !(P.px && P.py);
    compute_C(ya - 2, 4);
    __syncthreads();
    if (walls) {
        mirror_C(ya - 2, 4);
        __syncthreads();
    }
    compute_mu(ya - 1, 2);
    __syncthreads();

    const int tx = tid % L::TW, ty = tid / L::TW;
    const int x = x0 + tx;
    for (int t = 0; t < niter; ++t) {
        const int r = ya + t * RY;
        if (t + 2 <= niter) issue(t + 2);     // into the slot block t-1 used
        ok = wait_block(t + 1);
        if (!__syncthreads_and(ok)) {
            bail();
            return;
        }
        compute_C(r + 2, RY);
        __syncthreads();
        if (walls) {
            mirror_C(r + 2, RY);
            __syncthreads();
        }
        compute_mu(r + 1, RY);
        __syncthreads();

        const int y = r + ty;
        if (tx < W && x < P.nx && y < yb) {
            const long long o = P.org + (long long)y * P.pitch + x;
            SweepAcc<T, NP, TF> acc;
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                acc.st_r[d] = R.st_row(y - 1 + d) + tx;
                acc.lag_r[d] = R.lag_row(y - 1 + d) + tx;
                acc.C_r[d] = R.C_row(y - 1 + d, 0) + tx;
                acc.M_r[d] = R.M_row(y - 1 + d, 0) + tx;
            }
            acc.pop_r = R.pop_row(y) + tx;
            SweepSink<T, NP> sink;
            sink.o = o;
            sink.plane = P.plane;
            sink.gx_step = P.nx;
            sink.gy_step = (long long)P.ny * P.pitch;
            sink.pop = pop_out;
            sink.lout = lag_out;
#pragma unroll
            for (int p = 0; p < 9; ++p) {
                int tx2 = x + kSCx[p], ty2 = y + kSCy[p];
                bool bounce = false;
                if (tx2 < 0 || tx2 >= P.nx) {
                    if (P.px) tx2 = tx2 < 0 ? tx2 + P.nx : tx2 - P.nx;
                    else bounce = true;
                }
                if (ty2 < 0 || ty2 >= P.ny) {
                    if (P.py) ty2 = ty2 < 0 ? ty2 + P.ny : ty2 - P.ny;
                    else bounce = true;
                }
                if (bounce) {
                    tx2 = x;
                    ty2 = y;
                }
                sink.tgt[p] = P.org + (long long)ty2 * P.pitch + tx2;
                sink.dir[p] = bounce ? opposite(p) : p;
                unsigned char fl = 0;
                if (P.px) fl |= tx2 < 2 ? 1 : (tx2 >= P.nx - 2 ? 2 : 0);
                if (P.py) fl |= ty2 < 2 ? 4 : (ty2 >= P.ny - 2 ? 8 : 0);
                sink.gfl[p] = fl;
            }
            // ghost copies of a at distance 1 (periodic image or wall mirror)
            long long adx = 0, ady = 0;
            if (x == 0) adx = P.px ? (long long)P.nx : -1;
            else if (x == P.nx - 1) adx = P.px ? -(long long)P.nx : 1;
            if (y == 0) ady = P.py ? (long long)P.ny * P.pitch : -(long long)P.pitch;
            else if (y == P.ny - 1) ady = P.py ? -(long long)P.ny * P.pitch : (long long)P.pitch;
            sink.a_dx = adx;
            sink.a_dy = ady;
            sink.afl = (adx || ady) ? 1 : 0;
            dev::node_update<T, NP, 0>(P, acc, sink);
        }
        __syncthreads();
    }
}

template <typename T, int NP, bool TF>
cudaError_t sweep_n(const SweepArgs<T>& a, cudaStream_t s) {
    using L = Lay<T, NP, TF>;
    const cudaError_t e = cudaFuncSetAttribute(k_sweep<T, NP, TF>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)L::bytes);
    if (e != cudaSuccess) return e;
    k_sweep<T, NP, TF><<<a.plan.strips * a.plan.segs, L::NT, L::bytes, s>>>(
        *a.tm_pop, *a.tm_lag, *a.tm_st, *a.kp, a.pop_out, a.lag_out, a.err, a.plan);
    return cudaGetLastError();
}

}  // namespace

template <typename T>
size_t sweep_smem_bytes(int N, bool theta_field) {
    switch (N * 2 + (theta_field ? 1 : 0)) {
        case 4: return Lay<T, 2, false>::bytes;
        case 5: return Lay<T, 2, true>::bytes;
        case 6: return Lay<T, 3, false>::bytes;
        case 7: return Lay<T, 3, true>::bytes;
        case 8: return Lay<T, 4, false>::bytes;
        case 9: return Lay<T, 4, true>::bytes;
        default: return 0;
    }
}

template <typename T>
cudaError_t launch_sweep(const SweepArgs<T>& a, cudaStream_t s) {
    const bool tf = a.kp->has_cos_field != 0;
    switch (a.kp->N * 2 + (tf ? 1 : 0)) {
        case 4: return sweep_n<T, 2, false>(a, s);
        case 5: return sweep_n<T, 2, true>(a, s);
        case 6: return sweep_n<T, 3, false>(a, s);
        case 7: return sweep_n<T, 3, true>(a, s);
        case 8: return sweep_n<T, 4, false>(a, s);
        case 9: return sweep_n<T, 4, true>(a, s);
        default: return cudaErrorInvalidValue;
    }
}

template size_t sweep_smem_bytes<float>(int, bool);
template size_t sweep_smem_bytes<double>(int, bool);
template cudaError_t launch_sweep<float>(const SweepArgs<float>&, cudaStream_t);
template cudaError_t launch_sweep<double>(const SweepArgs<double>&, cudaStream_t);

}  // namespace ddcc
