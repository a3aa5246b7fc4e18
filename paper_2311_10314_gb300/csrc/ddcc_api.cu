// Host runtime and C ABI of the DD-CCLB stepper (declared in include/ddcc.h).
//
// The host side validates parameters, derives the kernel constants from the
// paper's relations, carves the caller's device workspace into fields,
// encodes the TMA tensor maps of the row-sweep kernel, stages host inputs,
// and sequences launches on the caller's stream.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include <cudaTypedefs.h>

#include "ddcc.h"
#include "ddcc_internal.h"

using namespace ddcc;

namespace {
// 0: order parameters, 1: tile collide-stream, 2: row sweep, 3: ghost-frame fills
constexpr int kKinds = 4;
}

struct ddcc_handle {
    ddcc_params prm;
    cudaStream_t stream;
    char* ws;
    size_t ws_bytes;
    int cur;
    int64_t steps;
    KParams<double> kd;
    KParams<float> kf;
    Fields<double> fd;
    Fields<float> ff;
    double* dev_mass;     // kMaxPhases doubles in the workspace
    // row-sweep kernel
    int use_sweep;
    SweepPlan plan;
    CUtensorMap tm_pop[2], tm_lag[2], tm_st;
    // TMA-staged tile kernel
    int n_walls;          // solids given by their own psi_k (ddcc_create_walls), else 0
    int use_tile_tma;     // 1: halo-staged tile kernel, 2: fused order parameters
    CUtensorMap tt_pop[2], tt_lag[2], tt_c, tt_st, tt_a[2], tt_fh[2], tt_g[2];
    // the fused tile step as a CUDA graph of two steps (from copy 0 back to
    // copy 0), captured on first use: 0 not tried, 1 ready, -1 unavailable
    int graph_state;
    cudaGraphExec_t step_graph;
    // the read-out planes (f.macro) hold the fields of the current state;
    // cleared by every call that may change the state
    int macro_valid;
    // reverse segments (ddcc_adjoint_segment, ddcc_adjoint_segment_pipelined)
    // replayed as CUDA graphs: the arguments of the last two plain calls,
    // and graphs captured for arguments seen again
    std::vector<std::vector<const void*>> seg_seen;
    struct SegGraph {
        std::vector<const void*> key;
        cudaGraphExec_t exec;
    };
    std::vector<SegGraph> seg_graphs;
    // the second stream a pipelined segment recomputes the next segment on,
    // and the events that fork it from and join it to the handle's stream
    // (created on first use)
    cudaStream_t side;
    cudaEvent_t fork_ev, join_ev;
    // profiling: event pairs recorded around launches while enabled
    int profiling;
    std::vector<cudaEvent_t> events;      // pool, reused
    std::vector<int> rec_kind;            // kind of pair i (events 2i, 2i+1)
};

namespace {

// Record a start event for a launch of `kind` (or nothing when not profiling).
int prof_begin(ddcc_handle* h, int kind) {
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

int prof_end(ddcc_handle* h) {
    if (!h->profiling) return DDCC_OK;
    const size_t i = h->rec_kind.size() - 1;
    return cudaEventRecord(h->events[2 * i + 1], h->stream) == cudaSuccess ? DDCC_OK : DDCC_ERR_CUDA;
}

constexpr size_t kAlign = 256;

inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Row pitch of a plane: the domain plus the ghost frame, rounded to 32.
int pitch_of(int nx) { return (nx + 2 * kGX + 31) / 32 * 32; }
int rows_of(int ny) { return ny + 2 * kGY; }

bool valid_params(const ddcc_params* p) {
    if (!p) return false;
    if (p->nx < 3 || p->ny < 3 || p->nx > (1 << 20) || p->ny > (1 << 20)) return false;
    if ((long long)p->nx * p->ny > (1LL << 31)) return false;
    if (p->nphase < 2 || p->nphase > DDCC_MAX_PHASES) return false;
    if (p->precision != DDCC_FP64 && p->precision != DDCC_FP32) return false;
    if (p->flags & ~(uint32_t)(DDCC_FLAG_TILE | DDCC_FLAG_SWEEP | DDCC_FLAG_OPEN_X)) return false;
    if ((p->flags & DDCC_FLAG_TILE) && (p->flags & DDCC_FLAG_SWEEP)) return false;
    if ((p->flags & DDCC_FLAG_OPEN_X) && (p->periodic_x || (p->flags & DDCC_FLAG_SWEEP))) return false;
    if (!(p->d0 > 0.0 && p->d0 < 1.0)) return false;
    if (!(p->width > 0.0) || !(p->eps0 > 0.0) || !(p->m0 > 0.0)) return false;
    const int N = p->nphase;
    for (int i = 0; i < N; ++i) {
        if (!(p->rho[i] > 0.0) || !(p->nu[i] > 0.0)) return false;
        for (int j = 0; j < N; ++j) {
            const double s = p->sigma[i][j];
            if (s != p->sigma[j][i]) return false;
            if (i == j ? s != 0.0 : !(s > 0.0)) return false;
        }
    }
    for (int i = 0; i < N - 1; ++i)
        if (!(p->eta[i] > 0.0)) return false;
    for (int k = 0; k < 5; ++k)
        if (!(p->s_f[k] > 0.0 && p->s_f[k] < 2.0)) return false;
    for (int k = 0; k < 4; ++k)
        if (!(p->s_g[k] > 0.0 && p->s_g[k] < 2.0)) return false;
    return true;
}

struct Layout {
    size_t pop[2], lag[2], st, C, macro, partial, stage, inflow, mass, flag, total;
    size_t plane_bytes;
};

// Workspace: per ping-pong copy the 9N population planes (f^1..f^{N-1},
// then g) contiguously and the 2N+3 lagged planes; the static planes psi
// and cos(theta_iN) contiguously; scratch.
Layout layout_of(const ddcc_params* p) {
    Layout L{};
    const int N = p->nphase;
    const size_t es = p->precision == DDCC_FP64 ? sizeof(double) : sizeof(float);
    const size_t plane = (size_t)pitch_of(p->nx) * rows_of(p->ny);
    const size_t pb = align_up(plane * es, kAlign);
    L.plane_bytes = pb;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = align_up(off + bytes, kAlign);
        return o;
    };
    for (int c = 0; c < 2; ++c) L.pop[c] = take(pb * 9 * N);
    for (int c = 0; c < 2; ++c) L.lag[c] = take(pb * lag_planes(N));
    L.st = take(pb * N);
    L.C = take(pb * (N - 1));
    L.macro = take(pb * (2 * N + 4));
    L.partial = take(sizeof(double) * kMassBlocks * kMaxPhases);
    L.stage = take(sizeof(double) * (size_t)p->nx * p->ny * (N - 1));
    L.inflow = take(es * (size_t)p->ny * N);
    L.mass = take(sizeof(double) * kMaxPhases);
    L.flag = take(sizeof(int) * 4);
    L.total = off;
    return L;
}

template <typename T>
void fill_kparams(const ddcc_params* p, KParams<T>& k) {
    std::memset(&k, 0, sizeof(k));
    const int N = p->nphase;
    const double d0 = p->d0, cs2 = d0;
    k.nx = p->nx;
    k.ny = p->ny;
    k.pitch = pitch_of(p->nx);
    k.N = N;
    k.px = p->periodic_x ? 1 : 0;
    k.py = p->periodic_y ? 1 : 0;
    // planes are 256-byte aligned, as carved by layout_of()
    k.plane = (long long)(align_up((size_t)k.pitch * rows_of(p->ny) * sizeof(T), kAlign) / sizeof(T));
    k.org = (long long)kGY * k.pitch + kGX;
    // D2Q9 weights of Sec. 3: w0 = (1-d0)^2, axis (d0-d0^2)/2, diagonal d0^2/4
    const double w0 = (1.0 - d0) * (1.0 - d0);
    const double wa = (d0 - d0 * d0) / 2.0, wd = d0 * d0 / 4.0;
    k.cs2 = (T)cs2;
    k.inv_cs2 = (T)(1.0 / cs2);
    k.gw1 = (T)(wa / cs2);
    k.gw2 = (T)(wd / cs2);
    k.lw1 = (T)(wa / cs2);
    k.lw2 = (T)(wd / cs2);
    k.w1d[0] = (T)(d0 / 2.0);
    k.w1d[1] = (T)(1.0 - d0);
    k.w1d[2] = (T)(d0 / 2.0);
    for (int i = 0; i < N; ++i) {
        k.rho[i] = (T)p->rho[i];
        k.nu[i] = (T)p->nu[i];
        k.sigN[i] = (T)p->sigma[i][N - 1];
        for (int j = 0; j < N; ++j) {
            const double s = p->sigma[i][j];
            k.beta2[i][j] = (T)(i == j ? 0.0 : 2.0 * 3.0 * s / p->width);  // 2 beta, beta = 3 sigma / eps
            k.kap[i][j] = (T)(0.75 * p->width * s);                       // -kappa_ij = 3 eps sigma / 4
            k.wet[i][j] = (T)(3.0 * s);
            k.invsig[i][j] = (T)(i == j ? 0.0 : 1.0 / s);
        }
    }
    k.m0 = (T)p->m0;
    // Hermite norms N_ab = n_a n_b, n = (1, d0, d0 (1 - d0)), order
    // (00, 10, 01, 20, 02, 11, 21, 12, 22)
    const double n1 = d0, n2 = d0 * (1.0 - d0);
    const double Nab[9] = {1.0, n1, n1, n2, n2, n1 * n1, n2 * n1, n1 * n2, n2 * n2};
    for (int a = 0; a < 9; ++a) k.invN[a] = (T)(1.0 / Nab[a]);
    for (int i = 0; i < N - 1; ++i) {
        k.eta[i] = (T)p->eta[i];
        // Eq. 17: m0 = (1/s1 - 1/2) eta_i cs2
        const double s1 = 1.0 / (p->m0 / (p->eta[i] * cs2) + 0.5);
        const double s[9] = {p->s_f[0], s1, s1, p->s_f[1], p->s_f[1], p->s_f[2],
                             p->s_f[3], p->s_f[3], p->s_f[4]};
        for (int a = 0; a < 9; ++a) k.lamf[i][a] = (T)(s[a] / Nab[a]);
    }
    k.lg00 = (T)(p->s_g[0]);
    k.lg1 = (T)(p->s_g[1] / n1);
    k.lg3 = (T)(p->s_g[2] / (n1 * n2));
    k.lg4 = (T)(p->s_g[3] / (n2 * n2));
    k.invN20 = (T)(1.0 / n2);
    k.invN11 = (T)(1.0 / (n1 * n1));
    // Eq. 16: nu = (1/s21 - 1/2)(1 - cs2)/2 = (1/s22 - 1/2) cs2
    k.nu_to_s21 = (T)(2.0 / (1.0 - cs2));
    k.nu_to_s22 = (T)(1.0 / cs2);
    k.damp = (T)(1.0 / (p->eps0 * p->eps0 * p->eps0));
    k.half_damp = (T)(0.5 / (p->eps0 * p->eps0 * p->eps0));
    // Eq. 19 (2D): K = 1 - d0, H = K (1 - 2 d0)(s21 - 2)
    const double K = 1.0 - d0, sg0 = p->s_g[0];
    k.A_P = (T)(0.5 + K * (1.0 - d0) * (2.0 - sg0) / (2.0 * sg0));
    k.Kh = (T)(K / 2.0);
    k.Hfac = (T)(K * (1.0 - 2.0 * d0));
    k.cP = (T)(cs2 / (1.0 - w0));
    // |u|^2 and m^C.u coefficient of Eq. 19 once s_0 = -w0 psi m.u / (1 - cs2)
    k.gam = (T)(K / 2.0 - w0 / (1.0 - cs2));
    k.c2m3cs2 = (T)(1.0 - 3.0 * cs2);
    k.body[0] = (T)p->body_force[0];
    k.body[1] = (T)p->body_force[1];
}

template <typename T>
KParams<T>& kp_of(ddcc_handle* h);
template <>
KParams<double>& kp_of<double>(ddcc_handle* h) { return h->kd; }
template <>
KParams<float>& kp_of<float>(ddcc_handle* h) { return h->kf; }
template <typename T>
Fields<T>& fd_of(ddcc_handle* h);
template <>
Fields<double>& fd_of<double>(ddcc_handle* h) { return h->fd; }
template <>
Fields<float>& fd_of<float>(ddcc_handle* h) { return h->ff; }

template <typename T>
void carve(ddcc_handle* h, const Layout& L, Fields<T>& f) {
    char* b = h->ws;
    const int N = h->prm.nphase;
    for (int c = 0; c < 2; ++c) {
        f.f[c] = reinterpret_cast<T*>(b + L.pop[c]);
        f.g[c] = reinterpret_cast<T*>(b + L.pop[c] + L.plane_bytes * 9 * (N - 1));
        f.lag[c] = reinterpret_cast<T*>(b + L.lag[c]);
    }
    f.psi = reinterpret_cast<T*>(b + L.st);
    f.cosf = reinterpret_cast<T*>(b + L.st + L.plane_bytes);
    f.C = reinterpret_cast<T*>(b + L.C);
    f.macro = reinterpret_cast<T*>(b + L.macro);
    f.partial = reinterpret_cast<double*>(b + L.partial);
    f.stage = reinterpret_cast<double*>(b + L.stage);
    f.inflow = reinterpret_cast<T*>(b + L.inflow);
    f.flag = reinterpret_cast<int*>(b + L.flag);
}

#define DDCC_CU(call)                                  \
    do {                                               \
        if ((call) != cudaSuccess) return DDCC_ERR_CUDA; \
    } while (0)

// --- TMA tensor maps of the sweep -------------------------------------------

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

// 3D map over `planes` planes of pitch x rows elements with a box of
// bx columns, by rows and bz planes.
template <typename T>
bool encode_box(CUtensorMap* tm, const T* base, const KParams<T>& k, int planes, int bx, int by, int bz) {
    PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
    if (!fn) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)k.pitch, (cuuint64_t)rows_of(k.ny), (cuuint64_t)planes};
    const cuuint64_t strides[2] = {(cuuint64_t)k.pitch * sizeof(T), (cuuint64_t)k.plane * sizeof(T)};
    const cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, (cuuint32_t)bz};
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUtensorMapDataType dt =
        sizeof(T) == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    const CUresult r = fn(tm, dt, 3, const_cast<T*>(base), dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

// Sweep boxes: strip plus 4 halo columns a side, kSweepRows rows, all planes.
template <typename T>
bool encode_planes(CUtensorMap* tm, const T* base, const KParams<T>& k, int planes, int box_planes) {
    return encode_box<T>(tm, base, k, planes, SweepWidth<T>::value + 8, kSweepRows, box_planes);
}

// Bands of rows per strip so that strips x bands fills whole waves of one
// CTA per SM, discounting each band's 2-row prologue.
SweepPlan make_plan(int nx, int ny, int W, int sms) {
    SweepPlan pl{};
    pl.strips = (nx + W - 1) / W;
    double best = -1.0;
    int best_s = 1;
    const int smax = ny / 16 > 1 ? ny / 16 : 1;
    for (int s = 1; s <= smax; ++s) {
        const long long items = (long long)pl.strips * s;
        const long long waves = (items + sms - 1) / sms;
        const double h = (double)ny / s;
        const double eff = (double)items / (double)(waves * sms) * (h / (h + 2.0));
        if (eff > best + 1e-9) {
            best = eff;
            best_s = s;
        }
    }
    pl.segs = best_s;
    pl.seg_base = ny / best_s;
    pl.seg_rem = ny % best_s;
    return pl;
}

template <typename T>
int setup_sweep(ddcc_handle* h) {
    const ddcc_params& p = h->prm;
    const int N = p.nphase;
    KParams<T>& k = kp_of<T>(h);
    Fields<T>& f = fd_of<T>(h);
    h->use_sweep = 0;
    if (!(p.flags & DDCC_FLAG_SWEEP)) return DDCC_OK;
    const int W = SweepWidth<T>::value;
    if (k.pitch < W + 8 || p.nx < 8 || p.ny < 8) return DDCC_OK;   // tile kernel for tiny grids
    int dev = 0, optin = 0, sms = 0;
    DDCC_CU(cudaGetDevice(&dev));
    DDCC_CU(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    DDCC_CU(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const bool tf = k.has_cos_field != 0;
    if (sweep_smem_bytes<T>(N, tf) > (size_t)optin) return DDCC_OK;
    for (int c = 0; c < 2; ++c) {
        if (!encode_planes<T>(&h->tm_pop[c], f.f[c], k, 9 * N, 9 * N)) return DDCC_OK;
        if (!encode_planes<T>(&h->tm_lag[c], f.lag[c], k, lag_planes(N), lag_planes(N))) return DDCC_OK;
    }
    const int nst = tf ? N : 1;
    if (!encode_planes<T>(&h->tm_st, f.psi, k, nst, nst)) return DDCC_OK;
    h->plan = make_plan(p.nx, p.ny, W, sms);
    h->use_sweep = 1;
    return DDCC_OK;
}

// Tensor maps of the TMA-staged tile kernel (tile path).
template <typename T>
int setup_tile_tma(ddcc_handle* h) {
    const ddcc_params& p = h->prm;
    const int N = p.nphase;
    KParams<T>& k = kp_of<T>(h);
    Fields<T>& f = fd_of<T>(h);
    h->use_tile_tma = 0;
    if (k.pitch < kTileHaloW) return DDCC_OK;                  // plain-load tile kernel
    int dev = 0, optin = 0;
    DDCC_CU(cudaGetDevice(&dev));
    DDCC_CU(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    const bool tf = k.has_cos_field != 0;
    if (tile_tma_smem_bytes<T>(N, tf) > (size_t)optin) return DDCC_OK;
    const int nst = tf ? N : 1;
    for (int c = 0; c < 2; ++c) {
        if (!encode_box<T>(&h->tt_pop[c], f.f[c], k, 9 * N, kTileX, kTileY, 9 * N)) return DDCC_OK;
        if (!encode_box<T>(&h->tt_lag[c], f.lag[c], k, lag_planes(N), kTileX, kTileY, lag_planes(N)))
            return DDCC_OK;
        if (!encode_box<T>(&h->tt_a[c], f.lag[c], k, lag_planes(N), kTileHaloW, kTileY + 2, 1)) return DDCC_OK;
    }
    if (!encode_box<T>(&h->tt_c, f.C, k, N - 1, kTileHaloW, kTileY + 4, N - 1)) return DDCC_OK;
    if (!encode_box<T>(&h->tt_st, f.psi, k, nst, kTileHaloW, kTileY + 4, nst)) return DDCC_OK;
    h->use_tile_tma = 1;
#ifndef DDCC_TILE_UNFUSED
    if (tile_fused_smem_bytes<T>(N, tf) > (size_t)optin) return DDCC_OK;
    for (int c = 0; c < 2; ++c) {
        if (!encode_box<T>(&h->tt_fh[c], f.f[c], k, 9 * (N - 1), kTileHaloW, kTileY + 4, 9 * (N - 1)))
            return DDCC_OK;
        if (!encode_box<T>(&h->tt_g[c], f.g[c], k, 9, kTileX, kTileY, 9)) return DDCC_OK;
    }
    h->use_tile_tma = 2;
#endif
    return DDCC_OK;
}

template <typename T>
int upload(ddcc_handle* h, const double* host, T* dst, int planes) {
    const ddcc_params& p = h->prm;
    Fields<T>& f = fd_of<T>(h);
    const KParams<T>& k = kp_of<T>(h);
    const size_t bytes = sizeof(double) * (size_t)p.nx * p.ny * planes;
    DDCC_CU(cudaMemcpyAsync(f.stage, host, bytes, cudaMemcpyHostToDevice, h->stream));
    DDCC_CU(launch_convert<T>(f.stage, dst, k, planes, h->stream));
    return DDCC_OK;
}

template <typename T>
int create_t(ddcc_handle* h, const double* psi, const double* cosf, const double* cosu,
             const double* C0, int n_walls = 0, const double* wall_psi = nullptr,
             const double* wall_cos = nullptr) {
    const ddcc_params& p = h->prm;
    const int N = p.nphase;
    KParams<T>& k = kp_of<T>(h);
    Fields<T>& f = fd_of<T>(h);
    fill_kparams<T>(&p, k);
    int st;
    if (n_walls > 0) {
        // psi = prod_k psi_k and e_j = sum_k cos(theta^k_jN) |grad psi_k| in
        // the angle planes; each solid is staged in the read-out scratch
        k.has_cos_field = 1;
        k.wet_field = 1;
        DDCC_CU(launch_walls_init<T>(k, f.psi, f.cosf, h->stream));
        const size_t plane = (size_t)p.nx * p.ny;
        for (int w = 0; w < n_walls; ++w) {
            if ((st = upload<T>(h, wall_psi + w * plane, f.macro, 1))) return st;
            if ((st = upload<T>(h, wall_cos + w * plane * (N - 1), f.macro + k.plane, N - 1))) return st;
            DDCC_CU(launch_fill_ghosts<T>(f.macro, 1, k, h->stream, 1, 1));
            DDCC_CU(launch_wall_accumulate<T>(k, f.macro, f.psi, f.cosf, h->stream));
        }
    } else {
        k.has_cos_field = cosf ? 1 : 0;
        for (int i = 0; i < N - 1; ++i) k.cos_uni[i] = cosf ? T(0) : (T)cosu[i];
        if ((st = upload<T>(h, psi, f.psi, 1))) return st;
        if (cosf && (st = upload<T>(h, cosf, f.cosf, N - 1))) return st;
    }
    DDCC_CU(launch_fill_ghosts<T>(f.psi, k.has_cos_field ? N : 1, k, h->stream));
    st = upload<T>(h, C0, f.C, N - 1);
    if (st) return st;
    DDCC_CU(launch_init<T>(k, f, 0, h->stream));
    DDCC_CU(launch_fill_ghosts<T>(f.f[0], 9 * N, k, h->stream));
    DDCC_CU(launch_fill_ghosts<T>(f.lag[0], lag_planes(N), k, h->stream));
    const int st2 = setup_sweep<T>(h);
    if (st2) return st2;
    return h->use_sweep ? DDCC_OK : setup_tile_tma<T>(h);
}

template <typename T>
int step_plain(ddcc_handle* h, int64_t n) {
    KParams<T>& k = kp_of<T>(h);
    Fields<T>& f = fd_of<T>(h);
    const int N = h->prm.nphase;
    for (int64_t s = 0; s < n; ++s) {
        const int c = h->cur;
        int st;
        if (h->use_sweep) {
            SweepArgs<T> a{&h->tm_pop[c], &h->tm_lag[c], &h->tm_st, &k, f.f[1 - c], f.lag[1 - c],
                           f.flag, h->plan};
            if ((st = prof_begin(h, 2))) return st;
            DDCC_CU(launch_sweep<T>(a, h->stream));
            if ((st = prof_end(h))) return st;
        } else if (h->use_tile_tma == 2) {
            TileTmaArgs<T> a{&h->tt_fh[c], &h->tt_g[c], &h->tt_lag[c], &h->tt_c, &h->tt_st, &h->tt_a[c], &k,
                             f.f[1 - c], f.lag[1 - c], f.flag};
            if ((st = prof_begin(h, 1))) return st;
            DDCC_CU(launch_collide_fused<T>(a, h->stream));
            if ((st = prof_end(h))) return st;
            if (h->prm.flags & DDCC_FLAG_OPEN_X)
                DDCC_CU(launch_open_bc<T>(k, f.f[1 - c], f.lag[1 - c], f.psi, f.inflow, h->stream));
            // the next step's halo boxes read the ghost frames of f and a
            if ((st = prof_begin(h, 3))) return st;
            DDCC_CU(launch_fill_ghosts2<T>(GhostRing<T>{f.f[1 - c], 9 * (N - 1), kFusedGhostF, kFusedGhostF},
                                           GhostRing<T>{f.lag[1 - c], 1, kFusedGhostA, kFusedGhostA}, k,
                                           h->stream));
            if ((st = prof_end(h))) return st;
        } else {
            if ((st = prof_begin(h, 0))) return st;
            DDCC_CU(launch_order_param<T>(k, f, c, h->stream));
            if ((st = prof_end(h))) return st;
            if (h->use_tile_tma) {
                // the C and a halo boxes read the ghost frame
                if ((st = prof_begin(h, 3))) return st;
                DDCC_CU(launch_fill_ghosts<T>(f.C, N - 1, k, h->stream));
                if ((st = prof_end(h))) return st;
                TileTmaArgs<T> a{&h->tt_pop[c], nullptr, &h->tt_lag[c], &h->tt_c, &h->tt_st, &h->tt_a[c],
                                 &k, f.f[1 - c], f.lag[1 - c], f.flag};
                if ((st = prof_begin(h, 1))) return st;
                DDCC_CU(launch_collide_tma<T>(a, h->stream));
                if ((st = prof_end(h))) return st;
                if (h->prm.flags & DDCC_FLAG_OPEN_X)
                    DDCC_CU(launch_open_bc<T>(k, f.f[1 - c], f.lag[1 - c], f.psi, f.inflow, h->stream));
                if ((st = prof_begin(h, 3))) return st;
                DDCC_CU(launch_fill_ghosts<T>(f.lag[1 - c], 1, k, h->stream));
                if ((st = prof_end(h))) return st;
            } else {
                if ((st = prof_begin(h, 1))) return st;
                DDCC_CU(launch_collide<T>(k, f, c, h->stream));
                if ((st = prof_end(h))) return st;
                if (h->prm.flags & DDCC_FLAG_OPEN_X)
                    DDCC_CU(launch_open_bc<T>(k, f.f[1 - c], f.lag[1 - c], f.psi, f.inflow, h->stream));
            }
        }
        h->cur = 1 - c;
        ++h->steps;
    }
    return DDCC_OK;
}

// The fused tile step's launches of two consecutive steps (copy 0 -> 1 -> 0)
// captured once into a CUDA graph on a private stream (the caller's stream
// may be the legacy default stream, which cannot be captured).  The kernels
// take the tensor maps and the parameters by value and the workspace never
// moves, so the graph stays valid for the handle's life.  Any failure leaves
// the plain launches in use.
template <typename T>
void build_step_graph(ddcc_handle* h) {
    h->graph_state = -1;
    cudaStream_t cs = nullptr;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return;
    const cudaStream_t user = h->stream;
    const int cur = h->cur;
    const int64_t steps = h->steps;
    h->stream = cs;
    h->cur = 0;
    cudaGraph_t g = nullptr;
    int rc = DDCC_ERR_CUDA;
    if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
        rc = step_plain<T>(h, 2);
        if (cudaStreamEndCapture(cs, &g) != cudaSuccess) rc = DDCC_ERR_CUDA;
    }
    h->stream = user;
    h->cur = cur;
    h->steps = steps;
    if (rc == DDCC_OK && g && cudaGraphInstantiate(&h->step_graph, g, 0) == cudaSuccess) h->graph_state = 1;
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cs);
    cudaGetLastError();   // a refused capture leaves no sticky error behind
}

template <typename T>
int step_t(ddcc_handle* h, int64_t n) {
    if (h->profiling || h->use_sweep || h->use_tile_tma != 2 || n < 4) return step_plain<T>(h, n);
    if (h->graph_state == 0) build_step_graph<T>(h);
    if (h->graph_state != 1) return step_plain<T>(h, n);
    int st;
    if (h->cur == 1) {
        if ((st = step_plain<T>(h, 1))) return st;
        --n;
    }
    for (int64_t i = 0; i < n / 2; ++i) DDCC_CU(cudaGraphLaunch(h->step_graph, h->stream));
    h->steps += 2 * (n / 2);
    return (n % 2) ? step_plain<T>(h, 1) : DDCC_OK;
}

// Error word of the kernels: bounded waits that ran out.
// A loaded state may come from a handle whose last step left the ghost frames
// of the population planes stale; the tile kernels read them, so refresh.
template <typename T>
int refresh_ghosts_t(ddcc_handle* h) {
    KParams<T>& k = kp_of<T>(h);
    Fields<T>& f = fd_of<T>(h);
    const int N = h->prm.nphase;
    DDCC_CU(launch_fill_ghosts<T>(f.f[h->cur], 9 * N, k, h->stream));
    DDCC_CU(launch_fill_ghosts<T>(f.lag[h->cur], lag_planes(N), k, h->stream));
    return DDCC_OK;
}

template <typename T>
int check_flag(ddcc_handle* h) {
    int flag = 0;
    DDCC_CU(cudaMemcpyAsync(&flag, fd_of<T>(h).flag, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    DDCC_CU(cudaStreamSynchronize(h->stream));
    return flag ? DDCC_ERR_TIMEOUT : DDCC_OK;
}

template <typename T>
int read_t(ddcc_handle* h, int field, double* out) {
    const ddcc_params& p = h->prm;
    const int N = p.nphase;
    KParams<T>& k = kp_of<T>(h);
    Fields<T>& f = fd_of<T>(h);
    const T* src = nullptr;
    if (field == DDCC_FIELD_PSI) {
        src = f.psi;
    } else {
        int plane = -1;
        if (field >= DDCC_FIELD_C && field < DDCC_FIELD_C + N) plane = field - DDCC_FIELD_C;
        else if (field == DDCC_FIELD_RHO) plane = N;
        else if (field == DDCC_FIELD_UX) plane = N + 1;
        else if (field == DDCC_FIELD_UY) plane = N + 2;
        else if (field == DDCC_FIELD_P) plane = N + 3;
        else if (field >= DDCC_FIELD_MU && field < DDCC_FIELD_MU + N) plane = N + 4 + field - DDCC_FIELD_MU;
        if (plane < 0) return DDCC_ERR_PARAM;
        if (!h->macro_valid) {
            DDCC_CU(launch_macro<T>(k, f, h->cur, h->stream));
            h->macro_valid = 1;
        }
        src = f.macro + (size_t)plane * k.plane;
    }
    DDCC_CU(launch_export<T>(src, f.stage, k, h->stream));
    DDCC_CU(cudaMemcpyAsync(out, f.stage, sizeof(double) * (size_t)p.nx * p.ny,
                            cudaMemcpyDeviceToHost, h->stream));
    DDCC_CU(cudaStreamSynchronize(h->stream));
    return check_flag<T>(h);
}

template <typename T>
int mass_t(ddcc_handle* h, double* out) {
    const int N = h->prm.nphase;
    KParams<T>& k = kp_of<T>(h);
    Fields<T>& f = fd_of<T>(h);
    DDCC_CU(launch_mass<T>(k, f, h->cur, h->dev_mass, h->stream));
    DDCC_CU(cudaMemcpyAsync(out, h->dev_mass, sizeof(double) * (N - 1), cudaMemcpyDeviceToHost,
                            h->stream));
    DDCC_CU(cudaStreamSynchronize(h->stream));
    const int st = check_flag<T>(h);
    if (st) return st;
    for (int i = 0; i < N - 1; ++i)
        if (!std::isfinite(out[i])) return DDCC_ERR_NONFINITE;
    return DDCC_OK;
}

// State = [int64 steps, padding to 256 bytes][populations][lagged] of the
// current copy (whole planes, ghost frame included).
size_t state_payload(const ddcc_handle* h, size_t* pb, size_t* lb) {
    const Layout L = layout_of(&h->prm);
    const int N = h->prm.nphase;
    *pb = L.plane_bytes * 9 * N;
    *lb = L.plane_bytes * lag_planes(N);
    return kAlign + *pb + *lb;
}

// Adjoint scratch: the planes of one reverse step, then the centroid
// reduction's block partials and its (J, M) pair.
size_t adjoint_planes_bytes(const ddcc_handle* h) {
    const Layout L = layout_of(&h->prm);
    const size_t planes = h->prm.precision == DDCC_FP64 ? adjoint_scratch_planes<double>(h->prm.nphase)
                                                        : adjoint_scratch_planes<float>(h->prm.nphase);
    return L.plane_bytes * planes;
}
size_t adjoint_total_bytes(const ddcc_handle* h) {
    return adjoint_planes_bytes(h) + align_up(sizeof(double) * 2 * kMassBlocks, kAlign) + kAlign;
}

bool adjoint_scratch_ok(const ddcc_handle* h, const void* scratch, size_t bytes) {
    return scratch && bytes >= adjoint_total_bytes(h) && reinterpret_cast<uintptr_t>(scratch) % kAlign == 0;
}

template <typename T>
AdjStepArgs<T> adjoint_args(ddcc_handle* h, void* scratch, double* dJ_dcos, double* dJ_dpsi) {
    Fields<T>& f = fd_of<T>(h);
    KParams<T>& k = kp_of<T>(h);
    AdjStepArgs<T> a{};
    a.kp = &k;
    a.psi = f.psi;
    a.cosf = k.has_cos_field ? f.cosf : nullptr;
    a.scratch = static_cast<T*>(scratch);
    a.dJ_dcos = dJ_dcos;
    a.dJ_dpsi = dJ_dpsi;
    return a;
}

template <typename T>
int adjoint_step_t(ddcc_handle* h, const void* state_n, const void* adj_next, void* adj_out, void* scratch,
                   double* dJ_dcos, double* dJ_dpsi) {
    size_t pb, lb;
    state_payload(h, &pb, &lb);
    AdjStepArgs<T> a = adjoint_args<T>(h, scratch, dJ_dcos, dJ_dpsi);
    const char* sn = static_cast<const char*>(state_n);
    const char* ai = static_cast<const char*>(adj_next);
    char* ao = static_cast<char*>(adj_out);
    a.st_pop = reinterpret_cast<const T*>(sn + kAlign);
    a.st_lag = reinterpret_cast<const T*>(sn + kAlign + pb);
    a.ad_pop_in = reinterpret_cast<const T*>(ai + kAlign);
    a.ad_lag_in = reinterpret_cast<const T*>(ai + kAlign + pb);
    a.ad_pop_out = reinterpret_cast<T*>(ao + kAlign);
    a.ad_lag_out = reinterpret_cast<T*>(ao + kAlign + pb);
    DDCC_CU(launch_adjoint_step<T>(a, h->stream));
    return DDCC_OK;
}

template <typename T>
int adjoint_initial_t(ddcc_handle* h, const double* C0, const void* adj0, void* scratch, double* dJ_dcos,
                      double* dJ_dpsi) {
    AdjStepArgs<T> a = adjoint_args<T>(h, scratch, dJ_dcos, dJ_dpsi);
    const char* ai = static_cast<const char*>(adj0);
    a.ad_pop_in = reinterpret_cast<const T*>(ai + kAlign);
    const int st = upload<T>(h, C0, adjoint_c_planes<T>(a.scratch), h->prm.nphase - 1);
    if (st) return st;
    DDCC_CU(launch_adjoint_initial<T>(a, h->stream));
    return DDCC_OK;
}

// One step of the fused tile path from the state in state_in to state_out
// (both in the saved-state layout), through tensor maps of those buffers.
template <typename T>
int step_between_t(ddcc_handle* h, const void* state_in, void* state_out) {
    if (h->use_sweep || h->use_tile_tma != 2 || (h->prm.flags & DDCC_FLAG_OPEN_X)) return DDCC_ERR_UNSUPPORTED;
    KParams<T>& k = kp_of<T>(h);
    Fields<T>& f = fd_of<T>(h);
    const int N = h->prm.nphase;
    size_t pb, lb;
    state_payload(h, &pb, &lb);
    const T* in_pop = reinterpret_cast<const T*>(static_cast<const char*>(state_in) + kAlign);
    const T* in_lag = reinterpret_cast<const T*>(static_cast<const char*>(state_in) + kAlign + pb);
    T* out_pop = reinterpret_cast<T*>(static_cast<char*>(state_out) + kAlign);
    T* out_lag = reinterpret_cast<T*>(static_cast<char*>(state_out) + kAlign + pb);
    CUtensorMap fh, g, lag, am;
    if (!encode_box<T>(&fh, in_pop, k, 9 * (N - 1), kTileHaloW, kTileY + 4, 9 * (N - 1)) ||
        !encode_box<T>(&g, in_pop + (size_t)9 * (N - 1) * k.plane, k, 9, kTileX, kTileY, 9) ||
        !encode_box<T>(&lag, in_lag, k, lag_planes(N), kTileX, kTileY, lag_planes(N)) ||
        !encode_box<T>(&am, in_lag, k, lag_planes(N), kTileHaloW, kTileY + 2, 1))
        return DDCC_ERR_CUDA;
    TileTmaArgs<T> a{&fh, &g, &lag, &h->tt_c, &h->tt_st, &am, &k, out_pop, out_lag, f.flag};
    DDCC_CU(launch_collide_fused<T>(a, h->stream));
    DDCC_CU(launch_fill_ghosts2<T>(GhostRing<T>{out_pop, 9 * (N - 1), kFusedGhostF, kFusedGhostF},
                                   GhostRing<T>{out_lag, 1, kFusedGhostA, kFusedGhostA}, k, h->stream));
    return DDCC_OK;
}

template <typename T>
int centroid_t(ddcc_handle* h, int phase, void* scratch, double* J_out, void* adj_seed) {
    Fields<T>& f = fd_of<T>(h);
    KParams<T>& k = kp_of<T>(h);
    char* sc = static_cast<char*>(scratch) + adjoint_planes_bytes(h);
    double* part = reinterpret_cast<double*>(sc);
    double* JM = reinterpret_cast<double*>(sc + align_up(sizeof(double) * 2 * kMassBlocks, kAlign));
    T* seed = nullptr;
    if (adj_seed) {
        size_t pb, lb;
        const size_t total = state_payload(h, &pb, &lb);
        DDCC_CU(cudaMemsetAsync(adj_seed, 0, total, h->stream));
        seed = reinterpret_cast<T*>(static_cast<char*>(adj_seed) + kAlign) + (size_t)9 * phase * k.plane;
    }
    DDCC_CU(launch_centroid<T>(k, f.f[h->cur] + (size_t)9 * phase * k.plane, part, JM, seed, h->stream));
    DDCC_CU(cudaMemcpyAsync(J_out, JM, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    DDCC_CU(cudaStreamSynchronize(h->stream));
    return check_flag<T>(h);
}

int create_handle(const ddcc_params* params, void* dev_workspace, size_t bytes, void* cuda_stream,
                  const double* psi, const double* cos_theta_field, const double* cos_theta_uniform,
                  const double* C0, int n_walls, const double* wall_psi, const double* wall_cos,
                  ddcc_handle** out);

}  // namespace

extern "C" {

size_t ddcc_workspace_bytes(const ddcc_params* params) {
    if (!valid_params(params)) return 0;
    return layout_of(params).total;
}

}  // extern "C"

namespace {

// Every value in (0, 1] (NaN fails).  Branch-free within blocks so that the
// compiler can vectorise the scan of a whole plane.
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

}  // namespace

extern "C" {

int ddcc_create(const ddcc_params* params, void* dev_workspace, size_t bytes, void* cuda_stream,
                const double* psi, const double* cos_theta_field,
                const double* cos_theta_uniform, const double* C0, ddcc_handle** out) {
    if (!out) return DDCC_ERR_PARAM;
    *out = nullptr;
    if (!valid_params(params) || !psi || !C0) return DDCC_ERR_PARAM;
    if (!cos_theta_field && !cos_theta_uniform) return DDCC_ERR_PARAM;
    if (!all_in_unit(psi, (long long)params->nx * params->ny)) return DDCC_ERR_PARAM;
    return create_handle(params, dev_workspace, bytes, cuda_stream, psi, cos_theta_field, cos_theta_uniform,
                         C0, 0, nullptr, nullptr, out);
}

int ddcc_create_walls(const ddcc_params* params, void* dev_workspace, size_t bytes, void* cuda_stream,
                      int n_walls, const double* wall_psi, const double* wall_cos_theta, const double* C0,
                      ddcc_handle** out) {
    if (!out) return DDCC_ERR_PARAM;
    *out = nullptr;
    if (!valid_params(params) || !wall_psi || !wall_cos_theta || !C0) return DDCC_ERR_PARAM;
    if (n_walls < 1 || n_walls > DDCC_MAX_WALLS) return DDCC_ERR_PARAM;
    const long long n = (long long)params->nx * params->ny;
    if (!all_in_unit(wall_psi, n * n_walls)) return DDCC_ERR_PARAM;
    for (long long i = 0; i < n * n_walls * (params->nphase - 1); ++i)
        if (!std::isfinite(wall_cos_theta[i])) return DDCC_ERR_PARAM;
    return create_handle(params, dev_workspace, bytes, cuda_stream, nullptr, nullptr, nullptr, C0, n_walls,
                         wall_psi, wall_cos_theta, out);
}

}  // extern "C"

namespace {
int create_handle(const ddcc_params* params, void* dev_workspace, size_t bytes, void* cuda_stream,
                  const double* psi, const double* cos_theta_field, const double* cos_theta_uniform,
                  const double* C0, int n_walls, const double* wall_psi, const double* wall_cos,
                  ddcc_handle** out) {
    const Layout L = layout_of(params);
    if (!dev_workspace || bytes < L.total || (reinterpret_cast<uintptr_t>(dev_workspace) % kAlign))
        return DDCC_ERR_WORKSPACE;
    ddcc_handle* h = new (std::nothrow) ddcc_handle();
    if (!h) return DDCC_ERR_NOMEM;
    h->prm = *params;
    h->stream = static_cast<cudaStream_t>(cuda_stream);
    h->ws = static_cast<char*>(dev_workspace);
    h->ws_bytes = bytes;
    h->cur = 0;
    h->steps = 0;
    h->dev_mass = reinterpret_cast<double*>(h->ws + L.mass);
    h->n_walls = n_walls;
    if (cudaMemsetAsync(h->ws, 0, L.total, h->stream) != cudaSuccess) {
        delete h;
        return DDCC_ERR_CUDA;
    }
    int st;
    if (params->precision == DDCC_FP64) {
        carve<double>(h, L, h->fd);
        st = create_t<double>(h, psi, cos_theta_field, cos_theta_uniform, C0, n_walls, wall_psi, wall_cos);
    } else {
        carve<float>(h, L, h->ff);
        st = create_t<float>(h, psi, cos_theta_field, cos_theta_uniform, C0, n_walls, wall_psi, wall_cos);
    }
    if (st == DDCC_OK && cudaStreamSynchronize(h->stream) != cudaSuccess) st = DDCC_ERR_CUDA;
    if (st != DDCC_OK) {
        delete h;
        return st;
    }
    *out = h;
    return DDCC_OK;
}
}  // namespace

namespace ddcc {
// ddcc_slab.cu: rows [y0, y0 + n) of npop population planes at pop and nlag
// lagged planes at lag, x in [0, nx), to (to_buf != 0) or from a dense
// buffer [plane][row][x].
template <typename T>
cudaError_t launch_rows_copy(T* pop, T* lag, int npop, int nlag, const KParams<T>& kp, int y0, int n, T* buf,
                             int to_buf, cudaStream_t s);
}  // namespace ddcc

namespace {
template <typename T>
int rows_t(ddcc_handle* h, int y0, int nrows, void* buf, int to_buf) {
    KParams<T>& k = kp_of<T>(h);
    Fields<T>& f = fd_of<T>(h);
    const int N = h->prm.nphase;
    DDCC_CU(launch_rows_copy<T>(f.f[h->cur], f.lag[h->cur], 9 * N, lag_planes(N), k, y0, nrows,
                                static_cast<T*>(buf), to_buf, h->stream));
    if (!to_buf) return refresh_ghosts_t<T>(h);
    return DDCC_OK;
}
bool rows_ok(const ddcc_handle* h, int y0, int nrows, const void* buf) {
    return h && buf && nrows > 0 && y0 >= 0 && y0 + nrows <= h->prm.ny;
}
}  // namespace

extern "C" {

int ddcc_step(ddcc_handle* h, int64_t nsteps) {
    if (!h || nsteps < 0) return DDCC_ERR_PARAM;
    h->macro_valid = 0;
    return h->prm.precision == DDCC_FP64 ? step_t<double>(h, nsteps) : step_t<float>(h, nsteps);
}

int ddcc_read(ddcc_handle* h, int field, double* host_out) {
    if (!h || !host_out) return DDCC_ERR_PARAM;
    return h->prm.precision == DDCC_FP64 ? read_t<double>(h, field, host_out)
                                         : read_t<float>(h, field, host_out);
}

int ddcc_mass(ddcc_handle* h, double* host_out) {
    if (!h || !host_out) return DDCC_ERR_PARAM;
    return h->prm.precision == DDCC_FP64 ? mass_t<double>(h, host_out) : mass_t<float>(h, host_out);
}

size_t ddcc_state_bytes(const ddcc_handle* h) {
    if (!h) return 0;
    size_t a, b;
    return state_payload(h, &a, &b);
}

int ddcc_save_state(ddcc_handle* h, void* buf, int on_device) {
    if (!h || !buf) return DDCC_ERR_PARAM;
    size_t pb, lb;
    state_payload(h, &pb, &lb);
    const Layout L = layout_of(&h->prm);
    char* dst = static_cast<char*>(buf);
    const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (on_device) {
        DDCC_CU(cudaMemcpyAsync(dst, &h->steps, sizeof(int64_t), cudaMemcpyHostToDevice, h->stream));
        DDCC_CU(cudaStreamSynchronize(h->stream));   // &h->steps is pageable host memory
    } else {
        std::memcpy(dst, &h->steps, sizeof(int64_t));
    }
    DDCC_CU(cudaMemcpyAsync(dst + kAlign, h->ws + L.pop[h->cur], pb, k, h->stream));
    DDCC_CU(cudaMemcpyAsync(dst + kAlign + pb, h->ws + L.lag[h->cur], lb, k, h->stream));
    if (!on_device) DDCC_CU(cudaStreamSynchronize(h->stream));
    return DDCC_OK;
}

int ddcc_load_state(ddcc_handle* h, const void* buf, int on_device) {
    if (!h || !buf) return DDCC_ERR_PARAM;
    h->macro_valid = 0;
    size_t pb, lb;
    state_payload(h, &pb, &lb);
    const Layout L = layout_of(&h->prm);
    const char* src = static_cast<const char*>(buf);
    const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    int64_t steps = 0;
    if (on_device) {
        DDCC_CU(cudaMemcpyAsync(&steps, src, sizeof(int64_t), cudaMemcpyDeviceToHost, h->stream));
        DDCC_CU(cudaStreamSynchronize(h->stream));
    } else {
        std::memcpy(&steps, src, sizeof(int64_t));
    }
    if (steps < 0) return DDCC_ERR_PARAM;
    DDCC_CU(cudaMemcpyAsync(h->ws + L.pop[h->cur], src + kAlign, pb, k, h->stream));
    DDCC_CU(cudaMemcpyAsync(h->ws + L.lag[h->cur], src + kAlign + pb, lb, k, h->stream));
    const int st = h->prm.precision == DDCC_FP64 ? refresh_ghosts_t<double>(h) : refresh_ghosts_t<float>(h);
    if (st) return st;
    if (!on_device) DDCC_CU(cudaStreamSynchronize(h->stream));
    h->steps = steps;
    return DDCC_OK;
}

int64_t ddcc_step_count(const ddcc_handle* h) { return h ? h->steps : -1; }

size_t ddcc_rows_bytes(const ddcc_handle* h, int nrows) {
    if (!h || nrows <= 0) return 0;
    const int N = h->prm.nphase;
    const size_t es = h->prm.precision == DDCC_FP64 ? sizeof(double) : sizeof(float);
    return es * (size_t)(9 * N + lag_planes(N)) * (size_t)nrows * (size_t)h->prm.nx;
}

int ddcc_get_rows(ddcc_handle* h, int y0, int nrows, void* dev_buf) {
    if (!rows_ok(h, y0, nrows, dev_buf)) return DDCC_ERR_PARAM;
    return h->prm.precision == DDCC_FP64 ? rows_t<double>(h, y0, nrows, dev_buf, 1)
                                         : rows_t<float>(h, y0, nrows, dev_buf, 1);
}

int ddcc_set_rows(ddcc_handle* h, int y0, int nrows, const void* dev_buf) {
    if (!rows_ok(h, y0, nrows, dev_buf)) return DDCC_ERR_PARAM;
    h->macro_valid = 0;
    void* b = const_cast<void*>(dev_buf);   // read only (to_buf = 0)
    return h->prm.precision == DDCC_FP64 ? rows_t<double>(h, y0, nrows, b, 0) : rows_t<float>(h, y0, nrows, b, 0);
}

int ddcc_set_inflow(ddcc_handle* h, const double* u_in, const double* C_in) {
    if (!h || !u_in || !C_in || !(h->prm.flags & DDCC_FLAG_OPEN_X)) return DDCC_ERR_PARAM;
    h->macro_valid = 0;
    const int ny = h->prm.ny, N = h->prm.nphase;
    std::vector<double> buf((size_t)ny * N);
    for (int y = 0; y < ny; ++y) buf[y] = u_in[y];
    for (size_t i = 0; i < (size_t)ny * (N - 1); ++i) buf[ny + i] = C_in[i];
    for (double v : buf)
        if (!std::isfinite(v)) return DDCC_ERR_PARAM;
    if (h->prm.precision == DDCC_FP64) {
        DDCC_CU(cudaMemcpyAsync(h->fd.inflow, buf.data(), sizeof(double) * buf.size(), cudaMemcpyHostToDevice,
                                h->stream));
    } else {
        std::vector<float> bf(buf.begin(), buf.end());
        DDCC_CU(cudaMemcpyAsync(h->ff.inflow, bf.data(), sizeof(float) * bf.size(), cudaMemcpyHostToDevice,
                                h->stream));
    }
    DDCC_CU(cudaStreamSynchronize(h->stream));   // the host vectors go out of scope
    return DDCC_OK;
}

int ddcc_step_between(ddcc_handle* h, const void* state_in, void* state_out) {
    if (!h || !state_in || !state_out || state_in == state_out) return DDCC_ERR_PARAM;
    h->macro_valid = 0;
    if ((reinterpret_cast<uintptr_t>(state_in) | reinterpret_cast<uintptr_t>(state_out)) % kAlign)
        return DDCC_ERR_PARAM;
    return h->prm.precision == DDCC_FP64 ? step_between_t<double>(h, state_in, state_out)
                                         : step_between_t<float>(h, state_in, state_out);
}

size_t ddcc_adjoint_bytes(const ddcc_handle* h) { return h ? adjoint_total_bytes(h) : 0; }

int ddcc_adjoint_step(ddcc_handle* h, const void* state_n, const void* adj_next, void* adj_out, void* scratch,
                      size_t scratch_bytes, double* dJ_dcos, double* dJ_dpsi) {
    if (!h || !state_n || !adj_next || !adj_out || adj_next == adj_out || !dJ_dcos || !dJ_dpsi)
        return DDCC_ERR_PARAM;
    h->macro_valid = 0;
    if (h->n_walls || (h->prm.flags & DDCC_FLAG_OPEN_X)) return DDCC_ERR_UNSUPPORTED;
    if (!adjoint_scratch_ok(h, scratch, scratch_bytes)) return DDCC_ERR_WORKSPACE;
    return h->prm.precision == DDCC_FP64
               ? adjoint_step_t<double>(h, state_n, adj_next, adj_out, scratch, dJ_dcos, dJ_dpsi)
               : adjoint_step_t<float>(h, state_n, adj_next, adj_out, scratch, dJ_dcos, dJ_dpsi);
}

}  // extern "C"

namespace {

// The launches of one reverse segment: the states 1..n-1 recomputed from
// states[0] (own), then the n reverse steps.  With n_next > 1 the states
// 1..n_next-1 of the next segment to reverse are recomputed from next[0]
// on the handle's second stream, forked from its stream before the reverse
// steps and joined after them; the two touch no common buffer, so the
// recompute runs in the gaps the reverse kernels leave on the GPU.
int segment_launches(ddcc_handle* h, const void* const* states, int n, bool own, const void* const* next,
                     int n_next, void* adj_cur, void* adj_other, void* scratch, double* dJ_dcos,
                     double* dJ_dpsi) {
    const bool f64 = h->prm.precision == DDCC_FP64;
    auto recompute = [&](const void* const* st, int m) {
        for (int s = 1; s < m; ++s) {
            const int r = f64 ? step_between_t<double>(h, st[s - 1], const_cast<void*>(st[s]))
                              : step_between_t<float>(h, st[s - 1], const_cast<void*>(st[s]));
            if (r) return r;
        }
        return static_cast<int>(DDCC_OK);
    };
    int st = own ? recompute(states, n) : static_cast<int>(DDCC_OK);
    if (st) return st;
    const bool fork = n_next > 1;
    if (fork) {
        DDCC_CU(cudaEventRecord(h->fork_ev, h->stream));
        DDCC_CU(cudaStreamWaitEvent(h->side, h->fork_ev, 0));
        const cudaStream_t main = h->stream;
        h->stream = h->side;
        st = recompute(next, n_next);
        h->stream = main;
        DDCC_CU(cudaEventRecord(h->join_ev, h->side));
    }
    void* cur = adj_cur;
    void* nxt = adj_other;
    for (int s = n - 1; s >= 0 && st == DDCC_OK; --s) {
        st = f64 ? adjoint_step_t<double>(h, states[s], cur, nxt, scratch, dJ_dcos, dJ_dpsi)
                 : adjoint_step_t<float>(h, states[s], cur, nxt, scratch, dJ_dcos, dJ_dpsi);
        void* t = cur;
        cur = nxt;
        nxt = t;
    }
    if (fork) DDCC_CU(cudaStreamWaitEvent(h->stream, h->join_ev, 0));
    return st;
}

// A segment's launches captured into a graph on a private stream (null
// when the capture is refused; the plain launches then stay in use).
template <class L>
cudaGraphExec_t capture_segment(ddcc_handle* h, L launches) {
    cudaStream_t cs = nullptr;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return nullptr;
    const cudaStream_t user = h->stream;
    h->stream = cs;
    cudaGraph_t g = nullptr;
    int rc = DDCC_ERR_CUDA;
    if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
        rc = launches();
        if (cudaStreamEndCapture(cs, &g) != cudaSuccess) rc = DDCC_ERR_CUDA;
    }
    h->stream = user;
    cudaGraphExec_t exec = nullptr;
    if (rc == DDCC_OK && g && cudaGraphInstantiate(&exec, g, 0) != cudaSuccess) exec = nullptr;
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cs);
    cudaGetLastError();
    return exec;
}

// Run a segment: replay the graph captured for these arguments; capture one
// when the arguments match one of the last two plain calls (a sweep that
// alternates two sets of buffers repeats every other call); else launch
// plainly.  At most four graphs are kept per handle.
template <class L>
int run_segment(ddcc_handle* h, const std::vector<const void*>& key, L launches) {
    if (h->profiling) return launches();
    for (const auto& sg : h->seg_graphs)
        if (sg.key == key) return cudaGraphLaunch(sg.exec, h->stream) == cudaSuccess ? DDCC_OK : DDCC_ERR_CUDA;
    bool seen = false;
    for (const auto& k : h->seg_seen) seen = seen || k == key;
    if (seen) {
        cudaGraphExec_t exec = capture_segment(h, launches);
        if (exec) {
            if (h->seg_graphs.size() >= 4) {
                cudaGraphExecDestroy(h->seg_graphs.front().exec);
                h->seg_graphs.erase(h->seg_graphs.begin());
            }
            h->seg_graphs.push_back({key, exec});
            return cudaGraphLaunch(exec, h->stream) == cudaSuccess ? DDCC_OK : DDCC_ERR_CUDA;
        }
    }
    h->seg_seen.push_back(key);
    if (h->seg_seen.size() > 2) h->seg_seen.erase(h->seg_seen.begin());
    return launches();
}

// The checks every segment call makes; DDCC_OK when the call may proceed.
int segment_args_ok(ddcc_handle* h, void* adj_cur, void* adj_other, void* scratch, size_t scratch_bytes,
                    double* dJ_dcos, double* dJ_dpsi, int* in_other) {
    if (!adj_cur || !adj_other || adj_cur == adj_other || !dJ_dcos || !dJ_dpsi || !in_other)
        return DDCC_ERR_PARAM;
    if (h->n_walls || (h->prm.flags & DDCC_FLAG_OPEN_X)) return DDCC_ERR_UNSUPPORTED;
    if (!adjoint_scratch_ok(h, scratch, scratch_bytes)) return DDCC_ERR_WORKSPACE;
    return DDCC_OK;
}

bool states_ok(const void* const* states, int n) {
    for (int s = 0; s < n; ++s)
        if (!states[s] || reinterpret_cast<uintptr_t>(states[s]) % kAlign) return false;
    return true;
}

}  // namespace

extern "C" {

int ddcc_adjoint_segment(ddcc_handle* h, const void* const* states, int n, void* adj_cur, void* adj_other,
                         void* scratch, size_t scratch_bytes, double* dJ_dcos, double* dJ_dpsi, int* in_other) {
    if (!h || !states || n < 1) return DDCC_ERR_PARAM;
    h->macro_valid = 0;
    int st = segment_args_ok(h, adj_cur, adj_other, scratch, scratch_bytes, dJ_dcos, dJ_dpsi, in_other);
    if (st) return st;
    if (!states_ok(states, n)) return DDCC_ERR_PARAM;
    // the result lands in adj_other when n is odd
    *in_other = n % 2;
    std::vector<const void*> key(states, states + n);
    key.insert(key.end(), {adj_cur, adj_other, scratch, dJ_dcos, dJ_dpsi, nullptr});
    return run_segment(h, key, [&] {
        return segment_launches(h, states, n, true, nullptr, 0, adj_cur, adj_other, scratch, dJ_dcos, dJ_dpsi);
    });
}

int ddcc_adjoint_segment_pipelined(ddcc_handle* h, const void* const* states, int n, const void* const* next,
                                   int n_next, void* adj_cur, void* adj_other, void* scratch,
                                   size_t scratch_bytes, double* dJ_dcos, double* dJ_dpsi, int* in_other) {
    if (!h || n < 0 || n_next < 0 || (n > 0 && !states) || (n_next > 0 && !next)) return DDCC_ERR_PARAM;
    h->macro_valid = 0;
    int st = segment_args_ok(h, adj_cur, adj_other, scratch, scratch_bytes, dJ_dcos, dJ_dpsi, in_other);
    if (st) return st;
    if (!states_ok(states, n) || !states_ok(next, n_next)) return DDCC_ERR_PARAM;
    // the recompute writes next[1..]: no buffer the reverse steps use
    for (int t = 1; t < n_next; ++t) {
        if (next[t] == adj_cur || next[t] == adj_other || next[t] == scratch) return DDCC_ERR_PARAM;
        for (int s = 0; s < n; ++s)
            if (next[t] == states[s]) return DDCC_ERR_PARAM;
    }
    if (n_next > 1 && (h->use_sweep || h->use_tile_tma != 2)) return DDCC_ERR_UNSUPPORTED;
    if (n_next > 1 && !h->side) {
        // all three or none
        cudaStream_t side = nullptr;
        cudaEvent_t fork = nullptr, join = nullptr;
        if (cudaStreamCreateWithFlags(&side, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&fork, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&join, cudaEventDisableTiming) != cudaSuccess) {
            if (side) cudaStreamDestroy(side);
            if (fork) cudaEventDestroy(fork);
            if (join) cudaEventDestroy(join);
            cudaGetLastError();
            return DDCC_ERR_CUDA;
        }
        h->side = side;
        h->fork_ev = fork;
        h->join_ev = join;
    }
    *in_other = n % 2;
    std::vector<const void*> key;
    if (n > 0) key.assign(states, states + n);
    key.push_back(nullptr);
    if (n_next > 0) key.insert(key.end(), next, next + n_next);
    key.insert(key.end(), {adj_cur, adj_other, scratch, dJ_dcos, dJ_dpsi, reinterpret_cast<const void*>(
                                                                              static_cast<uintptr_t>(n))});
    return run_segment(h, key, [&] {
        return segment_launches(h, states, n, false, next, n_next, adj_cur, adj_other, scratch, dJ_dcos,
                                dJ_dpsi);
    });
}

int ddcc_adjoint_initial(ddcc_handle* h, const double* C0, const void* adj0, void* scratch, size_t scratch_bytes,
                         double* dJ_dcos, double* dJ_dpsi) {
    if (!h || !C0 || !adj0 || !dJ_dcos || !dJ_dpsi) return DDCC_ERR_PARAM;
    h->macro_valid = 0;
    if (h->n_walls || (h->prm.flags & DDCC_FLAG_OPEN_X)) return DDCC_ERR_UNSUPPORTED;
    if (!adjoint_scratch_ok(h, scratch, scratch_bytes)) return DDCC_ERR_WORKSPACE;
    return h->prm.precision == DDCC_FP64 ? adjoint_initial_t<double>(h, C0, adj0, scratch, dJ_dcos, dJ_dpsi)
                                         : adjoint_initial_t<float>(h, C0, adj0, scratch, dJ_dcos, dJ_dpsi);
}

int ddcc_objective_centroid(ddcc_handle* h, int phase, void* scratch, size_t scratch_bytes, double* J_out,
                            void* adj_seed) {
    if (!h || !J_out || phase < 0 || phase >= h->prm.nphase - 1) return DDCC_ERR_PARAM;
    h->macro_valid = 0;
    if (!adjoint_scratch_ok(h, scratch, scratch_bytes)) return DDCC_ERR_WORKSPACE;
    return h->prm.precision == DDCC_FP64 ? centroid_t<double>(h, phase, scratch, J_out, adj_seed)
                                         : centroid_t<float>(h, phase, scratch, J_out, adj_seed);
}

int ddcc_profile(ddcc_handle* h, int enable) {
    if (!h) return DDCC_ERR_PARAM;
    h->profiling = enable ? 1 : 0;
    return DDCC_OK;
}

int ddcc_kernel_times(ddcc_handle* h, double* ms_out, int64_t* launches_out, int max_kinds) {
    if (!h || max_kinds < 0) return DDCC_ERR_PARAM;
    DDCC_CU(cudaStreamSynchronize(h->stream));
    double ms[kKinds] = {0.0, 0.0, 0.0, 0.0};
    int64_t cnt[kKinds] = {0, 0, 0, 0};
    for (size_t i = 0; i < h->rec_kind.size(); ++i) {
        float t = 0.f;
        DDCC_CU(cudaEventElapsedTime(&t, h->events[2 * i], h->events[2 * i + 1]));
        ms[h->rec_kind[i]] += t;
        cnt[h->rec_kind[i]] += 1;
    }
    h->rec_kind.clear();
    for (int k2 = 0; k2 < max_kinds && k2 < kKinds; ++k2) {
        if (ms_out) ms_out[k2] = ms[k2];
        if (launches_out) launches_out[k2] = cnt[k2];
    }
    return kKinds;
}

int ddcc_step_path(const ddcc_handle* h) {
    if (!h) return DDCC_ERR_PARAM;
    return h->use_sweep ? DDCC_PATH_SWEEP : DDCC_PATH_TILE;
}

void ddcc_destroy(ddcc_handle* h) {
    if (!h) return;
    if (h->graph_state == 1) cudaGraphExecDestroy(h->step_graph);
    for (const auto& sg : h->seg_graphs) cudaGraphExecDestroy(sg.exec);
    if (h->side) cudaStreamDestroy(h->side);
    if (h->fork_ev) cudaEventDestroy(h->fork_ev);
    if (h->join_ev) cudaEventDestroy(h->join_ev);
    for (cudaEvent_t e : h->events) cudaEventDestroy(e);
    delete h;
}

const char* ddcc_status_string(int status) {
    switch (status) {
        case DDCC_OK: return "ok";
        case DDCC_ERR_PARAM: return "invalid parameter";
        case DDCC_ERR_WORKSPACE: return "workspace missing, too small or misaligned";
        case DDCC_ERR_CUDA: return "CUDA runtime error";
        case DDCC_ERR_NONFINITE: return "non-finite population found";
        case DDCC_ERR_NOMEM: return "host allocation failed";
        case DDCC_ERR_UNSUPPORTED: return "unsupported";
        case DDCC_ERR_TIMEOUT: return "a kernel's bounded wait ran out; state is invalid";
        default: return "unknown status";
    }
}

int ddcc_version(void) { return 200; }

}  // extern "C"
