// Internal declarations shared by the host runtime and the kernels.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

namespace ddcc {

constexpr int kMaxPhases = 4;
constexpr int kTileX = 32;       // threads (and nodes) per tile row
constexpr int kTileY = 8;        // tile rows
constexpr int kMassBlocks = 304; // 2 x 152 SMs
// Ghost frame around every plane: node (x, y) lives at org + y * pitch + x
// with org = kGY * pitch + kGX.  Ghost cells hold periodic copies (or
// mirror copies at outer walls) so that row-block copies of the sweep
// kernel never wrap.
constexpr int kGX = 4;
constexpr int kGY = 6;

// Kernel constants in the arithmetic type T (all derived on the host from
// ddcc_params; see ddcc_api.cu for each formula's source).
template <typename T>
struct KParams {
    int nx, ny, pitch, N;
    int px, py;
    long long plane;              // elements per plane (pitch * (ny + 2 kGY), 256-byte aligned)
    long long org;                // offset of node (0, 0): kGY * pitch + kGX
    int has_cos_field;
    int wet_field;                // 1: the N-1 angle planes hold the wetting strengths
                                  //    e_j = sum_k cos(theta^k_jN) |grad psi_k| (several solids)
    T cs2, inv_cs2;
    T gw1, gw2;                   // w_axis / cs2, w_diag / cs2 (gradient stencil)
    T lw1, lw2;                   // w_axis / cs2, w_diag / cs2 (div(psi grad) stencil)
    T w1d[3];                     // 1D weights of c = -1, 0, +1: d0/2, 1-d0, d0/2
    T rho[kMaxPhases], nu[kMaxPhases];
    T beta2[kMaxPhases][kMaxPhases];   // 2 beta_ij = 6 sigma_ij / eps
    T kap[kMaxPhases][kMaxPhases];     // 3 eps sigma_ij / 4
    T wet[kMaxPhases][kMaxPhases];     // 3 sigma_ij
    T sigN[kMaxPhases];                // sigma_iN
    T invsig[kMaxPhases][kMaxPhases];  // 1 / sigma_ij (0 on the diagonal)
    T cos_uni[kMaxPhases];             // cos(theta_iN) when uniform
    T eta[kMaxPhases];
    T m0;
    // phase LB: lambda_ab = s_ab / N_ab in moment order
    // (00, 10, 01, 20, 02, 11, 21, 12, 22), and 1 / N_ab
    T lamf[kMaxPhases][9];
    T invN[9];
    // flow LB constant rates as lambda = s / N (00, 10, 01, 21, 12, 22)
    T lg00, lg1, lg3, lg4;
    T invN20, invN11;             // 1 / N for the per-node s21 and s22 rows
    T nu_to_s21, nu_to_s22;       // 2 / (1 - cs2) and 1 / cs2 (Eq. 16)
    T damp;                       // 1 / eps0^3
    T half_damp;
    T A_P;                        // 1/2 + K (1 - d0)(2 - s0) / (2 s0)
    T Kh;                         // K / 2
    T Hfac;                       // K (1 - 2 d0)
    T cP;                         // cs2 / (1 - w0)
    T gam;                        // K / 2 - w0 / (1 - cs2)
    T c2m3cs2;                    // 1 - 3 cs2
    T body[2];
};

// Device-side view of the fields carved out of the workspace.
template <typename T>
struct Fields {
    T* f[2];          // (N-1) x 9 planes each (ping-pong)
    T* g[2];          // 9 planes each, g_0 stored as g_0 - rho0
    T* lag[2];        // 2N+3 planes each: a, (psi C_i u)_{x,y}, T_xx, T_yy, T_xy, psi m.u
    T* psi;           // 1 plane
    T* cosf;          // N-1 planes or null
    T* C;             // N-1 planes (order-parameter scratch)
    T* macro;         // 2N+4 planes (read-out scratch)
    double* partial;  // kMassBlocks * kMaxPhases
    double* stage;    // host-input staging (double), max(N-1,1) planes
    T* inflow;        // open x ends: u_in (ny values), then C_in ((N-1) x ny)
    int* flag;        // device error word
};

inline int lag_planes(int N) { return 2 * N + 3; }

// Row-sweep kernel: strip width per precision, rows per iteration and
// threads per CTA.  With 60 columns the order-parameter pass (strip + 2
// halo columns a side = 64 columns x 4 rows) and the mu pass (62 x 4) each
// take one round of 256 threads.
template <typename T>
struct SweepWidth;
template <>
struct SweepWidth<float> {
    static constexpr int value = 60;
    static constexpr int threads = 256;
};
template <>
struct SweepWidth<double> {
    static constexpr int value = 28;
    static constexpr int threads = 128;
};
constexpr int kSweepRows = 4;

// Work split of the sweep: strips of SweepWidth columns times row bands;
// band k has seg_base (+1 for k < seg_rem) rows.
struct SweepPlan {
    int strips, segs, seg_base, seg_rem;
};

template <typename T>
struct SweepArgs {
    const CUtensorMap* tm_pop;   // 9N population planes (f then g) of the input copy
    const CUtensorMap* tm_lag;   // 2N+3 lagged planes of the input copy
    const CUtensorMap* tm_st;    // psi and, with a field, the N-1 cos(theta_iN) planes
    const KParams<T>* kp;
    T* pop_out;                  // population planes of the output copy
    T* lag_out;                  // lagged planes of the output copy
    int* err;                    // error word (bounded waits that ran out)
    SweepPlan plan;
};

// TMA-staged tile collide-stream kernel: 32 x 8 tiles whose populations,
// lagged planes and stencil halos arrive by tensor copies.
constexpr int kTileHaloW = kTileX + 8;   // halo box: tile + 4 columns a side
template <typename T>
struct TileTmaArgs {
    const CUtensorMap* tm_pop;   // box {32, 8, 9N} over the input population planes, or
                                 // (fused kernel) box {40, 12, 9(N-1)} over the f planes
    const CUtensorMap* tm_g;     // (fused kernel) box {32, 8, 9} over the input g planes
    const CUtensorMap* tm_lag;   // box {32, 8, 2N+3} over the input lagged planes
    const CUtensorMap* tm_c;     // box {40, 12, N-1} over the order-parameter planes
    const CUtensorMap* tm_st;    // box {40, 12, 1 or N} over psi (and cos(theta_iN))
    const CUtensorMap* tm_a;     // box {40, 10, 1} over lagged plane a of the input copy
    const KParams<T>* kp;
    T* pop_out;
    T* lag_out;
    int* err;
};
template <typename T>
size_t tile_tma_smem_bytes(int N, bool theta_field);
template <typename T>
cudaError_t launch_collide_tma(const TileTmaArgs<T>& a, cudaStream_t s);
template <typename T>
size_t tile_fused_smem_bytes(int N, bool theta_field);
template <typename T>
cudaError_t launch_collide_fused(const TileTmaArgs<T>& a, cudaStream_t s);

template <typename T>
size_t sweep_smem_bytes(int N, bool theta_field);
template <typename T>
cudaError_t launch_sweep(const SweepArgs<T>& a, cudaStream_t s);

// Launchers (ddcc_kernels.cu).  cur selects the input copy of the
// ping-pong buffers; outputs go to 1 - cur.
template <typename T>
cudaError_t launch_init(const KParams<T>& kp, const Fields<T>& fd, int cur, cudaStream_t s);
template <typename T>
cudaError_t launch_order_param(const KParams<T>& kp, const Fields<T>& fd, int cur, cudaStream_t s);
template <typename T>
cudaError_t launch_collide(const KParams<T>& kp, const Fields<T>& fd, int cur, cudaStream_t s);
template <typename T>
cudaError_t launch_macro(const KParams<T>& kp, const Fields<T>& fd, int cur, cudaStream_t s);
template <typename T>
cudaError_t launch_mass(const KParams<T>& kp, const Fields<T>& fd, int cur, double* dev_out,
                        cudaStream_t s);
template <typename T>
cudaError_t launch_convert(const double* src, T* dst, const KParams<T>& kp, int planes,
                           cudaStream_t s);
template <typename T>
cudaError_t launch_export(const T* src, double* dst, const KParams<T>& kp, cudaStream_t s);
// Fill the ghost frame of `planes` consecutive planes starting at base, gx
// columns and gy rows deep (at most kGX, kGY; the whole frame by default).
template <typename T>
cudaError_t launch_fill_ghosts(T* base, int planes, const KParams<T>& kp, cudaStream_t s, int gx = kGX,
                               int gy = kGY);
// Two rings in one launch: `planes` consecutive planes from base, gx
// columns and gy rows deep, each (planes = 0 leaves a ring out).
template <typename T>
struct GhostRing {
    T* base;
    int planes, gx, gy;
};
template <typename T>
cudaError_t launch_fill_ghosts2(const GhostRing<T>& g0, const GhostRing<T>& g1, const KParams<T>& kp,
                                cudaStream_t s);
// Ghost depth the fused tile kernel reads: the phase populations with a
// 2-node halo (order parameters for the chemical-potential halo) and the
// lagged plane a with a 1-node halo.
constexpr int kFusedGhostF = 2;
constexpr int kFusedGhostA = 1;

// Open x ends: reset the columns x = 0 and nx - 1 of the populations and
// lagged planes at pop/lag (a state just written by a step) to the inflow /
// outflow equilibrium.
template <typename T>
cudaError_t launch_open_bc(const KParams<T>& kp, T* pop, T* lag, const T* psi, const T* inflow,
                           cudaStream_t s);

// Several solids (Sec. 4.5): psi = prod_k psi_k and wetting strengths
// e_j = sum_k cos(theta^k_jN) |grad psi_k|.  walls_init sets psi = 1 and
// e = 0 on the domain; wall_accumulate folds in one solid whose psi_k
// (ghost frame filled) and N-1 angle planes sit at stage.
template <typename T>
cudaError_t launch_walls_init(const KParams<T>& kp, T* psi, T* e, cudaStream_t s);
template <typename T>
cudaError_t launch_wall_accumulate(const KParams<T>& kp, const T* stage, T* psi, T* e, cudaStream_t s);

// Adjoint of one step (ddcc_adjoint.cu).  All planes are padded planes of
// the handle's layout; the state and adjoint blocks are those of a saved
// state (9N population planes, f then g, and 2N+3 lagged planes).
template <typename T>
struct AdjStepArgs {
    const KParams<T>* kp;
    const T* psi;          // psi plane, ghost frame filled
    const T* cosf;         // N-1 cos(theta_iN) planes, or null when uniform
    const T* st_pop;       // state of step n
    const T* st_lag;
    const T* ad_pop_in;    // adjoint of the state of step n+1 (or of step 0)
    const T* ad_lag_in;
    T* ad_pop_out;         // adjoint of the state of step n
    T* ad_lag_out;
    T* scratch;            // adjoint_scratch_planes(N) planes
    double* dJ_dcos;       // (N-1) x ny x nx, accumulated
    double* dJ_dpsi;       // ny x nx, accumulated
};
template <typename T>
size_t adjoint_scratch_planes(int N);
template <typename T>
T* adjoint_c_planes(T* scratch);   // where the initial-state reverse expects C0
template <typename T>
cudaError_t launch_adjoint_step(const AdjStepArgs<T>& a, cudaStream_t s);
template <typename T>
cudaError_t launch_adjoint_initial(const AdjStepArgs<T>& a, cudaStream_t s);
// J = sum_x x m(x) / sum_x m(x), m = sum_p f_p over the 9 planes at f_phase;
// JM[0] = J, JM[1] = sum_x m(x); seed (9 planes, or null) = dJ/df_p = (x - J) / M.
template <typename T>
cudaError_t launch_centroid(const KParams<T>& kp, const T* f_phase, double* part, double* JM,
                            T* seed_f_phase, cudaStream_t s);

}  // namespace ddcc
