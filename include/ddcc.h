/*
 * ddcc.h -- C ABI of the GB300 (sm_103a) DD-CCLB time stepper.
 *
 * The library advances the lattice Boltzmann method of arXiv 2311.10314
 * (Liu, Zhan, Chen, Chai, Shi: a consistent and conservative diffuse-domain
 * LB method for N-phase flows in complex geometries) on a D2Q9 lattice:
 * N-1 phase-field populations f^i (Eq. 3.1) and one flow population g
 * (Eq. 3.2) per node, the Hermite-moment collision Lambda = H^-1 S H
 * (Sec. 3), the diffuse-domain sources built from the solid characteristic
 * function psi (the paper's phi, Sec. 2.3) and the wetting condition
 * (Eqs. 2.7, 2.9, 2.14), the isotropic finite-difference gradients those
 * sources need, and streaming.  Lattice units: dx = dt = c = 1, cs^2 = d0.
 *
 * Conventions shared by every call:
 *   - Arrays are row-major (y outer, x inner), nx * ny doubles per field,
 *     on the HOST unless a name says "dev".  The caller owns every buffer
 *     it passes; the library copies host inputs and never frees memory it
 *     did not allocate.
 *   - Device memory comes from the caller: ddcc_workspace_bytes() tells
 *     how much, ddcc_create() carves its fields out of it.  The workspace
 *     must stay allocated until ddcc_destroy().
 *   - All device work is issued on the CUDA stream given to ddcc_create()
 *     (a cudaStream_t passed as void*; NULL is the legacy default stream).
 *     Calls that return data to the host synchronise that stream.
 *   - Every call returns an int status: DDCC_OK (0) or a negative error
 *     code; no C++ exception crosses this interface.  ddcc_status_string()
 *     names a code.  After DDCC_ERR_CUDA the handle should be destroyed.
 *   - Handles are not thread-safe; distinct handles are independent.
 */
#ifndef DDCC_H
#define DDCC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DDCC_MAX_PHASES 4

/* status codes */
#define DDCC_OK                 0
#define DDCC_ERR_PARAM         -1   /* invalid parameter or size            */
#define DDCC_ERR_WORKSPACE     -2   /* workspace NULL, too small, misaligned */
#define DDCC_ERR_CUDA          -3   /* a CUDA runtime call failed           */
#define DDCC_ERR_NONFINITE     -4   /* NaN or Inf found by the FP64 reduction */
#define DDCC_ERR_NOMEM         -5   /* host allocation failed               */
#define DDCC_ERR_UNSUPPORTED   -6   /* build or device lacks a feature      */
#define DDCC_ERR_TIMEOUT       -7   /* a kernel's bounded wait ran out       */

/* ddcc_params.flags (default 0: the tile path) */
#define DDCC_FLAG_TILE  1u          /* step with the tile kernels (the default)  */
#define DDCC_FLAG_SWEEP 2u          /* step with the TMA row sweep where the grid
                                       allows it (one launch, no order-parameter
                                       round trip; slower on GB300 today)     */
#define DDCC_FLAG_OPEN_X 4u         /* inflow at x = 0, outflow at x = nx - 1
                                       (periodic_x must be 0; not with the row
                                       sweep; see ddcc_set_inflow)            */

/* step paths reported by ddcc_step_path() */
#define DDCC_PATH_TILE  1           /* order-parameter pass + tile collide-stream */
#define DDCC_PATH_SWEEP 2           /* TMA-fed row sweep (one launch per step)     */

/* arithmetic of the time step */
#define DDCC_FP64 0                 /* populations and arithmetic in double */
#define DDCC_FP32 1                 /* in float, g_0 stored as g_0 - rho0   */

/* fields for ddcc_read() */
#define DDCC_FIELD_C    0           /* + i (0..N-1): volume fraction C_{i+1} */
#define DDCC_FIELD_RHO  8           /* density rho = sum C_i rho_i           */
#define DDCC_FIELD_UX   9           /* velocity x                            */
#define DDCC_FIELD_UY  10           /* velocity y                            */
#define DDCC_FIELD_P   11           /* pressure P of Eq. 19                  */
#define DDCC_FIELD_MU  12           /* + i (0..N-1): chemical potential mu_{i+1} */
#define DDCC_FIELD_PSI 20           /* the characteristic function psi       */

/*
 * Physical and lattice parameters (Secs. 2-3).  Phase i = 1..N is index
 * i-1.  Only the first N (or N-1) entries of each array are read.
 */
typedef struct ddcc_params {
    int32_t nx, ny;           /* lattice size, each >= 3                        */
    int32_t nphase;           /* N, 2..DDCC_MAX_PHASES                          */
    int32_t periodic_x;       /* 1: periodic; 0: outer wall (halfway           */
    int32_t periodic_y;       /*    bounce-back, mirror ghost nodes; Sec. 2.3)  */
    int32_t precision;        /* DDCC_FP64 or DDCC_FP32                         */
    double  rho[DDCC_MAX_PHASES];   /* densities rho_i (Sec. 2.2)              */
    double  nu[DDCC_MAX_PHASES];    /* kinematic viscosities nu_i              */
    double  sigma[DDCC_MAX_PHASES][DDCC_MAX_PHASES]; /* surface tensions,
                                       symmetric, zero diagonal, > 0 off it     */
    double  width;            /* fluid-fluid interface width epsilon (Eq. 2.1)  */
    double  eps0;             /* solid diffuse-layer width epsilon_0 (Eq. 2.13c)*/
    double  d0;               /* free lattice parameter, cs^2 = d0 (Sec. 3)     */
    double  m0;               /* mobility m0 (Eqs. 2.5, 17)                     */
    double  eta[DDCC_MAX_PHASES];   /* eta_i of phases 1..N-1 (Eq. 3.5, 17)    */
    double  s_f[5];           /* phase-LB rates s0, s21, s22, s3, s4; s1 of
                                 phase i follows from m0 = (1/s1-1/2) eta_i d0 */
    double  s_g[4];           /* flow-LB rates s0, s1, s3, s4; s21 and s22 per
                                 node from nu = sum C_i nu_i by Eq. 16          */
    double  rho0;             /* constant of g_0^eq (Eq. 3.8)                   */
    double  body_force[2];    /* acceleration b; force density psi rho b        */
    uint32_t flags;           /* 0, DDCC_FLAG_TILE or DDCC_FLAG_SWEEP, optionally
                                 | DDCC_FLAG_OPEN_X                             */
} ddcc_params;

typedef struct ddcc_handle ddcc_handle;

/*
 * Bytes of device workspace ddcc_create() needs for these parameters, or 0
 * if they are invalid.  The workspace holds two copies of the populations
 * and of the lagged fields (ping-pong), psi, the contact-angle field, the
 * order-parameter scratch and reduction scratch.
 */
size_t ddcc_workspace_bytes(const ddcc_params* params);

/*
 * Validate the parameters, copy the host inputs to the device and set the
 * initial state (f = f^eq(C0, mu(C0), u = 0) by Eq. 3.5, g = g^eq(P = 0,
 * u = 0) by Eq. 3.8, lagged fields zero).
 *   params            : see ddcc_params.
 *   dev_workspace     : device pointer, >= ddcc_workspace_bytes(params)
 *                       bytes, 256-byte aligned.
 *   cuda_stream       : cudaStream_t (may be NULL).
 *   psi               : host, nx*ny, the solid characteristic function,
 *                       each value in (0, 1].
 *   cos_theta_field   : host, (N-1)*nx*ny values cos(theta_iN) per node
 *                       (Eq. 2.9), or NULL to use cos_theta_uniform.
 *   cos_theta_uniform : host, N-1 values cos(theta_iN); read only when the
 *                       field is NULL.
 *   C0                : host, (N-1)*nx*ny initial volume fractions of
 *                       phases 1..N-1 (C_N = 1 - sum).
 *   out               : receives the handle.
 * Errors: DDCC_ERR_PARAM, DDCC_ERR_WORKSPACE, DDCC_ERR_CUDA, DDCC_ERR_NOMEM.
 */
int ddcc_create(const ddcc_params* params, void* dev_workspace, size_t bytes,
                void* cuda_stream, const double* psi,
                const double* cos_theta_field, const double* cos_theta_uniform,
                const double* C0, ddcc_handle** out);

/*
 * ddcc_create() for a solid made of several parts, each given by its own
 * characteristic function and wetting angles (Sec. 4.5): psi = prod_k psi_k
 * and the wetting term of Eq. 2.14 becomes
 *   3 sigma_ij sum_{q != j} C_j C_q sum_k cos(theta^k_jq) |grad psi_k|,
 * with cos(theta^k_jq) from the solid's own angles theta^k_iN by Eq. 2.9
 * and |grad psi_k| by the step's gradient stencil (periodic copies or wall
 * mirrors at the box edge).  The per-node wetting strengths
 * sum_k cos(theta^k_iN) |grad psi_k| are formed once on the device; the
 * step kernels are the same.
 *   n_walls        : 1 <= n_walls <= DDCC_MAX_WALLS.
 *   wall_psi       : host, n_walls*nx*ny values, psi_k in (0, 1].
 *   wall_cos_theta : host, n_walls*(N-1)*nx*ny values cos(theta^k_iN),
 *                    solid k's block first (plane i-1 of the block for
 *                    phase i).
 * Other arguments and errors as ddcc_create().  The adjoint calls return
 * DDCC_ERR_UNSUPPORTED for such a handle.
 */
#define DDCC_MAX_WALLS 8
int ddcc_create_walls(const ddcc_params* params, void* dev_workspace, size_t bytes,
                      void* cuda_stream, int n_walls, const double* wall_psi,
                      const double* wall_cos_theta, const double* C0, ddcc_handle** out);

/*
 * Inflow and outflow along x (Sec. 4.5 imposes a parabolic velocity at the
 * inlet and the outlet of its channel), for a handle created with
 * DDCC_FLAG_OPEN_X.  After every step the columns x = 0 and x = nx - 1 are
 * reset to equilibrium (Eqs. 3.5 and 3.8 with mu = 0 and m^C = 0) at the
 * velocity (u_in(y), 0); the volume fractions are C_in(y) at the inlet and
 * those of the column x = nx - 2 at the outlet; the pressure is that of the
 * neighbouring column (Eq. 19 without its velocity terms:
 * psi P = c_P (sum_{p>0} g_p - K/2 psi m.u)); the lagged fields are those of
 * the boundary state.  C, psi, mu and a take zero-gradient (mirror) ghost
 * values across both ends.  Phase masses then change by the fluxes through
 * the ends.
 *   u_in : host, ny values (lattice units), the x velocity at both ends.
 *   C_in : host, (N-1)*ny values, the inflow volume fractions of phases
 *          1..N-1 (row-major: phase block first).
 * Until it is called u_in = 0 and C_in = 0.  Errors: DDCC_ERR_PARAM (NULL, or
 * a handle without DDCC_FLAG_OPEN_X), DDCC_ERR_CUDA.  The adjoint calls and
 * ddcc_step_between return DDCC_ERR_UNSUPPORTED for such a handle.
 */
int ddcc_set_inflow(ddcc_handle* h, const double* u_in, const double* C_in);

/*
 * Advance nsteps >= 0 time steps (Eqs. 3.1 and 3.2 with the equilibria,
 * sources, velocity and pressure of Sec. 3).  Asynchronous on the stream.
 * On the fused tile path, calls of four steps or more replay a CUDA graph of
 * two steps, captured on the first such call (not while profiling); the
 * arithmetic is the same as launching the kernels one by one.
 */
int ddcc_step(ddcc_handle* h, int64_t nsteps);

/*
 * Write one macroscopic field of the current state to host_out (nx*ny
 * doubles), computed as the next step would compute it: C_i = psi C_i /
 * psi with psi C_i = sum_p f^i_p, rho, the velocity and pressure of the
 * joint velocity / Eq. 19 solve, mu_i of Eq. 2.14.  Synchronises the stream.
 * field: one of the DDCC_FIELD_* values (C and MU take + phase index).
 * All fields of a state are formed by one pass on the first read and kept
 * until a call that may change the state (step, load_state, set_rows,
 * set_inflow, step_between or an adjoint call); later reads of the same
 * state only convert and copy.
 */
int ddcc_read(ddcc_handle* h, int field, double* host_out);

/*
 * Per-phase mass sum_x sum_p f^i_p (= sum_x psi C_i, conserved by the
 * method) for phases 1..N-1, reduced in FP64 on the device in a fixed
 * order.  host_out receives N-1 doubles.  Returns DDCC_ERR_NONFINITE if any
 * population is NaN or Inf.  Synchronises the stream.
 */
int ddcc_mass(ddcc_handle* h, double* host_out);

/*
 * Bytes of a saved state (populations and lagged fields in the step's
 * precision, plus the step counter).
 */
size_t ddcc_state_bytes(const ddcc_handle* h);

/*
 * Copy the full state to / from buf (ddcc_state_bytes() bytes), a device
 * pointer when on_device != 0, else host memory.  A state saved and loaded
 * resumes bit-exactly.  Save is asynchronous for device buffers and
 * synchronises the stream for host buffers; load likewise.
 * Layout of the buffer: the int64 step count in the first 256 bytes, then
 * (N-1)*9 phase-population planes (plane 9*(i-1)+p holds f^i_p), 9 flow
 * planes (g_p, with g_0 - rho0 stored for p = 0) and 2N+3 lagged planes,
 * each plane round_up(pitch*(ny+12)*e, 256) bytes with e the element size
 * of the precision and pitch = round_up(nx+8, 32); node (x, y) of a plane
 * is element (y+6)*pitch + (x+4) (a frame of 4 ghost columns and 6 ghost
 * rows surrounds the domain).
 */
int ddcc_save_state(ddcc_handle* h, void* buf, int on_device);
int ddcc_load_state(ddcc_handle* h, const void* buf, int on_device);

/* Steps taken since ddcc_create() (or the loaded state's count). */
int64_t ddcc_step_count(const ddcc_handle* h);

/*
 * Rows of the current state, for a decomposition of the grid into y slabs
 * over several GPUs (the paper has no counterpart; it computes on one
 * domain).  One step at node (x, y) reads the state at rows y - 3 .. y + 3
 * (the order parameters two rows out for the chemical potential one row
 * out, whose gradient the node needs, plus the populations streamed in from
 * one row out), so a slab that carries three extra rows on each side, run
 * as a periodic grid of its own, updates its inner rows exactly; after each
 * step the three edge rows on each side are replaced by the neighbouring
 * slabs' rows.
 *   ddcc_rows_bytes : bytes of nrows rows: (9N + 2N+3) planes x nrows x nx
 *                     elements of the handle's precision.
 *   ddcc_get_rows   : copies rows [y0, y0 + nrows) of every population plane
 *                     (f^1..f^{N-1}, then g) and every lagged plane, x in
 *                     [0, nx), into dev_buf (device, [plane][row][x]).
 *   ddcc_set_rows   : copies them back from dev_buf and refills the ghost
 *                     frame.
 * 0 <= y0, y0 + nrows <= ny, nrows >= 1, else DDCC_ERR_PARAM.  Both are
 * asynchronous on the handle's stream; the caller owns dev_buf.
 */
size_t ddcc_rows_bytes(const ddcc_handle* h, int nrows);
int ddcc_get_rows(ddcc_handle* h, int y0, int nrows, void* dev_buf);
int ddcc_set_rows(ddcc_handle* h, int y0, int nrows, const void* dev_buf);

/*
 * Per-kernel timing with CUDA events recorded on the handle's stream around
 * every launch that ddcc_step() issues while enabled (enable != 0).  The
 * events add no synchronisation.  ddcc_kernel_times() synchronises the
 * stream, writes for each kernel kind k < max_kinds the summed device time
 * in milliseconds (ms_out[k]) and the number of launches (launches_out[k]),
 * clears the record and returns the number of kinds (4: 0 = order
 * parameters and 1 = collide-stream of the tile path, 2 = row sweep,
 * 3 = ghost-frame fills of the tile path).
 * Either output may be NULL.
 */
int ddcc_profile(ddcc_handle* h, int enable);
int ddcc_kernel_times(ddcc_handle* h, double* ms_out, int64_t* launches_out, int max_kinds);

/*
 * Which kernels ddcc_step() runs for this handle: DDCC_PATH_TILE (the
 * default: one TMA-staged tile kernel that forms the order parameters from
 * the staged phase populations and makes the whole update, plus two small
 * ghost-frame fills; grids narrower than its halo boxes fall back to an
 * order-parameter pass and a plain-load tile kernel) or DDCC_PATH_SWEEP
 * (with DDCC_FLAG_SWEEP, when the grid is at least one sweep strip wide and
 * 8 rows high and the device has the shared memory).
 */
int ddcc_step_path(const ddcc_handle* h);

/*
 * Discrete adjoint of the step (reverse mode): the transpose of the
 * Jacobian of the arithmetic ddcc_step() performs (Sec. 3, Eqs. 3.1-3.10,
 * 2.14, 19, with the readings of the header of the oracle), used for
 * gradients of a scalar objective of the state after T steps with respect
 * to the per-node contact-angle field cos(theta_iN)(x) and psi(x).
 *
 * States and adjoint states are buffers of ddcc_state_bytes() in the layout
 * of ddcc_save_state() (device memory, 256-byte aligned; the adjoint of a
 * population or lagged plane sits where that plane sits).  scratch is a
 * device buffer of at least ddcc_adjoint_bytes() bytes, 256-byte aligned,
 * owned by the caller and free to reuse between calls.  dJ_dcos ((N-1) x ny
 * x nx doubles, plane i-1 for cos(theta_iN)) and dJ_dpsi (ny x nx doubles)
 * are device arrays, row-major without ghost frame, that the calls ADD to;
 * the caller zeroes them once.  A gradient with respect to a uniform angle
 * is the sum of its per-node entries.  All calls are asynchronous on the
 * handle's stream except ddcc_objective_centroid(), which synchronises it.
 * Errors: DDCC_ERR_PARAM for NULL or aliased buffers, DDCC_ERR_WORKSPACE
 * for a short or misaligned scratch, DDCC_ERR_CUDA for a failed launch.
 */
size_t ddcc_adjoint_bytes(const ddcc_handle* h);

/*
 * One step from the state in state_in to state_out (device buffers in the
 * ddcc_save_state() layout, 256-byte aligned, distinct), leaving the
 * handle's own state and step count untouched; the adjoint sweep uses it to
 * recompute a checkpointed segment without copying.  state_in must have
 * filled ghost frames, as every state the library writes has; state_out
 * gets them.  The step-count word of state_out is not written.  Only the
 * fused tile path provides it: DDCC_ERR_UNSUPPORTED otherwise (the caller
 * then loads, steps and saves).
 */
int ddcc_step_between(ddcc_handle* h, const void* state_in, void* state_out);

/*
 * One reverse step.  state_n: the state at step n (as saved before step
 * n+1 ran, or written by ddcc_step_between; its ghost frames filled);
 * adj_next: the adjoint of the state at step n+1; adj_out
 * (distinct from adj_next) receives the adjoint of the state at step n.
 * Contributions of step n+1 to dJ/dcos and dJ/dpsi are added.
 */
int ddcc_adjoint_step(ddcc_handle* h, const void* state_n, const void* adj_next, void* adj_out,
                      void* scratch, size_t scratch_bytes, double* dJ_dcos, double* dJ_dpsi);

/*
 * One checkpointed segment of the reverse sweep in a single call: states[0]
 * is the state at the segment's first step t0 (a checkpoint), states[1..n-1]
 * are buffers (ddcc_state_bytes(), 256-byte aligned) that receive the states
 * of steps t0+1 .. t0+n-1 by ddcc_step_between; then n reverse steps run from
 * adj_cur (the adjoint of the state at t0+n) down to the adjoint of the state
 * at t0, ping-ponging between adj_cur and adj_other.  *in_other = 1 when the
 * result ended in adj_other (n odd), else 0.  Adds to dJ_dcos and dJ_dpsi
 * like ddcc_adjoint_step.  DDCC_ERR_UNSUPPORTED where ddcc_step_between is
 * (the caller then recomputes with ddcc_load_state / ddcc_step /
 * ddcc_save_state and calls ddcc_adjoint_step).  Unless profiling is on,
 * a call with the arguments of one of the handle's last two calls captures
 * the segment's launches into a CUDA graph, and later calls with those
 * arguments replay it (at most four such graphs are kept per handle; the
 * arithmetic is the same).  A caller that passes the same buffers for
 * every segment (copying each checkpoint into states[0]) gets one graph for
 * the whole sweep.
 */
int ddcc_adjoint_segment(ddcc_handle* h, const void* const* states, int n, void* adj_cur,
                         void* adj_other, void* scratch, size_t scratch_bytes, double* dJ_dcos,
                         double* dJ_dpsi, int* in_other);

/*
 * One segment of a pipelined reverse sweep: the n reverse steps of a
 * segment whose states are all formed already (states[0..n-1], states[0]
 * at the segment's first step), as in ddcc_adjoint_segment; and, at the same
 * time on a second stream of the handle, the recompute of the next segment
 * to reverse: next[1..n_next-1] receive the states that follow next[0] (its
 * checkpoint), by ddcc_step_between.  The handle's stream waits for the
 * recompute after the reverse steps, so whatever is queued on it next (the
 * next call, reversing `next`) follows both.  A sweep
 * alternates two sets of segment buffers: the first call has n = 0 (the
 * last segment's recompute only) and the last n_next = 0.  next[1..] may
 * not be any of states[], adj_cur, adj_other or scratch (DDCC_ERR_PARAM).
 * The arithmetic is that of ddcc_adjoint_segment, so the gradients are the
 * same bit for bit; only the order of independent launches on the GPU
 * differs.  Graphs as for ddcc_adjoint_segment, captured when the arguments
 * repeat those of one of the last two plain calls.  DDCC_ERR_UNSUPPORTED
 * with n_next > 1 where ddcc_step_between is.
 */
int ddcc_adjoint_segment_pipelined(ddcc_handle* h, const void* const* states, int n,
                                   const void* const* next, int n_next, void* adj_cur,
                                   void* adj_other, void* scratch, size_t scratch_bytes,
                                   double* dJ_dcos, double* dJ_dpsi, int* in_other);

/*
 * Reverse of the initial state of ddcc_create() (f^i = f^i,eq(psi C0_i,
 * psi mu_i(C0), u = 0), g and lagged planes zero).  C0: host, the same
 * (N-1) x ny x nx doubles given to ddcc_create(); adj0: the adjoint of the
 * state at step 0.  Adds the initial state's contributions to dJ/dcos and
 * dJ/dpsi.
 */
int ddcc_adjoint_initial(ddcc_handle* h, const double* C0, const void* adj0, void* scratch,
                         size_t scratch_bytes, double* dJ_dcos, double* dJ_dpsi);

/*
 * Objective used by the adjoint: the x-centroid of phase `phase` + 1
 * (0 <= phase < N-1) of the handle's current state,
 *   J = sum_x x m(x) / sum_x m(x),  m(x) = sum_p f^(phase+1)_p(x) = psi C,
 * in FP64, written to *J_out (host).  The denominator is the phase mass,
 * which the step conserves.  If adj_seed (device, ddcc_state_bytes()) is
 * not NULL it receives dJ/dstate: (x - J) / sum_x m(x) in the planes of
 * f^(phase+1), zero elsewhere.
 */
int ddcc_objective_centroid(ddcc_handle* h, int phase, void* scratch, size_t scratch_bytes,
                            double* J_out, void* adj_seed);

/*
 * Per-phase mass sum_x sum_p f^i_p (i = 1..N-1) of caller-owned population
 * planes, reduced in FP64, without allocating anything.  This call has no
 * counterpart in the paper: it serves callers that cannot call cudaMalloc
 * (plugins whose host application owns every device allocation through its
 * own pool, real-time loops that cannot take the device synchronisation an
 * allocation implies).  Its scratch --
 * one double per (phase, row) -- is a static device array of
 * 3 x DDCC_NOALLOC_MAX_ROWS doubles (384 KiB) that every GPU loading the
 * library holds until the process exits.
 *   dev_populations : device, (N-1)*9 planes of T = double (DDCC_FP64) or
 *                     float (DDCC_FP32); element (x, y) of plane 9*(i-1)+p
 *                     at p_index*plane_stride + y*row_stride + x (elements).
 *   nx, ny          : 1 <= nx, 1 <= ny <= DDCC_NOALLOC_MAX_ROWS; larger ny
 *                     is rejected with DDCC_ERR_PARAM (beyond the static
 *                     scratch), as are row_stride < nx and
 *                     plane_stride < row_stride*ny.
 *   dev_out         : device, receives N-1 doubles.
 *   cuda_stream     : cudaStream_t (may be NULL); the call is asynchronous.
 * The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress, once per device, with that device current); make
 * that first call before any stream capture.  The address is kept for the
 * life of the process: after cudaDeviceReset on a device it is stale, and
 * the call must not be used on that device again.  All calls share the array,
 * which keeps the last call's contents; every partial a call reads is
 * written by that call first, so nothing needs clearing, but calls that
 * overlap on the GPU race and must be serialised by the caller.
 */
#define DDCC_NOALLOC_MAX_ROWS 16384
int ddcc_phase_mass_noalloc(const void* dev_populations, int precision, int nphase,
                            int nx, int ny, int64_t row_stride, int64_t plane_stride,
                            double* dev_out, void* cuda_stream);

/*
 * Self-test of the bounded waits of the library's TMA kernels.  With
 * deliver = 0 a one-block kernel waits (with a short poll limit) on an
 * mbarrier armed for bytes that no copy brings: the wait must run out, set
 * the error word at dev_flag and return, and the call returns
 * DDCC_ERR_TIMEOUT.  With deliver != 0 the barrier completes at once and the
 * call returns DDCC_OK.  dev_flag: device int owned by the caller; the call
 * synchronises cuda_stream.  Nothing is copied asynchronously, so nothing
 * lands after the kernel has returned.
 */
int ddcc_selftest_bounded_wait(void* cuda_stream, int* dev_flag, int deliver);

/*
 * Measured FP64 fused multiply-add rate of the current device in TFLOP/s
 * (2 flops per FMA), written to *tflops_out (host): the denominator of the
 * FP64 step's roofline, which the FP64 units bound on this GPU.  The paper
 * has no counterpart.  One warm-up and three timed launches of a kernel
 * whose threads run independent FMA chains on every SM; the best timed
 * launch counts.  dev_sink: device, at least 8 * (SM count) doubles, never
 * written in practice (it keeps the compiler from removing the chains).
 * Synchronises cuda_stream; takes about 0.1 s.
 */
int ddcc_measure_fp64_peak(void* cuda_stream, double* dev_sink, double* tflops_out);

/* Release the handle (not the caller's workspace).  NULL is allowed. */
void ddcc_destroy(ddcc_handle* h);

/* Static string naming a status code. */
const char* ddcc_status_string(int status);

/* Library version as major*10000 + minor*100 + patch. */
int ddcc_version(void);

#ifdef __cplusplus
}
#endif

#endif /* DDCC_H */
