/*
 * ddcc3d.h -- C ABI of the three-dimensional DD-CCLB time stepper (sm_103a).
 *
 * Sec. 3 of arXiv 2311.10314 runs its three-dimensional problems with the
 * D3Q7 lattice for the N-1 phase-field populations f^i (Eq. 3.1) and the
 * D3Q15 lattice for the flow population g (Eq. 3.2), with the weights and
 * relaxation orders printed there, the Hermite-moment collision
 * Lambda = H^-1 S H, and the 3D constants K = 1 - 2 d0 and
 * H = K (3 - 7 d0)(s21 - 2) / 2 of the pressure (Eq. 19).  Everything else
 * -- the chemical potential with the diffuse-domain wetting term (Eq. 2.14),
 * the mobility (Eq. 2.5), the sources (Eqs. 3.6, 3.10), the equilibria
 * (Eqs. 3.5, 3.8), the force and velocity -- is the dimension-free form of
 * Secs. 2-3 with three components.  The box is periodic along every axis;
 * solids enter through the characteristic function psi (Sec. 2.3) only.
 * Lattice units: dx = dt = c = 1, cs^2 = d0.
 *
 * Conventions (as ddcc.h): arrays are row-major with x fastest, then y, then
 * z (nx*ny*nz doubles per field) on the HOST; the caller owns every buffer
 * and the device workspace; all device work runs on the stream given to
 * ddcc3d_create(); calls that return data synchronise it; every call
 * returns DDCC_OK or a negative DDCC_ERR_* code of ddcc.h.  Handles are not
 * thread-safe.
 */
#ifndef DDCC3D_H
#define DDCC3D_H

#include <stddef.h>
#include <stdint.h>

#include "ddcc.h"

#ifdef __cplusplus
extern "C" {
#endif

/* extra field id of ddcc3d_read() (the others are the DDCC_FIELD_* of ddcc.h) */
#define DDCC_FIELD_UZ 21            /* velocity z                              */

/* ddcc3d_params.flags: how ddcc3d_step runs (the same arithmetic either
 * way).  0: the fused kernel in FP32, the three kernels in FP64 (where the
 * fused kernel's recomputed halo chemical potentials cost more FP64 work
 * than the saved traffic); SPLIT or FUSED force one; not both. */
#define DDCC3D_FLAG_SPLIT 1u
#define DDCC3D_FLAG_FUSED 2u

/*
 * Parameters (Secs. 2-3).  Phase i = 1..N is index i-1; only the first N
 * (or N-1) entries of each array are read.
 */
typedef struct ddcc3d_params {
    int32_t nx, ny, nz;       /* lattice size, each >= 3; nx*ny*nz < 2^31,
                                 ny <= 262140, nz <= 131070                      */
    int32_t nphase;           /* N, 2..DDCC_MAX_PHASES                           */
    int32_t precision;        /* DDCC_FP64 or DDCC_FP32                          */
    int32_t reserved;         /* must be 0                                       */
    double  rho[DDCC_MAX_PHASES];   /* densities rho_i                           */
    double  nu[DDCC_MAX_PHASES];    /* kinematic viscosities nu_i                */
    double  sigma[DDCC_MAX_PHASES][DDCC_MAX_PHASES]; /* symmetric, zero diagonal,
                                       > 0 off it                                */
    double  width;            /* interface width epsilon (Eq. 2.1)               */
    double  eps0;             /* solid diffuse-layer width epsilon_0             */
    double  d0;               /* cs^2 = d0, 0 < d0 < 1/2 (the D3Q15 rest weight
                                 (1-d0)(1-2d0) must be positive; the D3Q7 one,
                                 1 - 3 d0, may be negative, as at the d0 = 0.4
                                 of Sec. 4.4)                                    */
    double  m0;               /* mobility m0 (Eqs. 2.5, 17)                      */
    double  eta[DDCC_MAX_PHASES];   /* eta_i of phases 1..N-1                    */
    double  s_f[2];           /* D3Q7 rates s0, s21; s1 of phase i from
                                 m0 = (1/s1 - 1/2) eta_i d0 (Eq. 17)             */
    double  s_g[4];           /* D3Q15 rates s0, s1, s3, s4; s21 and s22 per node
                                 from nu = sum C_i nu_i by Eq. 16                */
    double  rho0;             /* constant of g_0^eq (Eq. 3.8)                    */
    double  body_force[3];    /* acceleration b; force density psi rho b         */
    uint32_t flags;           /* 0, DDCC3D_FLAG_SPLIT or DDCC3D_FLAG_FUSED       */
} ddcc3d_params;

typedef struct ddcc3d_handle ddcc3d_handle;

/*
 * Bytes of device workspace for these parameters, or 0 if they are
 * invalid: two copies of the populations (7(N-1) D3Q7 planes and 15
 * D3Q15 planes) and of the 3N + 7 lagged planes (a_xy, a_yz, a_zx, (psi C_i u)_{x,y,z},
 * T_{xx,yy,zz,xy,yz,zx}, psi m.u), psi, the angle field, the volume
 * fractions and chemical potentials of the current step, read-out and
 * reduction scratch.  Each plane is nx*ny*nz elements of the precision,
 * rounded up to 256 bytes.
 */
size_t ddcc3d_workspace_bytes(const ddcc3d_params* params);

/*
 * Validate, copy the host inputs and set the initial state: f^i = f^i,eq
 * (Eq. 3.5) at C0 with mu(C0) and u = 0; g = g^eq (Eq. 3.8) at P = 0,
 * u = 0; lagged fields zero.
 *   dev_workspace     : device, >= ddcc3d_workspace_bytes() bytes, 256-byte
 *                       aligned.
 *   cuda_stream       : cudaStream_t (may be NULL).
 *   psi               : host, nx*ny*nz values in (0, 1].
 *   cos_theta_field   : host, (N-1)*nx*ny*nz values cos(theta_iN) per node,
 *                       or NULL to use cos_theta_uniform (N-1 values).
 *   C0                : host, (N-1)*nx*ny*nz initial volume fractions.
 * Errors: DDCC_ERR_PARAM, DDCC_ERR_WORKSPACE, DDCC_ERR_CUDA, DDCC_ERR_NOMEM.
 */
int ddcc3d_create(const ddcc3d_params* params, void* dev_workspace, size_t bytes,
                  void* cuda_stream, const double* psi, const double* cos_theta_field,
                  const double* cos_theta_uniform, const double* C0, ddcc3d_handle** out);

/*
 * Advance nsteps >= 0 steps: the volume fractions C_i = sum_p f^i_p / psi,
 * the chemical potentials of Eq. 2.14, and the node update (gradients,
 * mobility, force, the joint velocity / Eq. 19 pressure solve, both
 * collisions, push streaming, lagged fields): one fused kernel per step,
 * which marches along z and keeps C and mu in shared memory, or three
 * kernels through C and mu planes in device memory (see the flags).
 * Asynchronous on the stream.
 */
int ddcc3d_step(ddcc3d_handle* h, int64_t nsteps);

/*
 * One macroscopic field of the current state as the next step would
 * compute it (nx*ny*nz doubles to host_out): DDCC_FIELD_C + i and
 * DDCC_FIELD_MU + i (i < N), DDCC_FIELD_RHO, DDCC_FIELD_UX, DDCC_FIELD_UY,
 * DDCC_FIELD_UZ, DDCC_FIELD_P, DDCC_FIELD_PSI.  Synchronises the stream.
 * C and mu of a state are formed on its first read and kept until the next
 * ddcc3d_step.
 */
int ddcc3d_read(ddcc3d_handle* h, int field, double* host_out);

/*
 * Per-phase mass sum_x sum_p f^i_p (phases 1..N-1, N-1 doubles), reduced in
 * FP64 on the device in a fixed order; DDCC_ERR_NONFINITE if a population
 * is NaN or Inf.  Synchronises the stream.
 */
int ddcc3d_mass(ddcc3d_handle* h, double* host_out);

/* Steps taken since ddcc3d_create(). */
int64_t ddcc3d_step_count(const ddcc3d_handle* h);

/*
 * Per-kernel timing with CUDA events on the handle's stream while enabled;
 * ddcc3d_kernel_times() synchronises, writes the summed milliseconds and
 * launch counts of each kind (0 = volume fractions, 1 = chemical
 * potentials, 2 = node update, 3 = fused step), clears the record and
 * returns 4.
 */
int ddcc3d_profile(ddcc3d_handle* h, int enable);
int ddcc3d_kernel_times(ddcc3d_handle* h, double* ms_out, int64_t* launches_out, int max_kinds);

/* Release the handle (not the caller's workspace).  NULL is a no-op. */
void ddcc3d_destroy(ddcc3d_handle* h);

#ifdef __cplusplus
}
#endif

#endif /* DDCC3D_H */
