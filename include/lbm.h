/*
 * lbm.h -- C ABI of the GB300 pseudopotential MRT lattice Boltzmann library (D2Q9).
 *
 * The library advances the per-time-step update of R. Huang, J. Huang, Q. Li,
 * "Improved third-order scheme in pseudopotential lattice Boltzmann model for
 * multiphase flows" (2026) on one CUDA device:
 *
 *   pull streaming, Eq. (lbe.str)                      -> f_i(x) = f_bar_i(x - e_i)
 *   density and momentum, Eq. (rho.rhou)               -> rho, j
 *   pseudopotential from the EOS (Sec. 2)              -> psi = sqrt(2 (p_EOS - rho/3)/G)
 *   pairwise force, Eq. (fint)                         -> F_int = -G psi(x) sum w psi(x+e) e
 *   velocity with the half force, Eq. (rho.rhou)       -> rho u = j + F/2
 *   MRT collision with the third-order source, Eq. (lbe.col), with Q_m original
 *   (Huang & Wu form, Sec. 2) or improved, Eqs. (qm.improved), (qm46.improved)
 *
 * Conventions used by every entry point:
 *   - Host and device arrays are row-major [ny][nx] with x fastest.  Vector fields are
 *     two consecutive planes (x component, then y).  Population arrays are nine planes
 *     [9][ny][nx] in the D2Q9 order e_0 = (0,0), e_1..e_4 = (1,0),(0,1),(-1,0),(0,-1),
 *     e_5..e_8 = (1,1),(-1,1),(-1,-1),(1,-1).
 *   - `on_device` = 0: pointers are host memory, copied synchronously.  `on_device` = 1:
 *     pointers are device memory of the context's device (e.g. a torch tensor's
 *     data_ptr()); they are read or written on the context stream, the call returns
 *     without waiting, and the caller must keep them alive until the stream reaches it.
 *   - The caller owns every pointer it passes.  The library owns every buffer it
 *     allocates internally (device memory from cudaMalloc) and frees it in lbm_destroy.
 *   - Every call returns an lbm_status.  No C++ exception crosses the ABI.  After a
 *     failure the message is kept by lbm_last_error(ctx) until the next failing call.
 *   - A context is not thread-safe: calls on one context must not overlap.
 *   - Lattice units: dx = dt = c = 1, c_s^2 = 1/3 (Sec. 3).
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define LBM_API __attribute__((visibility("default")))
#else
#define LBM_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_ctx lbm_ctx; /* opaque, owned by the library */

typedef enum {
    LBM_OK = 0,
    LBM_EINVAL = 1,   /* invalid argument or parameter */
    LBM_ENOMEM = 2,   /* device or host allocation failed */
    LBM_ECUDA = 3,    /* a CUDA runtime call failed */
    LBM_ESTATE = 4,   /* call not valid in the current state (e.g. fields not set) */
    LBM_ENAN = 5,     /* a non-finite density or velocity was detected */
    LBM_EBOUNDS = 6,  /* a device-side bounds check failed */
    LBM_ETIMEOUT = 7, /* a bounded device-side wait ran out */
    LBM_ENOTSUP = 8   /* combination of options not supported */
} lbm_status;

typedef enum {
    LBM_F64 = 0,     /* populations stored and updated in FP64 */
    LBM_F32 = 1,     /* populations stored and updated in FP32 */
    LBM_F16DEV = 2,  /* FP16 storage of f_i - w_i rho_ref, FP32 arithmetic */
    LBM_BF16DEV = 3  /* BF16 storage of f_i - w_i rho_ref, FP32 arithmetic */
} lbm_precision;

typedef enum {
    LBM_SCHEME_ORIGINAL = 0, /* Huang & Wu Q_m: Q2 = -Q1, Q4 = Q6 = 0 (Sec. 2) */
    LBM_SCHEME_IMPROVED = 1  /* Eqs. (qm.improved), (qm46.improved): Q2 = -Q1/2 (Sec. 2.2) */
} lbm_scheme;

typedef enum {
    LBM_EOS_VDW = 0, /* p = K (rho R T/(1 - b rho) - a rho^2), Sec. 3 */
    LBM_EOS_CS = 1   /* Carnahan-Starling, p = K (rho R T (1+h+h^2-h^3)/(1-h)^3 - a rho^2), h = b rho/4 */
} lbm_eos;

typedef enum {
    LBM_FORCE_CONST = 0,   /* external force density (Fx, Fy) at every fluid node */
    LBM_FORCE_BUOYANT = 1, /* (rho - rho_g) (Fx, Fy): gravity of Sec. 3.3 */
    LBM_FORCE_FIELD = 2    /* per-node force density set by lbm_set_geometry */
} lbm_force_mode;

typedef enum {
    LBM_KERNEL_AUTO = 0,     /* fused kernel when the geometry allows it, else two-pass */
    LBM_KERNEL_TWO_PASS = 1, /* psi pass + fused collide-and-pull-stream pass */
    LBM_KERNEL_FUSED = 2     /* one pass per step, psi recomputed on a staged halo */
} lbm_kernel;

/*
 * Problem parameters, in the paper's notation (Secs. 2-3).  Fill with
 * lbm_params_default() and override; struct_size must equal sizeof(lbm_params).
 */
typedef struct lbm_params {
    int32_t struct_size;
    int32_t nx, ny;                 /* lattice size, >= 1 */
    int32_t periodic_x, periodic_y; /* 1 periodic; 0 half-way bounce-back walls just
                                       outside the domain (at x = -1/2 and nx - 1/2) */
    int32_t precision;              /* lbm_precision */
    int32_t scheme;                 /* lbm_scheme */
    int32_t q2_original;            /* 1: improved Q4, Q6 with the original Q2 = -Q1 */
    int32_t eos;                    /* lbm_eos */
    int32_t force_mode;             /* lbm_force_mode */
    int32_t kernel;                 /* lbm_kernel */
    int32_t per_node_ref;           /* FP16/BF16 storage: 1 = deviations from w_i rho(x) of
                                       the writing node (extra FP32 plane), 0 = from
                                       w_i rho_ref */
    int32_t storage_scale_log2;     /* FP16/BF16 storage of (f_i - w_i rho_ref) 2^k; k in
                                       [-30, 30], for FP16 in [-15, 24] */
    int32_t storage_rounding;       /* FP16/BF16 storage, rounding of each stored deviation:
                                       0 to nearest (ties to even); 1 (default) stochastic (rounded up
                                       with probability equal to the discarded fraction of an
                                       ulp, from random bits that hash the node, the
                                       population and the step count: unbiased, and the same
                                       in every run and in both step kernels).  Rounding to
                                       nearest repeats the same error at every node of a
                                       uniform region, step after step, which drifts mass and
                                       momentum; stochastic rounding leaves a zero-mean error
                                       (but no longer keeps mirror-symmetric states exactly
                                       symmetric).  The initial state is rounded to nearest. */
    int32_t diag_every;             /* 0 (default): lbm_step never waits for the device.  D > 0:
                                       whenever the step count reaches a multiple of D, lbm_step
                                       waits, evaluates the diagnostics and returns LBM_ENAN (a
                                       non-finite density or velocity) or the status of the
                                       device error word; the steps after that point are not
                                       run.  The adjoint's forward sweep does not check. */
    double a, b, R, T, K_eos;       /* EOS coefficients */
    double G;                       /* interaction strength, < 0 (Sec. 2) */
    double k1, k2;                  /* source coefficients, epsilon = -8 (k1 + k2) */
    double tau_l, tau_g;            /* relaxation times of liquid and gas; when they differ
                                       nu = (tau - 1/2)/3 is interpolated linearly in rho
                                       between rho_g and rho_l (clamped) */
    double rho_l, rho_g;            /* reference liquid and gas densities */
    double Lambda;                  /* (1/s_q - 1/2)(1/s_p - 1/2), 1/12 in Sec. 3 */
    double Fx, Fy;                  /* force density (CONST) or gravity g (BUOYANT) */
    double rho_s;                   /* virtual wall density: psi at walls = psi(rho_s) */
    double rho_ref;                 /* FP16/BF16 storage reference density */
    double rho_max;                 /* create checks psi^2 > 0 on (0, rho_max] */
} lbm_params;

/* Number of doubles written by lbm_get_diagnostics. */
#define LBM_NDIAG 10

/* Parameters changeable after create (lbm_set_param). */
typedef enum {
    LBM_PARAM_FX = 0,
    LBM_PARAM_FY = 1,
    LBM_PARAM_G = 2,
    LBM_PARAM_T = 3
} lbm_param_id;

/* Objectives of lbm_adjoint_step: J = (1/n) sum_{t=1..n} J_t with J_t a linear
 * functional of the stored post-collision populations after step t. */
typedef enum {
    LBM_OBJ_WALL_FORCE_Y = 0, /* y momentum handed to the walls by the next streaming */
    LBM_OBJ_MEAN_JX = 1       /* (1/N_fluid) sum over fluid nodes of sum_i e_ix f_bar_i */
} lbm_objective;

/* Fill *p with defaults: 4 x 128 channel (periodic x, walls in y), FP64, improved
 * scheme, Carnahan-Starling a = 1, b = 4, R = 1, T = 0.7 T_c, G = -1,
 * k1 = k2 = -1.895/16, tau = 0.8, Lambda = 1/12, no force, kernel AUTO. */
LBM_API lbm_status lbm_params_default(lbm_params *p);

/* Validate parameters and allocate a context on the current CUDA device.
 * cuda_stream: a cudaStream_t to run on, or NULL for a stream the library creates.
 * Rejects (LBM_EINVAL): nx or ny < 1, ny > 65535, tau <= 1/2, G >= 0, Lambda <= 0,
 * p_EOS - rho/3 >= 0 somewhere on (0, rho_max], unknown enum values.
 * The populations are zero until lbm_init_fields or lbm_set_state. */
LBM_API lbm_status lbm_create(const lbm_params *p, void *cuda_stream, lbm_ctx **out);

/* Free every buffer of the context (waits for its stream first).  NULL is accepted. */
LBM_API lbm_status lbm_destroy(lbm_ctx *ctx);

/* Geometry, host arrays (each may be NULL):
 *   solid[ny*nx]          1 = solid node (wall); its psi is psi(rho_s), or that of its
 *                         own density when lbm_set_wall_density has set one
 *   wall_u[2*ny*nx]       velocity of each solid node; a link from a fluid node into a
 *                         moving solid gets the term 2 w rho_w (e.u_w)/c_s^2
 *   q[8*ny*nx]            q[(d-1)*ny*nx + node]: wall position on the link from a fluid
 *                         node along e_d, as a fraction of the link (0, 1]; 1/2 is
 *                         half-way bounce-back, other values interpolated bounce-back
 *                         (linear, Bouzidi: second order for the velocity but not mass
 *                         conserving; against a dense liquid the fluid mass drifts, while
 *                         half-way links conserve it to round-off)
 *   force_field[2*ny*nx]  force density of LBM_FORCE_FIELD
 * Passing NULL clears the corresponding array.  Call before stepping. */
LBM_API lbm_status lbm_set_geometry(lbm_ctx *ctx, const uint8_t *solid, const double *wall_u,
                            const double *q, const double *force_field);

/* Virtual density of each solid node, a host array [ny*nx] read at solid nodes only (the
 * wettability of each wall: Sec. 3 gives every wall psi(rho_s) with one rho_s; this sets
 * rho_s node by node, e.g. a gas-wetted inner and a liquid-wetted outer cylinder).  Every
 * entry must be positive with psi(entry) real (LBM_EINVAL otherwise; the previous field
 * is kept).  Walls beyond a non-periodic edge keep rho_s.  NULL restores rho_s at every
 * wall.  lbm_get_moments reports the field at solid nodes.  lbm_adjoint_step rejects a
 * context with a field set (LBM_ENOTSUP).  Call before stepping. */
LBM_API lbm_status lbm_set_wall_density(lbm_ctx *ctx, const double *wall_rho);

/* Set the populations to the equilibrium f_bar = M^-1 m_eq(rho, u) of each node.
 * rho, ux, uy: [ny*nx] doubles (ux, uy may be NULL for u = 0).  Resets the step count. */
LBM_API lbm_status lbm_init_fields(lbm_ctx *ctx, const double *rho, const double *ux, const double *uy,
                           int on_device);

/* Advance nsteps time steps on the context stream.  Launches the kernels and returns
 * without waiting for the device, unless lbm_params.diag_every = D > 0: then it waits at
 * every step count that is a multiple of D, and stops there with LBM_ENAN (non-finite
 * density or velocity) or the device error status.  A device-side failure of a launched
 * step (a bounded wait that ran out: LBM_ETIMEOUT; a bounds check: LBM_EBOUNDS) is
 * recorded in a device error word and reported by the next call that waits for the
 * stream: lbm_sync, lbm_get_moments / lbm_get_state with host buffers,
 * lbm_get_diagnostics, lbm_save_state, lbm_adjoint_step and the diag_every checks. */
LBM_API lbm_status lbm_step(lbm_ctx *ctx, int64_t nsteps);

/* Density and velocity of the current state (the state the next step pulls), computed
 * as the step computes them: rho = sum f_i, u = (j + F/2)/rho.  Solid nodes report
 * rho_s and u = 0.  Each output [ny*nx] doubles, may be NULL. */
LBM_API lbm_status lbm_get_moments(lbm_ctx *ctx, double *rho, double *ux, double *uy, int on_device);

/* FP64 diagnostics of the current state (sums over fluid nodes, accumulated in FP64):
 *   out[0] mass, out[1..2] sum of j = sum_i e_i f_i, out[3..4] sum of the total force,
 *   out[5..6] momentum handed to the walls by the streaming that produced the state,
 *   out[7] sum of rho u_y and out[8] sum of rho over the liquid region
 *   rho > (rho_l + rho_g)/2 (U_c = out[7]/out[8], Sec. 3.3), out[9] max |u|.
 * Waits for the stream.  Returns LBM_ENAN if the mass or max |u| is not finite. */
LBM_API lbm_status lbm_get_diagnostics(lbm_ctx *ctx, double out[LBM_NDIAG]);

/* Decoded populations of the current state as FP64, [9][ny][nx] (get) or set from
 * such an array (set; encoded into the storage precision). */
LBM_API lbm_status lbm_get_state(lbm_ctx *ctx, double *pops, int on_device);
LBM_API lbm_status lbm_set_state(lbm_ctx *ctx, const double *pops, int on_device);

/* Raw storage snapshot for checkpoint / resume in the storage precision.
 * lbm_save_state with buf = NULL writes the required size to *nbytes. */
LBM_API lbm_status lbm_save_state(lbm_ctx *ctx, void *host_buf, size_t *nbytes);
LBM_API lbm_status lbm_load_state(lbm_ctx *ctx, const void *host_buf, size_t nbytes);

/* Change one parameter (lbm_param_id) between steps. */
LBM_API lbm_status lbm_set_param(lbm_ctx *ctx, int32_t which, double value);

/* Adjoint of nsteps forward steps from the current state for the time-averaged
 * objective J = (1/nsteps) sum_{t=1..nsteps} J_t (lbm_objective); the paper has no
 * adjoint, this differentiates its step (Sec. 2) exactly.  The forward pass advances the
 * context nsteps steps, storing the populations every checkpoint_every steps and summing
 * J_t in FP64; the backward pass recomputes each segment from its checkpoint and runs the
 * transposed step back to the starting state.  On return *J holds the objective,
 * grad[0..3] = dJ/d(Fx, Fy, G, T) (summed in FP64; dJ/dG is zero up to round-off, since
 * psi ~ |G|^-1/2 makes the step independent of G), and the state is left at
 * step t0 + nsteps as if lbm_step(nsteps) had run.
 * grad and lambda0 both NULL: only the forward pass runs (the objective alone).
 * `lambda0` (may be NULL): receives dJ/d f_bar at the starting state, [9][ny][nx]
 * doubles on the host (zero at solid nodes).
 * Supported: every storage type, periodic directions, resting half-way walls (domain
 * edges and solid nodes), CONST and BUOYANT forces, one or two relaxation times;
 * LBM_ENOTSUP otherwise.  16-bit storage: the states are stored and recomputed as the
 * forward steps store them (the same stochastic rounding), and the transposed step runs in
 * FP32 on the decoded states, taking the storage's rounding as the identity (the gradient
 * of the unrounded step along the 16-bit run's trajectory).  Device memory (allocated on
 * the first call, kept until lbm_destroy or a larger call): ceil(nsteps/K) + 2 (K - 1)
 * population states (with their reference-density plane), 2 K psi fields and 15 planes of
 * the arithmetic type (FP64 for FP64 storage, FP32 otherwise), K = min(checkpoint_every,
 * nsteps) (the
 * recompute of a segment overlaps, on a second stream, the transposed steps of the segment
 * after it); LBM_ENOMEM when it does not fit (lower checkpoint_every).  LBM_EINVAL: nsteps or
 * checkpoint_every < 1, unknown objective. */
LBM_API lbm_status lbm_adjoint_step(lbm_ctx *ctx, int64_t nsteps, int32_t checkpoint_every,
                            int32_t objective, double *J, double grad[4], double *lambda0);

/* Block until the context stream is idle; returns the status recorded by the device
 * error word of the steps launched so far (see lbm_step). */
LBM_API lbm_status lbm_sync(lbm_ctx *ctx);

/* Number of steps since the last lbm_init_fields / lbm_set_state. */
LBM_API int64_t lbm_step_count(const lbm_ctx *ctx);

/* Kernel actually used by lbm_step (LBM_KERNEL_TWO_PASS or LBM_KERNEL_FUSED). */
LBM_API int32_t lbm_kernel_in_use(const lbm_ctx *ctx);

/* "LB-ana" (Sec. 3.1, Figs. 3-4): the steady velocity profile of two-phase Poiseuille flow that
 * the step itself predicts for a given density profile across the channel, from the
 * finite-difference velocity equation of the step, Eq. (fde.ali) (channel aligned with the
 * lattice, node spacing dx) or Eq. (fde.obl) (oblique != 0: the 45-degree channel, profile along
 * alpha = x - y with node spacing dx/sqrt 2), with the source term of p->scheme: Q_m,6 of
 * Eq. (qm6.ali) (aligned) or Q_m,4+6 of Eq. (obl.11) with K = (24 eps - 15)/32 (45 degrees) for
 * the improved scheme, none for the original.  The channel's walls are half-way no-slip walls
 * just beyond both ends of the profile.
 *   rho[n]    density of the n fluid nodes across the channel (n >= 3), host memory
 *   f_int[n]  the pairwise force along the profile (aligned: its component across the channel;
 *             45 degrees: its x component), or NULL to compute it from rho by Eq. (obl.10) with
 *             psi of p's EOS and psi(p->rho_s) at the walls (one wall node beyond each end,
 *             two for the 45-degree bands)
 *   F_drive   driving force density along the channel
 *   u[n]      receives the velocity along the channel
 * Uses p's EOS, G, k1, k2, scheme, rho_s and tau (tau_l == tau_g; nu = (tau - 1/2)/3).  Runs on
 * the host and needs no device.  LBM_EINVAL (message in lbm_last_error(NULL)): null pointers,
 * n < 3, tau_l != tau_g, G >= 0, a density where psi is not real and positive, a singular
 * system. */
LBM_API lbm_status lbm_lb_ana(const lbm_params *p, int32_t oblique, int32_t n, const double *rho,
                              const double *f_int, double F_drive, double *u);

/* Largest lattice (nx * ny) accepted by lbm_step_noalloc_f32. */
#define LBM_NOALLOC_MAX_NODES (1 << 20)

/* One FP32 time step that allocates nothing (this entry point has no counterpart in the
 * paper; it serves callers that cannot call cudaMalloc, e.g. while a stream is being
 * captured into a CUDA graph, or applications that hand all device memory to their own
 * pool).  Reads the populations of the current state from src and writes the next state
 * to dst, both caller-owned device memory holding nine planes [9][ny][pitch] of floats
 * (pitch >= nx elements per row); the step is the two-pass step of lbm_step with
 * precision LBM_F32 and no geometry arrays (periodic directions or half-way walls at the
 * domain edges, CONST or BUOYANT force).  Runs on cuda_stream (NULL: the legacy default
 * stream) and returns without waiting.
 * Scratch: the pseudopotential field lives in one file-scope device array of
 * LBM_NOALLOC_MAX_NODES floats (4 MiB) that every device loading the library holds until
 * exit.  The first call on each device looks up that array's device address with that
 * device current; make that first call before any stream capture.  The address is kept
 * per device together with the ID of its context: after cudaDeviceReset, or with another
 * context current, the next call looks it up again (and is then again a first call).
 * All calls on a device share the array, so calls that overlap on the GPU (other
 * streams, other threads) race: serialise them.  No call reads scratch left by an
 * earlier one.
 * Errors (message in lbm_last_error(NULL)): LBM_EINVAL for null or aliasing buffers, a
 * bad struct_size, pitch < nx, ny > 65535 or nx * ny > LBM_NOALLOC_MAX_NODES;
 * LBM_ENOTSUP for a precision other than LBM_F32 or LBM_FORCE_FIELD; LBM_ECUDA for a
 * failed launch. */
LBM_API lbm_status lbm_step_noalloc_f32(const lbm_params *p, const float *src, float *dst, int64_t pitch,
                                        void *cuda_stream);

/* Message of the last failure on ctx (or of the last failed lbm_create when ctx is
 * NULL); never NULL. */
LBM_API const char *lbm_last_error(const lbm_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* LBM_H */
