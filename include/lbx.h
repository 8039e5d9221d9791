/*
 * lbx.h - C ABI of the B300 (sm_103a) kinetic-relaxation lattice Boltzmann library.
 *
 * The library advances the discrete-velocity kinetic relaxation scheme that the paper
 * "Automated Derivation of Lattice Boltzmann Methods for Systems of Conservation Laws"
 * derives for a system dQ/dt + div Phi(Q) = S(Q) (Eq. pde_target): one population set
 * f_{k,i} per conserved or gradient-tracker component k (Sec. 2.2.1), the exact-flux
 * equilibrium f^eq_{k,i} = w_i (Q_k + c_i . [(dt/dx) Phi_k] / c_s^2) (Eq. feq) and the
 * BGK collide-and-stream update (Eq. lbe_update)
 *     f_{k,i}(x + c_i dx, t + dt) = f - (f - f^eq)/tau_k + dt w_i S_k(x, t + dt/2).
 * The workflow follows the paper's statement of the problem (Algorithm 1, Fig. 1):
 * declare the system, derive the lattice and grid scaling, then init / step(n) /
 * moments / sub-characteristic check.
 *
 * Conventions shared by every call
 *  - Status: every call returns an lbx_status; nothing calls exit() or abort().  The
 *    message of the last failure on the calling thread is lbx_last_error().
 *  - Fields: Q arrays are float64 [K][cells], cells = nz*ny*nx with x fastest (C order),
 *    node coordinates x_i = i/N on the periodic unit domain.  Values are the
 *    nondimensional physical ones: the flux factor dt/dx and the source factor dt are
 *    applied inside the library (Eq. feq, Eq. lbe_update).
 *  - Host arrays passed in or out are only accessed during the call.  Device pointers
 *    must be device memory of the current CUDA device.
 *  - Streams: device work is enqueued on the state's stream and is asynchronous unless
 *    the call returns host values (those calls synchronise that stream).
 *  - Ownership: handles are created and destroyed by the library.  Buffers the caller
 *    passes in (f_buf_a/f_buf_b) stay owned by the caller and must outlive the state.
 */
#ifndef LBX_H
#define LBX_H

#include <stdint.h>
#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LBX_OK = 0,
    LBX_ERR_ARG = 1,          /* invalid argument, combination or size               */
    LBX_ERR_CUDA = 2,         /* a CUDA runtime call failed                           */
    LBX_ERR_OOM = 3,          /* device allocation failed                             */
    LBX_ERR_SUBCHAR = 4,      /* sub-characteristic bound violated (Sec. 2.3.2)       */
    LBX_ERR_NONFINITE = 5,    /* a NaN/Inf was detected in the state                  */
    LBX_ERR_TIMEOUT = 6,      /* a device-side wait ran out of its iteration budget   */
    LBX_ERR_STATE = 7,        /* call not valid for this state (e.g. flag raised)     */
    LBX_ERR_IO = 8,           /* file error, bad magic, hash or CRC mismatch          */
    LBX_ERR_UNSUPPORTED = 9   /* combination not compiled into this library           */
} lbx_status;

/* System families (Sec. 3).  Component orders:
 *   ADR_CASCADE      (u, G_x, G_y)                                        K = 3, 2D
 *   NSF_PRIM_TRACK   (rho, m_x, m_y, E, G_u(2), G_v(2), G_T(2))           K = 10, 2D
 *   MHD_J_TRACK      (rho, m(3), B(3), E, j(3))                           K = 11, 3D
 *   BURGERS (u), EULER (rho, m_x, m_y, E), MAXWELL_TM (E_z, H_x, H_y)     2D
 *   NSF_CONS_TRACK   (rho, m_x, m_y, E, G_rho(2), G_mx(2), G_my(2), G_E(2))       K = 12, 2D
 *                    the paper's own cascade: trackers of the conserved fields, the chain
 *                    rule for grad u and grad T (Sec. 2.1.1)
 *   MHD_POWELL_2D    (rho, m_x, m_y, E, B_x, B_y, G_rho(2), G_mx(2), G_my(2), G_E(2),
 *                     G_Bx(2), G_By(2))                                         K = 18, 2D
 *                    the paper's own MHD: viscous, heat-conducting (T = p/rho), resistive,
 *                    Powell source -(tr G_B)(0, B, u.B, u)
 *   HCNSF_3D         (rho, m_x, m_y, m_z, E, G_11, G_22, G_T(3), G_00, G_01, G_02, G_12)
 *                                                                            K = 14, 3D
 *                    3D homogenized compressible NSF (Sec. 3, HCNSF) in the paper's order:
 *                    G ~ sym grad u, G_T ~ grad T (T = p/rho), porosity alpha and solid
 *                    velocity u_s prescribed (lbx_prescribed); Phi_m = m u + p I - alpha tau_v,
 *                    Phi_E = (E + p) u - alpha tau_v u - alpha kappa G_T,
 *                    S_m = (1 - alpha)/eta (rho u_s - m), S_E = S_m . u.  The background Q0
 *                    must have zero tracker components.
 * Trackers G_{V,b} ~ dV/dx_b follow Eq. gradient_advection with tau_grad = g_tau dt. */
typedef enum {
    LBX_ADR_CASCADE = 1,
    LBX_NSF_PRIM_TRACK = 2,
    LBX_MHD_J_TRACK = 3,
    LBX_BURGERS = 4,
    LBX_EULER = 5,
    LBX_MAXWELL_TM = 6,
    LBX_NSF_CONS_TRACK = 7,
    LBX_MHD_POWELL_2D = 8,
    LBX_HCNSF_3D = 9
} lbx_family;

typedef enum { LBX_D2Q5 = 1, LBX_D2Q9 = 2, LBX_D3Q7 = 3, LBX_D3Q19 = 4 } lbx_lattice;
typedef enum { LBX_ACOUSTIC = 1, LBX_DIFFUSIVE = 2 } lbx_scaling;

/* Storage and arithmetic (Sec. 2.4.3 reference/equilibrium shift):
 *   FP64         populations f in float64, float64 arithmetic;
 *   FP32_SHIFT   f* = f - f^eq(Q0, F0) stored and computed in float32;
 *   FP16_SCALED  f* divided by s_k stored as IEEE binary16 (round to nearest), s_k a power of two
 *                per component fixed at init (s_k = 2^ceil(log2(4 max|f*_k|))),
 *                float32 arithmetic.
 * Init and the moment/norm reductions are float64 in every mode. */
typedef enum { LBX_FP64 = 1, LBX_FP32_SHIFT = 2, LBX_FP16_SCALED = 3 } lbx_precision;

/* Manufactured forcing S_MMS = d_t Q_ex + div Phi(Q_ex) - S(Q_ex) (Sec. 4), added to the
 * conserved components at t + dt/2 (node coordinates x = (i, j, l) dx, dx = 1/nx):
 *   NONE          no forcing;
 *   ADR_SEPARABLE u_ex = 1 + A sin(2 pi x) cos(2 pi y) exp(-t) for the ADR cascade with
 *                 R = 0; mms_amp = A; closed form, conserved component only;
 *   FOURIER       every primitive field V_p of the family is mms_mean[p] plus a sum of
 *                 modes (lbx_mms_mode, at most LBX_MMS_MAX_MODES).  The exact augmented
 *                 state is assembled from the primitives and their derivatives, and S_MMS
 *                 is evaluated at every node and step from the modes' analytic
 *                 derivatives, carried through the family's own flux by forward-mode dual
 *                 numbers.  Primitives p per family, and the state built from them:
 *                   ADR_CASCADE (u)                  Q = (u, du/dx, du/dy)
 *                   NSF (rho, u, v, p)               Q = (rho, rho u, rho v,
 *                                                        p/(gamma-1) + rho|u|^2/2,
 *                                                        grad u, grad v, grad T), T = p/(rho R)
 *                   MHD (rho, u_x, u_y, u_z, B_x, B_y, B_z, p)
 *                                                    Q = (rho, rho u, B, p/(gamma-1) +
 *                                                        rho|u|^2/2 + |B|^2/2, curl B)
 *                   NSF_CONS_TRACK (rho, u, v, p)    as NSF, trackers grad rho, grad(rho u),
 *                                                        grad(rho v), grad E
 *                   MHD_POWELL_2D (rho, u, v, p, B_x, B_y)
 *                                                    Q = (rho, rho u, rho v, p/(gamma-1) +
 *                                                        rho|u|^2/2 + |B|^2/2, B, gradients
 *                                                        of the six conserved fields)
 *                   HCNSF_3D (rho, u_x, u_y, u_z, p) Q = (rho, rho u, p/(gamma-1) + rho|u|^2/2,
 *                                                        sym grad u, grad(p/rho)), the
 *                                                        paper's order
 *                   BURGERS (u), MAXWELL_TM (E_z, H_x, H_y): Q = V
 *                   EULER (rho, u, v, p)             Q = (rho, rho u, rho v,
 *                                                        p/(gamma-1) + rho|u|^2/2)
 *                 S_MMS is the residual of the whole augmented state (the paper's Sec. 4
 *                 definition on Q+): each tracker is forced with d_t G_ex + div Phi_G(Q_ex)
 *                 - S_G(Q_ex), G_ex its exact gradient (or curl B), so it carries no
 *                 relaxation lag; mms_conserved_only = 1 forces the conserved components
 *                 alone.  The table is copied by lbx_scheme_derive. */
typedef enum { LBX_MMS_NONE = 0, LBX_MMS_ADR_SEPARABLE = 1, LBX_MMS_FOURIER = 2 } lbx_mms;

/* Prescribed coefficient fields of HCNSF_3D (Sec. 3, HCNSF; supplement, HCNSF MMS): the
 * porosity alpha (1 fluid, 0 solid) and the solid velocity u_s, evaluated in the step kernel
 * at every node x = (i, j, l) dx from closed forms, at the time level t^n = n dt of the state
 * they multiply (t + dt/2 inside the manufactured forcing, whose flux divergence includes
 * the fields' gradient):
 *   NONE      alpha = 1, u_s = 0 (plain compressible NSF);
 *   UNIFORM   alpha = pf[0], u_s = (pf[1], pf[2], pf[3]);
 *   ADVECTED  a moving solid: with s_d = sin(2 pi x_d), c_d = cos(2 pi x_d), the rotation
 *             pattern r = rot (s_0 c_1 c_2, -c_0 s_1 c_2, c_0 c_1 s_2), translation c and
 *             oscillation osc,
 *               u_s = (r_0 cos t + c_0 + osc sin t c_2, r_1 cos t + c_1 + osc cos t c_0,
 *                      r_2 sin t + c_2 + osc sin t c_1),
 *               alpha = a_mean + a_amp [z_0 + z_1 + z_2 + 2 z_0 z_1 z_2], z_d = sin(2 pi xi_d),
 *               xi = x - r sin t - c t;
 *             pf = (a_mean, a_amp, rot, osc, c_0, c_1, c_2, theta_S, theta_Phi).  The
 *             paper's values are (0.5, 0.1, 0.2, 0.1, 0.1, -0.1, 0.05), for which alpha stays
 *             in [0, 1].  theta_S and theta_Phi move the fields' time level inside the drag
 *             source and inside the equilibrium flux to t^n + theta dt (0: the state's time
 *             level; 1/2: the step's midpoint, where the manufactured forcing is taken). */
typedef enum { LBX_PRESCRIBED_NONE = 0, LBX_PRESCRIBED_UNIFORM = 1, LBX_PRESCRIBED_ADVECTED = 2 } lbx_prescribed;

/* Population storage of a state:
 *   TWO_BUFFERS  two buffers A, B; each step pulls from one and writes the other;
 *   IN_PLACE     one buffer (half the memory).  Steps alternate between two kinds whose reads
 *                and writes of a node cover the same addresses (kind 1 pulls from the
 *                neighbours and stores each post-collision population into the slot of the
 *                opposite velocity it just emptied; kind 2 reads the node's own swapped
 *                slots and stores in the standard slots).  After an even number of steps the
 *                populations are bitwise those of TWO_BUFFERS.  After an odd number the
 *                layout is the pair's intermediate one: every call that reads or writes the
 *                populations (moments, populations, norms, sums, finite and sub-characteristic
 *                checks, save) fails with LBX_ERR_STATE until one more step is taken; lbx_load
 *                restores a standard layout.
 *                Staged systems use bulk row copies where the staging resolves to them
 *                (lbx_state_set_staging, blocks of lbx_state_set_block), else per-thread
 *                copies in 128-thread blocks; no tuning, batches or adjoint. */
typedef enum { LBX_STREAM_TWO_BUFFERS = 0, LBX_STREAM_IN_PLACE = 1 } lbx_streaming;

#define LBX_MMS_MAX_MODES 64
/* One term of a manufactured primitive field:
 *   V_p(x, t) += amp sin(2 pi (k . x) + phase) exp(sigma t) cos(omega t + psi). */
typedef struct {
    int p;                 /* primitive index (see LBX_MMS_FOURIER)                      */
    int k[3];              /* integer wave numbers (k[2] = 0 in 2D)                      */
    double amp, phase, sigma, omega, psi;
} lbx_mms_mode;

typedef struct {
    int family;            /* lbx_family                                                */
    /* Physical parameters, by family:
     *   ADR_CASCADE  {a_x, a_y, nu, R}
     *   NSF          {gamma, R_gas, mu, kappa}
     *   MHD          {gamma, eta}
     *   BURGERS      {}            EULER {gamma}            MAXWELL_TM {c}
     *   NSF_CONS_TRACK {gamma, R_gas, mu, kappa}   MHD_POWELL_2D {gamma, mu, kappa, eta}
     *   HCNSF_3D     {gamma, mu, kappa, eta}  (eta > 0: drag time scale) */
    double params[8];
    /* Reference (background) state Q0 [K] for the shifted storage modes; F0 = Phi(Q0). */
    double Q0[24];
} lbx_system_desc;

typedef struct {
    int lattice;           /* lbx_lattice; must match the family's dimension           */
    int64_t extent[3];     /* nx, ny, nz (nz = 1 in 2D); each >= 2                      */
    int scaling;           /* lbx_scaling: dt = f dx (acoustic) or f dx^2 (diffusive)   */
    double f;              /* time-step factor f                                       */
    double tau_lb;         /* > 0: tau_LB of the conserved fields, used directly        */
    double tau_R;          /* used when tau_lb <= 0: tau_LB = 1/2 + tau_R dt (Sec. 2.3.1)*/
    double g_tau;          /* tracker steps: tau_grad = g_tau dt, tracker tau_LB = g_tau+1 */
    int precision;         /* lbx_precision                                             */
    int mms;               /* lbx_mms                                                   */
    double mms_amp;        /* amplitude A of the ADR manufactured solution              */
    int allow_subchar_violation; /* nonzero: lbx_init does not fail on a violated bound */
    const lbx_mms_mode* mms_modes; /* FOURIER: the mode table (read during the call)    */
    int mms_n_modes;       /* FOURIER: 1 .. LBX_MMS_MAX_MODES                           */
    double mms_mean[8];    /* FOURIER: mean of each primitive                           */
    int mms_conserved_only; /* FOURIER: nonzero leaves the tracker components unforced */
    int prescribed;        /* lbx_prescribed (HCNSF_3D only; NONE for every other family) */
    double prescribed_params[10]; /* pf of the prescribed fields                         */
    int streaming;         /* lbx_streaming                                             */
    /* Slab of a larger periodic grid cut along its last axis (y in 2D, z in 3D), for a
     * domain decomposition with one slab per process or GPU (see lbx_halo_pack).
     * slab_planes_global: planes of the whole grid along that axis; 0 (the default) means
     * this scheme is the whole grid.  slab_origin: global index of the slab's first plane
     * (0 <= slab_origin and slab_origin + local planes <= slab_planes_global).  The extents
     * are the slab's own; dx = 1/nx is the whole grid's (a slab spans the whole x extent,
     * and the whole y extent in 3D), and node coordinates (manufactured forcing, prescribed
     * fields) use the global plane index.  TWO_BUFFERS streaming only. */
    int64_t slab_origin;
    int64_t slab_planes_global;
    /* FP16_SCALED only: when every one of the K values is > 0, the storage scales s_k
     * lbx_init uses instead of deriving them from the initial populations (slabs of one
     * grid must share their scales; powers of two keep the scaling exact).  All zero (the
     * default): derived at init as described for LBX_FP16_SCALED. */
    double fp16_scales[24];
} lbx_scheme_desc;

typedef struct lbx_system lbx_system;
typedef struct lbx_scheme lbx_scheme;
typedef struct lbx_state lbx_state;
typedef struct lbx_batch lbx_batch;

/* Message of the last failed call on this thread ("" if none).  Owned by the library. */
const char* lbx_last_error(void);

/* Library version as major*10000 + minor*100 + patch. */
int lbx_version(void);

/* ---- 1. declare the system (Eq. pde_target, Sec. 2.1.1 cascade) ------------------- */
lbx_status lbx_system_declare(const lbx_system_desc* desc, lbx_system** out);
/* K = component count (conserved + trackers), n_cons = conserved count, dim = D. */
lbx_status lbx_system_info(const lbx_system* sys, int* K, int* n_cons, int* dim);
/* Name of component k (static string), or NULL if k is out of range. */
const char* lbx_component_name(const lbx_system* sys, int k);
void lbx_system_destroy(lbx_system* sys);

/* ---- 2. derive the lattice scheme and grid scaling (Sec. 2.3.1, supplement recipes) - */
/* Copies what it needs from sys; sys may be destroyed afterwards. */
lbx_status lbx_scheme_derive(const lbx_system* sys, const lbx_scheme_desc* desc, lbx_scheme** out);
/* dx = 1/nx, dt from the refinement law, lam = dt/dx, tau[K] the per-component tau_LB,
 * q the velocity count.  Any output pointer may be NULL. */
lbx_status lbx_scheme_info(const lbx_scheme* sch, double* dx, double* dt, double* lam,
                           double* tau, int* q);
void lbx_scheme_destroy(lbx_scheme* sch);

/* Velocities (q x 3 ints, unused components 0) and weights of a lattice in the order
 * the library stores populations.  c and w may be NULL to query q only. */
lbx_status lbx_lattice_velocities(int lattice, int* q, int* c, double* w);

/* ---- 3. state: init / step / moments / checks ---------------------------------------- */
/* Populations start at the (shifted) equilibrium of Q (supplement, recipes paragraph).
 * Q: float64 [K][cells], on the host (q_on_device = 0) or device (1).  Page-locked host
 * fields (pinned or registered) are read by the init kernel directly over the bus, with
 * no staging copy.  Pageable host fields are copied in chunks of planes of the last axis
 * on a second stream of the state, each chunk's equilibrium computed while the next one
 * is copied (FP16_SCALED without given scales copies them whole first, since the scales
 * need every field).
 * stream: a cudaStream_t (NULL = the legacy default stream).
 * f_buf_a, f_buf_b: NULL to let the library allocate the two population buffers, or
 * two device buffers of lbx_state_buffer_bytes() bytes each, owned by the caller.  An
 * IN_PLACE scheme uses f_buf_a alone (f_buf_b must be NULL): NULL lets the library
 * allocate its one buffer.
 * Runs the sub-characteristic check and fails with LBX_ERR_SUBCHAR on a violation
 * unless the scheme allows it.  On failure *out is NULL and nothing is leaked. */
lbx_status lbx_init(const lbx_scheme* sch, const double* Q, int q_on_device, void* stream,
                    void* f_buf_a, void* f_buf_b, lbx_state** out);
/* Bytes of one population buffer for this scheme (K*q*cells*storage size). */
size_t lbx_state_buffer_bytes(const lbx_scheme* sch);

/* Advance 0 <= n <= 2^30 steps of Eq. lbe_update (fused pull collide-and-stream),
 * asynchronous: one step kernel per step (FP64 states with an advected solid also launch
 * a one-thread kernel before each step, which computes the sines of the step's field
 * times).  Fails with LBX_ERR_NONFINITE without stepping if a previous check found a
 * NaN/Inf.  With graph replay enabled, the launches are recorded into a CUDA graph the
 * first time this (n, buffer parity) occurs and replayed afterwards. */
lbx_status lbx_step(lbx_state* st, int64_t n);
/* Threads per block (32, 64 or 128; default 128) of the step kernels that stage a node's
 * populations in shared memory (K q s > 360 bytes or K > 12: MHD on D3Q19, FP64 NSF, the
 * 18-component MHD, the homogenized NSF), in-place bulk steps included; the other kernels
 * always use 128.  Only speed changes, never results. */
lbx_status lbx_state_set_block(lbx_state* st, int block);
/* How the staged step kernels (K q s > 360 bytes or K > 12) bring a node's pulled populations into
 * shared memory; only speed changes, except LBX_STAGE_LANES2, whose moment sums add in
 * another order (results change by rounding only).
 *   LBX_STAGE_AUTO     bulk row copies when they apply, else per-thread copies (default)
 *   LBX_STAGE_THREAD   each thread copies its node's K q values (cp.async)
 *   LBX_STAGE_LANES2   two adjacent lanes share a node: one takes the rest population, and
 *                      of every opposite velocity pair each takes one velocity; partial
 *                      moments are combined by a warp shuffle
 *   LBX_STAGE_BULK     warp 0 of a block issues one bulk copy (TMA engine) per population
 *                      row segment the block pulls; needs nx % 8 == 0 and 16-byte aligned
 *                      population buffers (LBX_ERR_UNSUPPORTED otherwise).  Its wait on the
 *                      copies is bounded: a timeout sets a device error word that
 *                      lbx_synchronize and lbx_check_finite report as LBX_ERR_TIMEOUT.
 *   LBX_STAGE_PIPE     per-thread copies in a persistent grid (a multiple of the SM count)
 *                      that walks row segments: each thread stages its next node while it
 *                      updates the current one (two private columns, cp.async groups).
 *                      It uses the largest block up to the set one whose two columns fit
 *                      in shared memory.
 * The register-resident kernels ignore it.  LBX_ERR_ARG for unknown values. */
typedef enum {
    LBX_STAGE_AUTO = 0,
    LBX_STAGE_THREAD = 1,
    LBX_STAGE_LANES2 = 2,
    LBX_STAGE_BULK = 3,
    LBX_STAGE_PIPE = 4
} lbx_staging;
lbx_status lbx_state_set_staging(lbx_state* st, int staging);
/* Limit of the bounded wait of the bulk-staged step kernels (LBX_STAGE_BULK, and the
 * in-place bulk steps) for their row copies, in nanoseconds of the GPU's global timer;
 * the default is 1e9 (1 s).  When it runs out, a block raises the state's device error
 * word, waits once more (at most 1 s) for the copies it issued to land, and leaves the
 * populations of its nodes unwritten for that step; lbx_synchronize and
 * lbx_check_finite then return LBX_ERR_TIMEOUT and clear the word.  ns = 0 makes every
 * bulk-staged block give up before its first try while its copies complete normally,
 * which exercises that path without any fault; the populations of such a step are not
 * valid (restore them, e.g. with lbx_set_populations or lbx_load, before stepping on).
 * Other kernels never wait.  Drops the state's recorded graphs when the limit changes. */
lbx_status lbx_state_set_wait_limit(lbx_state* st, uint64_t ns);
/* Autotune the staged step kernel of this state: time per-thread copies and (where they
 * apply) bulk row copies, each with blocks of 32, 64 and 128 threads, over `trials`
 * launches (1..1000) after one warm-up launch, and keep the fastest.  Every timed launch
 * reads the current populations and writes the other buffer, which the next step
 * rewrites anyway, so neither the populations nor the time change; all candidates give
 * bitwise identical results (two lanes per node and the pipelined copies, measured slower
 * on every bench system, are not candidates).  Register-resident
 * kernels have one launch shape: nothing is timed and *ms_per_step is -1.  Synchronous.
 * Outputs (each may be NULL): the chosen staging and block, the best time per launch. */
lbx_status lbx_state_tune(lbx_state* st, int trials, int* staging, int* block, double* ms_per_step);
/* Enable (1) or disable (0) graph replay in lbx_step; needs a non-default stream. */
lbx_status lbx_state_use_graph(lbx_state* st, int enable);

/* Q_k = sum_i f_{k,i} (Eq. moments) at the current time, float64 [K][cells] into host
 * (out_on_device = 0, synchronous: the moments kernel writes page-locked host memory
 * directly over the bus; for pageable memory chunks of planes are copied back on the
 * state's second stream while the next chunk's moments are computed) or device memory
 * (1, asynchronous). */
lbx_status lbx_moments(lbx_state* st, double* Q_out, int out_on_device);

/* sum over nodes of Q_k, float64, fixed reduction order (deterministic). */
lbx_status lbx_conserved_sums(lbx_state* st, double* sums /* [K] host */);

/* Relative L2 ((N^-1 sum e^2)^1/2 over the same for Q_ref) and relative Linf
 * (max|e| / max|Q_ref|) per component against Q_ref [K][cells] (Sec. 4).  Q_ref on host
 * (ref_on_device = 0) or device (1).  Outputs are host arrays [K]; either may be NULL. */
lbx_status lbx_error_norms(lbx_state* st, const double* Q_ref, int ref_on_device,
                           double* relL2, double* relLinf);

/* Sets *finite to 1 if every moment is finite, else 0 and raises the state's flag. */
lbx_status lbx_check_finite(lbx_state* st, int* finite);

/* Sub-characteristic check (Sec. 2.3.2, Eq. subchar_system) in lattice form:
 * max_speed = (dt/dx) max over nodes of a closed-form bound of the spectral radius of
 * sum_a n_a dPhi_a/dQ over unit n (exact for ADR, Burgers, Euler, Maxwell; an upper
 * bound for NSF and MHD, including the tracker speeds); bound_cs = c_s;
 * bound_monotone = c_s^2 (monotone equilibria, Sec. 3 Burgers); ok = max_speed <= c_s. */
lbx_status lbx_subchar_check(lbx_state* st, double* max_speed, double* bound_cs,
                             double* bound_monotone, int* ok);

/* Pre-collision populations f_{k,i}(x, t) at the current time, float64 [K][q][cells]
 * host arrays, in the unshifted and unscaled representation (f = f* + f^eq(Q0) and
 * f* = s_k h).  Population order as lbx_lattice_velocities. */
lbx_status lbx_get_populations(lbx_state* st, double* f_out);
lbx_status lbx_set_populations(lbx_state* st, const double* f_in);

/* Step counter and time t = step * dt. */
lbx_status lbx_state_time(const lbx_state* st, int64_t* step, double* t);
/* Device pointer to the buffer holding the current populations (storage type).  For an
 * IN_PLACE state after an odd number of steps the buffer holds the step pair's
 * intermediate layout (see lbx_streaming). */
void* lbx_state_populations(const lbx_state* st);
/* Wait for all work queued on the state's stream. */
lbx_status lbx_synchronize(lbx_state* st);

/* Checkpoint: header (magic, version, shape, precision, step, scheme hash), populations
 * and a CRC32.  lbx_load checks all of them (LBX_ERR_IO on mismatch). */
lbx_status lbx_save(lbx_state* st, const char* path);
lbx_status lbx_load(lbx_state* st, const char* path);

void lbx_state_destroy(lbx_state* st);

/* ---- slabs of one grid: the face exchange (domain decomposition) ----------------------
 * A slab (lbx_scheme_desc.slab_planes_global > 0) steps with the periodic wrap of its own
 * planes along the slab axis a (y in 2D, z in 3D).  In the pull layout that wrap makes the
 * nodes of plane 0 read their c_a = +1 populations from the slots of the last plane P - 1,
 * and the nodes of plane P - 1 read their c_a = -1 populations from the slots of plane 0;
 * nothing else reads those slots.  After a step they hold the populations that leave the
 * slab through its upper and its lower face, and Eq. lbe_update across the faces needs
 * them exchanged with the neighbouring slabs: after EVERY lbx_step(st, 1) of a slab, and
 * before its next step or any call that reads its populations, the caller runs
 *     lbx_halo_pack(st, to_upper, to_lower);      exchange;
 *     lbx_halo_unpack(st, from_lower, from_upper);
 * where from_lower is the lower neighbour's to_upper and from_upper the upper neighbour's
 * to_lower (periodic: the first slab's lower neighbour is the last slab).  lbx_init and
 * lbx_set_populations leave the slots consistent (they hold the nodes' own pre-collision
 * values), so no exchange is needed before the first step; lbx_load restores the slots as
 * they were saved.  One velocity
 * plane of one face per velocity crossing it: 3 of 9 on D2Q9, 1 of 5 on D2Q5, 1 of 7 on
 * D3Q7, 5 of 19 on D3Q19, for all K components.  Reductions (sums, norms, checks) are per
 * slab: add the sums (lbx_conserved_sums, lbx_error_stats) over the slabs in float64.
 * With a single slab (the whole grid) the exchange is from_lower = to_upper and
 * from_upper = to_lower.  These calls also accept a whole-grid two-buffer state. */
/* Bytes of each face buffer: (velocities crossing a face) x K x (nodes of a plane) x the
 * storage size; 0 for a NULL scheme. */
size_t lbx_halo_bytes(const lbx_scheme* sch);
/* Copy the two faces' outgoing slots of the current populations into device buffers of
 * lbx_halo_bytes() bytes, 16-byte aligned: to_upper (plane P - 1, c_a = +1) and to_lower
 * (plane 0, c_a = -1).  Asynchronous on the state's stream (one kernel launch). */
lbx_status lbx_halo_pack(lbx_state* st, void* to_upper, void* to_lower);
/* Copy the neighbours' face buffers into the slots the next step pulls across the faces:
 * from_lower into plane P - 1's c_a = +1 slots, from_upper into plane 0's c_a = -1 slots.
 * Asynchronous on the state's stream (one kernel launch).  The face buffers' contents are
 * in the state's storage representation (shifted and scaled), so slabs that exchange must
 * share the scheme's storage, background state and (FP16) scales. */
lbx_status lbx_halo_unpack(lbx_state* st, const void* from_lower, const void* from_upper);
/* The exchange hidden behind the interior: a step in pieces.  Only the nodes of planes 0
 * and P - 1 write the face slots, and the interior planes never read them, so a slab can
 * step its two boundary planes first, exchange their faces on a second stream while the
 * interior planes step, and join before the next step:
 *     lbx_step_planes(st, 0, 1, side);  lbx_step_planes(st, P - 1, 1, side);
 *     lbx_step_planes(st, 1, P - 2, NULL);              (the state's stream)
 *     lbx_halo_pack_next(st, to_upper, to_lower, side);  transport on side;
 *     lbx_halo_unpack_next(st, from_lower, from_upper, side);
 *     the state's stream waits for side;  lbx_step_commit(st);
 * lbx_step_planes updates planes [plane0, plane0 + nplanes) of the last axis from the
 * current populations into the other buffer on `stream` (NULL: the state's stream),
 * asynchronously, without swapping the buffers; the same kernels and arithmetic as
 * lbx_step, so the pieces of a step are bitwise one lbx_step(st, 1).  LBX_ERR_ARG for a
 * range outside the grid, LBX_ERR_UNSUPPORTED for in-place states and the persistent
 * LBX_STAGE_PIPE kernel.  lbx_step_commit makes the other buffer current and advances the
 * step count (the device counter of time-dependent systems on the state's stream, so
 * every piece of the step must be ordered before it).  The _next face calls act on the
 * buffer being written (before lbx_step_commit), on `stream` (NULL: the state's). */
lbx_status lbx_step_planes(lbx_state* st, int64_t plane0, int64_t nplanes, void* stream);
lbx_status lbx_step_commit(lbx_state* st);
lbx_status lbx_halo_pack_next(lbx_state* st, void* to_upper, void* to_lower, void* stream);
lbx_status lbx_halo_unpack_next(lbx_state* st, const void* from_lower, const void* from_upper, void* stream);
/* The storage scales s_k of the state (1 unless FP16_SCALED), float64 [K] host array. */
lbx_status lbx_state_scales(const lbx_state* st, double* scales);
/* Raw error statistics per component against Q_ref [K][cells] (host or device): stats[k][0]
 * = sum_x e^2, [k][1] = sum_x Q_ref^2, [k][2] = max_x |e|, [k][3] = max_x |Q_ref|, e = Q_k -
 * Q_ref,k, float64 [K][4] host array.  The relative norms of lbx_error_norms follow from
 * them; slabs add [0], [1] and take the maximum of [2], [3] over the grid. */
lbx_status lbx_error_stats(lbx_state* st, const double* Q_ref, int ref_on_device, double* stats);

/* ---- batched states: many independent grids, one persistent launch per step ---------
 * n 2D schemes of the same family, lattice, storage (FP64 or FP32_SHIFT) and forcing,
 * each with its own extents, parameters and relaxation times, share two population
 * buffers (instance j at its own 256-byte aligned offset).  One launch of a persistent
 * kernel advances every instance by one step of Eq. lbe_update: blocks walk a list of
 * tiles of `block` consecutive cells with a grid-size stride (grid = SMs x ctas_per_sm).
 * lbx_batch_step records the n launches (plus the step-counter advance) into a CUDA graph
 * on first use and replays it afterwards (use_graph = 1).
 * Q[j]: host float64 [K][cells_j].  stream: NULL = a private non-blocking stream.  */
typedef struct {
    int block;             /* threads per block and cells per tile (multiple of 32)      */
    int ctas_per_sm;       /* persistent grid = SM count x ctas_per_sm                    */
    int steps_per_launch;  /* 1: a step needs every neighbour's previous step             */
    int use_graph;         /* nonzero: lbx_batch_step replays a captured CUDA graph       */
} lbx_batch_config;

lbx_status lbx_batch_create(const lbx_scheme* const* schemes, int n, const double* const* Q,
                            void* stream, lbx_batch** out);
lbx_status lbx_batch_info(const lbx_batch* b, int* n, int64_t* total_cells, size_t* buffer_bytes);
/* Advance every instance by n steps (asynchronous on the batch's stream). */
lbx_status lbx_batch_step(lbx_batch* b, int64_t n);
/* finite[j] = 1 when every stored population of instance j is finite, else 0 (one launch,
 * one block per instance; synchronous).  Instances step independently, so a diverged
 * instance does not disturb the others: the batched form of a stability sweep. */
lbx_status lbx_batch_check_finite(lbx_batch* b, int* finite);
lbx_status lbx_batch_synchronize(lbx_batch* b);
/* Moments of instance j, float64 [K][cells_j] host array (synchronous). */
lbx_status lbx_batch_moments(lbx_batch* b, int j, double* Q_out);
lbx_status lbx_batch_get_config(const lbx_batch* b, lbx_batch_config* cfg);
lbx_status lbx_batch_set_config(lbx_batch* b, const lbx_batch_config* cfg);
/* Autotuner: times `trials` launches of every (block, ctas_per_sm) candidate with CUDA
 * events (each launch reads the current buffer and writes the other one without
 * swapping, so the state does not advance), keeps the fastest and writes a JSON report
 * of all trials into `report` (may be NULL). */
lbx_status lbx_batch_tune(lbx_batch* b, int trials, char* report, size_t report_len);
void lbx_batch_destroy(lbx_batch* b);

/* ---- adjoint: gradient of a final-time density misfit -------------------------------
 * J = 1/2 sum_x (rho(x, T) - rho*(x))^2 after n_steps steps from populations at the
 * (shifted) equilibrium of Q_init.  Computes J, dJ/dQ_init (float64 [K][cells], every
 * component of the initial fields, trackers included) and dJ/dtau, tau the tau_LB
 * shared by the conserved fields.  The discrete adjoint of Eq. lbe_update runs on the
 * GPU (reverse pull along -c_i with the node-local flux and source Jacobians taken by
 * forward-mode dual numbers); the forward state is checkpointed every ckpt_every steps
 * and each segment is recomputed bitwise before its reverse sweep, so device memory
 * holds about (n_steps/ckpt_every + ckpt_every) population buffers.  The relaxation-time
 * term is accumulated per node in float64.  Storage FP64 or FP32_SHIFT (the adjoint runs
 * in the same arithmetic).  Q_init and rho_target are host arrays; outputs are host
 * pointers (any may be NULL); synchronous. */
lbx_status lbx_adjoint(const lbx_scheme* sch, const double* Q_init, int64_t n_steps, int ckpt_every,
                       const double* rho_target, void* stream, double* J, double* dJ_dQ0,
                       double* dJ_dtau);

/* Device time (CUDA events on the adjoint's stream, milliseconds) of the phases of the
 * last lbx_adjoint call that succeeded on the calling thread: ms[0] the forward sweep,
 * ms[1] the recomputation of the checkpointed segments, ms[2] the reverse (adjoint)
 * steps, ms[3] everything else between the first and the last timed point (misfit,
 * adjoint seed, segment restores and their host synchronisations, initial VJP, dJ/dtau
 * reduction).  Allocation, the host-to-device copies of the inputs and the copies of the
 * results back to the host are outside all four.  -1 before any call. */
lbx_status lbx_adjoint_timings(double* ms /* [4] host */);

/* ---- step-wise adjoint: the reverse sweep driven by the caller -----------------------
 * The pieces of lbx_adjoint, for a caller that runs the sweep itself, above all the slabs
 * of a grid cut across processes (lbx_adjoint refuses slab schemes).  With Lam_n = dJ/dA_n
 * in the pull layout, the reverse step of Eq. lbe_update is
 *     Lam_n[k][i][x - c_i] = (1 - w_k) Lam_{n+1}[k][i][x] + h_k(x)
 * (h: the node-local VJP of the equilibrium's flux and source), a push along -c_i.  An
 * adjoint buffer holds Lam in the compute type (double for FP64, float for FP32_SHIFT
 * storage) as [K][q][cells], lbx_adjoint_lam_bytes() bytes.  All calls run on the state's
 * stream; they need a two-buffer state of an lbx_adjoint family and storage, else
 * LBX_ERR_UNSUPPORTED.  Device pointers throughout.
 *
 * Sweep (one slab; a whole grid is the one-slab case, exchange = local copy):
 *   forward: before each segment of k steps lbx_adjoint_checkpoint(st, ckpt[c]); step and
 *            exchange the population faces as usual (lbx_halo_pack / unpack);
 *   seed:    lbx_adjoint_seed(st, rho_target, lamA, &J_slab); reverse face exchange;
 *   reverse, per segment from the last: lbx_adjoint_restore(st, ckpt[c], c k); keep the
 *            segment's states A_m (lbx_adjoint_checkpoint before each forward step with
 *            its exchange), then for m from the last down: lbx_adjoint_step(st, A_m,
 *            lam_next, lam_out, tau_acc); reverse face exchange of lam_out; swap;
 *   finish:  forward face exchange of Lam_0; lbx_adjoint_finish(st, Lam_0, Q_init,
 *            dJ_dQ0, tau_acc, &dJ_dtau_slab).
 * J and dJ/dtau add over the slabs; dJ/dQ_init is per node.
 *
 * Faces.  lbx_adjoint_halo_pack copies the slots of the upper face (plane P - 1, c_a = +1)
 * and the lower face (plane 0, c_a = -1) of an adjoint buffer into face buffers of
 * lbx_adjoint_halo_bytes() bytes ([face velocities][K][plane cells]); _unpack copies them
 * back into the same slots.  After lbx_adjoint_seed and after every lbx_adjoint_step the
 * transport is REVERSED: the push of plane 0's nodes has left the lower neighbour's values
 * in this slab's upper-face slots, so each slab unpacks face_upper = its UPPER neighbour's
 * packed face_upper and face_lower = its LOWER neighbour's packed face_lower.  Before
 * lbx_adjoint_finish (whose initial VJP pulls Lam_0 at x - c_i) the transport runs
 * FORWARD: face_upper = the LOWER neighbour's face_upper, face_lower = the UPPER
 * neighbour's face_lower. */
size_t lbx_adjoint_lam_bytes(const lbx_scheme* sch);     /* 0: NULL or no adjoint */
size_t lbx_adjoint_halo_bytes(const lbx_scheme* sch);    /* 0: NULL or no adjoint */
/* Copy the current populations (lbx_state_buffer_bytes() bytes, the storage layout as it
 * is) into dst, asynchronously. */
lbx_status lbx_adjoint_checkpoint(lbx_state* st, void* dst);
/* Make src (a checkpoint) the current populations and `step` the state's step count (the
 * time of time-dependent forcing and prescribed fields); synchronous. */
lbx_status lbx_adjoint_restore(lbx_state* st, const void* src, int64_t step);
/* The misfit of the current populations against rho_target ([cells], device) into *J
 * (host, may be NULL; synchronous reduction) and the seed Lam_N into lam. */
lbx_status lbx_adjoint_seed(lbx_state* st, const double* rho_target, void* lam, double* J);
/* One reverse step from the forward populations An (before step n) and Lam_{n+1} =
 * lam_next into lam_out = Lam_n (every slot written); tau_acc [cells] (float64, zeroed by
 * the caller before the sweep) accumulates the relaxation-time term.  Asynchronous. */
lbx_status lbx_adjoint_step(lbx_state* st, const void* An, const void* lam_next, void* lam_out,
                            double* tau_acc);
lbx_status lbx_adjoint_halo_pack(lbx_state* st, const void* lam, void* face_upper, void* face_lower);
lbx_status lbx_adjoint_halo_unpack(lbx_state* st, void* lam, const void* face_upper, const void* face_lower);
/* dJ/dQ_init [K][cells] (device) from Lam_0 and the initial fields Q_init ([K][cells],
 * device), and this state's share of dJ/dtau (host) from tau_acc; synchronous. */
lbx_status lbx_adjoint_finish(lbx_state* st, const void* lam0, const double* Q_init, double* dJ_dQ0,
                              const double* tau_acc, double* dJ_dtau);

/* ---- conserved sums without any device allocation --------------------------------------
 * The paper has no counterpart to this call; it exists for callers that must not
 * allocate device memory: code recorded into a CUDA graph or running under a latency
 * budget (cudaMalloc and cudaFree synchronise the device), and programs whose device
 * memory is entirely owned by another allocator (a framework's caching allocator or a
 * hard memory cap).  It computes what lbx_conserved_sums computes, sum over nodes of Q_k,
 * with the same deterministic FP64 reduction, but allocates nothing: its scratch is one
 * file-scope device array of LBX_STATIC_REDUCE_SCRATCH_DOUBLES doubles that every GPU
 * which loads the library holds until the process exits.
 *   sch          scheme the populations belong to (host handle only).
 *   populations  device buffer in the library's storage layout, e.g. the pointer from
 *                lbx_state_populations() or a buffer the caller passed to lbx_init();
 *                FP64 or FP32_SHIFT storage (FP16_SCALED -> LBX_ERR_UNSUPPORTED, its
 *                scales belong to the state).
 *   sums         device output, K float64 values, written on `stream`.
 *   nblocks      reduction blocks, 1..LBX_STATIC_REDUCE_MAX_BLOCKS, or 0 for 2 x SMs
 *                (capped); larger values fail with LBX_ERR_ARG.
 *   stream       cudaStream_t (NULL = legacy default stream); the call is asynchronous.
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress,
 * with that device current) and caches it; make that first call before any stream
 * capture.  All calls share the one array and it keeps the last call's contents (every
 * value a call reads is written earlier in the same call, so nothing is cleared); calls
 * whose work overlaps on the GPU race on it and must be ordered, e.g. on one stream. */
#define LBX_STATIC_REDUCE_MAX_BLOCKS 512
#define LBX_STATIC_REDUCE_SCRATCH_DOUBLES (LBX_STATIC_REDUCE_MAX_BLOCKS * 18 * 4 + 18 * 4)
lbx_status lbx_conserved_sums_static(const lbx_scheme* sch, const void* populations, double* sums,
                                     int nblocks, void* stream);

/* ---- peak probes used for the roofline denominators ---------------------------------- */
/* Streams a copy of `bytes` bytes (read + write counted) and a dependent FP64 FMA loop on
 * the given stream; returns measured GB/s and FP64 GFLOP/s (CUDA events).  Either output
 * may be NULL to skip that probe. */
lbx_status lbx_probe_peaks(size_t bytes, void* stream, double* copy_gbs, double* fp64_gflops,
                           double* fp32_gflops);

#ifdef __cplusplus
}
#endif
#endif /* LBX_H */
