/*
 * lbm.h -- C ABI of the GB300 Shan-Chen multiphase lattice Boltzmann library.
 *
 * One time step follows arXiv 2506.17713 (JAX-LaB), Section 2:
 *   density rho^k = sum_i f_i^k (Eq. macroeq / macroeq_mcp),
 *   improved virtual density at solid nodes (Section 2.4, Eq. improved_virtual_density),
 *   pseudopotential psi^k, U^k from an equation of state (Eq. eos_potential),
 *   mixed Shan-Chen / Zhang-Chen interaction force with cross-component terms
 *   (Eq. software_ff_force_mcmp) plus a body force,
 *   BGK or MRT collision (Eq. collision_model) with Exact Difference Method forcing (Eq. edm),
 *   streaming with halfway bounce-back at solids (Eq. lbe_steps),
 *   optional constant-density x faces.
 *
 * Conventions (all entry points):
 *   - Node index n = x + nx*(y + ny*z), x fastest. N = nx*ny*nz. D2Q9 has nz = 1.
 *   - Scalar fields are [N]; vector fields are [D][N] (D = 2 for D2Q9, 3 for D3Q19);
 *     populations are [Q][N] in the library's velocity order (lbm_velocity_set).
 *   - Arguments tagged `where` are host pointers (LBM_HOST) or device pointers
 *     (LBM_DEVICE) of the current CUDA device. The library copies inputs; the caller
 *     keeps ownership of every buffer it passes.
 *   - The library never allocates device memory: the caller allocates one device
 *     workspace of lbm_workspace_size() bytes and keeps it alive until lbm_destroy().
 *   - All device work is enqueued on the caller's stream (cudaStream_t passed as void*,
 *     NULL = legacy default stream). Entry points that return data to the host
 *     synchronise that stream.
 *   - No exception crosses the ABI. A context is not thread safe.
 *   - Errors are sticky: after a CUDA error or a detected instability every later
 *     call on the context returns the same status until it is destroyed.
 *   - Precision: LBM_FP32 and LBM_FP64 store and compute in that type. LBM_FP16S and
 *     LBM_BF16S compute in FP32 and store each population as the 16-bit (FP16 / BF16)
 *     deviation f_i - w_i rho_ref[k] from the lattice weights times a reference density,
 *     rounded to nearest. This halves the bytes of a step. The global mass and momentum sums
 *     and the residual stay FP64 in every mode.
 */
#ifndef GB300_LBM_H
#define GB300_LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LBM_OK = 0,
    LBM_ERR_INVALID_ARG = 1, /* a pointer, size, enum or parameter is out of range */
    LBM_ERR_WORKSPACE = 2,   /* workspace missing, misaligned (256 B) or too small */
    LBM_ERR_CUDA = 3,        /* a CUDA runtime call or kernel launch failed */
    LBM_ERR_UNSTABLE = 4,    /* non-finite or non-positive density met in a step */
    LBM_ERR_TIMEOUT = 5,     /* a bounded device-side wait gave up */
    LBM_ERR_STATE = 6        /* call out of order (e.g. step before init) */
} lbm_status;

enum { LBM_D2Q9 = 0, LBM_D3Q19 = 1 };
enum { LBM_FP32 = 0, LBM_FP64 = 1, LBM_FP16S = 2, LBM_BF16S = 3 };
enum { LBM_BGK = 0, LBM_MRT = 1 };
/* equilibrium velocity of a component: its own bare velocity j^k / rho^k
 * (Eq. macroeq_mcp) or the Shan-Chen common velocity sum_k j^k/tau_k / sum_k rho^k/tau_k */
enum { LBM_UEQ_COMPONENT = 0, LBM_UEQ_COMMON = 1 };
/* pseudopotential: from an EOS (Eq. eos_potential), psi = rho (Section 3.3.2),
 * psi = exp(-1/rho) (Section 5) */
enum { LBM_PSI_EOS = 0, LBM_PSI_RHO = 1, LBM_PSI_EXP = 2 };
/* equations of state named in Section 2.2 */
enum { LBM_EOS_CS = 0, LBM_EOS_PR = 1, LBM_EOS_VDW = 2, LBM_EOS_RK = 3, LBM_EOS_RKS = 4 };
/* face kinds: periodic; wall (halfway bounce-back, neutral wetting); constant density
 * (x faces only) */
enum { LBM_BC_PERIODIC = 0, LBM_BC_WALL = 1, LBM_BC_PRESSURE = 2 };
enum { LBM_HOST = 0, LBM_DEVICE = 1 };
/* forcing of the collision: the Exact Difference Method of Eq. edm (default), or the
 * moment-space forcing F_m that Eq. mrt_surface (Section 2.3) places inside M^-1[...] next
 * to the relaxation -- the scheme of Li et al. (2013) for the surface-tension adjustment,
 * i.e. the forcing of Guo et al. (2002) in moment space: equilibrium at the physical
 * velocity v = u + F/(2 rho), source (I - S/2) M S_i with
 * S_i = w_i [(e_i - v)/c_s^2 + (e_i.v) e_i/c_s^4].F. It equals the EDM update minus S
 * applied to the moments of rho du du / 4 (du = F/rho), so it lacks EDM's F F / rho stress,
 * and with it the surface tension scales with 1 - kappa as Section 2.3 states. D2Q9 only
 * (LBM_ERR_INVALID_ARG for D3Q19), BGK or MRT. */
enum { LBM_FORCING_EDM = 0, LBM_FORCING_MOMENT = 1 };
/* kernel schedule of a step. AUTO and TWO_PASS: a density pass (psi to HBM) and a collide
 * pass, back to back. SLAB_OVERLAP (D3Q19 lattices of 64 or more planes without solids,
 * else TWO_PASS): the same two passes over z slabs of about 32 planes, overlapped on two
 * internal streams forked from and joined back to the caller's stream (the collide of a
 * slab starts once the density of its neighbour slabs is done); on GB300 at 256^3 it
 * measured 6% slower than TWO_PASS, because the collide pass already occupies every SM.
 * SINGLE_PASS (periodic D3Q19 lattices without solids only, else two passes): psi is
 * recomputed on chip from the populations, which are read and written once; on GB300 the
 * accurate FP32 arithmetic makes that recompute cost more issue slots than the HBM traffic
 * it saves. All give the same values bit for bit. */
enum { LBM_SCHEDULE_AUTO = 0, LBM_SCHEDULE_TWO_PASS = 1, LBM_SCHEDULE_SINGLE_PASS = 2,
       LBM_SCHEDULE_SLAB_OVERLAP = 3 };

/*
 * Problem parameters (all per component k = 0, 1; entries of absent components are ignored).
 *
 *   tau[k]            relaxation time; kinematic viscosity c_s^2 (tau - 1/2).
 *   mrt_s[k][m]       MRT relaxation rate of moment m of the Gram-Schmidt basis
 *                     (D2Q9: Lallemand & Luo order rho,e,eps,jx,qx,jy,qy,pxx,pxy;
 *                     D3Q19: d'Humieres 2002 order rho,e,eps,jx,qx,jy,qy,jz,qz,
 *                     3pxx,3pixx,pww,piww,pxy,pyz,pxz,mx,my,mz). The stress rates are
 *                     replaced by 1/tau[k] and the conserved ones by 0.
 *   eos_a/b/R/omega   EOS parameters a, b, R and acentric factor omega (PR, RKS).
 *   T_red[k]          temperature T / Tc, Tc being the exact critical temperature of
 *                     the EOS (where dp/drho = d2p/drho2 = 0).
 *   alpha[k]          pressure scaling alpha^k of Eq. eos_potential.
 *   A[k]              Zhang-Chen / Shan-Chen mixing weight A_kk of Eq. software_ff_force_mcmp.
 *   g[k][k']          interaction strengths g_kk'; g_kk = -1 for an EOS pseudopotential.
 *   wet_phi, wet_drho virtual solid density rho_s = wet_phi * rho_ave - wet_drho
 *                     (phi >= 1 with drho = 0 for theta <= 90 deg, phi = 1 with drho >= 0
 *                     above), limited to [rho_min, rho_max].
 *   body_accel[k][d]  body acceleration a^k: the body force is rho^k a^k. On D2Q9 the z
 *                     component must be 0 (LBM_ERR_INVALID_ARG otherwise).
 *   bc[f]             face kinds, faces -x,+x,-y,+y,-z,+z (z faces ignored in 2-D).
 *   bc_rho[f][k]      densities of constant-density faces.
 *
 * Interaction weights G_i = w_i / c_s^2 on all Q-1 links; psi = sqrt(max(0, 2 U / g_kk))
 * with U = alpha p_EOS - c_s^2 rho for the EOS kind, and U = g_kk psi^2 / 2 otherwise.
 * Across non-periodic faces the force and wetting stencils read the coordinate-clamped
 * in-domain node.
 */
typedef struct lbm_params {
    int lattice;     /* LBM_D2Q9 | LBM_D3Q19 */
    int nx, ny, nz;  /* nz = 1 for D2Q9 */
    int ncomp;       /* 1 | 2 */
    int real;        /* LBM_FP32 | LBM_FP64 | LBM_FP16S | LBM_BF16S */
    int collision;   /* LBM_BGK | LBM_MRT */
    int velocity;    /* LBM_UEQ_COMPONENT | LBM_UEQ_COMMON */
    double tau[2];
    double mrt_s[2][19];
    int psi_kind[2];
    int eos[2];
    double eos_a[2], eos_b[2], eos_R[2], eos_omega[2], T_red[2];
    double alpha[2];
    double A[2];
    double g[2][2];
    double wet_phi[2], wet_drho[2];
    double rho_min[2], rho_max[2];
    double body_accel[2][3];
    int bc[6];
    double bc_rho[6][2];
    int schedule;    /* LBM_SCHEDULE_AUTO | _TWO_PASS | _SINGLE_PASS | _SLAB_OVERLAP */
    double rho_ref[2]; /* LBM_FP16S / LBM_BF16S: reference density of the stored deviation
                          f_i - w_i rho_ref[k] (1 = the lattice weights); ignored otherwise */
    double kappa[2];   /* surface-tension adjustment (Section 2.3, Eqs. mrt_surface and
                          li_surface_adjust): the MRT collision gains the moment source
                          C = [0, 1.5 s_e (Qxx+Qyy), -1.5 s_eps (Qxx+Qyy), 0, 0, 0, 0,
                          -s_nu (Qxx-Qyy), -s_nu Qxy] with
                          Q = kappa g_kk/2 [(1-A) psi sum_i G_i (psi(x+e_i)-psi) e_i e_i
                                            + A/2 sum_i G_i (psi(x+e_i)^2-psi^2) e_i e_i].
                          0 = off. Nonzero only with D2Q9 and MRT (the paper gives no D3Q19
                          form): LBM_ERR_INVALID_ARG otherwise. */
    int forcing;       /* LBM_FORCING_EDM (0) | LBM_FORCING_MOMENT (D2Q9) */
} lbm_params;

typedef struct lbm_ctx lbm_ctx;

/* Bytes of device workspace needed for these parameters (Section 2.6 data layout:
 * one population array per component, here two of them for pull streaming).
 * Returns LBM_ERR_INVALID_ARG for invalid parameters. */
lbm_status lbm_workspace_size(const lbm_params* p, size_t* bytes);

/* Create a context on the current CUDA device: the lattice, EOS, wetting and boundary
 * parameters of one problem (Section 2: Eqs. lbe, collision_model, eos_potential,
 * software_ff_force_mcmp, improved_virtual_density; the critical temperature of each
 * EOS is found from its definition, Section 3.1). d_workspace: device pointer, 256-byte
 * aligned, at least lbm_workspace_size() bytes, owned by the caller; stream: the
 * caller's cudaStream_t. On success *out receives the context (host memory owned by
 * the library, freed by lbm_destroy). The geometry starts all-fluid. Returns
 * LBM_ERR_INVALID_ARG for invalid parameters or pointers, LBM_ERR_WORKSPACE for a
 * missing, misaligned or small workspace, LBM_ERR_CUDA if the device set-up fails. */
lbm_status lbm_create(const lbm_params* p, void* d_workspace, size_t bytes, void* stream,
                      lbm_ctx** out);

/* Solid mask, N bytes, 1 = solid, 0 = fluid (Sections 3.4, 2.4). Builds the list of
 * boundary solids (solids read by a fluid node's stencil). Invalidates the fields:
 * call lbm_init_fields or lbm_set_populations afterwards. */
lbm_status lbm_set_geometry(lbm_ctx* ctx, const uint8_t* solid, int where);

/* Populations of component comp := f^eq(rho, u) at fluid nodes (Eq. macroeq with the
 * second-order equilibrium). rho: [N] doubles; u: [D][N] doubles or NULL for rest.
 * u is the velocity of the equilibrium populations, i.e. the bare velocity
 * sum_i f_i e_i / rho; lbm_macroscopic reports (sum_i f_i e_i + F/2) / rho, which is
 * F/(2 rho) higher. To restart from a reported field, subtract F/(2 rho) first. */
lbm_status lbm_init_fields(lbm_ctx* ctx, int comp, const double* rho, const double* u,
                           int where);

/* Advance nsteps time steps (Eq. lbe_steps), enqueued on the context stream. */
lbm_status lbm_step(lbm_ctx* ctx, int nsteps);

/* Density and velocity u = (sum_i f_i e_i + F/2) / rho of component comp, or of the
 * mixture (sum over components) for comp = -1, at the current time (Eq. after Eq. edm).
 * Element type = the context's compute type (double for LBM_FP64, float otherwise).
 * rho: [N], u: [D][N]; either may be NULL; solids give 0. */
lbm_status lbm_macroscopic(lbm_ctx* ctx, int comp, void* rho, void* u, int where);

/* Total mass sum_x rho^k and momentum sum_x (j^k + F^k/2) per component (Eq. macroeq_mcp
 * and the velocity after Eq. edm; mass is conserved exactly by the step, Section 3.1),
 * summed in FP64 in a fixed order (deterministic). mass: [ncomp]; momentum: [ncomp][3].
 * residual (may be NULL): ||u - u_prev||_2 / ||u||_2 of the mixture velocity over fluid
 * nodes, u_prev being the velocity at the previous call that asked for a residual
 * (1.0 on the first such call). The paper runs its steady cases to a steady state
 * (Sections 3.1 and 3.4.1) without naming a criterion; this residual, taken every k steps
 * and compared with a threshold such as 1e-6, is the reading used here.
 * Synchronises; reports LBM_ERR_UNSTABLE if a step met a non-finite or non-positive
 * density. */
lbm_status lbm_diagnostics(lbm_ctx* ctx, double* mass, double* momentum, double* residual);

/* Post-stream populations of component comp, [Q][N] of the compute type (checkpoint /
 * inspection; the paper has no passage on checkpoints: this is the state f_i of
 * Eq. lbe_steps after streaming). lbm_set_populations restores them exactly (bit for bit), except for the
 * populations that constant-density faces recompute. With 16-bit storage the values are
 * the stored deviations plus w_i rho_ref in FP32, and lbm_set_populations rounds
 * f_i - w_i rho_ref back to the storage type (the values lbm_get_populations returned
 * round back to the stored bits). */
lbm_status lbm_get_populations(lbm_ctx* ctx, int comp, void* f, int where);
lbm_status lbm_set_populations(lbm_ctx* ctx, int comp, const void* f, int where);

/* Velocity set in the library's order: e: [Q][3] ints, w: [Q] doubles (either NULL). */
lbm_status lbm_velocity_set(const lbm_ctx* ctx, int* q, int* e, double* w);

/* Wait for the context stream; returns the sticky status. */
lbm_status lbm_sync(lbm_ctx* ctx);

/* Advance nsteps time steps like lbm_step, recording CUDA events on the context
 * stream between the kernels of every step, then synchronise. ms[0], ms[1], ms[2]
 * receive the summed device time (milliseconds) of the density, virtual-density and
 * collide kernels; launches[0..2] the number of launches of each. Timing aid for the
 * benchmark; the arithmetic is that of lbm_step. The kernels run back to back here (no
 * slab overlap). With the single-pass schedule the density slot stays 0 and the collide
 * slot holds the single-pass kernel. */
lbm_status lbm_profile_step(lbm_ctx* ctx, int nsteps, double* ms, long long* launches);

/* Bandwidth probe of the collide pass's access pattern: nsteps launches of a kernel that
 * gathers the post-stream populations of every fluid node exactly as the collide pass
 * does (pull streaming, bounce-back, the same launch shape) and stores them unchanged in
 * the other buffer -- free streaming, no collision, force or psi. *ms receives the summed
 * device time (milliseconds, CUDA events on the context stream, synchronised after each
 * launch). The populations end streamed nsteps times: this replaces the state of the
 * lattice, so it is for benchmarks on a context that is not needed afterwards. No
 * counterpart in the paper. */
lbm_status lbm_stream_probe(lbm_ctx* ctx, int nsteps, double* ms);

/* Number of kernels this context has launched since creation. */
long long lbm_kernel_launches(const lbm_ctx* ctx);

/* Absolute temperature T_red * Tc used for component comp (EOS pseudopotential). */
lbm_status lbm_temperature(const lbm_ctx* ctx, int comp, double* T);

/* Release the context (not the caller's workspace). NULL is ignored. */
void lbm_destroy(lbm_ctx* ctx);

/* Static string naming a status. */
const char* lbm_status_str(lbm_status s);

/*
 * Batches (the paper advances many porous samples, Section 3.4; its code does
 * not batch them). A batch advances several lattices in lock step with one
 * persistent kernel launch per pass (density, virtual density, collide) for all of
 * them, two time steps per replay of a CUDA graph captured on the first call.
 * The lattices of a batch may differ in size and geometry, but must share
 * lattice, real, ncomp, collision and whether they have solids or closed faces.
 * Every context must outlive the batch, and the caller orders work on the
 * contexts' streams and the batch stream (e.g. by using one stream for all).
 * Results are those of lbm_step on each lattice, bit for bit.
 *
 * lbm_batch_workspace_size: device bytes of the batch's lattice table for ctxs[0..n).
 *   LBM_ERR_INVALID_ARG if n < 1, a context is NULL or the contexts differ in the
 *   properties above.
 * lbm_batch_create: d_workspace (device, 256-byte aligned, >= that many bytes, owned
 *   by the caller), stream = the stream every batch step is enqueued on. Each context
 *   may appear once. The batch itself allocates no device memory; the CUDA graph it
 *   instantiates holds driver resources until lbm_batch_destroy.
 * lbm_batch_autotune: times each pass over the current state for CTA sizes 128 and
 *   256 and persistent grids of 2 to 16 CTAs (of 256 threads) per SM, and keeps the
 *   fastest. The passes it repeats are idempotent, so the state does not change
 *   (only the status counters of a lattice whose density is already out of range
 *   count again). config (may be NULL): [3][2] int, the chosen (CTA size, grid) of
 *   the density, virtual-density and collide passes. Synchronises the batch stream.
 * lbm_batch_step: nsteps time steps of every lattice, enqueued on the batch stream.
 *   Returns the sticky error of any lattice (LBM_ERR_STATE before its fields are
 *   initialised); a CUDA failure makes every lattice of the batch sticky.
 * lbm_batch_launches: kernel launches issued by batch steps so far (graph replays
 *   count their kernels); per-context launch counters do not include them.
 */
typedef struct lbm_batch lbm_batch;
lbm_status lbm_batch_workspace_size(lbm_ctx* const* ctxs, int n, size_t* bytes);
lbm_status lbm_batch_create(lbm_ctx* const* ctxs, int n, void* d_workspace, size_t bytes, void* stream,
                            lbm_batch** out);
lbm_status lbm_batch_autotune(lbm_batch* b, int* config);
lbm_status lbm_batch_step(lbm_batch* b, int nsteps);
long long lbm_batch_launches(const lbm_batch* b);
void lbm_batch_destroy(lbm_batch* b);

/*
 * Mass without allocation. The paper has no counterpart: this is a service for callers
 * that cannot allocate device memory at all -- processes where a framework owns every
 * allocation, or callers whose memory is used up by the lattice itself. It returns the
 * same sums as the mass part of lbm_diagnostics, from populations the caller already
 * holds. It copies its totals to host memory and synchronises the stream, which a stream
 * being captured into a CUDA graph cannot do: on such a stream it returns
 * LBM_ERR_INVALID_ARG before enqueuing anything, and the capture stays valid.
 *
 *   p     lattice parameters; lattice, nx, ny, nz, ncomp and real are used.
 *   d_f   device pointer, post-stream populations [ncomp][Q][N] of the real type of p,
 *         the layout lbm_get_populations writes (solid nodes hold 0). Only LBM_FP32 and
 *         LBM_FP64 are accepted (LBM_ERR_INVALID_ARG for the 16-bit storage modes).
 *   mass  host pointer, ncomp doubles: sum over nodes of sum_i f_i, per component, summed
 *         in FP64 in a fixed order.
 *   stream  cudaStream_t (NULL = legacy default stream); the call synchronises it.
 *
 * No cudaMalloc, cudaFree or allocating library routine is called. The reduction's
 * scratch is one file-scope device array of 16 KB, held by every GPU that loads the
 * library until the process exits; it holds the partial sums of at most
 * LBM_NOALLOC_MAX_NODES nodes (256^3), and larger lattices are rejected with
 * LBM_ERR_INVALID_ARG before any device work. The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress) with that device current and caches it
 * for later calls (the cache is safe to fill from several host threads). Every call
 * shares the array and leaves its last contents there; each call overwrites all it
 * reads. Calls that overlap on the GPU (different streams, or different host threads)
 * race on the array.
 */
#define LBM_NOALLOC_MAX_NODES (256 * 256 * 256)
lbm_status lbm_mass_noalloc(const lbm_params* p, const void* d_f, double* mass, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* GB300_LBM_H */
