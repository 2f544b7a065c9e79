/*
 * ffe.h - C ABI of the GB300 library for the general-relativistic force-free
 * electrodynamics (GRFFE) DG-FD hybrid scheme of arXiv:2404.01531.
 *
 * What the library computes (section numbers are the paper's):
 *   - the conservative 3+1 force-free system in densitised variables
 *     U = (E~^i, B~^i, psi~, phi~, q~), fluxes F^j and sources S (Sec. II.A),
 *     with the driver-term current (drift + eta parallel/rectifier) (Sec. II.B);
 *   - nodal DG-SEM on Legendre-Gauss-Lobatto points with mass lumping,
 *     Rusanov face fluxes and the exponential filter (Sec. III.A);
 *   - conservative FD on (2P+1)^3 subcells with WENO5-Z, Rusanov and the
 *     4th-order derivative corrector (Sec. III.C.2);
 *   - IMEX-SSP3(4,3,3) stepping with the stiff current and the cleaning damping
 *     implicit (Sec. III.B), and the algebraic E.B = 0 / E < B clamp
 *     (Sec. II.B, conventional approach) as an option;
 *   - the modal troubled-cell indicator on |B~| with DG<->FD switching and
 *     rollback of a troubled DG substep (Sec. III.C.1, III.C.3).
 *
 * Conventions for every entry point:
 *   - Every function returns ffe_status.  FFE_OK = 0.  On error a thread-local
 *     message is available from ffe_last_error(); no exception, longjmp or
 *     device trap crosses the ABI (a host allocation or thread start that
 *     fails inside the library is FFE_ENOMEM).
 *   - Arguments are validated before anything is enqueued (FFE_EINVAL).
 *   - "_dev" pointers are device pointers owned by the caller (for example a
 *     torch tensor's data_ptr()); "_host" pointers are host memory owned by the
 *     caller.  The library owns the context and everything it allocates.
 *   - All work is enqueued on the CUDA stream given to ffe_create (NULL = the
 *     legacy default stream).  Functions that return host data synchronise
 *     that stream.
 *   - State layout ("state vector", doubles): the DG block [9][n_dg] followed
 *     by the FD block [9][n_fd].  Element e owns DG nodes
 *     [e*(P+1)^3, (e+1)*(P+1)^3) with node index i + (P+1)(j + (P+1) k), i along
 *     xi^1 (fastest), and FD cells [e*(2P+1)^3, (e+1)*(2P+1)^3) ordered the same
 *     way.  Variable order: E~x E~y E~z B~x B~y B~z psi~ phi~ q~.  Only the block
 *     matching an element's mask (0 = DG, 1 = FD) is meaningful.
 */
#ifndef FFE_H
#define FFE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    FFE_OK = 0,
    FFE_EINVAL = 1,     /* invalid argument or configuration                   */
    FFE_ENOMEM = 2,     /* device or host allocation failed                    */
    FFE_ECUDA = 3,      /* a CUDA runtime call failed                          */
    FFE_ETIMEOUT = 4,   /* a bounded device wait gave up                       */
    FFE_ENUMERIC = 5,   /* NaN/Inf produced or the stiff solve did not converge */
    FFE_ESTATE = 6,     /* call not valid in the context's current state       */
    FFE_ENOTIMPL = 7    /* combination not implemented                         */
} ffe_status;

typedef struct ffe_ctx ffe_ctx;

/* domain kinds, boundary kinds, metric kinds, initial data, constraint modes */
enum { FFE_DOMAIN_BOX = 0, FFE_DOMAIN_SHELL6 = 1 };
enum { FFE_BC_PERIODIC = 1, FFE_BC_DIRICHLET = 2, FFE_BC_NO_INCOMING = 3, FFE_BC_STAR = 4,
       FFE_BC_OUTFLOW = 5   /* exterior state = interior state: an excision surface inside a
                               horizon, where the paper imposes no condition (Sec. IV.B.2) */ };
enum { FFE_METRIC_MINKOWSKI = 0, FFE_METRIC_KERR_SCHILD = 1 };
enum { FFE_ID_FAST_WAVE = 0, FFE_ID_BREAKDOWN = 1, FFE_ID_CLEANING_MODE = 2,
       FFE_ID_WALD = 3, FFE_ID_DIPOLE = 4,
       /* the paper's one-dimensional tests (App. A): fast wave with two kinks,
        * stationary Alfven wave, FFE breakdown */
       FFE_ID_FAST_WAVE_KINK = 5, FFE_ID_ALFVEN = 6, FFE_ID_BREAKDOWN_1D = 7 };
enum { FFE_RELAX = 0, FFE_HARD = 1, FFE_RELAX_THEN_HARD = 2 };
enum { FFE_INIT_KEEP_MASK = 1,     /* ffe_set_initial flags */
       FFE_INIT_VIA_FD = 2 };

/* Domain (Sec. III.A; shell: Sec. IV.B).  BOX: [lo, hi], boundary kind per axis
 * (periodic or a physical kind applied at both ends).  SHELL6: six cubed-sphere
 * wedges between r_in and r_out, equiangular angular map, logarithmic radial map;
 * bc_lo[0] applies at r_in, bc_hi[0] at r_out. */
typedef struct {
    int kind;
    double lo[3], hi[3];
    int bc_lo[3], bc_hi[3];
    double r_in, r_out;
    int shell_ks;   /* SHELL6 on FFE_METRIC_KERR_SCHILD: 1 = r_in, r_out and the
                       logarithmic radial map are in the spherical Kerr-Schild
                       radius r of the metric's spin a (App. B), the point of
                       unit direction v at radius r being x = r v + a (z^ x v),
                       so r = const is the spheroid (x^2+y^2)/(r^2+a^2) + z^2/r^2 = 1
                       (r_in between the horizons puts the whole inner surface
                       where every characteristic leaves the domain); 0 = the
                       sphere |x| = r.  With 1, FD subcells are FFE_ENOTIMPL
                       (tci_on must be 0; FFE_INIT_VIA_FD and FD masks are refused).
                       FFE_EINVAL on a box or a Minkowski metric. */
} ffe_domain;

/* Elements: BOX n[0] x n[1] x n[2]; SHELL6 n[0] = n[1] angular, n[2] radial per wedge. */
typedef struct { int n[3]; } ffe_elements;

/* Background metric (Sec. II.A; Kerr-Schild: App. B): mass M, spin a. */
typedef struct { int kind; double M, a; } ffe_metric;

/* Scheme parameters.  dt = 0 selects the CFL step
 * dt = cfl (dx)_min / lambda_max * c_over_D (Sec. III.B). */
typedef struct {
    double eta, kappa_psi, kappa_phi;   /* driver-term conductivity, cleaning damping  */
    double cfl, c_over_D, dt;
    int filter_on; double filter_a, filter_b;        /* exponential filter (Sec. III.A) */
    int tci_on, tci_M; double tci_alpha;             /* troubled-cell indicator          */
    double weno_eps; int fd_corrector;               /* FD subcell scheme                */
    int constraint_mode;                             /* FFE_RELAX | FFE_HARD | ...        */
    double omega_star;                               /* star rotation (FFE_BC_STAR)       */
    int recon;                                       /* FFE_RECON_WENO5Z | FFE_RECON_MP5  */
    int fd_chunk;                                    /* FD elements per scratch chunk: the FD
                                                        kernels walk the FD list in chunks of this
                                                        many elements (0 = 2048); bounds the FD
                                                        scratch whatever the FD population      */
    int fd_capacity;                                 /* ffe_create: FD slots of the context's
                                                        FD block (0 or >= elements: one per
                                                        element, FD block of element e at slot e);
                                                        fewer: a pool of slots that elements take
                                                        when they switch to FD and return when they
                                                        switch back (see ffe_get_layout); an element
                                                        flagged when none is free stays on DG and
                                                        status bit 2 is raised.  Ignored by
                                                        ffe_create_batch (its own argument)      */
} ffe_params;

/* FD reconstruction: WENO5-Z with q = 2 (the paper's, Sec. III.C.2) or MP5
 * (Suresh & Huynh's monotonicity-preserving limiter on the 5-point
 * interpolant); the adjoint is built for WENO5-Z only. */
enum { FFE_RECON_WENO5Z = 0, FFE_RECON_MP5 = 1 };

/* Sizes of the state vector. */
typedef struct {
    int n_elem, P, np1, nc;       /* elements, order, DG points and FD cells per direction */
    int64_t n_dg, n_fd;           /* DG nodes, FD cells in the whole context              */
    int64_t n_state;              /* doubles in a state vector: 9 (n_dg + n_fd)           */
    double dt, dxmin, t;          /* time step, (dx)_min, current time                    */
    int64_t steps;                /* steps taken                                          */
    int n_fd_elem;                /* elements currently on FD                             */
    int64_t node_updates;         /* DG nodes + FD cells advanced through an explicit RHS
                                     and its stage update, summed since ffe_set_initial     */
    int64_t fd_elem_updates;      /* FD elements advanced through an RHS and stage update
                                     (rollback redos included), since ffe_set_initial      */
    int64_t dg_elem_updates;      /* DG elements advanced likewise                         */
    int dg_ctas_per_sm[3];        /* persistent DG launch shapes the autotuner chose (CTAs per
                                     SM) for the highest order and, in a batch, the next two
                                     lower orders; 0 = not tuned (the first ffe_step tunes)   */
} ffe_info;

/* Create a context: builds the mesh, operator tables and geometry, allocates
 * the state and work buffers on the current device and binds `cuda_stream`
 * (a cudaStream_t, or NULL).  *out receives the context on success. */
ffe_status ffe_create(const ffe_domain* domain, const ffe_elements* elements, int P,
                      const ffe_metric* metric, const ffe_params* params,
                      void* cuda_stream, ffe_ctx** out);

/* Batched context (Sec. IV.C workloads, many independent magnetospheres): n_inst
 * six-wedge shells in flat space, each with its own domain (r_in, r_out,
 * boundary kinds), elements (n[0] angular, n[2] radial per wedge), order
 * P[i] in {3, 4, 5} and parameters params[i] (time step from its own CFL
 * condition, star rotation omega_star); every other scheme parameter must
 * equal params[0].  All instances advance together: one launch per kernel and
 * substep covers every element of every instance (the DG substep kernel: one
 * launch per element order present, each in CTAs sized for its order).
 * fd_capacity bounds the number of elements on FD subcells at any time
 * (0 = every element); an element the indicator flags when no FD slot is left
 * stays on DG and status bit 2 is raised.  State layout: every element owns a
 * DG slot of (Pmax+1)^3 nodes (its own (P+1)^3 at the front) and an FD element
 * owns one of fd_capacity FD slots of (2 Pmax+1)^3 cells (see ffe_get_layout). */
ffe_status ffe_create_batch(int n_inst, const ffe_domain* domains, const ffe_elements* elements, const int* P,
                            const ffe_metric* metric, const ffe_params* params, int fd_capacity,
                            void* cuda_stream, ffe_ctx** out);

/* Per-element layout (host copies, synchronising; any pointer may be NULL):
 * order of each element [n_elem], FD slot of each element [n_elem] (-1 when it
 * has none), instance of each element [n_elem], first element of each
 * instance [n_inst + 1], and the number of instances. */
ffe_status ffe_get_layout(ffe_ctx* ctx, int* elem_P, int* fd_slot, int* elem_inst, int* inst_first, int* n_inst);

/* Initial data for every instance of a context: id_params holds n_inst blocks
 * of n_params values, one block per instance (same meaning as ffe_set_initial). */
ffe_status ffe_set_initial_batch(ffe_ctx* ctx, int id_kind, const double* id_params, int n_params, int flags);

/* Set analytic initial data.  id_params (may be NULL when n_params = 0):
 *   FAST_WAVE      {amp}                 B=(1,b,0), E=(0,0,-b), b = 1 + amp sin(pi x)
 *   BREAKDOWN      {}                    current sheet of the breakdown workload
 *   CLEANING_MODE  {eps}                 B=(1+eps sin(pi x),0,0)
 *   WALD           {M, a, B0[, e]}       Wald's field (Kerr-Schild metric); E~ times e (default
 *                                        1; e = 0: the vacuum Wald problem's start, Sec. IV.B.2)
 *   DIPOLE         {mu, delta, chi}      B~ = curl[mu m x x/(r^2+delta^2)^(3/2)], m = (sin chi, 0, cos chi)
 *   FAST_WAVE_KINK {}                    B=(1,b,0), E=(0,0,-b), b = 1 | 0.85-1.5x | 0.7 across |x|<0.1
 *   ALFVEN         {}                    B=(1,1,b), E=(-b,0,1), b = 1 | 1.15+0.15 sin(5 pi x) | 1.3,
 *                                        q~ = -db/dx (Gauss's law)
 *   BREAKDOWN_1D   {}                    B=(1,b,b), E=(0,0.5,-0.5), b = 1 | -10x | -1
 * The data are set on the LGL nodes, then the troubled-cell indicator runs and
 * flagged elements take the data at their subcell centres (Sec. III.C.1/III.C.3).
 * flags & FFE_INIT_KEEP_MASK: no indicator; the context's current mask is kept
 * and its FD elements take the data at their subcell centres (fixed-mask runs).
 * flags & FFE_INIT_VIA_FD: the paper's start (Sec. III.C.1): every element on
 * FD with the data at its subcell centres; the FD indicator at the end of each
 * step returns smooth elements to DG.  Needs the indicator on and a flat
 * metric (FFE_EINVAL otherwise); excludes FFE_INIT_KEEP_MASK; not built for
 * batches (FFE_ENOTIMPL from ffe_set_initial_batch).
 * Resets time and step counters. */
ffe_status ffe_set_initial(ffe_ctx* ctx, int id_kind, const double* id_params, int n_params, int flags);

/* Explicit right-hand side F(U) (volume + boundary correction + explicit
 * sources; no stiff part) of the state vector U_dev under the context's
 * current mask, written to dUdt_dev (state-vector layout).  No state change. */
ffe_status ffe_rhs(ffe_ctx* ctx, const double* U_dev, double* dUdt_dev);

/* Advance the internal state by nsteps IMEX-SSP3(4,3,3) steps including the
 * troubled-cell indicator, rollback and FD->DG switching. */
ffe_status ffe_step(ffe_ctx* ctx, int nsteps);

/* Borrowed device view of the current state vector and mask (uint8 per element,
 * 0 = DG, 1 = FD); valid until the next mutating call.  Writes through the
 * view are not checked: a mask written there must hold 0 and 1 only (and, in
 * a batched context, match its FD slot map, see ffe_set_state). */
ffe_status ffe_get_state(ffe_ctx* ctx, double** U_dev, unsigned char** mask_dev);

/* Replace the state and mask from caller device buffers (state-vector layout);
 * either pointer may be NULL.  The mask is checked on the host first (one
 * E-byte copy, synchronising the context stream): bytes other than 0 and 1,
 * or, in a batched context, an element on FD without an FD pool slot or on DG
 * while holding one (pool slots change only through the indicator's
 * switches), give FFE_EINVAL with nothing replaced.  ffe_upload applies the
 * same check to its host mask. */
ffe_status ffe_set_state(ffe_ctx* ctx, const double* U_dev, const unsigned char* mask_dev);

/* Host copies of the state (synchronising); either pointer may be NULL. */
ffe_status ffe_download(ffe_ctx* ctx, double* U_host, unsigned char* mask_host);
ffe_status ffe_upload(ffe_ctx* ctx, const double* U_host, const unsigned char* mask_host);

/* Sizes, time step and counters. */
ffe_status ffe_get_info(ffe_ctx* ctx, ffe_info* info);

/* Device-side status bits accumulated since the last call (synchronising):
 * bit 0 NaN/Inf seen, bit 1 stiff solve hit its iteration cap.  Cleared on read. */
ffe_status ffe_get_status(ffe_ctx* ctx, int* status_bits);

/* Troubled-cell indicator ratio sqrt(sum u^2 / sum u^) per element for the DG
 * data of U_dev (all elements, whatever the mask), written to ratio_dev[n_elem]. */
ffe_status ffe_tci_ratio(ffe_ctx* ctx, const double* U_dev, double* ratio_dev);

/* Elements whose last indicator ratio was within 1e-12 (relative) of the
 * threshold during the last ffe_step call: copies up to `cap` indices to
 * idx_host and the count to *n (synchronising). */
ffe_status ffe_near_threshold(ffe_ctx* ctx, int* idx_host, int cap, int* n);

/* Kernel launches enqueued by the library since creation (for accounting);
 * graph replays count the kernel nodes of the captured step. */
ffe_status ffe_launch_count(ffe_ctx* ctx, int64_t* n);

/* Per-kernel timing.  With on = 1, ffe_step launches eagerly (no graph) and
 * brackets every kernel with CUDA events on the context stream, synchronising
 * once per step; totals accumulate until read.  ffe_profile_read writes a JSON
 * object {"kernel": [launches, total_ms, max_ms], ...} into buf (NUL-terminated,
 * truncated to cap) and clears the totals. */
ffe_status ffe_set_profiling(ffe_ctx* ctx, int on);
ffe_status ffe_profile_read(ffe_ctx* ctx, char* buf, size_t cap);

/* FD-subcell right-hand side that allocates no memory.  The paper has no
 * counterpart: this is a service for callers that cannot call cudaMalloc --
 * host applications that own all device memory and forbid allocations behind
 * their back, latency-critical paths where an allocation would stall.
 * ffe_create allocates a whole context, so those callers cannot reach
 * ffe_rhs; this entry point computes the explicit FD right-hand side (flat
 * metric, affine element of widths h_host[0..2]) of caller-built extended
 * blocks from caller-owned buffers:
 *   Uext_dev  [9][n_elem][(2P+7)^3]  the 9 evolved variables on each element's
 *             (2P+1)^3 subcells plus 3 ghost layers on every face (edge and
 *             corner ghost regions are never read), x fastest;
 *   dUdt_dev  [9][n_elem][(2P+1)^3]  output, same cell order as the FD block.
 * The current J~ of every cell, ghosts included, is computed from that cell's
 * state.  This is what ffe_rhs does for ghosts that hold an FD neighbour's
 * data or a boundary state; ghosts across a DG neighbour's face get that
 * neighbour's nodal current from ffe_rhs instead, so for them the two differ.
 * Its intermediate data (J~ at every extended cell and the face fluxes) live
 * in one fixed device array of 2^20 doubles (8 MiB) that every GPU loading the
 * library holds until exit; calls needing more (per element 3 (2P+7)^3 +
 * 27 (2P+2)(2P+1)^2 doubles, e.g. at most 19 elements at P = 5) are rejected
 * with FFE_EINVAL, as are P outside [3, 6], n_elem < 0, NULL buffers, widths that
 * are not positive and finite, eta < 0 or weno_eps <= 0 (non-finite values
 * included); these checks make no CUDA call, and n_elem = 0 returns FFE_OK
 * without one.  Devices 0 to 63 are served (FFE_EINVAL on a higher index).
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current and keeps it for the life
 * of the process: after a cudaDeviceReset of that device the kept address is
 * stale, so do not call this entry point again after such a reset.  All
 * calls share the array and each overwrites every entry it reads (nothing
 * needs clearing), so calls that overlap on the GPU (different streams, no
 * ordering between them) race.  Enqueued on cuda_stream. */
ffe_status ffe_fd_rhs_noalloc(int P, int n_elem, const double* h_host, double eta, double weno_eps,
                              int fd_corrector, const double* Uext_dev, double* dUdt_dev, void* cuda_stream);

/* ---- adjoint (reverse mode) ------------------------------------------------
 * Hand-written vector-Jacobian products of the hybrid DG-FD step with every
 * discrete decision frozen as the forward pass took it (piecewise
 * differentiability): the DG/FD mask (which must be frozen, ffe_freeze_mask:
 * FFE_ESTATE otherwise), the rectifier max(E^2-B^2,0), the stiff-solve branch
 * and the sign of S.n at a no-incoming-Poynting face, and in the HARD modes
 * the clamp's branch (E^2 > B^2 after the projection).  WENO5-Z weights are
 * differentiated (they are smooth).  Flat-metric shells (FFE_DOMAIN_SHELL6),
 * every constraint mode, WENO5-Z reconstruction (FFE_ENOTIMPL for MP5, the
 * Kerr-Schild metric and batches).  All buffers are device state vectors; lambda and the
 * outputs live on the representation each element uses (DG nodes of DG
 * elements, cells of FD elements) and are zero on the other one. */

/* Freeze (on != 0) or release the DG/FD mask: while frozen the troubled-cell
 * indicator is not evaluated, no element switches, and ffe_step advances the
 * hybrid operator with the current mask.  Released, the indicator setting of
 * ffe_create applies again.  Invalidates the captured step graph. */
ffe_status ffe_freeze_mask(ffe_ctx* ctx, int on);

/* out_dev = lambda^T dF/dU at U_dev (F the explicit right-hand side of ffe_rhs);
 * *omega_bar (host, may be NULL) += lambda^T dF/dOmega (star rotation). */
ffe_status ffe_rhs_vjp(ffe_ctx* ctx, const double* U_dev, const double* lam_dev, double* out_dev, double* omega_bar);

/* One IMEX step backward: given the step's input state U_n (U_dev) and
 * lambda_{n+1} = dL/du_{n+1}, writes lambda_n = dL/du_n (lam_out_dev, may alias
 * nothing else) and adds the step's d L/d Omega to *omega_bar (may be NULL).  The
 * step's internal stages are recomputed from U_n (checkpointed recomputation). */
ffe_status ffe_adjoint_step(ffe_ctx* ctx, const double* U_dev, const double* lam_in_dev, double* lam_out_dev,
                            double* omega_bar);

/* The two halves of ffe_adjoint_step, for callers that keep a segment's stages
 * in device memory instead of recomputing them (Sec. III.B stages; checkpointed
 * recomputation with the stage states stored):
 * ffe_adjoint_forward recomputes the step's stages from U_n; when stages_dev is
 * not NULL it receives them as five consecutive state vectors [U2][T3][U3][T4]
 * [U4] (T_s the filtered explicit part of stage s), and when U_next_dev is not
 * NULL it receives u_{n+1} (must not alias U_dev).
 * ffe_adjoint_reverse runs the backward sweep from those stages: same result
 * as ffe_adjoint_step(U_dev, lam_in, lam_out, omega_bar).  In the HARD modes
 * the clamp at the step's end needs the pre-clamp state, which the stages do
 * not hold, so the reverse recomputes the step (as ffe_adjoint_step does). */
ffe_status ffe_adjoint_forward(ffe_ctx* ctx, const double* U_dev, double* stages_dev, double* U_next_dev);
ffe_status ffe_adjoint_reverse(ffe_ctx* ctx, const double* U_dev, const double* stages_dev, const double* lam_in_dev,
                               double* lam_out_dev, double* omega_bar);

/* Spin-down luminosity through the shell's coordinate surface r = r_L (Sec.
 * IV.C.2; the sphere |x| = r_L unless shell_ks): L = closed integral of
 * (E x B).n^ dA on the radial element layer containing r_L (xi^3
 * interpolation, LGL quadrature, exact area element and outward normal).  *L_host receives L;
 * when grad_dev is not NULL, scale * dL/dU is added to it.  Single contexts
 * (batches: FFE_DIAG_LUMINOSITY with an instance index). */
ffe_status ffe_luminosity(ffe_ctx* ctx, const double* U_dev, double r_L, double* L_host, double* grad_dev,
                          double scale);

/* Derivative of the initial DG state set by ffe_set_initial with respect to its
 * parameter `which` (DIPOLE: 0 = mu, 2 = chi) at the nodes, into dU_dev. */
ffe_status ffe_initial_tangent(ffe_ctx* ctx, int which, double* dU_dev);

/* Checkpoint / resume.  ffe_save writes the context's evolving state to a
 * caller-owned host buffer: time, step count, initial-data kind and
 * parameters (the boundary data are rebuilt from them), the state vector, the
 * DG/FD mask, the FD slot pool of a batched context and the update counters.
 * With host_buf = NULL it only stores the size needed in *bytes; otherwise
 * *bytes is the buffer's size on entry (FFE_EINVAL if too small) and the
 * bytes written on return; synchronises the context stream.  ffe_load
 * restores such a checkpoint into a context created with the same domain,
 * elements, orders, metric and FD pool (FFE_EINVAL otherwise); stepping on
 * from it gives the same results as the saved context would.  Every count
 * and index of the buffer (parameter count, mask bytes 0/1, the FD pool's
 * element <-> slot maps and free list) is checked on the host first: a
 * truncated, foreign or corrupt buffer is FFE_EINVAL and leaves the context
 * unchanged.  Adjoint work fields are not part of a checkpoint. */
ffe_status ffe_save(ffe_ctx* ctx, void* host_buf, size_t* bytes);
ffe_status ffe_load(ffe_ctx* ctx, const void* host_buf, size_t bytes);

/* Pointwise constraint diagnostics (flat metric; FFE_ENOTIMPL on
 * Kerr-Schild) of a state vector U_dev (NULL: the context's state), over the
 * DG nodes of DG elements and the subcells of FD elements: out_host[0] =
 * max |E~.B~|, [1] = min (B~^2 - E~^2), [2] = max |psi~|, [3] = max |phi~|.
 * Synchronises the context stream. */
ffe_status ffe_constraints(ffe_ctx* ctx, const double* U_dev, double* out_host);

/* Borrowed device view of the DG/FD mask (uint8 per element, 0 = DG,
 * 1 = FD; Sec. III.C.3) and, when n_elem is not NULL, the element count;
 * valid until the context is destroyed, contents current after the context
 * stream reaches the point of the call. */
ffe_status ffe_get_mask(ffe_ctx* ctx, const unsigned char** mask_dev, int* n_elem);

/* Same as ffe_freeze_mask (declared with the adjoint below): on != 0 replays
 * the current mask, with no troubled-cell indicator and no switching, in
 * every following step (the frozen-branch runs of finite-difference and
 * complex-step checks); on = 0 restores the indicator setting of ffe_create. */
ffe_status ffe_set_frozen_masks(ffe_ctx* ctx, int on);

/* Diagnostics of the context's current state, written to out_host
 * (synchronising the context stream):
 *   FFE_DIAG_L2_ERR      the L2 error norm of Sec. IV.B.1 (Table II),
 *                        L2 = sqrt((1/n) sum_k sum_v (U_v,k - R_v,k)^2) over the
 *                        n points k (DG nodes of DG elements, subcells of FD
 *                        elements) and the variables v0 <= v < v0 + nv, where
 *                        R is the analytic initial data of ffe_set_initial at
 *                        those points (the exact solution of a stationary
 *                        problem such as the Wald field); args = {v0, nv}
 *                        (NULL: {3, 3}, the magnetic field B~); out_host[0] = L2,
 *                        out_host[1] = n.  FFE_ESTATE before ffe_set_initial.
 *                        The reference is evaluated on the host and kept on the
 *                        device until the mask or the initial data change; the
 *                        sum is reduced on the device (deterministic).
 *   FFE_DIAG_LUMINOSITY  args[0] = r_L: out_host[0] = the luminosity of
 *                        ffe_luminosity through r = r_L (shells).  Batched
 *                        contexts: args[1] = the instance (an integer index),
 *                        whose shell and elements the surface covers; the
 *                        instance must have the batch's top order
 *                        (FFE_ENOTIMPL else).  A radius outside the shell is
 *                        FFE_EINVAL.
 *   FFE_DIAG_CONSTRAINTS out_host[0..3] as ffe_constraints (flat metric).
 *   FFE_DIAG_BFLUX_UPPER args[0] = R: out_host[0] = the magnetic flux of B~
 *                        through the upper half (z > 0) of the shell's
 *                        coordinate surface of radius R (the sphere |x| = R;
 *                        with shell_ks the spheroid of Kerr-Schild radius R, so
 *                        R = r+ is the outer horizon itself), on the radial
 *                        element layer containing R (xi^3 interpolation, LGL
 *                        quadrature, exact area element and outward normal).
 *                        B~ has zero coordinate divergence, so on a shell
 *                        of spheres R = sqrt(r+^2 + a^2) gives the same flux
 *                        (same equator), the quantity of Sec. IV.B.2.
 *                        Shells with n[0] even
 *                        (the equator on element boundaries), FFE_EINVAL else;
 *                        batched contexts take args[1] as for the luminosity. */
enum { FFE_DIAG_L2_ERR = 0, FFE_DIAG_LUMINOSITY = 1, FFE_DIAG_CONSTRAINTS = 2, FFE_DIAG_BFLUX_UPPER = 3 };
ffe_status ffe_diagnostic(ffe_ctx* ctx, int kind, const double* args, double* out_host);

/* Cartesian coordinates of the DG nodes [3][n_dg] and of the FD subcell
 * centres [3][n_fd] (every element's block, in state-vector order), copied
 * into caller-owned device arrays (either may be NULL) on the context stream.
 * FD centres of batched contexts are not stored (FFE_ENOTIMPL when
 * xyz_fd_dev is not NULL). */
ffe_status ffe_get_coords(ffe_ctx* ctx, double* xyz_dg_dev, double* xyz_fd_dev);

/* Reciprocal 1/x that the WENO5-Z weights use (the hardware approximation
 * rcp.approx.ftz.f64 refined by two Newton-Raphson steps), evaluated
 * elementwise: y_dev[i] = 1/x_dev[i], i < n, both device arrays of doubles
 * (caller-owned; x_dev and y_dev may be the same).  Defined for positive
 * normal x whose reciprocal is normal (below 2^1022); within about one ulp of
 * the correctly rounded quotient.  For accuracy tests; enqueued on
 * cuda_stream.  FFE_EINVAL for n < 0 or a NULL array with n > 0. */
ffe_status ffe_eval_recip(const double* x_dev, double* y_dev, int64_t n, void* cuda_stream);

/* FP64 FMA throughput of the current device, measured: a register-only
 * loop of independent fused multiply-adds (4 CTAs of 256 threads per SM, 8
 * chains per thread, 2^16 steps each, no memory traffic) timed with CUDA
 * events on cuda_stream (synchronising it); *tflops_host receives the rate in
 * TFLOP/s (an FMA counts 2).  The measured denominator of the FP64 roofline
 * reported beside the one derived from the SM count and clock.  Not part of
 * the method. */
ffe_status ffe_fp64_fma_rate(void* cuda_stream, double* tflops_host);

/* Thread-local message of the last failed call ("" if none). */
const char* ffe_last_error(void);

/* Free the context and everything it owns (synchronises its stream). */
void ffe_destroy(ffe_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* FFE_H */
