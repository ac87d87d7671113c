/*
 * acmhd_fr.h - C ABI of the GB300 (sm_103a) flux-reconstruction library for
 * the artificial-compressibility Navier-Stokes equations with hyperbolised
 * diffusion (ACM-HD).
 *
 * What is computed (paper: Trojak, Watson & Witherden, "Hyperbolic Diffusion
 * in Flux Reconstruction: Optimisation through Kernel Fusion within
 * Tensor-Product Elements"):
 *   R = -div F(U) + S(U)
 * for the ACM-HD system of Sec. 2.2 (Eq. acmhd_2d for d = 2, Eq. acmhd_nd for
 * d = 3), discretised by flux reconstruction (Sec. 2.1, FR divergence
 * equation) on a periodic, uniform, axis-aligned mesh of affine quadrilateral
 * or hexahedral elements with (p+1)^d Gauss-Legendre solution points, using
 * the six stages of Table fr_adv.  Common interface flux: Rusanov on the
 * hyperbolic (P, V) equations and the mean flux on the auxiliary equations
 * (Sec. 5).
 *
 * Variables (n_v = 1 + d + d^2): P, V = (u, v[, w]), then d(V_i)/dx_b at
 * index 1 + d + i*d + b.  3-D: P,u,v,w,qx,qy,qz,rx,ry,rz,sx,sy,sz.
 *
 * State layout ("SoA, elements fastest"): a state is one device buffer of
 * n_v * (p+1)^d * elem_stride values of the context's precision (float or
 * double), value (v, pt, e) at offset (v * (p+1)^d + pt) * elem_stride + e,
 * with pt = i + m j + m^2 k (i along x, m = p + 1) and
 * e = ex + nx (ey + ny ez).  elem_stride >= n_elem is a multiple of 32
 * (fr_layout reports it); padding entries are read but never influence
 * entries e < n_elem, and are written with unspecified values.  Device
 * pointers must be 16-byte aligned.
 *
 * Ownership: the caller owns every state buffer it passes.  The context owns
 * its operator constants, face-trace scratch and time-stepping registers,
 * which fr_destroy releases.  A context is bound to the device that was
 * current when fr_create ran; calls must be made with that device current.
 *
 * Streams: `stream` is a cudaStream_t (NULL = legacy default stream).  Unless
 * stated otherwise, calls only enqueue work and do not synchronise the host.
 * Calls on one context must not overlap on different streams (the context's
 * scratch is shared).
 *
 * Errors: every call returns FR_OK (0) or a negative code; nothing throws
 * across the ABI.  FR_ECUDA carries the last CUDA error text, readable with
 * fr_last_error(); fr_strerror() maps a code to a fixed string.
 */
#ifndef ACMHD_FR_H
#define ACMHD_FR_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FR_ABI_VERSION 1

typedef struct fr_ctx fr_ctx;

/* Periodic, uniform, axis-aligned mesh: n[a] elements on [lo[a], hi[a]]
 * along direction a (a < dim).  Entries a >= dim are ignored. */
typedef struct fr_mesh {
    int dim;          /* 2 or 3 */
    int n[3];         /* elements per direction, each >= 1 */
    double lo[3];
    double hi[3];     /* hi[a] > lo[a] */
} fr_mesh;

enum {
    FR_OK = 0,
    FR_EINVAL = -1,      /* bad argument: mesh, order, nvars, parameters, pointer */
    FR_ECUDA = -2,       /* a CUDA runtime call or kernel launch failed */
    FR_ENOCONV = -3,     /* pseudo-time iteration hit max_iter above tolerance */
    FR_ENONFINITE = -4,  /* a residual norm was NaN or Inf */
    FR_ENOMEM = -5       /* device or host allocation failed */
};

/* arithmetic precision.  FR_DF64: states stored in FP64 (exactly as FR_F64),
 * the trace and volume kernels computing in double-float arithmetic - each
 * value an unevaluated sum of two FP32 numbers, about 48 significant bits
 * (relative rounding about 3.6e-15) in FP32's exponent range - which runs on
 * the FP32 pipes, 74 times faster than GB300's FP64 pipe; the update,
 * residual and BDF kernels stay FP64.  Contexts report FR_F64 storage. */
enum { FR_F32 = 32, FR_F64 = 64, FR_DF64 = 65 };
enum { FR_GUESS_PREVIOUS = 0, FR_GUESS_EXTRAPOLATE = 1, FR_GUESS_MLP = 2 };  /* fr_dual_step guess */

typedef struct fr_mlp fr_mlp;
enum { FR_CORR_DG = 0, FR_CORR_G2 = 1 };     /* correction function (Sec. 2.1) */
enum {
  FR_SCHEDULE_AUTO = 0,
  FR_SCHEDULE_TWO_KERNELS = 1,
  FR_SCHEDULE_FUSED_STAGE = 3     /* (2 is not used) */
};

/* Create a context.
 *   order       p, 1..6 (m = p + 1 solution points per direction)
 *   nvars       must equal 1 + dim + dim^2 (7 in 2-D, 13 in 3-D)
 *   zeta        artificial compressibility zeta > 0 (Sec. 2.2)
 *   nu          kinematic viscosity nu >= 0
 *   t_r         relaxation time T_r > 0 of the auxiliary equations
 *   precision   FR_F32, FR_F64 or FR_DF64
 *   correction  FR_CORR_DG (right Radau, h_l = R_{R,p+1}) or FR_CORR_G2 (Huynh)
 * Allocates the context's device scratch on the current device.
 * Returns FR_EINVAL for bad arguments, FR_ENOMEM/FR_ECUDA on allocation
 * failure; *out is set only on success. */
int fr_create(const fr_mesh* mesh, int order, int nvars, double zeta, double nu,
              double t_r, int precision, int correction, fr_ctx** out);

/* Release a context and its device memory (NULL is a no-op).  Synchronises
 * the device before freeing. */
void fr_destroy(fr_ctx* ctx);

/* Layout of a state: elements per row (padded), number of real elements,
 * and the byte size of one state buffer.  Any output pointer may be NULL. */
int fr_layout(const fr_ctx* ctx, size_t* elem_stride, size_t* n_elem,
              size_t* bytes_per_state);

/* Fused right-hand side R = -div F(U) + S(U) (Table fr_adv stages 1-6):
 * a trace kernel stores the face traces (stage 1; only the 1 + 2d variables
 * the normal flux needs), then one volume kernel evaluates per element the
 * flux (stage 2), the partially corrected divergence (3), the Rusanov/mean
 * common flux (4), the correction (5) and negation plus source (6).
 * U, R: device state buffers (must not alias).  Uses the context's trace
 * scratch.  Asynchronous on `stream`. */
int fr_rhs(fr_ctx* ctx, const void* U, void* R, void* stream);

/* Selects the schedule of the pseudo steps (fr_rk_step, fr_pseudo_solve).
 *   FR_SCHEDULE_TWO_KERNELS  each RK4 stage is fr_rhs (trace kernel + volume
 *                            kernel) followed by a separate update kernel.
 *   FR_SCHEDULE_FUSED_STAGE  one trace kernel per call, then each RK4 stage
 *                            is one kernel: the volume work with the stage
 *                            combination (and the FP64 velocity rows, BDF
 *                            source and residual partials of fr_pseudo_solve)
 *                            in its epilogue, writing the face traces of the
 *                            stage it leaves behind; R is never stored.  Same
 *                            arithmetic in the same order as the separate
 *                            update: identical results.
 *   FR_SCHEDULE_AUTO         (default) the fused stage at p <= 2, where it is
 *                            faster on GB300, the separate update at p >= 3,
 *                            where the volume kernel's occupancy serves the
 *                            update traffic at lower bandwidth than a
 *                            streaming kernel.
 * fr_rhs always runs the trace kernel and the volume kernel.  FR_EINVAL for
 * an unknown schedule. */
int fr_set_schedule(fr_ctx* ctx, int schedule);

/* The two halves of fr_rhs, for callers that time or schedule them apart.
 * fr_trace: stage 1 only - interpolates U to the faces of every element
 * (the 1 + 2d slots each face needs) into the context's trace scratch.
 * fr_rhs_volume: stages 2-6 - the fused kernel, reading U and the traces
 * that the last fr_trace on this context wrote.  The caller must pass the
 * same U to both and keep it unchanged in between; fr_rhs(U, R) is
 * fr_trace(U) followed by fr_rhs_volume(U, R). */
int fr_trace(fr_ctx* ctx, const void* U, void* stream);
int fr_rhs_volume(fr_ctx* ctx, const void* U, void* R, void* stream);

/* The same R computed by six separate stage kernels with HBM intermediates,
 * exactly as laid out in Table fr_adv (dense flux array F_s[d n_v n_s],
 * traces of all n_v variables).  The unfused baseline.  Allocates its
 * intermediates on first use (FR_ENOMEM on failure). */
int fr_rhs_unfused(fr_ctx* ctx, const void* U, void* R, void* stream);

/* fr_rhs on HOST buffers: copies U (bytes_per_state bytes, host memory,
 * preferably pinned) to context-owned device staging, evaluates the fused
 * RHS and copies R back to host memory.  Synchronises `stream` before
 * returning.  Allocates the staging on first use.  Meshes of at least two
 * slabs (element ranges of whole 32-element tiles, each one element layer
 * plus a tile; up to 4) are pipelined: each slab is copied in, traced,
 * computed and copied out as soon as its data and its neighbours' traces
 * are there, on three internal streams ordered after `stream`, so copies in
 * both directions overlap each other and the kernels.  Only the real
 * elements' columns of R_host are written (the padding to elem_stride is
 * left as it was). */
int fr_rhs_host(fr_ctx* ctx, const void* U_host, void* R_host, void* stream);

/* One classical RK4 step in pseudo time of dU/dtau = R(U) (Sec. 5, read as
 * RK4 with a fixed step): U <- U + dtau/6 (k1 + 2 k2 + 2 k3 + k4), in place.
 * Uses the context's RK registers (allocated on first use; the fused-stage
 * schedule of fr_set_schedule adds a second stage buffer and a second trace
 * buffer).  Asynchronous. */
int fr_rk_step(fr_ctx* ctx, void* U, double dtau, void* stream);

/* fr_rhs for callers that cannot allocate device memory.  The paper has no
 * counterpart: this is a deployment variant of fr_rhs with the same kernels
 * and the same results, bit for bit.  Some callers must not allocate device
 * memory once running - e.g. a host application whose own pool allocator
 * reserved the device's memory at start-up, or a time-critical loop in which
 * a device allocation (which can synchronise the whole device) is not
 * allowed - and fr_create allocates.  This call needs no context: it takes
 * the mesh and parameters of fr_create (same meaning and checks) and the
 * state buffers of fr_rhs (same layout; elem_stride = n_elem rounded up to a
 * multiple of 32), and calls no cudaMalloc, cudaFree or other allocating
 * routine.  Its face-trace scratch is one fixed 16 MiB array in the
 * library's device image, held by every GPU that loads it until the process
 * exits.
 * Limit: 2d (1+2d) (p+1)^(d-1) * elem_stride * sizeof(value) <= 16 MiB
 * (e.g. 6,240 hexahedra at p = 3 in FP32, 3,104 in FP64); larger problems
 * return FR_EINVAL with the reason in fr_last_error() and launch nothing.
 * First call on each device: it looks up the array's device address
 * (cudaGetSymbolAddress, with that device current) and caches it.  With
 * CUDA's default lazy module loading, that lookup and the first launches
 * also load the library's device code and the 16 MiB array onto the device,
 * which the driver does by allocating device memory: make one call on each
 * device before the caller's pool reserves the device's memory (or before
 * the region that must not allocate, and before any stream capture), or run
 * with CUDA_MODULE_LOADING=EAGER so that loading happens when the CUDA
 * context is created.  Later calls allocate nothing.  The cached address
 * does not survive a reset of the device (cudaDeviceReset) in the process.
 * All calls share the one array and it keeps the previous call's contents
 * (nothing needs clearing: every entry read is first written by the same
 * call), so calls whose kernels overlap on the GPU - other streams or host
 * threads - race on it and must be serialised by the caller.  Asynchronous
 * on `stream`. */
int fr_rhs_static(const fr_mesh* mesh, int order, int nvars, double zeta, double nu,
                  double t_r, int precision, int correction, const void* U, void* R,
                  void* stream);

/* Pseudo-time iteration of one physical time step (Sec. 5, dual time
 * stepping): classical RK4 in pseudo time tau on
 *     dU/dtau = R_tau(U) = R(U) - I_V (a0 V + a1 V^n + a2 V^{n-1}) / dt,
 * where I_V selects the velocity equations (Eq. acmhd_nd: the physical time
 * derivative acts on V only) and (a0, a1, a2) = (1, -1, 0) for BDF1 or
 * (3/2, -2, 1/2) for BDF2, until the residual - the RMS over all velocity
 * degrees of freedom of R_tau(U) - is below tol.
 *   U        work state (context precision; device), in/out.  Its P and
 *            auxiliary rows are the initial guess; its velocity rows are
 *            overwritten from V.
 *   V        velocity master in FP64: rows 1..d of a state, i.e.
 *            d * (p+1)^d * elem_stride doubles (device), in/out: the initial
 *            guess on entry, the converged velocity on return.  The BDF source,
 *            the velocity part of the RK4 update and the residual are FP64.
 *   Vn, Vnm1 FP64 velocity at t^n and t^{n-1} (same layout; Vnm1 unused for
 *            bdf_order 1).  dt > 0, dtau > 0 the physical and pseudo steps.
 *   check_every  the residual is evaluated (from the first RK stage of the
 *            step, no extra RHS) every check_every iterations and after the
 *            last; each check reads one double back to the host and is the
 *            call's only synchronisation.
 *   stall    if > 0, also stop (FR_ENOCONV) when a check finds the residual
 *            above stall times the previous check's (0 disables).
 * Returns FR_OK (converged, *res < tol), FR_ENOCONV (max_iter reached or
 * stalled; U and V hold the last iterate), FR_ENONFINITE (residual NaN/Inf).  *iters
 * and *res (if non-NULL) receive the iteration count and last residual.
 * Allocates its FP64 registers on first use. */
int fr_pseudo_solve(fr_ctx* ctx, void* U, double* V, const double* Vn, const double* Vnm1,
                    double dt, int bdf_order, double dtau, double tol, int max_iter,
                    int check_every, double stall, int* iters, double* res, void* stream);

/* Physical time stepping with context-owned history (three levels of the
 * state and of the FP64 velocity).  fr_dual_init stores U as level n (its
 * velocity widened to FP64) and allocates the history on first use.
 * fr_dual_step advances one step: initial guess (FR_GUESS_PREVIOUS: level
 * n; FR_GUESS_EXTRAPOLATE: the extrapolation through the stored levels,
 * 2U^n - U^{n-1} or 3U^n - 3U^{n-1} + U^{n-2}), fr_pseudo_solve with BDF1 on
 * the first step and BDF2 afterwards, then the new level enters the history
 * (also when the solve returns FR_ENOCONV, which is passed on).  U receives
 * the new level.  FR_GUESS_MLP: the extrapolated guess and the network's
 * guess (opts->mlp, three stored levels needed) are both evaluated - one RHS
 * and residual each - and so is the point of the segment between them,
 * (1 - alpha) extrapolation + alpha network with alpha in (0, 1) the
 * minimiser of the linearised residual |r0 + alpha (r1 - r0)| (r0, r1 the
 * two FP64 velocity residuals; one more RHS and residual).  The candidate
 * with the smallest residual is iterated, so the tolerance decides
 * convergence exactly as without the network.
 *
 * Mixed precision: FP32 arithmetic cannot bring the residual below its own
 * rounding floor (the FP32 RHS of the stored state).  With `refine` set to
 * an FR_F64 context on the same mesh, order, correction and parameters, the
 * iterations in ctx stop at tol_switch (or when the residual stalls: a check
 * finds it above 0.99 times the previous check's) and
 * continue on `refine` (work state U_refine, device, refine's layout) from
 * the widened state until tol; the result is narrowed back into U.  The
 * FP64 velocity master and the history stay in ctx.
 * fr_dual_velocity copies the newest FP64 velocity level into V (device). */
/* P-multigrid pseudo solver (Sec. 5: the Taylor-Green runs accelerate their
 * pseudo-iterations by P-multigrid over the orders of the same mesh, in an
 * asymmetric cycle of (order, iterations) pairs - (4,1) (3,1) (2,1) (1,4)
 * (2,1) (3,1) (4,7) at p = 4 - with the pseudo step enlarged by a constant
 * factor, 1.75, per order below the finest).  Full approximation scheme
 * with N(U) = R(U) - I_V (a0/dt) V: going down from order q to q - 1 the
 * state and the residual N + g are restricted (per element and direction,
 * L2 projection onto degree q - 1) and the coarse forcing is
 * g = I_r (N_q(U) + g_q) - N_{q-1}(I_r U); going up the coarse correction
 * U_{q-1} - I_r U_q is interpolated and added (to the FP64 velocity master
 * on the finest level).  Each entry of the cycle moves one order (restrict
 * or prolong) and then takes its iterations of classical RK4 in pseudo time
 * on dU/dtau = D (N(U) + g), D = 1 on P, 1 / (1 + dtau a0/dt) on the
 * velocity and 1 / (1 + dtau / T_r) on the gradient rows (point-implicit
 * scaling of the two linear stiff terms; it does not change the converged
 * state; fr_pmg_set_dtau can switch it off).
 *   fr_pmg_create      levels of order coarsest_order .. p - 1 of ctx's
 *                      discretization (internal contexts and four state
 *                      buffers each, allocated here); default cycle: one
 *                      iteration per order down, 4 on the coarsest, one
 *                      per order up, 7 on the finest; pseudo step of order
 *                      q: dtau 1.75^(p - q); scaling on.
 *   fr_pmg_set_cycle   n entries (orders[i], iters[i]): starts and ends at
 *                      p with iters[0] >= 1, consecutive orders differ by
 *                      at most one, orders within coarsest .. p.
 *   fr_pmg_set_dtau    factor[q] (q = coarsest .. p; array indexed by
 *                      order) multiplies dtau on order q; NULL keeps the
 *                      factors; implicit 0/1 switches the scaling.
 *   fr_pmg_solve       the pseudo-iteration of fr_pseudo_solve with cycles
 *                      instead of RK4 steps: the residual (RMS of R_tau over
 *                      the velocity DOFs, FP64) of the state at the start of
 *                      each cycle decides convergence (tol), max_cycles and
 *                      stall as fr_pseudo_solve's max_iter and stall; one
 *                      host synchronisation per cycle; *cycles and *res as
 *                      there.  U, V, Vn, Vnm1, dt, bdf_order, dtau: as
 *                      fr_pseudo_solve (dtau is the finest level's step).
 * All levels run in the precision of ctx. */
typedef struct fr_pmg fr_pmg;
int fr_pmg_create(fr_ctx* ctx, int coarsest_order, fr_pmg** out);
void fr_pmg_destroy(fr_pmg* pmg);
int fr_pmg_set_cycle(fr_pmg* pmg, int n, const int* orders, const int* iters);
int fr_pmg_set_dtau(fr_pmg* pmg, const double* factor, int implicit);
/* Anderson mixing over the cycles of fr_pmg_solve (not in the paper; Walker
 * & Ni 2011): after cycle k, with G(x_j) the state a cycle produced from
 * x_j and f_j = G(x_j) - x_j over the last memory + 1 cycles of this solve,
 * the next state is G(x_k) - dG gamma, gamma minimising || f_k - dF gamma ||
 * (dF, dG: successive differences; inner products over the real elements,
 * the velocity through its FP64 master; normal equations, regularised by
 * 1e-13 of their largest diagonal entry, oldest columns dropped while they
 * are singular).  memory 0 switches it off; memory < 16.  Allocates
 * 2 (memory + 1) + 1 copies of the state and the velocity (freed by
 * fr_pmg_destroy or the next call); one host synchronisation per cycle. */
int fr_pmg_set_anderson(fr_pmg* pmg, int memory);
int fr_pmg_solve(fr_pmg* pmg, void* U, double* V, const double* Vn, const double* Vnm1,
                 double dt, int bdf_order, double dtau, double tol, int max_cycles,
                 double stall, int* cycles, double* res, void* stream);

typedef struct fr_dual_opts {
    double dt, dtau;      /* physical and pseudo time steps (> 0) */
    double tol;           /* residual tolerance (RMS of R_tau over velocity DOFs) */
    int max_iter;         /* pseudo iterations per physical step, both phases */
    int check_every;      /* residual check interval (>= 1) */
    int guess;            /* FR_GUESS_* */
    fr_ctx* refine;       /* NULL, or the FP64 refinement context */
    void* U_refine;       /* refine's work state */
    double tol_switch;    /* residual at which ctx hands over to refine */
    fr_mlp* mlp;          /* trained network for FR_GUESS_MLP (created on this
                             context or one of the same discretization; the
                             guess comes from this context's history) */
    fr_pmg* pmg;          /* NULL, or a P-multigrid solver created on ctx: the
                             pseudo-iteration runs fr_pmg_solve, max_iter
                             counting cycles */
    fr_pmg* refine_pmg;   /* the same for the refinement context */
} fr_dual_opts;

typedef struct fr_dual_stats {
    int iters;            /* pseudo iterations (cycles with P-multigrid) in ctx */
    int iters_refine;     /* pseudo iterations (cycles) in refine */
    double res;           /* final residual */
    double res_switch;    /* residual when ctx handed over (or final) */
    int guess_used;       /* FR_GUESS_* actually used (the MLP guess falls back) */
    double res_guess[2];  /* FR_GUESS_MLP: initial residual of [extrapolation, network] */
    double mlp_weight;    /* FR_GUESS_MLP: weight alpha of the network's guess in the
                             state iterated: 0 extrapolation, 1 network, between: blend */
    double res_blend;     /* FR_GUESS_MLP: residual of the blend (NaN if not tried) */
} fr_dual_stats;

int fr_dual_init(fr_ctx* ctx, const void* U, void* stream);
int fr_dual_step(fr_ctx* ctx, void* U, const fr_dual_opts* opts, fr_dual_stats* stats,
                 void* stream);
int fr_dual_velocity(const fr_ctx* ctx, double* V, void* stream);

/* Copies the physical-time history (all stored levels) of src into dst, a
 * context on the same mesh, order and precision: dst continues from exactly
 * src's state ("forks" the solver).  Allocates dst's history on first use. */
int fr_dual_copy(fr_ctx* dst, const fr_ctx* src, void* stream);

/* Learned initial guess (no counterpart in the paper).  A per-element MLP,
 * on the tensor cores (BF16 operands, FP32 accumulation, FP32 master
 * weights), maps the element's last three levels - fed as U^n, the first
 * and the second difference, each scaled per variable by its RMS - through
 * two hidden ReLU layers to the correction of the plain extrapolation
 * 3U^n - 3U^{n-1} + U^{n-2}, scaled per variable by the RMS of the collected
 * corrections.
 *   fr_mlp_create   network of `hidden` units per layer bound to ctx, with
 *                   room for `capacity` element samples; weights drawn from
 *                   a splitmix64 stream seeded with `seed`.
 *   fr_mlp_collect  after an fr_dual_step that left four levels in ctx's
 *                   history: stores `count` element samples (elements drawn
 *                   from a splitmix64 stream; written to elems if non-NULL)
 *                   of inputs (the three older levels) and target (the
 *                   newest).  The first call fixes the input scales.
 *                   Synchronises `stream`.
 *   fr_mlp_loss_grad  MSE and its gradients over the collected samples.
 *   fr_mlp_train    `epochs` full-batch Adam steps (beta 0.9/0.999, eps
 *                   1e-8, step lr); *loss is the loss before the last step.
 *   fr_mlp_predict  guess of the next level from ctx's three newest levels:
 *                   U (context precision) and V (FP64 velocity rows).
 *   fr_mlp_predict_for  the same from the history of another context `ctx`
 *                   of the same discretization (dimension, order, elements,
 *                   precision; FR_EINVAL otherwise), e.g. a second solver
 *                   that shares the trained network.  fr_dual_step with
 *                   FR_GUESS_MLP uses its own context's history this way.
 *   fr_mlp_params   copy to (set = 0) or from (set != 0) host memory:
 *                   which 0 = parameters, 1 = gradients (count = the total
 *                   from fr_mlp_info, order W1 b1 W2 b2 W3 b3, W row-major
 *                   (out x in)); which 2 = scales (3 nv input + nv output);
 *                   which 3 / 4 (read only) = the collected samples'
 *                   features (n_in x n_samples, row-major) / raw targets
 *                   (n_out x n_samples).
 * Buffers are allocated by fr_mlp_create (and by the first fr_mlp_predict);
 * FR_EINVAL when the history, samples or training a call needs are missing. */
int fr_mlp_create(fr_ctx* ctx, int hidden, int capacity, unsigned long long seed, fr_mlp** out);
void fr_mlp_destroy(fr_mlp* mlp);
int fr_mlp_info(const fr_mlp* mlp, int* n_in, int* hidden, int* n_out, int* n_samples,
                size_t* n_params);
int fr_mlp_collect(fr_mlp* mlp, int count, unsigned long long seed, int* elems, void* stream);
int fr_mlp_loss_grad(fr_mlp* mlp, double* loss, void* stream);
int fr_mlp_train(fr_mlp* mlp, int epochs, double lr, double* loss, void* stream);
int fr_mlp_predict(fr_mlp* mlp, void* U, double* V, void* stream);
int fr_mlp_predict_for(fr_mlp* mlp, fr_ctx* ctx, void* U, double* V, void* stream);
int fr_mlp_params(fr_mlp* mlp, int which, float* host, size_t count, int set);

/* Training options.  n_val: the newest n_val collected samples are held out
 * of training (fr_mlp_loss_grad, fr_mlp_train, fr_mlp_train_step use the
 * others) and fr_mlp_validation_loss reports the loss on them; weight_decay:
 * decoupled weight decay of Adam (AdamW: every step also subtracts
 * lr * weight_decay * w from each weight; biases are not decayed).  Both 0
 * by default.  FR_EINVAL for negative values or n_val beyond the capacity;
 * training needs at least one training sample. */
int fr_mlp_set_training(fr_mlp* mlp, int n_val, double weight_decay);
int fr_mlp_validation_loss(fr_mlp* mlp, double* loss, void* stream);

/* One full-batch Adam step over the collected samples (fr_mlp_train with
 * one epoch); *loss (if non-NULL) is the loss before the step.  Synchronises
 * `stream`. */
int fr_mlp_train_step(fr_mlp* mlp, double lr, double* loss, void* stream);

/* Save / load a network.  The file holds a magic word, a format version, the
 * discretization it was built for (dimension, order, variables, points per
 * element), its sizes, the Adam step count, the feature and output scales,
 * the FP32 master weights and Adam's moments, and a checksum (FNV-1a 64 over
 * all preceding bytes); little-endian.  fr_mlp_load creates a network bound
 * to ctx with room for `capacity` samples and restores all of that, so
 * predictions are bit-identical to the saved network's and training resumes
 * where it stopped.  The collected samples are not saved.  FR_EINVAL (reason
 * in fr_last_error) for a missing, corrupt or foreign file, or a network of
 * another discretization (dimension, order or variable count). */
int fr_mlp_save(const fr_mlp* mlp, const char* path);

/* Smoothing of the learned correction (no counterpart in the paper): with
 * degree q >= 0, every correction the network learns from (the targets that
 * fr_mlp_collect gathers from then on) and every correction it predicts is
 * projected, per element and variable, onto the polynomials of degree <= q
 * in each direction (the L2 projection on the element's Gauss-Legendre
 * points, applied along each axis).  The network then neither learns nor
 * adds element-scale detail, which the pseudo-time residual penalises, and
 * keeps the smooth part of the correction, which the extrapolated guess
 * carries forward.  degree -1 (the default) turns it off; q = order is the
 * identity.  FR_EINVAL outside [-1, order].  The setting is not saved by
 * fr_mlp_save. */
int fr_mlp_set_output_degree(fr_mlp* mlp, int degree);
int fr_mlp_load(fr_ctx* ctx, const char* path, int capacity, fr_mlp** out);

/* The tensor-core GEMM of the MLP as a utility: C[N x M] = A . B in FP32
 * from BF16 operands.  amode 0: A[n * lda + k]; 1: A[k * lda + n].
 * bmode 0: B[k * ldb + m]; 1: B[m * ldb + k].  C[n * ldc + m].  Device
 * pointers; asynchronous. */
int fr_gemm_bf16(int amode, int bmode, int N, int M, int K, const void* A, long long lda,
                 const void* B, long long ldb, float* C, long long ldc, void* stream);

/* Kernel choice for the network's GEMMs (fr_gemm_bf16 and the MLP's
 * forward and backward products, every orientation), process-wide.
 * FR_GEMM_AUTO (the default): the fifth-generation tensor-core kernel
 * (tcgen05.mma with the accumulators in tensor memory, operands brought in
 * by TMA) whenever A and B start on 16-byte boundaries and lda, ldb are
 * multiples of 8; the warp-level mma.sync kernels otherwise.
 * FR_GEMM_MMA_SYNC: always the mma.sync kernels (for comparison).
 * FR_EINVAL for another value. */
enum { FR_GEMM_AUTO = 0, FR_GEMM_MMA_SYNC = 1 };
int fr_gemm_set_kernel(int kind);

/* Synchronises `stream`; FR_ECUDA (text in fr_last_error) if a kernel
 * failed or a tensor-memory GEMM gave up one of its bounded waits (about two
 * seconds each; the GEMM's output is then invalid), FR_OK otherwise.  The
 * give-up record is cleared by the call. */
int fr_gemm_check(void* stream);

/* Arithmetic peak probe (a measuring utility; no counterpart in the
 * paper): launches one kernel that does only fused multiply-adds in FP32 or
 * FP64 (precision FR_F32 / FR_F64), `iters` x 128 per thread on every SM,
 * and stores *flops, the floating-point operations it performs (2 per FMA).
 * The caller times it (CUDA events on `stream`) to obtain this GPU's FMA
 * throughput, the roofline denominator of an arithmetic-bound kernel.
 * `out` is a device buffer of at least 8 * (SM count) * 8 bytes that the
 * kernel may write (it never does for valid inputs).  Asynchronous. */
int fr_fma_probe(int precision, int iters, void* out, double* flops, void* stream);

/* Synchronises `stream` and reports an asynchronous CUDA error (a failed
 * kernel) as FR_ECUDA with its text in fr_last_error(); FR_OK otherwise. */
int fr_check(fr_ctx* ctx, void* stream);

/* Static text for a status code. */
const char* fr_strerror(int status);

/* Text of the last CUDA error seen by this library in the calling thread
 * (empty if none). */
const char* fr_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* ACMHD_FR_H */
