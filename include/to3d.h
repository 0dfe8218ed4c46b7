/*
 * to3d.h -- C interface of the GB300 SIMP / Optimality Criteria hot path.
 *
 * The library solves the compliance-minimisation problem of Kim & Kang,
 * "PyTopo3D" (arXiv 2504.05604): a structured grid of nelx x nely x nelz unit
 * 8-node hexahedra (Section 2.2), SIMP moduli E_e = Emin + x_e^p (E0 - Emin)
 * (Section 2.3), the linear-decay rmin filter (Section 2.4) and the OC update
 * with bisection on the volume multiplier (Section 2.3), iterated as in
 * Section 2.5.  Every step runs in the library's own CUDA kernels on one GPU.
 *
 * Numbering (all arrays at this interface are unpadded):
 *   element (i,j,k) -> e = i + nelx*(j + nely*k)              [nel]
 *   node    (i,j,k) -> n = i + (nelx+1)*(j + (nely+1)*k)      [N]
 *   dof             -> 3*n + c, c = 0 (x), 1 (y), 2 (z)       [3N]
 *   element-local node a + 2b + 4c sits at corner (i+a, j+b, k+c).
 *
 * Conventions:
 *   - Status codes only; no exceptions or aborts cross this boundary.
 *     to3d_last_error() gives a message for the last failure on a context.
 *   - Inputs to to3d_create are copied; the caller keeps ownership of its
 *     buffers.  Outputs go to caller-allocated buffers.
 *   - `on_device` = 1: the pointers are CUDA device pointers (e.g. torch
 *     tensor data_ptr()) on the context's device; 0: host pointers.  Host
 *     pointers are copied through the context's stream and the call
 *     returns after the copy back has completed.
 *   - All GPU work is enqueued on the stream given at create (NULL = the
 *     legacy default stream).  A context is used by one host thread at a time.
 *   - Clamped dofs: the operator is K restricted to the free dofs with unit
 *     rows/columns on the clamped ones (Section 2.2, "modifying the system
 *     matrix and load vector"); loads on clamped dofs are ignored.
 */
#ifndef TO3D_H
#define TO3D_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define TO3D_API __attribute__((visibility("default")))
#else
#define TO3D_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    TO3D_OK = 0,
    TO3D_EINVAL = 1,    /* bad argument or size                                */
    TO3D_ENOMEM = 2,    /* device or host allocation failed                    */
    TO3D_ECUDA = 3,     /* a CUDA runtime call failed                          */
    TO3D_ENOCONV = 4,   /* solver reached its iteration limit                  */
    TO3D_ENUMERIC = 5,  /* NaN/Inf or non-positive curvature in a solver       */
    TO3D_ETIMEOUT = 6,  /* a bounded device-side wait gave up                  */
    TO3D_ESTATE = 7     /* call not valid in the context's current state       */
} to3d_status;

/* Arithmetic of the equilibrium solve.  The *_DC forms run an inner
 * conjugate-gradient solve with FP32 vectors and a tensor-core element
 * matvec (integer-exact stiffness, 16-bit displacement operands, FP32
 * accumulation) inside an FP64 defect-correction loop: r = f - K u in FP64,
 * FP64 dot products and norms, u += d in FP64. */
typedef enum {
    TO3D_F64 = 0,        /* FP64 Jacobi-PCG with the FP64 element matvec      */
    TO3D_BF16_DC = 1,    /* BF16 operand (one slice); after 8 outer stalls in a
                          * solve it switches to the two-slice form           */
    TO3D_BF16X2_DC = 2,  /* BF16 hi + lo slices (about 16 mantissa bits)      */
    TO3D_FP16_DC = 3,    /* FP16 operand with per-element power-of-two scale
                          * (same escalation to two slices)                   */
    TO3D_FP16X2_DC = 4   /* scaled FP16 hi + lo slices (about 22 bits)        */
} to3d_precision;

/* Preconditioner of the equilibrium solve (none is in the paper, which uses
 * a sparse direct solver, Section 2.2).  TO3D_LMG: the learned multigrid
 * V-cycle (to3d_mg_*); with TO3D_F64 it preconditions FP64 flexible CG,
 * with a *_DC precision the FP32 inner CG of the defect correction. */
typedef enum { TO3D_JACOBI = 0, TO3D_CNN_FCG = 1, TO3D_LMG = 2 } to3d_precond;
typedef enum { TO3D_FILTER_SENS = 0, TO3D_FILTER_DENS = 1 } to3d_filter;

typedef struct {
    int32_t nelx, nely, nelz;
    double volfrac;      /* volume fraction of the design elements            */
    double penal;        /* SIMP power p                                      */
    double rmin;         /* filter radius in element lengths                  */
    double E0, Emin, nu; /* solid modulus, void modulus, Poisson ratio        */
    double move;         /* OC move limit                                     */
    double bisect_tol;   /* stop bisection when (l2-l1)/(l1+l2) <= tol        */
    double cg_rtol;      /* stop when ||f - K u||_2 <= cg_rtol ||f||_2        */
    double inner_rtol;   /* *_DC forms: the FP32 residual is replaced by the  */
                         /* true FP64 one each time it has dropped by this    */
                         /* factor (0 < inner_rtol < 1)                       */
    int32_t cg_maxit;    /* iteration limit of one solve (all inner steps)    */
    int32_t filter;      /* to3d_filter                                       */
    int32_t precision;   /* to3d_precision                                    */
    int32_t precond;     /* to3d_precond                                      */
    int32_t oc_levels;   /* bisection levels resolved per reduction pass, 1-6 */
    int32_t warm_start;  /* 1: start each solve from the previous u           */
    int32_t fcg_ref_iters; /* TO3D_CNN_FCG: Jacobi-PCG iterations at cg_rtol
                            * that flexible CG must keep pace with before the
                            * context has timed a plain solve of its own (0:
                            * no such bound until then)                       */
    int32_t mg_sweeps;   /* TO3D_LMG: Jacobi sweeps on the coarsest level
                          * (0: 6)                                            */
    int32_t fp64_tc;     /* 1: every FP64 K p (the FP64 forms' matvec, the
                          * defect correction's residual, flexible CG) and
                          * the element energies u_e^T KE u_e on the tensor
                          * cores by exact integer slicing (FP64 accuracy;
                          * needs a nu whose lambda / mu is a small rational,
                          * else the CUDA-core FP64 kernels run);
                          * 0 (default): the CUDA-core FP64 kernels           */
    int32_t mg_keep_dir; /* TO3D_LMG with a *_DC precision: 1 keeps the inner
                          * CG's direction across FP64 residual replacements
                          * (Fletcher-Reeves beta right after one), 0 restarts
                          * it at each replacement                            */
    int32_t mg_nu;       /* TO3D_LMG: damped-Jacobi sweeps before and after
                          * each coarse correction (0: 1)                     */
    int32_t reserved[1];
} to3d_params;

typedef struct {
    int32_t iter;        /* 0-based OC iteration index                        */
    int32_t status;      /* to3d_status of the iteration                      */
    double compliance;   /* c = f^T u = sum_e E_e u_e^T KE u_e                 */
    double volume;       /* design volume fraction after the update           */
    double change;       /* max_e |x_new - x|                                 */
    double lambda;       /* last bisection midpoint                           */
    double relres;       /* final true relative residual of the solve         */
    int32_t cg_iters;    /* inner (or plain) CG iterations of the solve       */
    int32_t outer_iters; /* defect-correction steps (1 for TO3D_F64)          */
    int32_t halvings;    /* bisection halvings                                */
    int32_t pad;
    double ms_solve, ms_sens, ms_filter, ms_oc;   /* CUDA-event phase times   */
} to3d_iter_info;

typedef struct {
    int32_t iters, outer, status, pad;
    double relres;
} to3d_solve_info;

typedef struct to3d_ctx to3d_ctx;

/* Fill *p with the defaults: E0 = 1, Emin = 1e-9, nu = 0.3, penal = 3,
 * volfrac = 0.3, rmin = 1.5, move = 0.2, bisect_tol = 1e-3, cg_rtol = 1e-8,
 * inner_rtol = 0.3, cg_maxit = 200000, sensitivity filter, TO3D_F64,
 * Jacobi, oc_levels = 3, warm_start = 1.  Grid sizes are set to 0. */
TO3D_API to3d_status to3d_default_params(to3d_params* p);

/* Create a context for one problem.
 *   fixed   [3N] uint8, host: nonzero = clamped dof (Section 2.2).
 *   load    [3N] double, host: nodal forces F (Section 2.2, K U = F).
 *   passive [nel] uint8, host, may be NULL: 0 design, 1 void (x pinned at 0),
 *           2 solid (x pinned at 1); pinned elements are excluded from the
 *           volume constraint (Section 2.3, passive regions).
 *   stream  cudaStream_t (as void*) on which all work is enqueued.
 * The density starts at volfrac on design elements.
 * Errors: EINVAL for non-positive sizes or parameters out of range, ENOMEM,
 * ECUDA.  *out is NULL on failure. */
TO3D_API to3d_status to3d_create(const to3d_params* p, const uint8_t* fixed, const double* load,
                        const uint8_t* passive, void* stream, to3d_ctx** out);

TO3D_API void to3d_destroy(to3d_ctx* ctx);
TO3D_API const char* to3d_last_error(const to3d_ctx* ctx);
TO3D_API const char* to3d_status_string(to3d_status s);
/* Number of this library's kernel launches issued on the context so far. */
TO3D_API int64_t to3d_launch_count(const to3d_ctx* ctx);

/* Sampled device durations of the solver's dominant kernel launches, taken
 * with CUDA events recorded inside the captured solver chunks (one launch in
 * four, launches that did work only).  which = 0: tensor-core matvec of the
 * defect-correction forms; 1: FP64 matvec.  *ms_total = summed duration,
 * *samples = number of launches timed; reset = 1 clears the counters. */
TO3D_API to3d_status to3d_kernel_stats(to3d_ctx* ctx, int32_t which, double* ms_total,
                                       int64_t* samples, int32_t reset);

/* One OC iteration (Section 2.5): solve K(x) u = f, element energies and
 * sensitivities, filter, OC update of x.  With params.filter =
 * TO3D_FILTER_DENS (Section 2.4, density filter) the analysis runs on
 * xphys = H x / Hs with passive elements pinned, the sensitivities are
 * carried back by H^T (dc / Hs), and the OC update and its volume act on x.
 * `info` may be NULL. */
TO3D_API to3d_status to3d_step(to3d_ctx* ctx, to3d_iter_info* info);
/* `iters` OC iterations; hist [iters] may be NULL. */
TO3D_API to3d_status to3d_run(to3d_ctx* ctx, int32_t iters, to3d_iter_info* hist);

/* Current design x [nel] (FP64) and last displacement u [3N] (FP64). */
TO3D_API to3d_status to3d_get_density(to3d_ctx* ctx, double* x, int32_t on_device);
TO3D_API to3d_status to3d_set_density(to3d_ctx* ctx, const double* x, int32_t on_device);
TO3D_API to3d_status to3d_get_displacement(to3d_ctx* ctx, double* u, int32_t on_device);
/* Checkpoint / resume: x (set_density; host values must lie in [0, 1], else
 * EINVAL and x is left unchanged; they are checked on the GPU after the
 * copy; device values are taken as given), u (the next solve's warm start)
 * and the OC iteration counter of a context.  A context given the x, u and iteration of another one repeats
 * that one's next OC iteration exactly. */
TO3D_API to3d_status to3d_set_displacement(to3d_ctx* ctx, const double* u, int32_t on_device);
TO3D_API to3d_status to3d_get_iteration(const to3d_ctx* ctx, int32_t* iter);
TO3D_API to3d_status to3d_set_iteration(to3d_ctx* ctx, int32_t iter);

/* ---- single steps of the path (also used by the parity tests) ---------- */

/* y = Kbar(x) p in FP64 (Section 2.2 operator with clamped dofs as identity
 * rows/columns).  x [nel] densities, p, y [3N].  Matrix-free: K is never
 * formed. */
TO3D_API to3d_status to3d_matvec(to3d_ctx* ctx, const double* x, const double* p, double* y,
                        int32_t on_device);

/* y = Kbar(x) p with the tensor-core element matvec of precision `prec`
 * (TO3D_BF16_DC, TO3D_BF16X2_DC, TO3D_FP16_DC or TO3D_FP16X2_DC): p rounded per element to
 * the 16-bit operand format, integer-exact element stiffness, FP32
 * accumulation, FP32 scaling by E_e.  p, y [3N] FP32. */
TO3D_API to3d_status to3d_matvec_lowp(to3d_ctx* ctx, const double* x, const float* p, float* y,
                             int32_t prec, int32_t on_device);

/* Solve Kbar(x) u = f to ||f - Kbar u|| <= cg_rtol ||f|| with the context's
 * precision and preconditioner.  f may be NULL (the context's load).
 * u [3N] is the result (its input value is the initial guess when
 * warm_start = 1, else ignored). */
TO3D_API to3d_status to3d_solve(to3d_ctx* ctx, const double* x, const double* f, double* u,
                       int32_t on_device, to3d_solve_info* info);

/* ce_e = u_e^T KE u_e, dc_e = -p x_e^(p-1) (E0 - Emin) ce_e and
 * c = sum_e E_e ce_e (Section 2.3).  ce, dc [nel]; *compliance on host.
 * With params.fp64_tc the energies come from the sliced tensor-core path
 * (the element's exact products B V dotted with u_e in FP64). */
TO3D_API to3d_status to3d_sensitivity(to3d_ctx* ctx, const double* x, const double* u, double* ce,
                             double* dc, double* compliance, int32_t on_device);

/* Filter (Section 2.4) with H_ei = max(0, rmin - |c_e - c_i|), Hs_e its
 * in-grid row sum.  Sensitivity filter: out = H(x dc) / (Hs max(1e-3, x));
 * density filter (TO3D_FILTER_DENS): out = H v / Hs, and its transpose
 * (chain rule) when `transpose` = 1: out = H^T (v / Hs). */
TO3D_API to3d_status to3d_filter_apply(to3d_ctx* ctx, int32_t kind, const double* x, const double* v,
                              double* out, int32_t transpose, int32_t on_device);

/* OC update (Section 2.3) of x with filtered sensitivities dcf:
 * x_new = clamp(x sqrt(-dcf/lambda), max(0, x - move), min(1, x + move)),
 * lambda by bisection on [0, 1e9] until (l2-l1)/(l1+l2) <= bisect_tol, the
 * design volume sum_design x_new > volfrac * n_design raising l1.
 * Passive elements are pinned.  Outputs on host: lambda, design volume
 * (absolute), halvings; xnew [nel] as `on_device` says. */
TO3D_API to3d_status to3d_oc_update(to3d_ctx* ctx, const double* x, const double* dcf, double* xnew,
                           double* lambda, double* volume, int32_t* halvings,
                           int32_t on_device);

/* ---- learned preconditioner ----------------------------------------------
 * Not in the paper, which solves K U = F with a sparse direct solver
 * (Section 2.2): an optional preconditioner for the library's iterative
 * solve of the same FP64 state equation.
 * A four-level U-Net on the node grid (16/32/64/64 channels, 3x3x3
 * convolutions with zero padding, 2x2x2 average pooling, nearest x2
 * upsampling with skip concatenation, ReLU), applied as z = M(r) inside
 * flexible CG when params.precond = TO3D_CNN_FCG.  Inputs: the Jacobi-scaled
 * residual rt = D^-1/2 r (D = diag K) divided by s = RMS(rt), three
 * channels, and log10 of the node density; output: a correction on top of
 * Jacobi, z = D^-1 r + s D^-1/2 out (a zero network is plain Jacobi).
 * Clamped dofs are zero in and out.  Parameters
 * are FP32 (flat vector, per layer: weights [27][C_out][C_in] with tap =
 * 9 dz + 3 dy + dx, then bias [C_out]); the convolutions run on the tensor
 * cores in BF16 with FP32 accumulation.  Flexible CG (FP64 vectors,
 * Polak-Ribiere beta, exact line search) takes z = D^-1 r (Jacobi) in any
 * iteration where the network's r^T z <= 0, and falls back to Jacobi-PCG
 * when a curvature p^T K p is non-positive, when the smallest residual seen
 * drops by less than 10 % over 200 iterations, or when, past 50
 * iterations, it is 10x above where the context's last plain Jacobi-PCG
 * solve (its iteration count at the same tolerance; before there is one,
 * params.fcg_ref_iters) would have been at its average rate; to3d_solve_info.outer is then 2 (the fallback starts from
 * zero unless the true residual is already below 1e-2 |f|).  The true FP64
 * residual decides convergence. */

/* (Re)initialise the network's parameters (He-normal, counter-based hash
 * of `seed`); clears the optimiser state.  Network not trained afterwards. */
TO3D_API to3d_status to3d_cnn_init(to3d_ctx* ctx, uint64_t seed);
/* Number of FP32 parameters (allocates the network if needed). */
TO3D_API to3d_status to3d_cnn_param_count(to3d_ctx* ctx, int64_t* n);
/* Copy the parameters out (host buffer of n floats; EINVAL if n differs). */
TO3D_API to3d_status to3d_cnn_get_params(to3d_ctx* ctx, float* p, int64_t n);
/* Load parameters (host buffer of n floats); marks the network trained. */
TO3D_API to3d_status to3d_cnn_set_params(to3d_ctx* ctx, const float* p, int64_t n);
/* z = M(r) for densities x [nel] and residual r [3N]; z [3N].  EINVAL if
 * the network does not exist yet (call to3d_cnn_init first). */
TO3D_API to3d_status to3d_cnn_apply(to3d_ctx* ctx, const double* x, const double* r, double* z,
                                    int32_t on_device);
/* Train on the GPU.  Snapshots: `nsnap` residuals r = f - K u of FP64
 * Jacobi-PCG (source 0) or of flexible CG with the current network
 * (source 1: the residuals the network itself leaves) from u = 0 on the
 * context's design, the first of every `per_design` taken before any
 * iteration (r = f), the others after a random 1..200 iterations; each stores r, the design and r^T K^-1 r (FP64
 * solve to 1e-10).  After every `per_design` snapshots the design advances
 * by one plain OC iteration (FP64 Jacobi-PCG).  Then `steps` Adam steps
 * (lr, betas 0.9 / 0.999), one snapshot per step, on the energy-norm loss
 * L = ||M(r) - K^-1 r||_K^2 / ||K^-1 r||_K^2 = (z^T K z - 2 z^T r + r^T e) /
 * (r^T e), z = M(r), e = K^-1 r (L < 1 implies r^T z > 0).  loss_first /
 * loss_last (host, may be NULL): mean loss of the first and last tenth of
 * the steps.  Snapshots stay resident and accumulate over calls (nsnap = 0
 * trains on those already taken; steps = 0 only takes snapshots).
 * Continues from the current parameters (initialised from `seed` if none
 * were set).  The context's displacement is not kept (the next solve
 * starts from zero). */
TO3D_API to3d_status to3d_cnn_train(to3d_ctx* ctx, int32_t nsnap, int32_t per_design,
                                    int32_t steps, double lr, uint64_t seed, int32_t source,
                                    double* loss_first, double* loss_last);
/* The training loss of one sample and its gradient with respect to every
 * parameter (same layout as to3d_cnn_get_params), without an optimiser
 * step: x [nel] densities, r [3N] residual (clamped entries ignored), e [3N]
 * its error K^-1 r, needed only for r^T e > 0 (EINVAL otherwise), all as
 * `on_device`; grad: host buffer of ngrad floats (NULL to skip); *loss on
 * host. */
TO3D_API to3d_status to3d_cnn_loss_grad(to3d_ctx* ctx, const double* x, const double* r,
                                        const double* e, int32_t on_device, float* grad,
                                        int64_t ngrad, double* loss);
/* One 3x3x3 convolution on caller device buffers (channels-last, zero
 * padding): out[v][Cout] (FP32) = bias + W * concat(in1[v][C1], in2[v][C2]),
 * ReLU if relu.  in1, in2 BF16; W BF16 [27][Cout][C1+C2]; bias FP32 or NULL.
 * C1 >= 16 and C2 >= 0 multiples of 16, Cout/8 in {1,2,4,6,8,12,16}.
 * Enqueued on `stream` (cudaStream_t as void*), not synchronised. */
TO3D_API to3d_status to3d_conv3d_forward(int32_t Z, int32_t Y, int32_t X, int32_t C1, int32_t C2,
                                         int32_t Cout, const void* in1, const void* in2,
                                         const void* W, const float* bias, int32_t relu,
                                         float* out, void* stream);
/* Backward of the same convolution for upstream gradient gy [v][Cout]
 * (FP32), masked by act > 0 where act (BF16 [v][Cout], the forward ReLU
 * output) is not NULL: gw [27][Cout][C1+C2] and gb [Cout] (FP32, added to
 * what they hold; gb may be NULL) and, if gx is not NULL, gx [v][C1+C2]
 * (FP32, overwritten).  x1, x2 BF16 forward inputs.  Cout in 16..64 a
 * multiple of 16, C1 + C2 <= 128.  Enqueued on `stream`. */
TO3D_API to3d_status to3d_conv3d_backward(int32_t Z, int32_t Y, int32_t X, int32_t C1, int32_t C2,
                                          int32_t Cout, const void* x1, const void* x2,
                                          const void* W, const float* gy, const void* act,
                                          float* gx, float* gw, float* gb, void* stream);

/* ---- many independent problems ------------------------------------------ */

/* ---- learned multigrid preconditioner (params.precond = TO3D_LMG) ----------
 * Not in the paper, which solves K U = F with a sparse direct solver
 * (Section 2.2): a preconditioner for the library's iterative solve of the
 * same state equation, K = sum_e E_e KE with E_e from the SIMP law of
 * Section 2.3.  A geometric multigrid V-cycle:
 *   levels     element counts halved (rounded up) until the largest is at
 *              most 4 or the smallest below 2; coarse node C on fine node
 *              2C; a coarse dof is clamped when the fine dof at 2C is;
 *   coarse K   coarse element modulus s_l (mean over its 8 child slots of
 *              E^q_l)^(1/q_l), children past the grid counted as 0, times
 *              the unit KE (s = 2 gives the Galerkin operator for a uniform
 *              modulus);
 *   transfer   trilinear prolongation P, restriction P^T, clamped dofs 0;
 *   smoother   damped Jacobi, one sweep before and one after the coarse
 *              correction, params.mg_sweeps sweeps (default 6) on the
 *              coarsest level; damping w_l * 2 / lam_l, lam_l = min(1.2 rq,
 *              l1) with rq the Rayleigh quotient of D^-1 K after 16 power
 *              steps from a fixed hashed start and l1 = max_a sum_b
 *              |KE_ab| / KE_aa, so every sweep converges for 0 < w < 1.
 * The cycle runs in FP32 with the tensor-core operator (the context's
 * operand form; BF16 for TO3D_F64) on every level.  With TO3D_F64 it
 * preconditions FP64 flexible CG (the Jacobi-PCG fallback as for
 * TO3D_CNN_FCG); with a *_DC precision it preconditions the FP32 inner CG,
 * which restarts at each FP64 residual replacement (every drop by
 * params.inner_rtol).
 * Parameters theta (10 doubles, to3d_mg_param_count): w_0, w_1, w_2, w_3,
 * q_1, q_2, q_3, s_1, s_2, s_3, where index g applies to level min(l, 3), so
 * parameters learned on one grid size apply to any other.  Defaults: w = 2/3,
 * q = 1, s = 2.  Valid ranges: 0 < w < 1, 1/8 <= q <= 8, 0 < s <= 64
 * (TO3D_EINVAL otherwise).  The first call that needs the hierarchy creates
 * one coarse context per level (device allocations). */
TO3D_API to3d_status to3d_mg_param_count(to3d_ctx* ctx, int64_t* n);
TO3D_API to3d_status to3d_mg_get_params(to3d_ctx* ctx, double* theta, int64_t n);
TO3D_API to3d_status to3d_mg_set_params(to3d_ctx* ctx, const double* theta, int64_t n);
/* Number of levels of the hierarchy (1 = the design grid only). */
TO3D_API to3d_status to3d_mg_levels(to3d_ctx* ctx, int32_t* nlev);
/* z = V r for densities x [nel] and a residual r [3N] (FP64, clamped
 * entries ignored; z is 0 there), host or device as `on_device` says. */
TO3D_API to3d_status to3d_mg_apply(to3d_ctx* ctx, const double* x, const double* r, double* z,
                                   int32_t on_device);
/* Learn theta from snapshots of the method's own solves.  Takes `nsnap`
 * snapshots on the context's current design: residuals of FP64 Jacobi-PCG
 * from u = 0 after a random number (0..200) of iterations (seed `seed`),
 * each with r^T K^-1 r from an FP64 solve to 1e-10; with append = 1 they are
 * added to those of earlier calls (other designs of the trajectory; at most
 * 256 in all), else they replace them.  Then `steps` Adam steps (rate lr) on
 * central-difference gradients of the mean energy-norm error
 * ||e - V r||_K^2 / ||e||_K^2, e = K^-1 r, each snapshot with the operator
 * of its own design.  Keeps the best parameters seen; *loss_first /
 * *loss_last: mean loss before and after.  Overwrites the context's
 * displacement. */
TO3D_API to3d_status to3d_mg_train(to3d_ctx* ctx, int32_t nsnap, int32_t steps, double lr,
                                   uint64_t seed, int32_t append, double* loss_first,
                                   double* loss_last);

typedef struct to3d_batch to3d_batch;

/* Create `nprob` independent problems (each as for to3d_create; params[i],
 * fixed[i], load[i], passive[i] (passive may be NULL, or hold NULL entries)).
 * Every problem's OC iteration is captured once as a CUDA graph whose solver
 * and bisection loops run on the device (conditional graph nodes); the
 * tensor-core kernel's z-segment length is autotuned per grid shape.  Only
 * the tensor-core defect-correction precisions are accepted (EINVAL for
 * TO3D_F64), with either filter; the device-side solver has no single- to
 * two-slice escalation,
 * so the two-slice forms are the robust choice here (a single-slice solve
 * that stalls ends in TO3D_ENOCONV).  `stream`: the caller's stream that each step is ordered on. */
TO3D_API to3d_status to3d_batch_create(int32_t nprob, const to3d_params* params,
                                       const uint8_t* const* fixed, const double* const* load,
                                       const uint8_t* const* passive, void* stream,
                                       to3d_batch** out);
/* One OC iteration of every problem (the graphs run side by side on a pool
 * of streams); info [nprob] may be NULL.  Returns the worst status. */
TO3D_API to3d_status to3d_batch_step(to3d_batch* b, to3d_iter_info* info);
TO3D_API to3d_status to3d_batch_get_density(to3d_batch* b, int32_t i, double* x, int32_t on_device);
TO3D_API int32_t to3d_batch_size(const to3d_batch* b);
/* Learned-multigrid parameters (see to3d_mg_set_params) for every problem of
 * a batch created with params.precond = TO3D_LMG; the problems' OC-iteration
 * graphs are captured again.  TO3D_ESTATE if a problem uses another
 * preconditioner, TO3D_EINVAL for invalid parameters. */
TO3D_API to3d_status to3d_batch_set_mg_params(to3d_batch* b, const double* theta, int64_t n);
TO3D_API void to3d_batch_destroy(to3d_batch* b);

/* Failure-detection self-test: one thread waits, with the bounded
 * suspend-and-poll loop every wait of the tensor-core kernel uses, on an
 * mbarrier phase that nothing completes; after `polls` polls (1 .. 65536, at
 * most ~1 us each) it gives up and *status receives TO3D_ETIMEOUT, the code
 * the tensor-core kernel reports when one of its waits runs out.  Nothing
 * hangs and the CUDA context stays usable.  `stream`: cudaStream_t as void*. */
TO3D_API to3d_status to3d_selftest_wait_timeout(int32_t polls, int32_t* status, void* stream);

/* Same results as to3d_sensitivity, but the library allocates nothing, and
 * no context is needed.  The paper has no counterpart: this entry point
 * exists for callers that cannot let a library call cudaMalloc.  Examples are
 * programs whose own pool or arena holds all device memory, where an outside
 * allocation falls outside that budget and may fail, and latency-critical
 * loops that must not enter the driver's allocator, which can synchronise the
 * device.
 *   x [nel], u [3N]       device pointers, inputs (densities, displacements)
 *   ce, dc [nel]          device pointers, outputs
 *   *compliance           host pointer, output
 *   stream                cudaStream_t (as void*) the work is enqueued on;
 *                         the call returns after the stream has finished it.
 * The grid-wide compliance sum uses one fixed scratch array compiled into
 * the library: 256 KiB + 256 B, which every GPU that loads the library
 * holds until the process exits.  It limits nel to 8,388,608 elements
 * (32768 blocks of 256); larger grids return TO3D_EINVAL, as do non-positive
 * sizes, null pointers and out-of-range parameters.  The first call on each
 * device looks up the array's device address; make that first call before
 * any stream capture.  That address belongs to the device's primary
 * context: after cudaDeviceReset (or any other release and re-creation of
 * that context) in the same process it is stale, so do not call this entry
 * point again in a process that has reset the device.  All calls share the array, and each call leaves its
 * contents behind (the call clears what must start at zero), so calls that
 * overlap on the GPU -- on different streams or from different threads --
 * race on it and must be serialised by the caller.
 * Errors: TO3D_EINVAL as above, TO3D_ECUDA if a CUDA call fails. */
TO3D_API to3d_status to3d_sensitivity_noalloc(int32_t nelx, int32_t nely, int32_t nelz,
                                              double penal, double E0, double Emin, double nu,
                                              const double* x, const double* u, double* ce,
                                              double* dc, double* compliance, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* TO3D_H */
