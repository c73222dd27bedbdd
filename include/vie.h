/*
 * vie.h -- C ABI of libvie: the FFT-accelerated J-VIE operator of
 * "Adiabatic absorbers in photonics simulations with the volume integral
 * equation method" (arXiv:1803.06237) on one NVIDIA GB300 (sm_103a).
 *
 * The library solves the discrete J-VIE of Sec. 3.1,
 *     (I - M_eps N) w = c_e M_eps e_inc,
 * on a uniform voxel grid with piecewise-constant currents and materials
 * (Sec. 3.1).  N is block-Toeplitz with six unique tensor components and is
 * applied with FFTs (Sec. 5.4); M_eps = (eps_r - 1)/eps_r per voxel (Sec. 3)
 * carries the material and the graded absorber loss (Sec. 4.1-4.2).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Grid n = {nx, ny, nz}.  A current vector holds 3 components per voxel in
 *    the layout [c][z][y][x] (x fastest), complex interleaved (re, im).  Its
 *    length is 3*nx*ny*nz complex numbers.  A per-voxel field is [z][y][x].
 *  - Units: h and 1/k0 are in the same length unit.  An exterior medium eps_bg
 *    is scaled out (Sec. 2): the operator uses k = k0 sqrt(eps_bg) and the
 *    contrast is taken relative to eps_bg.
 *  - Complex types: VIE_C64 = two float32 per number, VIE_C128 = two float64.
 *  - Pointers named *_host are host memory; *_dev are device memory on the
 *    device that was current when the plan was created.  The caller owns every
 *    buffer it passes; the library never keeps a caller pointer after a call
 *    returns.  `stream` is a cudaStream_t passed as void* (NULL = legacy
 *    default stream); device work is enqueued on it and the call returns
 *    without synchronising unless stated.
 *  - Every call returns a vie_status.  Nothing is printed; vie_last_error()
 *    returns a thread-local description of the last failure.
 */
#ifndef VIE_H_
#define VIE_H_

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct vie_plan vie_plan;

typedef enum {
  VIE_OK = 0,
  VIE_ERR_INVALID = 1,        /* bad argument: null pointer, size, flag */
  VIE_ERR_OOM = 2,            /* device allocation failed */
  VIE_ERR_CUDA = 3,           /* a CUDA runtime call or kernel launch failed */
  VIE_ERR_NOT_CONVERGED = 4,  /* solver stopped before the tolerance */
  VIE_ERR_TIMEOUT = 5,        /* a bounded device wait ran out */
  VIE_ERR_NONFINITE = 6       /* NaN/Inf met in an input or an iterate */
} vie_status;

enum { VIE_C64 = 1, VIE_C128 = 2 };

/* Flags for vie_plan_create. */
enum {
  VIE_PLAN_DEFAULT = 0,
  VIE_PLAN_CIRC_2N = 1,       /* circulant sizes exactly 2n (else the smallest
                                 5-smooth size >= 2n - 1) */
  VIE_PLAN_AUTOTUNE = 2       /* time complex64 operator applications for the
                                 three smallest 5-smooth sizes >= 2n - 1 per axis
                                 and the x-pass variants (four-step with 2 or 4
                                 lines per block, three-factor with 1 or 2)
                                 of the forward and the inverse pass, keep the
                                 fastest (any M >= 2n - 1 embeds the operator
                                 exactly); ignored with VIE_PLAN_CIRC_2N */
};

typedef struct {
  int n[3];                   /* grid nx, ny, nz */
  int m[3];                   /* circulant sizes Mx, My, Mz (each >= 2n-1) */
  double h, k0, eps_bg, kappa;/* kappa = k0 sqrt(eps_bg) h */
  size_t device_bytes;        /* device memory held by the plan */
  double setup_ms;            /* device time of entries + spectrum */
  double tune_ms;             /* host time spent by VIE_PLAN_AUTOTUNE (0 without) */
  int tune_candidates;        /* configurations timed (0 without) */
  int x_lines_per_block;      /* forward x pass chosen by the tuner: > 0 four-step
                                 register FFT with that many lines per block,
                                 < 0 three-factor register FFT with -value lines
                                 per block, 0 the default (three-factor where
                                 compiled for Mx, else four-step; five lines
                                 per block in complex64 when that makes one
                                 block per SM, e.g. nx = 600 with 759 lines) */
  int x_lines_per_block_inverse; /* the same for the inverse x pass (its default:
                                    four-step where compiled for Mx) */
} vie_plan_info;

/* Graded absorber of Sec. 4.1-4.2: eps'' = eps2_max * u^degree with
 * u = (x_c - x0)/length (direction +1) or (x0 - x_c)/length (direction -1),
 * x_c = ix + 1/2 the voxel centre in units of h, 0 <= u <= 1; applied to voxels
 * whose permittivity differs from eps_bg (the core).  eps'' = sigma/(w eps_0)
 * (the reading under which the round-trip formula of Sec. 4.3 holds). */
typedef struct {
  double x0;
  double length;
  int degree;                 /* 0..3 in the paper; any >= 0 accepted */
  int direction;              /* +1 or -1 */
  double eps2_max;
} vie_absorber;

/* Create a plan for grid n with voxel size h, free-space wavenumber k0 and
 * background permittivity eps_bg (Sec. 2 scaling).  Computes on the device,
 * in FP64, the Galerkin Toeplitz entries T_pq(Delta) of N (Sec. 3.1,
 * N_ij = <N P_j, P_i>) for Delta in [0,n) and the spectra of their circulant
 * embedding (Sec. 5.4), stored once in complex128 and once in complex64.
 * The plan's workspace holds 3*ny*nz*Mx complex128 values, plus Mx*My*3*nz
 * when the y-z plane is too large for one thread block (e.g. 1200 x 24: a
 * ring resonator's 600 x 11 cross-section), where the operator transforms y,
 * then z, then y back in separate passes; device_bytes reports the total.
 * Synchronises the device before returning.  The contrast starts at zero
 * (operator = identity).  Errors: VIE_ERR_INVALID (n < 1, h <= 0, k0 < 0,
 * eps_bg <= 0), VIE_ERR_OOM, VIE_ERR_CUDA.  *out is NULL on error. */
vie_status vie_plan_create(vie_plan** out, const int n[3], double h, double k0,
                           double eps_bg, int flags);

/* Release every device buffer of the plan.  NULL is accepted.  Always
 * VIE_OK. */
vie_status vie_plan_destroy(vie_plan* plan);

/* Fill *info (sizes, memory, setup and tuning figures above).  Host only.
 * Errors: VIE_ERR_INVALID (NULL argument). */
vie_status vie_plan_get_info(const vie_plan* plan, vie_plan_info* info);

/* Contrast from a relative permittivity map (step a1; Sec. 3, M_eps):
 * eps_host holds nx*ny*nz complex128 values (eps' - j eps'', relative to
 * vacuum) in [z][y][x] order.  Each absorber adds -j eps''(x) on core voxels;
 * then chi = eps/eps_bg - 1 and M = chi/(1 + chi) are formed on the device
 * and kept in complex128 and complex64.  n_abs may be 0 (absorbers NULL).
 * Synchronous.  Errors: VIE_ERR_INVALID, VIE_ERR_NONFINITE (eps = 0 after the
 * absorber, or non-finite), VIE_ERR_CUDA. */
vie_status vie_set_permittivity(vie_plan* plan, const double* eps_host,
                                const vie_absorber* absorbers, int n_abs);

/* Contrast directly from chi = eps_r/eps_bg - 1 (nx*ny*nz complex128, host).
 * M = chi/(1 + chi).  Synchronous.  Errors as vie_set_permittivity. */
vie_status vie_set_contrast(vie_plan* plan, const double* chi_host);

/* y = w - M (N w): one application of the J-VIE operator I - M_eps N
 * (Sec. 5.4 MVP): pad to the circulant, 3-D FFT, symmetric 3x3 spectral
 * multiply, inverse FFT, crop, contrast.  x_dev and y_dev are device vectors
 * of 3*nx*ny*nz complex numbers of type `dtype`; they must not overlap.
 * Asynchronous on `stream`.  Uses the plan's workspace, so calls on one plan
 * must not run concurrently on different streams.  Errors: VIE_ERR_INVALID,
 * VIE_ERR_CUDA. */
vie_status vie_matvec(vie_plan* plan, const void* x_dev, void* y_dev, int dtype,
                      void* stream);

/* Right-hand side of the J-VIE for an impressed current w_src radiating in
 * the background (Sec. 3, integral representation: e_inc = (1/c_e)(N - I) w_src):
 * b = c_e M e_inc = M ((N - I) w_src).  Same layout, types, rules and errors
 * as vie_matvec. */
vie_status vie_rhs_from_source(vie_plan* plan, const void* src_dev, void* b_dev,
                               int dtype, void* stream);

/* Copy the FP64 Toeplitz octant T_pq(Delta), Delta in [0,nx)x[0,ny)x[0,nz),
 * to the host: 6*nx*ny*nz complex128 in [comp][z][y][x] order with the
 * component order xx, yy, zz, xy, xz, yz.  out_host is caller-owned.
 * Synchronous.  Errors: VIE_ERR_INVALID (NULL argument), VIE_ERR_CUDA. */
vie_status vie_get_toeplitz(const vie_plan* plan, double* out_host);

/* eps''_max for a target round-trip reflection (Sec. 4.3 closed form with
 * p = d): -(d+1) ln(R_rt) sqrt(eps_r) / (D L eta k0).  Host-only arithmetic;
 * length and 1/k0 in the same unit.  Errors: VIE_ERR_INVALID. */
vie_status vie_eps2_from_round_trip(double r_rt, int degree, double length,
                                    double k0, double eps_r, double D, double eta,
                                    double* eps2_max);

/* ------------------------------------------------------------------------ */
/* Iterative solution of (I - M_eps N) w = b (Sec. 3.1 discrete J-VIE; the paper
 * uses GMRES at relative tolerance 1e-8, Sec. 5).                            */
/* ------------------------------------------------------------------------ */
enum {
  VIE_SOLVE_FP64 = 0,   /* restarted GMRES on the complex128 operator */
  VIE_SOLVE_MIXED = 1   /* iterative refinement: residual b - A x with the
                           complex128 operator, correction by restarted
                           (flexible) GMRES on the complex64 operator to a
                           loose tolerance, x accumulated in complex128 */
};

typedef struct {
  int mode;               /* VIE_SOLVE_FP64 or VIE_SOLVE_MIXED */
  int restart;            /* Krylov dimension m per cycle (<= 1000; 0 -> 100) */
  int max_iters;          /* cap on Arnoldi steps over the solve (0 -> 5000) */
  double inner_tol;       /* mixed: relative residual reduction asked of each
                             complex64 cycle (0 -> 1e-4) */
  int max_outer;          /* cap on cycles / refinement steps (0 -> 200) */
  int x0_given;           /* 1: x_dev holds an initial guess on entry */
  int use_preconditioner; /* 1: right-precondition with the learned network
                             set by vie_set_preconditioner (flexible GMRES) */
  int check_every;        /* host reads the device status every k steps (0 -> 4) */
  double timeout_s;       /* host wall-clock limit (0 -> 600 s) */
  int host_buffers;       /* 0: b and x are device pointers; 1: host pointers
                             (pageable or pinned), staged through device
                             buffers of 2 x 3N complex128 that the plan
                             allocates on first use and keeps */
  int resident;           /* 1: without a preconditioner, run the whole solve
                             (true residuals, refinement steps, cycles and
                             their decisions) as one CUDA graph launch with
                             device-side control (conditional WHILE/IF nodes;
                             the time limit is checked on the device at each
                             refinement step); 0: one graph launch per cycle,
                             decisions on the host between cycles.  Falls
                             back to 0 where conditional nodes are missing. */
} vie_solve_opts;

typedef struct {
  int iterations;         /* Arnoldi steps (Krylov operator applications) */
  int outer;              /* GMRES cycles (plain mode) or refinement steps
                             (mixed mode; each step may run several
                             complex64 cycles restarted from the complex64
                             residual) */
  int matvecs64;          /* complex128 operator applications */
  int matvecs32;          /* complex64 operator applications */
  int converged;          /* 1 if ||b - A x|| <= tol ||b|| (true FP64 residual) */
  int fallback;           /* 1 if the preconditioner was dropped during the solve
                             (a cycle it did not help, or network outputs that
                             were not finite and were replaced by the input) */
  double residual;        /* final true relative residual ||b - A x|| / ||b|| */
  double time_ms;         /* device time of the solve */
  int history_len;        /* entries used in history */
  double history[64];     /* true relative residual at the start of each cycle */
  int graph_cycles;       /* cycles run as one CUDA graph launch (the steps'
                             control flow on the device); the others ran from
                             the host loop */
  int reorth_steps;       /* Arnoldi steps that took the second Gram-Schmidt pass */
} vie_solve_info;

/* Solve (I - M N) x = b on the device (the paper's system of Sec. 3.1,
 * solved with GMRES as in Sec. 5).  b and x are complex128 vectors of
 * 3*nx*ny*nz entries, device pointers, or host pointers when
 * opts->host_buffers = 1 (b is copied in, x copied in if opts->x0_given and
 * copied out after the solve).  x: initial guess if opts->x0_given, the
 * solution on return; b is not modified.  Convergence is judged on the true
 * FP64 residual.  The solver workspace is allocated on the first call for a
 * given (restart, mode) and kept by the plan.  Synchronises `stream` before
 * returning.  Errors: VIE_ERR_INVALID, VIE_ERR_OOM, VIE_ERR_CUDA,
 * VIE_ERR_NONFINITE, VIE_ERR_TIMEOUT (x holds the best iterate),
 * VIE_ERR_NOT_CONVERGED (caps reached; x and info hold the last iterate). */
vie_status vie_solve(vie_plan* plan, const void* b, void* x, double tol,
                     const vie_solve_opts* opts, vie_solve_info* info, void* stream);

/* ------------------------------------------------------------------------ */
/* Batches of problems (many absorbers, profiles and right-hand sides of     */
/* uneven grid sizes solved together).                                       */
/* ------------------------------------------------------------------------ */

/* A plan with the same grid, h, k0 and eps_bg as `base` that shares base's
 * Toeplitz entries, spectra and twiddle tables (read-only, reference
 * counted) and owns its contrast (zero on return) and workspace.  Either plan
 * may be destroyed first.  Errors: VIE_ERR_INVALID, VIE_ERR_OOM, VIE_ERR_CUDA. */
vie_status vie_plan_clone(const vie_plan* base, vie_plan** out);

/* y_i = x_i - M_i (N_i x_i) for count plans.  Plans of equal grid and
 * circulant sizes are applied together, up to 16 per launch of each pass; a
 * plan may appear once.  x[i], y[i]: device vectors of plan i of type dtype.
 * Asynchronous on `stream`.  Errors: VIE_ERR_INVALID, VIE_ERR_CUDA. */
vie_status vie_matvec_batch(vie_plan* const* plans, int count, const void* const* x,
                            void* const* y, int dtype, void* stream);

/* vie_solve for count problems at once: every step advances all open
 * problems with one launch per kernel (the operator per group of equal
 * shape); each problem stops when its own true FP64 residual reaches tol.
 * b[i], x[i]: complex128 vectors of plan i (device pointers, or host pointers
 * with opts->host_buffers = 1, staged as in vie_solve); infos[i] its
 * report.  Synchronises `stream`.  Returns the first non-OK status of any
 * problem (VIE_ERR_NOT_CONVERGED etc.; every x[i] then holds its last
 * iterate).  Errors: as vie_solve. */
vie_status vie_solve_batch(vie_plan* const* plans, int count, const void* const* b,
                           void* const* x, double tol, const vie_solve_opts* opts,
                           vie_solve_info* infos, void* stream);

/* ------------------------------------------------------------------------ */
/* Learned right preconditioner (not in the paper, whose preconditioner is   */
/* block-circulant, Sec. 5.4): a 3-D convolutional network z = Net(v, chi)     */
/* trained on the device.  8 input channels (re/im of the three components  */
/* of v scaled to unit RMS, re/im of chi), 4 levels (2x2 average pooling in  */
/* x and y), 32 channels, 3x3x3 convolutions with zero padding, ReLU,        */
/* nearest upsampling with additive skips, 6 output channels; BF16 weights,  */
/* FP32 master weights and Adam.  Inference and (by default) training run   */
/* every convolution on the tcgen05 tensor cores with channels-last BF16    */
/* activations and FP32 accumulation: forward and input-gradient            */
/* convolutions as implicit GEMMs over positions, weight gradients as GEMMs */
/* over positions with 27 taps x 32 x 32 outputs.  VIE_TRAIN_FP32 selects   */
/* the FP32 SIMT training kernels instead (FP32 activations).               */
/* The preconditioner is z = v + Net(v): an untrained network (output layer */
/* at zero) is the identity.                                                */
/* Parameter layout (FP32): per layer enc0..enc3, dec2, dec1, dec0, out:     */
/* w[co][ci][27] (tap = 9 dz + 3 dy + dx) then b[co].                        */
/* ------------------------------------------------------------------------ */
typedef struct vie_net vie_net;

/* Number of FP32 parameters of the network. */
size_t vie_net_param_count(void);

/* New network on the current device: parameters copied from params_host
 * (count == vie_net_param_count()) or, if params_host is NULL, He-initialised
 * from `seed`.  Errors: VIE_ERR_INVALID, VIE_ERR_OOM, VIE_ERR_CUDA. */
vie_status vie_net_create(vie_net** out, const float* params_host, size_t count,
                          unsigned long long seed);
/* Release the network (NULL accepted; always VIE_OK).  It must not be set
 * as a plan's preconditioner (vie_set_preconditioner_net) at the time. */
vie_status vie_net_destroy(vie_net* net);

/* Copy the FP32 parameters / accumulated gradients (vie_net_param_count()
 * floats, caller-owned host array) to the host.  Synchronous.  Errors:
 * VIE_ERR_INVALID (NULL argument), VIE_ERR_CUDA. */
vie_status vie_net_get_params(const vie_net* net, float* out_host);
vie_status vie_net_get_grads(const vie_net* net, float* out_host);

/* z = v + |v|_rms Net(v / |v|_rms, chi of the plan) on the plan's grid; v_dev
 * and z_dev are device vectors (3*nx*ny*nz of dtype, not overlapping).  A
 * non-finite output entry is replaced by v and recorded (vie_net_status).
 * Asynchronous on `stream`.  Errors: VIE_ERR_INVALID (NULL argument, dtype,
 * a grid whose tensor maps cannot be encoded), VIE_ERR_OOM (first use on a
 * grid: activation workspace), VIE_ERR_CUDA; non-finite outputs and
 * timed-out waits are reported by vie_net_status, not here. */
vie_status vie_net_apply(vie_net* net, const vie_plan* plan, const void* v_dev,
                         void* z_dev, int dtype, void* stream);

/* One training sample (r, e) with A e = r (complex64 device vectors): forward
 * pass on r, loss |r + Net(r) - e|^2 / |e|^2 (all scaled by the RMS of r),
 * backward pass; gradients are ADDED to the network's accumulators.  *loss
 * receives the sample's loss.  Synchronises `stream`.  Errors:
 * VIE_ERR_INVALID (NULL argument, a grid whose tensor maps cannot be
 * encoded), VIE_ERR_OOM (first use on a grid: training workspace),
 * VIE_ERR_CUDA.  A bounded wait inside a tensor-core kernel that ran out is
 * recorded for vie_net_status (flag 2); the sample's gradients are then not
 * valid. */
vie_status vie_net_accumulate(vie_net* net, const vie_plan* plan, const void* r_dev,
                              const void* e_dev, double* loss, void* stream);
/* Clear the accumulated gradients.  Synchronous.  Errors: VIE_ERR_INVALID
 * (NULL), VIE_ERR_CUDA. */
vie_status vie_net_zero_grad(vie_net* net);

/* Precision of vie_net_accumulate: VIE_TRAIN_TENSOR_BF16 (default; BF16
 * activations and gradient tensors, tensor cores, FP32 accumulation) or
 * VIE_TRAIN_FP32 (FP32 activations, SIMT kernels).  Errors: VIE_ERR_INVALID. */
#define VIE_TRAIN_TENSOR_BF16 0
#define VIE_TRAIN_FP32 1
vie_status vie_net_set_training(vie_net* net, int mode);

/* Adam step (beta1 0.9, beta2 0.999, eps 1e-8) on the accumulated gradients
 * times grad_scale, refresh of the BF16 weights, gradients cleared.
 * Asynchronous on `stream`.  Errors: VIE_ERR_INVALID (NULL), VIE_ERR_CUDA. */
vie_status vie_net_adam_step(vie_net* net, float lr, float grad_scale, void* stream);

/* Status of the applications since the last clear (synchronises the device):
 * *flag = 0 all fine, 1 a non-finite output was replaced by v, 2 a wait inside
 * a tensor-core convolution timed out (its output is not valid).  clear != 0
 * resets it.  Errors: VIE_ERR_INVALID (NULL argument), VIE_ERR_CUDA. */
vie_status vie_net_status(vie_net* net, int* flag, int clear);

/* ------------------------------------------------------------------------ */
/* Block-circulant preconditioner (Sec. 5.4): W, the matrix nearest to        */
/* A = I - M N in the Frobenius norm among those that are circulant along x */
/* (dense (3 ny nz)^2 blocks, rows and columns ordered (component, z, y)):   */
/* W = circ(c_0 .. c_{nx-1}), c_k = (1/nx) sum_i A[i][(i - k) mod nx].  The  */
/* DFT along x makes W block diagonal; the nx blocks are LU-factored        */
/* (partial pivoting) in complex64 on the device.  Applied as a right        */
/* preconditioner of flexible GMRES (the paper writes the left form         */
/* W^{-1} A; the two preconditioned matrices are similar).                   */
/* Device memory: nx (3 ny nz)^2 complex64 (2.8 GB for the 600 x 23 x 11     */
/* guide).                                                                   */
/* ------------------------------------------------------------------------ */
typedef struct vie_circulant vie_circulant;

/* Flags of vie_circulant_create. */
#define VIE_CIRC_DEFAULT 0
#define VIE_CIRC_FP16_FACTORS 1   /* keep the LU factors in complex half precision (half the memory and
                                     half the bytes per application); the factorisation runs in complex64 */

/* Build W from the plan's current Toeplitz entries and contrast (the plan's
 * contrast must have been set) and factor it; synchronises `stream`.  The
 * preconditioner keeps a pointer to the plan: destroy it before the plan.
 * If the plan's contrast changes afterwards, applications fail with
 * VIE_ERR_INVALID (stale).  Errors: VIE_ERR_INVALID (no contrast, cross
 * section above ~1600 unknowns), VIE_ERR_OOM, VIE_ERR_CUDA,
 * VIE_ERR_NONFINITE (a singular block). */
vie_status vie_circulant_create(vie_plan* plan, int flags, vie_circulant** out, void* stream);

/* z = W^{-1} v for device vectors of 3*nx*ny*nz entries of dtype (VIE_C64
 * or VIE_C128; computed in complex64 either way, with complex-half factors
 * if built with VIE_CIRC_FP16_FACTORS), not overlapping.
 * Asynchronous on `stream`.  Errors: VIE_ERR_INVALID (NULL argument, dtype,
 * the plan's contrast changed since the build), VIE_ERR_CUDA. */
vie_status vie_circulant_apply(vie_circulant* c, const void* v_dev, void* z_dev, int dtype, void* stream);

/* Setup time (ms, host clock around the build) and device bytes held
 * (either pointer may be NULL).  Host only.  Errors: VIE_ERR_INVALID (NULL
 * c). */
vie_status vie_circulant_info(const vie_circulant* c, double* build_ms, size_t* device_bytes);
/* Release the factors (NULL accepted; always VIE_OK).  It must not be set as
 * a plan's preconditioner at the time. */
vie_status vie_circulant_destroy(vie_circulant* c);

/* Use `c` (NULL: none) as the right preconditioner of this plan's solves
 * with opts->use_preconditioner = 1, replacing any network set with
 * vie_set_preconditioner.  `c` must have been built for this plan; the plan
 * keeps a reference, not a copy.  Errors: VIE_ERR_INVALID (NULL plan, `c`
 * built for another plan). */
vie_status vie_set_circulant_preconditioner(vie_plan* plan, vie_circulant* c);

/* Use the learned network with the given FP32 parameters as the right
 * preconditioner of this plan's solves with opts->use_preconditioner = 1
 * (flexible GMRES).  weights: host array of vie_net_param_count() floats in
 * the parameter layout above (e.g. from vie_net_get_params after training);
 * bytes must be 4 * vie_net_param_count().  The plan builds and owns a
 * network from a copy (the caller's array is not kept) and releases it when
 * the preconditioner is replaced or the plan destroyed.  weights = NULL:
 * unpreconditioned (any preconditioner set before is removed).  Errors:
 * VIE_ERR_INVALID (bytes), VIE_ERR_OOM, VIE_ERR_CUDA. */
vie_status vie_set_preconditioner(vie_plan* plan, const void* weights, size_t bytes);

/* Same, with a network object the caller keeps (e.g. while training it):
 * `net` (NULL: none) becomes the right preconditioner; the plan keeps a
 * reference, and the caller must not destroy the network while it is set.
 * Errors: VIE_ERR_INVALID (NULL plan). */
vie_status vie_set_preconditioner_net(vie_plan* plan, vie_net* net);

/* ------------------------------------------------------------------------ */
/* JM-VIE (Sec. 3, discrete form Sec. 3.1): electric and magnetic currents,  */
/* for magnetic loss matched to the electric absorber (Sec. 4.2).  With      */
/* u_e = J/c_e and u_m = eta M/c_m (both in units of the electric field,   */
/* eta the background impedance) the system (I - M T)(J, M) = C M (E, H)    */
/* reads                                                                     */
/*   u_e - M_eps (N u_e) + j kappa M_eps (C x u_m) = M_eps e_inc             */
/*   u_m - M_mu  (N u_m) - j kappa M_mu  (C x u_e) = M_mu  eta h_inc         */
/* with K = curl S = h C x (the curl Toeplitz operator, three unique odd     */
/* components C_a = <P_i, d_a S P_j>/h), kappa = k h, M_mu = (mu_r-1)/mu_r.  */
/* A JM vector holds 6 components per voxel, [c][z][y][x] with c = 0..2     */
/* the electric and c = 3..5 the magnetic current, 6*nx*ny*nz complex       */
/* numbers.  The plane of one kx (6 x My x Mz values) must fit in one       */
/* thread block's shared memory (e.g. the 23 x 11 guide cross-section).     */
/* ------------------------------------------------------------------------ */

/* Permeability of the plan's voxels for the JM-VIE: mu_host holds
 * nx*ny*nz complex128 mu_r = mu' - j mu'' in [z][y][x] order, or NULL for
 * the impedance-matched permeability of Sec. 4.2, mu'' = eps''/eps' with
 * eps' - j eps'' the plan's current permittivity (mu_r = 1 where it is
 * lossless, i.e. outside the absorbers).  The first call computes, in FP64,
 * the curl entries C_a(Delta) and their folded spectra and allocates the
 * JM workspace (6 ny nz Mx complex128).  Call it again after the
 * permittivity changes.  Synchronous.  Errors: VIE_ERR_INVALID,
 * VIE_ERR_NONFINITE (mu = 0 or non-finite), VIE_ERR_OOM, VIE_ERR_CUDA. */
vie_status vie_set_permeability(vie_plan* plan, const double* mu_host);

/* y = u - M (T u) for 6N device vectors x = u and y of type dtype (not
 * overlapping).  Asynchronous on `stream`; uses the plan's JM workspace.
 * Errors: VIE_ERR_INVALID (no permeability set, stale, overlap),
 * VIE_ERR_CUDA. */
vie_status vie_jm_matvec(vie_plan* plan, const void* x_dev, void* y_dev, int dtype, void* stream);

/* Right-hand side for impressed currents (w_e, w_m) (6N, scaled like u)
 * radiating in the background: e_inc = (N - I) w_e - j kappa C x w_m,
 * eta h_inc = (N - I) w_m + j kappa C x w_e, b = (M_eps e_inc, M_mu eta h_inc).
 * Same rules and errors as vie_jm_matvec. */
vie_status vie_jm_rhs_from_source(vie_plan* plan, const void* src_dev, void* b_dev, int dtype, void* stream);

/* Solve the JM-VIE for 6N complex128 vectors b and x (device pointers, or
 * host pointers with opts->host_buffers = 1), as vie_solve does for the
 * J-VIE: restarted GMRES on the complex128 operator or mixed-precision
 * refinement; no preconditioner (opts->use_preconditioner must be 0).
 * The field on the axis is vie_axis_field of the electric half (E =
 * u_e / chi_e).  Errors: as vie_solve. */
vie_status vie_jm_solve(vie_plan* plan, const void* b, void* x, double tol, const vie_solve_opts* opts,
                        vie_solve_info* info, void* stream);

/* Field on the centre axis (step a12; Sec. 3 equivalent currents J =
 * c_e chi E, so E = J/(c_e chi); the factor c_e h^(3/2) common to every
 * field is not applied).  w_dev: complex128 solution (3*nx*ny*nz); e_dev:
 * complex128 output of 3*n_keep values [c][ix] for ix < n_keep on the voxel
 * row (ny/2, nz/2), using the plan's chi.  Synchronous.  Errors:
 * VIE_ERR_INVALID, VIE_ERR_NONFINITE (chi = 0 on the axis), VIE_ERR_CUDA. */
vie_status vie_axis_field(const vie_plan* plan, const void* w_dev, int n_keep,
                          void* e_dev, void* stream);

/* Reflection coefficient of Sec. 5.1: R = sum |E_ref - E|^2 / sum |E_ref|^2
 * over `count` complex128 device values (e.g. two vie_axis_field outputs
 * cut to the guide before the absorber).  FP64 sums.  Synchronous.  Errors:
 * VIE_ERR_INVALID, VIE_ERR_NONFINITE (zero reference), VIE_ERR_CUDA. */
vie_status vie_reflection(const void* eref_dev, const void* e_dev, int count,
                          double* r_out, void* stream);

/* Transmission through the voxel plane ix (Sec. 5.2): T = sum of |E|^2 over
 * the plane's voxels with chi != 0 (the structure's cross-section), E =
 * w / chi per component (the common factor |c_e|^2 h^3 is not applied).
 * w_dev: complex128 solution (3*nx*ny*nz).  FP64 sums.  Synchronous.
 * Errors: VIE_ERR_INVALID, VIE_ERR_CUDA. */
vie_status vie_slice_power(const vie_plan* plan, const void* w_dev, int ix, double* t_out, void* stream);

/* Same operator application as vie_matvec, for callers that cannot allocate
 * device memory where they apply the operator (their memory is owned by
 * another allocator or held to a fixed budget after start-up, so they cannot
 * make a second plan or a second workspace).  The paper has no counterpart:
 * this is a deployment variant of the Sec. 5.4 product.
 *
 * It allocates nothing.  Its workspace is a static device array of 16 MiB
 * inside the library (every GPU that loads the library holds it until the
 * process exits) instead of the plan's workspace, so it may run on another
 * stream while vie_matvec runs on the same plan.  The plan is only read.
 * Limit: 3*ny*nz*Mx complex values of `dtype` (Mx from vie_plan_get_info) must
 * fit in 16 MiB; larger plans are rejected with VIE_ERR_INVALID.  Where the
 * y-z plane is too large for one thread block and the y-pass buffer
 * (Mx*My*3*nz values) does not fit behind it in the 16 MiB, the plane is
 * transformed by clusters of thread blocks sharing it in distributed shared
 * memory (same result, slower).  The plan's
 * device must be current.  vie_plan_create and vie_plan_clone look up the
 * array's device address (cudaGetSymbolAddress) on the plan's device, which
 * also makes the CUDA runtime load the part of the library that holds the
 * array; so under lazy module loading (the CUDA default) the memory is
 * reserved when a plan is made, not by the first call here, and the calls
 * only read the cached address.  Every call shares the one array and it keeps the previous
 * call's contents; nothing in it needs to start at zero (the first pass writes
 * every element the later passes read).  Calls whose execution overlaps on the
 * GPU race on the array: order them on one stream or with events.
 * Asynchronous on `stream`.  Errors: VIE_ERR_INVALID, VIE_ERR_CUDA. */
vie_status vie_matvec_static_scratch(const vie_plan* plan, const void* x_dev,
                                     void* y_dev, int dtype, void* stream);

/* Measured fused multiply-add throughput of the current GPU in TFLOP/s
 * (2 flops per FMA): FP32 for dtype VIE_C64, FP64 for VIE_C128.  Runs two
 * short FMA-chain kernels (a few ms) on `stream` and synchronises it.  The
 * paper has no counterpart: this is the ALU roofline against which the
 * operator's FP32 (complex64) and FP64 (complex128) passes are reported.
 * Errors: VIE_ERR_INVALID, VIE_ERR_OOM, VIE_ERR_CUDA. */
vie_status vie_probe_fma_tflops(int dtype, double* tflops, void* stream);

/* Failure detection of the solver's grid barrier (the cooperative
 * Gram-Schmidt step; no counterpart in the paper): one barrier over one
 * block per SM in which block absent_block (-1: none) does not take part.
 * The other blocks give up after wait_ms (0 < wait_ms <= 2000) and set the
 * abort word; *aborted = 1 then, 0 when the barrier completed.  Synchronous.
 * Errors: VIE_ERR_INVALID, VIE_ERR_CUDA. */
vie_status vie_probe_grid_barrier(int absent_block, double wait_ms, int* aborted);

/* Thread-local description of the last error ("" if none). */
const char* vie_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* VIE_H_ */
