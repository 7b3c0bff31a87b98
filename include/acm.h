/*
 * acm.h -- C ABI of the GB300 (sm_103a) implementation of accelerated
 * computational micromechanics (ACM) for periodic porous unit cells
 * (Karimi & Bhattacharya, arXiv 2312.15554).
 *
 * Problem (Section 2, Eq. 1): in the periodic unit cube Y = Y_p (pore) + Y_s (solid),
 *   Stokes flow   -grad p + nu Lap u + g = 0, div u = 0 in Y_p, u = 0 in Y_s;
 *   solute        Pe u.(grad chi) - Lap chi = Pe (ubar - u).g_chi in Y_p,
 *                 zero-flux condition on the pore boundary;
 * with effective permeability K (Eq. 2) and diffusivity D (Eq. 3).
 *
 * Method (Section 3): Stokes by ADMM on an augmented Lagrangian (Eq. 6-13) with
 * adaptive penalties (Eq. 22); solute by a Lippmann-Schwinger fixed point with a
 * fictitious solid diffusivity (Eq. 14-21). Every iteration is a voxelwise local
 * step plus a constant-coefficient solve in Fourier space.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Grid      (n0, n1, n2): n1 and n2 powers of two in [8, 512], n0 the same or 1
 *           (then n1 >= 32); axis 2 is contiguous. The cell is the unit cube; h_c = 1/n_c;
 *           V = n0*n1*n2 voxels. n0 = 1 is a single plane: the two-dimensional
 *           cell of the paper's experiments (Section 4), with the symbols of
 *           axis 0 equal to zero (no variation along it); vector fields keep
 *           three components (component 0, the flow along the cylinders of an
 *           extruded geometry, decouples from the in-plane ones).
 * H         uint8_t[n0][n1][n2], 1 = solid, 0 = pore (Eq. 4).
 * Vectors   component-planar [3][n0][n1][n2]; component c is along array axis c.
 *           Load direction e_j therefore means array axis j.
 * Reals     float when the precision is ACM_FP32, double otherwise (the
 *           "real type" below).
 * Pointers  every array argument may be a device pointer or a host pointer.
 *           Device pointers are used in place; host buffers (pageable or
 *           pinned) are staged through the context's device workspace with
 *           copies on the context's stream, so a host call includes the
 *           host<->device transfers. Scalars and reports are host memory.
 * Ownership the library never frees or retains caller memory. A context owns
 *           its workspace (allocated on first use of a precision, freed by
 *           acm_destroy); an acm_batch and an acm_fno own theirs likewise
 *           (freed by acm_batch_destroy / acm_fno_destroy). Calls on one object
 *           are not thread safe; distinct objects are independent.
 * Streams   all device work of a context is ordered on the stream given at
 *           acm_create (NULL = legacy default stream). Every solver entry point
 *           returns after its results are complete on the host side (K, D,
 *           reports) and enqueued on the stream (fields).
 * Errors    every entry point returns an acm_status and never aborts. On any
 *           status other than ACM_OK and ACM_ERR_MAXITER the output fields are
 *           unspecified; ACM_ERR_MAXITER still writes every output.
 */
#ifndef ACM_H
#define ACM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct acm_ctx acm_ctx;

typedef enum acm_status {
  ACM_OK = 0,
  ACM_ERR_ARG = -1,              /* invalid argument (null pointer, bad size or parameter) */
  ACM_ERR_NOMEM = -2,            /* device allocation failed */
  ACM_ERR_CUDA = -3,             /* a CUDA runtime call failed */
  ACM_ERR_MAXITER = -4,          /* max_iter reached before the tolerance; outputs written */
  ACM_ERR_DIVERGED = -5,         /* residual grew 1e3x above its running minimum */
  ACM_ERR_NONFINITE = -6,        /* a residual became NaN or infinite */
  ACM_ERR_NO_SOLID = -7,         /* Stokes: H has no solid voxel (mean flow unbounded) */
  ACM_ERR_NO_FLUID = -8,         /* H has no pore voxel */
  ACM_ERR_TIMEOUT = -9,          /* a bounded device wait gave up */
  ACM_ERR_UNSUPPORTED_SIZE = -10 /* grid size outside the supported set */
} acm_status;

typedef enum acm_deriv {
  ACM_DERIV_EXACT = 0,   /* d_c = k_c (0 on the Nyquist plane), L = |k|^2 (Eq. 13) */
  ACM_DERIV_CENTRAL = 1  /* d_c = sin(h k_c)/h, L = sum 4 sin^2(h k_c/2)/h^2 (Eq. 21) */
} acm_deriv;

typedef enum acm_precision {
  ACM_FP32 = 0,           /* FP32 fields and FFTs, FP64 reductions */
  ACM_FP64 = 1,           /* FP64 throughout */
  ACM_FP32_THEN_FP64 = 2  /* FP32 iterations to eps32, then FP64 iterations to eps */
} acm_precision;

/* Stokes (ADMM) parameters, Section 3.1 and Eq. 22. */
typedef struct acm_stokes_params {
  double nu;           /* viscosity (default 1) */
  double eps;          /* eps_abs = eps_rel of Eq. 11-12 (default 1e-5) */
  double alpha0;       /* initial penalty alpha (solid constraint); <= 0 selects the default */
  double beta0;        /* initial penalty beta (incompressibility); <= 0 selects the default */
  double b0;           /* initial penalty b (u = u~); <= 0 selects the default */
  double phi[3];       /* Eq. 22 growth factors for (alpha, beta, b) (default 1.1) */
  double tau[3];       /* Eq. 22 residual-balance ratios (default {5, 10, 5}) */
  double psi_min_frac; /* psi_min = psi_min_frac * psi0 (default 1e-3) */
  double eps32;        /* FP32 phase tolerance of ACM_FP32_THEN_FP64 (default 1e-5); a load
                          whose FP32 residuals stop gaining on it (no 2 % gain in 500
                          iterations: the FP32 rounding floor) moves on to FP64 early */
  int max_iter;        /* iteration cap (default 20000) */
  int adaptive;        /* 1: Eq. 22 penalty updates; 0: fixed penalties (default 1) */
  int deriv;           /* acm_deriv (default ACM_DERIV_EXACT) */
  int precision;       /* acm_precision (default ACM_FP32) */
  int check_every;     /* iterations between host checks of the stop flag (default 16) */
  int device_loop;     /* 1: the whole iteration loop is one device-resident CUDA graph
                          launch (default); 0: host-launched chunks of check_every */
  double pore_scale;   /* > 0: every penalty not given explicitly starts at
                          pore_scale / l^2 times its default, l = (pore voxels) /
                          (solid-pore voxel faces) of the cell, in voxels (per cell in
                          a batch). Not part of the paper: Eq. 22 compares a velocity
                          with a penalty times a velocity, so the best fixed penalty
                          follows the pore scale; 9 with adaptive = 0 is the measured
                          choice for time to permeability. 0 (default): off */
} acm_stokes_params;

/* Solute (Lippmann-Schwinger) parameters, Section 3.2. */
typedef struct acm_advdiff_params {
  double eta;          /* fictitious solid diffusivity (default 0.01) */
  double A0;           /* comparison medium A0 > 0 (default 0.55) */
  double B0[3];        /* comparison medium B0, used when B0_explicit = 1 */
  int B0_explicit;     /* 0: B0 = mean over Y of B = Pe (1-H) u (default); 1: B0 as given */
  double eps;          /* tolerance of Eq. 19 (default 1e-5) */
  int max_iter;        /* iteration cap (default 20000) */
  int deriv;           /* acm_deriv (default ACM_DERIV_CENTRAL) */
  int precision;       /* acm_precision (default ACM_FP32); with ACM_FP32_THEN_FP64 the
                          FP32 iterations run to max(eps, 1e-5) (or until they stop
                          gaining on it, their rounding floor), then FP64 ones to eps */
  int check_every;     /* iterations between host checks of the stop flag when the
                          loop is host-launched (default 16) */
  int device_loop;     /* 1: the whole iteration loop is one device-resident CUDA graph
                          launch (default); 0: host-launched chunks of check_every */
} acm_advdiff_params;

/* Per-solve report. For Stokes res/tol hold r_p1, r_d1, r_p2, r_d2, r_p3, r_d3
 * (Eq. 10) and their tolerances (Eq. 11-12) of the last iteration; psi the
 * penalties alpha, beta, b of that iteration. For the solute res[0..1] hold
 * r1, r2 (Eq. 19) and tol[0..1] their tolerances. */
typedef struct acm_report {
  int iters;           /* total iterations */
  int iters_fp64;      /* iterations of those run in FP64 */
  int converged;       /* 1 when every residual passed its tolerance */
  int status;          /* acm_status of this solve */
  double res[6];
  double tol[6];
  double psi[3];
  double time_ms;      /* wall time of the solve (host clock, stream synchronised) */
} acm_report;

/* Fill defaults (documented in the structs above). Returns ACM_ERR_ARG on NULL. */
acm_status acm_stokes_default_params(acm_stokes_params* p);
acm_status acm_advdiff_default_params(acm_advdiff_params* p);

/* Create a context for grids of shape (n0, n1, n2) whose device work runs on
 * `cuda_stream` (a cudaStream_t, NULL for the default stream) of the current
 * device. Returns ACM_ERR_UNSUPPORTED_SIZE unless n1 and n2 are powers of two
 * in [8, 512] and n0 is one too, or 1 with n1 >= 32. */
acm_status acm_create(acm_ctx** ctx, int n0, int n1, int n2, void* cuda_stream);
acm_status acm_destroy(acm_ctx* ctx);

/* Problem 1 of Algorithm 1 (Section 3.1): Stokes flow for the body force g
 * (g = -g_p, the negative average pressure gradient of Eq. 1).
 *   init_u, init_lambda  optional warm start (NULL = zero): X^0 = {u, u~ = u,
 *                        q, a = H lambda, lambda = H lambda}; real type. q is 0
 *                        without init_lambda; with it, q is the pressure of a
 *                        fixed point with that a: the divergence of Eq. 7 at
 *                        u = u~, div u = 0 gives |d|^2 q^ = i d.a^ (k != 0).
 *   u       out [3][V] velocity u^{n} of the last iteration (real type).
 *   p       out [V] pressure q - mean(q) (nullable; real type).
 *   lambda  out [3][V] solid multiplier H lambda (nullable; real type).
 *   K_col   out (host, 3 doubles, nullable) volume average of u, i.e. K g for
 *           nu = 1 (the average-velocity form of Eq. 2).
 *   rep     out (host, nullable).
 * Returns ACM_ERR_NO_SOLID when H has no solid voxel (the mean flow is then
 * unbounded) and ACM_ERR_NO_FLUID when H is all solid. */
acm_status acm_stokes(acm_ctx* ctx, const uint8_t* H, const double g[3],
                      const acm_stokes_params* prm,
                      const void* init_u, const void* init_lambda,
                      void* u, void* p, void* lambda,
                      double K_col[3], acm_report* rep);

/* The three unit loads e_j solved together (superposition, Section 2).
 *   u3      out [3 loads][3][V] (real type; nullable).
 *   K       out (host, 9 doubles, row-major K[i][j] = mean of u^j_i).
 *   K_grad  out (host, 9 doubles, nullable): Eq. 2 literally, the integral over
 *           Y_p of grad u^i : grad u^j with the spectral gradient of prm->deriv.
 *   rep     out (host, 3 reports, nullable). */
acm_status acm_stokes_tensor(acm_ctx* ctx, const uint8_t* H, const acm_stokes_params* prm,
                             void* u3, double K[9], double K_grad[9], acm_report rep[3]);

/* Problem 2 of Algorithm 1 (Section 3.2): the concentration corrector chi for
 * the composition gradient g_chi, advected by the velocity u (real type
 * [3][V], e.g. the output of acm_stokes) at Peclet number Pe.
 *   chi       out [V] (real type, nullable), mean zero.
 *   grad_chi  out [3][V] (real type, nullable), spectral gradient.
 *   Dg        out (host, 3 doubles): Eq. 3 contracted with g_chi,
 *             (D g)_i = (1/V) sum_pore [g_i + Pe (ubar - u)_i chi + d_i chi].
 *   Dg_ext    out (host, 3 doubles, nullable): extended-domain average
 *             (1/V) sum_Y A (g + grad chi)_i + the same Pe term.
 * The real type of u, chi and grad_chi follows prm->precision (double for the
 * mixed mode). A device u aligned to 16 bytes is read in place; any other u
 * is first copied into the context's workspace. */
acm_status acm_advdiff(acm_ctx* ctx, const uint8_t* H, const void* u, double Pe,
                       const double g_chi[3], const acm_advdiff_params* prm,
                       void* chi, void* grad_chi, double Dg[3], double Dg_ext[3],
                       acm_report* rep);

/* The three composition loads e_j: D (host, 9 doubles, row-major D[i][j] =
 * (D e_j)_i), D_ext (nullable), chi3 out [3 loads][V] (nullable). */
acm_status acm_advdiff_tensor(acm_ctx* ctx, const uint8_t* H, const void* u, double Pe,
                              const acm_advdiff_params* prm, void* chi3,
                              double D[9], double D_ext[9], acm_report rep[3]);

/* The 3D real-to-complex transform used by both solvers, exposed for testing:
 * f^(m) = sum_x f(x) exp(-2 pi i m.x), unnormalised.
 *   in   real [nbatch][V] (float when fp64 = 0, double otherwise).
 *   out  complex interleaved (re, im) [nbatch][n0][n1][n2/2 + 1].
 * acm_fft_c2r is the exact inverse: it divides by V. */
acm_status acm_fft_r2c(acm_ctx* ctx, int fp64, int nbatch, const void* in, void* out);
acm_status acm_fft_c2r(acm_ctx* ctx, int fp64, int nbatch, const void* in, void* out);

/* Batched Stokes (the unit-cell problem of Section 2 for many cells at once):
 * the three unit loads of every cell, solved in one device-resident loop. Cells
 * of one shape share every kernel launch; each problem keeps its own penalties
 * (Eq. 22) and stop flag, and converged problems stop doing work.
 *   acm_batch_create  ncells cells with shapes dims[ncells][3] (host), each
 *                     a grid acm_create accepts; the workspace of all cells is
 *                     allocated here (about 95 MB per 128^3 cell in FP32).
 *   acm_batch_stokes  H: host array of ncells indicator pointers (device or
 *                     host); prm: precision ACM_FP32 or ACM_FP64 (the mixed
 *                     mode is not batched); init_u, init_lambda: nullable host
 *                     arrays of ncells nullable pointers to [3 loads][3][V]
 *                     (real type), the warm start X^0 of each load as in
 *                     acm_stokes (u~ = u, lambda masked by H, a = H lambda);
 *                     u_out, lambda_out: nullable host arrays of ncells
 *                     nullable pointers to [3 loads][3][V] (real type);
 *                     K: host [ncells][9], row-major K[i][j] of each cell (NaN
 *                     for a cell without solid or without pore voxels, whose
 *                     reports carry ACM_ERR_NO_SOLID / ACM_ERR_NO_FLUID);
 *                     rep: nullable host [ncells][3].
 * Returns ACM_OK when every problem ran (check the per-problem statuses in rep). */
typedef struct acm_batch acm_batch;
acm_status acm_batch_create(acm_batch** batch, int ncells, const int* dims, void* cuda_stream);
acm_status acm_batch_destroy(acm_batch* batch);
acm_status acm_batch_stokes(acm_batch* batch, const uint8_t* const* H, const acm_stokes_params* prm,
                            const void* const* init_u, const void* const* init_lambda, void* const* u_out,
                            void* const* lambda_out, double* K, acm_report* rep);
/* Tile autotuner. The strided FFT passes of the solver loops (y forward and
 * inverse of the Stokes iteration, the z pass with the Green step of Eq. 13,
 * the y forward, z pass (Eq. 20) and y inverse of the solute iteration) exist in up to
 * three tile widths (columns per block). acm_autotune times each candidate on
 * the context's workspace and stream and keeps the fastest for that precision
 * (fp64 0/1) and derivative symbol; acm_batch_autotune does so per cell shape
 * with the batch's problem count. Fields do not depend on the choice; only the
 * summation order of the FP64 residual partials does. tiles (out, nullable):
 * the widths in the order y-forward Stokes, z Stokes, y-inverse Stokes,
 * y-forward solute, z solute, y-inverse solute (0 where a pass does not apply). acm_set_tiles sets them explicitly
 * (ACM_ERR_ARG for a width that has no compiled variant); acm_get_tiles reads
 * the current widths. Call between solves. */
acm_status acm_autotune(acm_ctx* ctx, int fp64, int deriv, int tiles[6]);
acm_status acm_set_tiles(acm_ctx* ctx, int fp64, const int tiles[6]);
acm_status acm_get_tiles(acm_ctx* ctx, int fp64, int tiles[6]);
acm_status acm_batch_autotune(acm_batch* batch, int fp64, int deriv);
acm_status acm_batch_tiles(acm_batch* batch, int cell, int fp64, int tiles[6]);

/* Per-iteration records of every problem of a batch (the Stokes record of
 * acm_history: residuals, tolerances, penalties, mean velocity), off by default.
 *   acm_batch_history_enable  cap > 0 allocates cap records per problem
 *                     (160 bytes each; 3 problems per cell), cap = 0 frees them.
 *   acm_batch_history  the records of (cell, load) from the last acm_batch_stokes
 *                     into out [min(cap, count)][20]; count = records kept. */
acm_status acm_batch_history_enable(acm_batch* batch, int cap);
acm_status acm_batch_history(acm_batch* batch, int cell, int load, double* out, int cap, int* count);
/* The profiler of acm_profile_enable / acm_profile_read over all cells of a batch. */
acm_status acm_batch_profile_enable(acm_batch* batch, int on);
acm_status acm_batch_profile_read(acm_batch* batch, double* ms, long long* launches);

/* Learned warm start: a 3D Fourier neural operator mapping an indicator H to
 * an initial velocity and solid multiplier for acm_stokes (warm-start inputs
 * init_u, init_lambda), trained on solutions of the method itself.
 *   features (H, x0, x1, x2) with x_c = (i_c + 1/2)/n_c; lift v = P a + p;
 *   L layers v <- gelu(G(R_l F(v)) + M_l v + m_l), F the forward DFT on the
 *   kept modes (k2 < modes; k0, k1 in [0, modes) or [n - modes, n)), R_l a
 *   width x width complex matrix per kept mode, G(Y) = (1/V) sum w_k Re[Y e^{2 pi i k.x}]
 *   (w_k = 1 on k2 = 0, else 2); projection out = Q v + q to 6 channels
 *   (u, lambda). Loss (1/(B V)) sum |out_u - t_u|^2 + H |out_lambda - t_lambda|^2.
 * Weights and stored activations are BF16; arithmetic and accumulation FP32.
 * Parameters form one FP32 vector: P [W][4], p [W], per layer R [M][W][W][2]
 * (M = 4 modes^3), M [W][W], m [W]; then Q [6][W], q [6].
 *   acm_fno_create    width in {4, 8, 16, 32}; 1 <= max_batch <= 64; parameters zero.
 *   acm_fno_forward   H [batch][V] (device or host), out [batch][6][V] FP32 (device
 *                     or host, nullable).
 *   acm_fno_backward  forward with targets t [batch][6][V] FP32, loss (host,
 *                     nullable), gradient kept for acm_fno_adamw and copied to
 *                     grad [nparams] (nullable).
 *   acm_fno_warm_start  cubic grids only: the warm start of all three unit
 *                     loads, init_u and init_lambda [batch][3 loads][3][V]
 *                     FP32 on the device (the layout acm_batch_stokes takes).
 *                     The network predicts the load e_0; the load e_j uses the
 *                     cell with axes 0 and j swapped and swaps them back
 *                     (with the vector components), which is exact for the
 *                     Stokes problem itself.
 *   acm_fno_adamw     one AdamW step on the FP32 master parameters. */
typedef struct acm_fno acm_fno;
acm_status acm_fno_create(acm_fno** fno, int n0, int n1, int n2, int width, int modes, int layers, int max_batch,
                          void* cuda_stream);
acm_status acm_fno_destroy(acm_fno* fno);
acm_status acm_fno_num_params(acm_fno* fno, long long* n);
acm_status acm_fno_set_params(acm_fno* fno, const float* theta);
acm_status acm_fno_get_params(acm_fno* fno, float* theta);
acm_status acm_fno_forward(acm_fno* fno, int batch, const uint8_t* H, float* out);
acm_status acm_fno_warm_start(acm_fno* fno, int batch, const uint8_t* H, float* init_u, float* init_lambda);
acm_status acm_fno_backward(acm_fno* fno, int batch, const uint8_t* H, const float* target, double* loss,
                            float* grad);
acm_status acm_fno_adamw(acm_fno* fno, double lr, double beta1, double beta2, double eps, double weight_decay);

/* Convergence history of the last solve on this context for problem `index`
 * (0 for acm_stokes and acm_advdiff; the load index 0..2 for the tensor calls).
 * Copies up to `cap` records, record-major, into `out` (host) and returns the
 * number of recorded iterations in *count (nullable) and the record length in
 * *record_len (nullable); records are kept for the first 20000 iterations.
 * Stokes records hold 20 doubles: r_p1, r_d1, r_p2, r_d2, r_p3, r_d3 (Eq. 10),
 * their tolerances (Eq. 11-12), the penalties alpha, beta, b of the iteration,
 * the volume average of u^{n+1} (3 components, the k = 0 coefficient of the
 * Fourier solve; with a unit load e_j it is column j of K), and 2 unused.
 * Solute records hold 4 doubles: r1, r2 (Eq. 19) and their tolerances. */
acm_status acm_history(acm_ctx* ctx, int index, double* out, int cap, int* count, int* record_len);

/* Kernel kinds of the per-kernel profiler. */
typedef enum acm_kernel_kind {
  ACM_K_X_STOKES_LOCAL = 0,  /* C2R along axis 2 + ADMM steps 2-3 (Eq. 8-9) + residual partial sums */
  ACM_K_X_STOKES_RHS = 1,    /* known part of Eq. 7 + R2C along axis 2 */
  ACM_K_Y_FWD_STOKES = 2,    /* forward FFT along axis 1, 3 components */
  ACM_K_Z_STOKES = 3,        /* FFT along axis 0 + Eq. 13 solve + q update + inverse FFT */
  ACM_K_Y_INV_STOKES = 4,    /* inverse FFT along axis 1, 3 components */
  ACM_K_X_SOLUTE = 5,        /* C2R of grad chi + Eq. 18 local terms + R2C, axis 2 */
  ACM_K_Y_FWD_SOLUTE = 6,    /* forward FFT along axis 1, 4 components */
  ACM_K_Z_SOLUTE = 7,        /* FFT along axis 0 + Eq. 20 solve + inverse FFT */
  ACM_K_Y_INV_SOLUTE = 8,    /* inverse FFT along axis 1, 3 components */
  ACM_K_FINALIZE = 9,        /* FP64 residuals, tolerances, stop test, Eq. 22 */
  ACM_K_OTHER = 10,          /* set-up, outputs, reductions, standalone transforms */
  ACM_K_COUNT = 11
} acm_kernel_kind;

/* Per-kernel device timing. While enabled (on = 1), every kernel the context
 * launches is bracketed by CUDA events recorded on the context's stream.
 * acm_profile_read synchronises that stream and returns, per acm_kernel_kind,
 * the summed device time in milliseconds (ms, nullable; zero for kinds launched
 * while profiling was off) and the number of launches (launches, nullable;
 * counted whether or not profiling is enabled) since the previous read, then
 * resets both. Arrays have ACM_K_COUNT entries (host memory). */
acm_status acm_profile_enable(acm_ctx* ctx, int on);
acm_status acm_profile_read(acm_ctx* ctx, double* ms, long long* launches);

/* Size of the fixed device scratch array used by acm_fft_r2c_static. */
#define ACM_STATIC_SCRATCH_BYTES ((size_t)16 << 20)

/* acm_fft_r2c_static: the transform of acm_fft_r2c for one field, for callers
 * that cannot let a library allocate device memory (an application that gives
 * each component a fixed device-memory budget under its own allocator, or a
 * latency-critical loop that must not call cudaMalloc/cudaFree, which can
 * synchronise the device). It needs no context and allocates nothing: its
 * working spectrum lives in a fixed __device__ array of
 * ACM_STATIC_SCRATCH_BYTES that every GPU loading this library holds until the
 * process exits. The paper has no counterpart; it is a deployment variant.
 *   n0, n1, n2   grid, powers of two in [8, 512], with
 *                n0 * n1 * (n2/2 + 4) * (8 or 16 bytes) <= ACM_STATIC_SCRATCH_BYTES
 *                (128^3 in FP32, 128 x 128 x 64 in FP64); larger grids return
 *                ACM_ERR_UNSUPPORTED_SIZE before any device work.
 *   fp64         0: float input, 1: double input.
 *   in           device pointer, real [n0][n1][n2]; out: device pointer,
 *                complex interleaved [n0][n1][n2/2 + 1]; both in memory of the
 *                current device (or managed memory). Host pointers and memory
 *                of another device return ACM_ERR_ARG before any device work.
 *   cuda_stream  stream of the work (NULL = default stream); the call returns
 *                once the work is enqueued.
 * The first call on a device (with that device current) resolves the array's
 * device address with cudaGetSymbolAddress, uploads a twiddle table and
 * synchronises the device; make that first call before any stream capture. Every call
 * on a device shares the one array and overwrites every part of it that it
 * later reads, so nothing has to start at zero; calls whose work overlaps on the
 * GPU (other streams, other host threads) race on the array. */
acm_status acm_fft_r2c_static(int n0, int n1, int n2, int fp64, const void* in, void* out, void* cuda_stream);

/* Description of the last CUDA runtime failure seen by this thread in the
 * library (empty if none): error name, message and the failing call. The
 * string is thread-local and stays valid until the next failure. */
const char* acm_last_error(void);

/* Human-readable name of a status code (static string). */
const char* acm_status_str(acm_status s);

#ifdef __cplusplus
}
#endif

#endif /* ACM_H */
