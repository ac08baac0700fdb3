/*
 * rte.h -- C ABI of the GB300 (sm_103a) implementation of the homogeneous-
 * medium fast method of Fan, An & Ying, "Fast algorithms for integral
 * formulations of steady-state radiative transfer equation" (arXiv 1802.03061).
 *
 * The library applies the Nystrom-discretised Fredholm operators of the
 * paper with FFTs on the zero-padded (circulant-embedded) grid and solves the
 * second-kind equation with a device GMRES.
 *
 *   2D, angular Fourier modes |k| <= L (Sec. 3.1.1, Eq. ani_2d_Fredholm;
 *   discretisation Sec. 3.3, Eq. ani_discretization / ani_AU):
 *       u = K u + b,     b = K~ g,  g = f delta_{k,0}
 *       (K u)_{i,k} = mu_s sum_j sum_{k'=-L..L} K~_{(i,k),(j,k')} sigma_hat_{|k'|} u_{j,k'}
 *       K~_{(i,k),(j,k')} = h^2 kappa(x_i - x_j) exp(i (k'-k) theta(x_i - x_j)),  i != j
 *       kappa(r) = exp(-mu_t |r|) / (2 pi |r|)                      (Sec. 2.3.1)
 *       K~_{(i,k),(i,k')} = integral over cell i of the same kernel  (Sec. 2.3)
 *   3D isotropic (Sec. 2.1, Eq. iso_Fredholm; Sec. 2.3.1 with d = 3):
 *       kappa(r) = exp(-mu_t |r|) / (4 pi |r|^2), h^3 cell volume.
 *
 * Grid: n cells per side on [0,1]^d (h = 1/n is usual but any h > 0 is
 * accepted), cell centres x_i = ((i1+1/2)h, (i2+1/2)h[, (i3+1/2)h]).
 *
 * Field layouts (all arrays are dense, C order, x index fastest):
 *   2D: "mode field"  double2 (or float2) [L+1][n][n]: modes k = 0..L,
 *       interleaved (re, im).  Modes k < 0 are implied by u_{-k} = conj(u_k),
 *       which holds for every field the solver produces (real f, real even
 *       sigma_hat).  The imaginary part of mode 0 must be zero.
 *   3D: double (or float) [n][n][n] real mean density.
 *   Source f: double [n][n] (2D) or [n][n][n] (3D).
 *
 * Ownership: the plan owns every device buffer it allocates (kernel spectra,
 * FFT intermediates, Krylov workspace), freed by rte_destroy.  The caller
 * owns x, y, f, u and the stream.  Pointers named *_dev are device pointers;
 * *_host are host pointers.  Calls are stream-ordered on `cuda_stream`
 * (a cudaStream_t; NULL = legacy default stream).  A plan is not thread-safe.
 *
 * Errors: every call returns an rte_status; nothing else crosses the ABI.
 * RTE_EINVAL for bad arguments (null pointers, n < 1, h <= 0, mu_t < 0,
 * mu_s < 0, mu_s > mu_t (assumption (C2), Sec. 2.2), L < 0 or L > 64,
 * |sigma_hat_0 - 1| > 1e-12 (the scattering kernel averages to one, Sec. 1),
 * |sigma_hat_k| > 1 (needed by the contraction argument, Sec. 3.2)),
 * RTE_EUNSUPPORTED for 3D with L > 0, RTE_ENOMEM when a device allocation
 * fails, RTE_ECUDA for any other CUDA error, RTE_ENOCONV when the solve
 * stops at maxit (u then holds the best iterate), RTE_ENAN when the source
 * or the residual is not finite.
 */
#ifndef RTE_H
#define RTE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int dim;   /* 2 or 3 */
    int n[3];  /* cells per side; only n[0] is used (square/cubic grids) */
} rte_grid;

typedef enum {
    RTE_OK = 0,
    RTE_EINVAL = 1,
    RTE_EUNSUPPORTED = 2,
    RTE_ENOMEM = 3,
    RTE_ECUDA = 4,
    RTE_ENOCONV = 5,
    RTE_ETIMEOUT = 6,
    RTE_ENAN = 7
} rte_status;

typedef enum {
    RTE_PREC_FP64 = 0,          /* FP64 FFTs, FP64 spectra, FP64 GMRES               */
    RTE_PREC_MIXED_FP32 = 1,    /* FP32 inner GMRES / FFTs / spectra + FP64 refinement */
    RTE_PREC_MIXED_BF16SPEC = 2 /* as above with the inner spectra stored in BF16      */
} rte_prec;

/* Krylov method of the FP32 inner solves of the mixed modes.  GMRES (the
 * default); MINRES (Paige-Saunders, three-term recurrence) where the operator
 * is symmetric, i.e. L = 0 (Sec. 2.3.1: the isotropic Nystrom matrix is
 * symmetric and the paper solves that case with MINRES) -- for L > 0, or a
 * restart length below 5, MINRES requests run GMRES.  The plain FP64 mode
 * always uses GMRES. */
typedef enum { RTE_INNER_GMRES = 0, RTE_INNER_MINRES = 1 } rte_inner_solver;

/* Solver options.  A zero-initialised struct selects the defaults given in
 * brackets.  tol is the relative residual ||b - (I-K)u|| / ||b|| in the
 * 2-norm over all modes -L..L, measured with the FP64 operator (the paper
 * leaves the stopping rule to GMRES/MINRES, Sec. 2.4). */
typedef struct {
    rte_prec prec;     /* [RTE_PREC_FP64] */
    double tol;        /* [1e-8] */
    int restart;       /* [40] GMRES restart length, 1..128 */
    int maxit;         /* [2000] total inner iterations */
    double inner_tol;  /* [1e-4] relative tolerance of each inner (FP32) solve */
    int use_guess;     /* [0] 1: u_dev holds an initial guess on entry */
    int q_policy;      /* [0] 0: smallest even 2^a 3^b >= 2n-1; else Q itself */
    int inner_solver;  /* [RTE_INNER_GMRES] Krylov method of the FP32 inner solves */
    int precond;       /* [0] 1: periodic preconditioner for the inner GMRES (mixed modes; 2D up to
                          Q = 1024, else it is not used): GMRES on (I-K) M with M built from
                          (I - C)^{-1}, C the convolution on the periodic padded grid, inverted per
                          frequency; same answer, fewer inner iterations.  Not in the paper.  Built
                          on the first solve that asks for it (allocates). */
    int precond_lmax;  /* [0] 2D: the preconditioner inverts the modes |k| <= lmax (block lower
                          triangular: the higher modes keep their coupling to those, not among
                          themselves); 0 = the smallest lmax with (mu_s/mu_t) max_{k>lmax}
                          |sigma_hat_k| <= 0.03, >= L = all modes.  Read when the preconditioner
                          is built. */
    int mode_mix;      /* [0] 2D: how the column pass forms the mode coupling sum_k' S_{k-k'} w_k'
                          per frequency (the kernel depends only on k - k', Sec. 3.3.1):
                          0 = the direct (2L+1)^2 sum for L <= 8 and a circular convolution along
                          the mode axis by FFTs of length P >= 4L+1 above; 1 = direct (L <= 8 only,
                          else RTE_EINVAL); 2 = the mode-axis FFT at every L.  Read at plan
                          creation; plans with the mode-axis FFT have no preconditioner. */
} rte_opts;

typedef struct {
    int iters;            /* GMRES iterations (inner ones for the mixed modes) */
    int outer;            /* FP64 refinement steps (mixed modes), 0 for FP64  */
    int converged;        /* 1 if relres_true <= tol                            */
    double relres_true;   /* FP64 ||b - (I-K)u|| / ||b|| at exit                */
    double ms_total;      /* wall time of the call (events on the stream)      */
    double ms_pre;        /* plan creation time of this plan                   */
    double est_err_bound; /* cond_est * relres_true, cond_est = (1+r)/(1-r), r = mu_s/mu_t */
} rte_stats;

typedef struct rte_plan_s* rte_plan;

/* Create a plan: computes the singular-cell weights (Sec. 2.3), samples the
 * kernels on the periodic zero-padded grid and stores their spectra
 * (Sec. 2.3.1 "calculate the Fourier modes of kappa"; Sec. 3.3.1 for the
 * mode-coupled kernels), all on the device.  sigma_hat: host array of L+1
 * coefficients sigma_hat_0..L (sigma_hat_0 == 1).  opts may be NULL.
 * The work is enqueued on cuda_stream and synchronised before return. */
rte_status rte_plan_create(rte_plan* out, rte_grid grid, double h, double mu_t, double mu_s, int L,
                           const double* sigma_hat, const rte_opts* opts, void* cuda_stream);

/* y = K x (T.2's operator, Sec. 3.3).  x_dev, y_dev: FP64 fields in the
 * layout above (2D double2 [L+1][n][n], 3D double [n]^3); may not alias. */
rte_status rte_apply_K(rte_plan plan, const void* x_dev, void* y_dev, void* cuda_stream);

/* y = x - K x, the matrix A = I - K of Eq. ani_AU. */
rte_status rte_apply_A(rte_plan plan, const void* x_dev, void* y_dev, void* cuda_stream);

/* y = K x to FP64 accuracy computed in float-float arithmetic (pairs of
 * FP32 numbers, ~48 significant bits) on the FP32 units; this is how the
 * mixed-precision solve forms its residuals, because FP64 units are scarce on
 * this GPU.  Same layouts as rte_apply_K. */
rte_status rte_apply_K64e(rte_plan plan, const void* x_dev, void* y_dev, void* cuda_stream);

/* FP32 versions used by the inner solves of the mixed modes: x_dev, y_dev are
 * float2 [L+1][n][n] (2D) or float [n]^3 (3D); the spectra are FP32 or BF16
 * as the plan's prec selects (FP32 for an FP64 plan). */
rte_status rte_apply_K32(rte_plan plan, const void* x_dev, void* y_dev, void* cuda_stream);
/* The periodic preconditioner of the inner solves (see rte_opts.precond) on an
 * FP32 field.  C is the convolution with the plan's kernel samples on the Q^d
 * periodic grid, diagonal in Fourier space.  3D: y = M x = crop((I - C)^{-1}
 * pad(x)), a scalar per frequency.  2D: with T(xi) the (2L+1) x (2L+1) mode
 * coupling of C and "low" the channels of the modes |k| <= lmax
 * (rte_opts.precond_lmax, rte_precond_info), y = x + crop(P pad(x_low)) with
 * P = T[:, low] (I - T_ll)^{-1} per frequency, stored in BF16: for lmax = L
 * this is crop((I - C)^{-1} pad(x)); for smaller lmax the higher modes keep
 * their coupling to the inverted ones.  Layout as rte_apply_K32.  Builds the
 * preconditioner data on the first call (allocates device memory).
 * RTE_EUNSUPPORTED for 2D plans whose column spectra do not fit the column
 * passes (Q above 1024 at L = 8).  Not in the paper. */
rte_status rte_apply_precond32(rte_plan plan, const void* x_dev, void* y_dev, void* cuda_stream);
/* The built preconditioner's inverted modes: *lmax_out = lmax (2D, |k| <=
 * lmax; see rte_opts.precond_lmax), 0 for 3D.  RTE_EINVAL before it is built
 * (the first preconditioned solve or rte_apply_precond32 builds it). */
rte_status rte_precond_info(rte_plan plan, int* lmax_out);

/* b = K~ g (step T.1 / S.1): f_dev double [n]^d real source, b_dev an FP64
 * field (all modes 0..L in 2D). */
rte_status rte_rhs(rte_plan plan, const double* f_dev, void* b_dev, void* cuda_stream);

/* Solve (I - K) u = K~ g (step T.2) for u.  f_dev: source; u_dev: FP64
 * field, read as the initial guess when opts->use_guess, else zeroed.
 * Mixed modes: b = K~ g is formed in FP32 (the first inner right-hand side
 * and ||b||), every residual in float-float as K~ (mu_s sigma_hat u + g) - u,
 * which is b - (I - K) u for the exact b; stats->relres_true is its norm over
 * ||b||.
 * opts NULL = the plan's options.  stats may be NULL.  Synchronises the
 * stream once at exit to fill stats.  Once the solve graph has run, u_dev
 * holds its last iterate whatever the status (RTE_ENOCONV, RTE_ENAN). */
rte_status rte_solve(rte_plan plan, const double* f_dev, void* u_dev, const rte_opts* opts,
                     rte_stats* stats, void* cuda_stream);

/* Same as rte_solve with host buffers: copies f_host to the device, solves,
 * copies u back to u_host (FP64 field layout above, host memory; pinned
 * memory keeps the copies asynchronous).  The copy back is queued behind the
 * solve graph and the statistics, and one synchronisation covers all three. */
rte_status rte_solve_host(rte_plan plan, const double* f_host, void* u_host, const rte_opts* opts,
                          rte_stats* stats, void* cuda_stream);

/* Sizes of this plan: n, Q, L, reals per field vector. Any pointer may be NULL. */
rte_status rte_plan_info(rte_plan plan, int* n, int* Q, int* L, long* nreal);

/* Cell weights the plan computed: D_m for m = 0..2L (2D) or D (3D) into
 * host array out (2L+1 doubles, or 1). */
rte_status rte_plan_cell_weights(rte_plan plan, double* out_host);

/* ---- Batched solves (task extension: many sources and coefficient sets on
 * grids of uneven size solved by one graph launch; no counterpart in the
 * paper, which solves one problem at a time) ---- */
typedef struct {
    int n;                    /* cells per side (2D) */
    double h, mu_t, mu_s;     /* as rte_plan_create */
    int L;
    const double* sigma_hat;  /* host, L+1 values, sigma_hat[0] == 1 */
    int q;                    /* padded FFT length, 0 = default (see rte_autotune) */
    int rows_per_block;       /* row-pass tile, 0 = default (see rte_autotune) */
} rte_instance_desc;
typedef struct rte_batch_s* rte_batch;

/* Create plans for `count` 2D instances and capture one CUDA graph holding
 * every instance's whole solve (T.1 + refinement + GMRES, device-controlled)
 * as independent branches.  opts: precision, tolerance, restart, maxit,
 * inner_tol shared by all instances (use_guess is ignored: zero start).
 * Owns all device memory; RTE_ENOMEM if it does not fit. */
rte_status rte_batch_create(rte_batch* out, int count, const rte_instance_desc* descs, const rte_opts* opts,
                            void* cuda_stream);
/* Solve every instance: f[i] (device, n_i^2 doubles) is instance i's source
 * and u[i] (device, 2(L_i+1) n_i^2 doubles, the FP64 mode-field layout)
 * receives its solution; f and u are host arrays of `count` device pointers,
 * caller-owned (one device buffer per instance).  The
 * sources are gathered into the batch's packed buffer by one kernel, the
 * graph runs, one kernel scatters the solutions.  stats_host (count entries,
 * may be NULL) receives each instance's statistics (ms_total = the graph
 * launch's device time).  Synchronises the stream once at exit.  Returns the
 * first non-OK instance status; RTE_EINVAL for a null pointer. */
rte_status rte_batch_solve(rte_batch b, const double* const* f, void* const* u, rte_stats* stats_host,
                           void* cuda_stream);
/* Offsets (in doubles) of instance i's source f (n^2 doubles) and solution u
 * (2(L+1)n^2 doubles, the FP64 mode-field layout) in the packed arrays that
 * rte_batch_solve_packed takes; arrays of count+1 entries (last = total). */
rte_status rte_batch_layout(rte_batch b, long* f_offsets_host, long* u_offsets_host);
/* The same solve on packed arrays: f_packed_dev / u_packed_dev are
 * caller-owned device arrays in the rte_batch_layout packing (one copy in,
 * one copy out instead of the gather / scatter kernels); ms_out (may be
 * NULL) receives the device time of the graph launch. */
rte_status rte_batch_solve_packed(rte_batch b, const double* f_packed_dev, double* u_packed_dev,
                                  rte_stats* stats_host, double* ms_out, void* cuda_stream);
rte_status rte_batch_destroy(rte_batch b);
/* The plan of instance i (owned by the batch; valid until rte_batch_destroy). */
rte_status rte_batch_plan(rte_batch b, int i, rte_plan* out);

/* Autotuner: for a 2D grid of n cells per side and truncation L, time the
 * FP32 operator application (prec = RTE_PREC_MIXED_FP32 or _BF16SPEC) for
 * the candidate padded lengths Q (the smallest even 2^a 3^b >= 2n-1, the
 * next two, and the smallest power of two in 64..1024 that is >= 2n-1, whose
 * column passes use the warp-register FFT) and row passes {0 = default: one warp per line with the FFT in
 * registers when Q = 32 * 2^j, 64 <= Q <= 512 (the column passes also at
 * Q = 1024), else the shared-memory FFT
 * with 8 rows per block; or the shared-memory FFT with 2, 4, 8, 16 rows per
 * block}, `reps` applications each, with CUDA
 * events on cuda_stream; returns the fastest (Q, rows per block) and its time
 * in ms per application.  Allocates temporary plans. */
rte_status rte_autotune(int n, int L, int prec, int reps, int* Q_out, int* rows_per_block_out, double* ms_out,
                        void* cuda_stream);

/* ---- Learned initial guess (task extension; no counterpart in the paper) ----
 * A 3x3 convolutional network on the 2D grid: NHWC BF16 activations with 16
 * input channels (the 2L+1 real channels of b = K~ g scaled by s_b, f / fmax,
 * log(mu_t)/4, mu_s/mu_t, sigma_hat_1, zero padding), hidden width 64, 16
 * output channels of which the first 2L+1 are the scaled correction:
 * u0 = b + s_b * net.  FP32 accumulation on the BF16 tensor cores; trained on
 * the GPU by the library's own forward, data-gradient and weight-gradient
 * kernels with Adam.  The solve uses u0 through opts->use_guess and falls
 * back to the zero start when ||b - (I-K) u0|| >= ||b||. */
typedef struct rte_cnn_s* rte_cnn;
/* cin, cout in {16, 32}; width = 64; depth >= 2. */
rte_status rte_cnn_create(rte_cnn* out, int cin, int width, int depth, int cout, unsigned long long seed,
                          void* cuda_stream);
rte_status rte_cnn_destroy(rte_cnn net);
/* y_dev (f32 [B][H][W][cout]) = net(X_dev), X_dev bf16 [B][H][W][cin]. */
rte_status rte_cnn_forward(rte_cnn net, const void* X_dev, int B, int H, int W, float* y_dev, void* cuda_stream);
/* One training step on a batch: loss = mean over pixels and the first `used`
 * output channels of (net(X) - T)^2 (T bf16 [B][H][W][cout]); weight and bias
 * gradients are left in the layers; an Adam step with rate lr when lr > 0.
 * loss_out (host, may be NULL) receives the loss (synchronises). */
rte_status rte_cnn_train_step(rte_cnn net, const void* X_dev, const void* T_dev, int B, int H, int W, int used,
                              float lr, float* loss_out, void* cuda_stream);
/* Device pointers of layer l: weights f32 [9][cin][cout] (tap = 3(dy+1)+(dx+1)),
 * bias f32 [cout], and their gradients from the last training step. */
rte_status rte_cnn_layer(rte_cnn net, int l, int* cin, int* cout, float** w_dev, float** bias_dev, float** gw_dev,
                         float** gb_dev);
/* Refresh the BF16 weight copies after the FP32 weights were written. */
rte_status rte_cnn_sync_weights(rte_cnn net, void* cuda_stream);
/* Write the FP32 weights and biases to a file (host path): "RTECNN01", int32
 * cin, width, depth, cout, then per layer int32 cin_l, cout_l, f32
 * w[9][cin_l][cout_l], f32 bias[cout_l], host byte order.  Synchronises the
 * device.  RTE_EINVAL if the file cannot be written. */
rte_status rte_cnn_save(rte_cnn net, const char* path);
/* Read a file written by rte_cnn_save into a network of the same shape
 * (cin, width, depth, cout, per-layer sizes) and refresh the BF16 copies on
 * cuda_stream.  RTE_EINVAL (network unchanged) if the file is missing,
 * truncated, or of another shape. */
rte_status rte_cnn_load(rte_cnn net, const char* path, void* cuda_stream);
/* Training checkpoint (resume): everything rte_cnn_save writes plus the
 * optimizer's state -- per layer the Adam first and second moments of the
 * weights and biases -- and its step count (the bias correction), so that
 * training steps after rte_cnn_load_state repeat those of the run that saved
 * it.  File: "RTECNS01", int32 cin, width, depth, cout, int64 step, per layer
 * int32 cin_l, cout_l, f32 w, bias, m_w, v_w, m_b, v_b (host byte order).
 * save synchronises the device; load refreshes the BF16 copies on
 * cuda_stream.  RTE_EINVAL (network unchanged) for an unwritable, missing,
 * truncated or other-shaped file. */
rte_status rte_cnn_save_state(rte_cnn net, const char* path);
rte_status rte_cnn_load_state(rte_cnn net, const char* path, void* cuda_stream);
/* Network input (cin channels, 2L+5 <= cin) / training target (cout
 * channels, 2L+1 <= cout) of plan p (2D) from the source f (double [n][n]),
 * b = K~ g and, for targets, the solution u (FP64 mode fields).  The scales
 * s_b = RMS of b's real channels and fmax = max |f| are computed on the
 * device.  X_dev / T_dev: bf16 [n][n][cin|cout]. */
rte_status rte_guess_features(rte_plan p, int cin, const double* f_dev, const double* b_dev, void* X_dev,
                              void* cuda_stream);
rte_status rte_guess_targets(rte_plan p, int cout, const double* f_dev, const double* u_dev, const double* b_dev,
                             void* T_dev, void* cuda_stream);
/* The learned initial guess with caller-provided buffers: b_out_dev = K~ g
 * (step T.1, FP64 mode field), then u0_dev = b + s_b * net(features).
 * X_scratch_dev: bf16 [n][n][cin].  Pass u0 to rte_solve with
 * opts->use_guess = 1. */
rte_status rte_cnn_guess_apply(rte_cnn net, rte_plan p, const double* f_dev, double* b_out_dev, void* X_scratch_dev,
                               void* u0_dev, void* cuda_stream);

/* The learned guess as the boundary's handle (task extension (4): the
 * network predicts the GMRES initial guess from the source and mu_t, mu_s,
 * g; the paper has no counterpart).  rte_guess_load creates the network of
 * the shape recorded in a weights file written by rte_cnn_save and loads it
 * (synchronous, legacy default stream); RTE_EINVAL if the file is missing,
 * truncated or not a weights file, RTE_ENOMEM when the device is full.  The
 * handle owns the network and its scratch (the features and b = K~ g of the
 * largest grid it has been applied to). */
typedef struct rte_guess_s* rte_guess;
rte_status rte_guess_load(rte_guess* out, const char* weights_path);
/* u0_dev (FP64 mode field of plan p, device) = the learned initial guess for
 * the source f_dev (double [n][n], device); pass it to rte_solve with
 * opts->use_guess = 1 (the solve falls back to the zero start when the guess
 * does not lower the residual).  The first call for a grid larger than any
 * before allocates the handle's scratch (and synchronises the device); later
 * calls are asynchronous on cuda_stream.  RTE_EINVAL for a 3D plan or when
 * the plan's 2L+1 channels exceed the network's inputs or outputs. */
rte_status rte_guess_apply(rte_guess g, rte_plan p, const double* f_dev, void* u0_dev, void* cuda_stream);
rte_status rte_guess_destroy(rte_guess g);

/* ---- Inhomogeneous medium, isotropic scattering, 2D (Sec. 2.3,
 * Eq. iso_discretization): the Nystrom matrix K~ applied directly, O(N^2).
 * K~_ij = h^2 E(x_i, x_j) / (2 pi |x_i - x_j|) for i != j, with
 * E(x, y) = exp(-|x - y| int_0^1 mu_t(x - s(x - y)) ds) by 5-point
 * Gauss-Legendre along the segment; K~_ii = (2h/pi) ln(1 + sqrt 2) plus the
 * smooth part (E - 1)/(2 pi r) integrated over the cell by the 15 x 15
 * Gauss-Legendre rule (the split the paper describes after Eq. iso_AU).
 * mu_t between its cell-centred samples: bilinear, index clamped to the grid.
 * The solve of Eq. iso_AU needs A = diag(1/mu_s) - K~ on top of this apply. ---- */
typedef struct rte_inhom_s* rte_inhom;
/* mu_t_host: n*n cell values [i2][i1] (x fastest), >= 0 and finite, host
 * memory, copied.  Computes the diagonal on the device (FP64).  RTE_EINVAL on
 * bad arguments; RTE_ENOMEM when the device buffers cannot be allocated. */
rte_status rte_inhom_create(rte_inhom* out, int n, double h, const double* mu_t_host, void* cuda_stream);
/* y = K~ x, FP32 (x_dev, y_dev: float [n*n], device, must not alias;
 * compensated summation) or FP64.  A block owns 32 output cells and splits
 * the sources over 8 warps; mu_t staged in shared memory for n <= 110 (FP32)
 * / 78 (FP64). */
rte_status rte_inhom_apply32(rte_inhom op, const float* x_dev, float* y_dev, void* cuda_stream);
rte_status rte_inhom_apply64(rte_inhom op, const double* x_dev, double* y_dev, void* cuda_stream);
/* the diagonal K~_ii into diag_host (n*n doubles, host) */
rte_status rte_inhom_diag(rte_inhom op, double* diag_host);
rte_status rte_inhom_destroy(rte_inhom op);

/* ---------------------------------------------------------------------------
 * 3D anisotropic scattering in real spherical harmonics (Sec. 3.1.2).
 *
 * The angular density is expanded in the real orthonormal harmonics Y_a,
 * a = l^2 + l + m, |m| <= l <= L (no Condon-Shortley phase: Y_{l,0} = N P_l(z),
 * Y_{l,+-m} = sqrt2 N_lm P_l^m(z)/(1-z^2)^{m/2} {Re, Im}(x + i y)^m, so
 * Y_{1,-1}, Y_{1,0}, Y_{1,1} = sqrt(3/4pi) (y, z, x)), M = (L+1)^2 channels.
 * The moments u_a = (4 pi)^{-1/2} int Phi Y_a dv (u_0 = the mean density)
 * solve u = K u + b with
 *   (K u)_a = sum_b K~^{ab} mu_s sigma_hat_{l_b} u_b,   b_a = K~^{a0} f,
 *   K~^{ab}_{ij} = h^3 exp(-mu_t r)/(4 pi r^2) 4 pi Y_a(v) Y_b(v), v = (x_i - x_j)/r,
 *   K~^{ab}_{ii} = the same kernel integrated over the cell (D_ab);
 * sigma_hat_l: the phase function's Legendre moments (sigma_hat_0 = 1,
 * |sigma_hat_l| <= 1; Henyey-Greenstein: g^l) -- the paper's coefficient of
 * Y_l^0 times sqrt(4 pi/(2l+1)).  L = 0 is the isotropic equation.
 * Fields: double (float for apply_K32) [M][n][n][n], x fastest, device memory;
 * the source f: double [n][n][n].  Applied with FFTs on the zero-padded Q^3
 * grid: for 17 <= n <= 128 Q is the power of two 64, 128 or 256 >= 2n - 1 and
 * each pass transforms all M channels in one launch with warp-register FFTs;
 * otherwise Q is the smallest even 2^a 3^b >= 2n - 1 and the passes run channel
 * by channel.  FP64 spectra for the FP64 calls, FP32 for apply_K32, a
 * float-float copy of the FP64 spectra for apply_K64e.  Limits: L <= 4,
 * n <= 1024, and the M channels of one Z line must fit in shared memory
 * (RTE_EUNSUPPORTED otherwise; n = 128 takes L <= 4).  Inputs and outputs may
 * not alias.
 * ------------------------------------------------------------------------- */
typedef struct rte_aniso3d_s* rte_aniso3d;
/* Computes D_ab and the M(M+1)/2 spectra on the device (synchronises). */
rte_status rte_aniso3d_create(rte_aniso3d* out, int n, double h, double mu_t, double mu_s, int L,
                              const double* sigma_hat, void* cuda_stream);
rte_status rte_aniso3d_info(rte_aniso3d op, int* M_out, int* Q_out);
/* Host only (no device call): the M x M channel-pair table the spectra are
 * stored by, row-major into out_host: pair index (unordered pairs a <= b
 * numbered row by row) | 1 << 16 if the pair's spectrum is imaginary (W_ab odd
 * under v -> -v) | 1 << 17 if W_ab is odd in y | 1 << 18 if odd in z. */
rte_status rte_aniso3d_pair_table(int L, int* out_host);
/* D_ab, row-major M x M, into host memory. */
rte_status rte_aniso3d_cell_weights(rte_aniso3d op, double* out_host);
/* y = K x: native FP64 / FP64-accurate in float-float arithmetic on the FP32
 * units (native FP64 when Q is not a power of two) / in FP32. */
rte_status rte_aniso3d_apply_K(rte_aniso3d op, const double* x_dev, double* y_dev, void* cuda_stream);
rte_status rte_aniso3d_apply_K64e(rte_aniso3d op, const double* x_dev, double* y_dev, void* cuda_stream);
rte_status rte_aniso3d_apply_K32(rte_aniso3d op, const float* x_dev, float* y_dev, void* cuda_stream);
/* b = K~^{.0} f (Sec. 3.3, T.1). */
rte_status rte_aniso3d_rhs(rte_aniso3d op, const double* f_dev, double* b_dev, void* cuda_stream);
/* (I - K) u = b (Sec. 3.3, T.2) until ||b - (I - K) u|| <= tol ||b|| (FP64
 * residual), zero start: the same device solver as rte_solve (one CUDA graph
 * with device-side loop control; the host only launches it and reads the
 * statistics).  prec = RTE_PREC_FP64: restarted FP64 GMRES(restart)
 * (classical Gram-Schmidt twice), native FP64; RTE_PREC_MIXED_FP32: refinement
 * steps, each an FP32 GMRES(restart) solve of (I - K) d = r/||r|| to
 * max(1e-4, tol/(2 relres)) followed by u += ||r|| d and an FP64-accurate
 * residual r = K~ (mu_s sigma_hat u + f) - u (float-float, native FP64 when Q
 * is not a power of two).  restart 1..128.  RTE_ENOCONV after maxit (inner)
 * iterations, u holding the last iterate; RTE_ENAN for a non-finite residual;
 * RTE_EINVAL for another prec.  The first solve of a precision and restart
 * allocates its workspace and builds its graph (RTE_ENOMEM on a failed
 * allocation; a later call retries).  stats: iters (inner), outer (mixed:
 * refinement steps; FP64: 0), converged, relres_true, ms_total (the graph),
 * ms_pre = creation time.  Synchronises. */
rte_status rte_aniso3d_solve(rte_aniso3d op, const double* f_dev, double* u_dev, double tol, int restart,
                             int maxit, int prec, rte_stats* stats, void* cuda_stream);
rte_status rte_aniso3d_destroy(rte_aniso3d op);

/* Diagnostics (no counterpart in the paper).
 * rte_time_passes: average duration in ms of each FFT pass of one K
 * application -- ms_out[0] row pass, [1] column pass (FFT, mode mix, inverse
 * FFT), [2] inverse row pass -- over `reps` back-to-back launches, timed with
 * CUDA events on cuda_stream.  inner = 0 times the FP64 passes, inner = 1 the
 * FP32 passes with the plan's inner spectra, inner = 2 the float-float passes
 * of rte_apply_K64e, inner = 3 the passes of rte_apply_precond32 (building
 * the preconditioner first if needed: allocates).  Operates on plan-owned
 * scratch vectors.  2D plans only (RTE_EUNSUPPORTED for 3D).
 * rte_kernel_launches: number of kernels this library has launched so far in
 * the process (host-side counter; a replayed graph adds its kernel nodes). */
rte_status rte_time_passes(rte_plan plan, int inner, int reps, double* ms_out_host, void* cuda_stream);
long long rte_kernel_launches(void);
/* Fault injection for tests of the error paths (no counterpart in the
 * paper): every device and pinned-host allocation the library makes is
 * counted; after this call the k-th one (k >= 1, counting from this call)
 * fails as if the device were full (RTE_ENOMEM from the call that made it),
 * and k <= 0 turns that off.  Outputs (any may be NULL), read before the
 * reset: the allocations made since the previous call, and the library's
 * live device and pinned-host allocations (a create call that failed must
 * leave these where they were). */
rte_status rte_debug_fail_alloc(long k, long* seen_out, long* live_dev_out, long* live_host_out);

/* y = K x for a small 2D grid with no device allocation at all.  For
 * callers that may not allocate device memory where they call: plug-ins
 * whose host application owns and caps all device memory, real-time loops
 * that forbid allocator calls after start-up, code that runs while another
 * component holds the whole device allocator.  Such callers cannot create a
 * plan (rte_plan_create allocates), so this call rebuilds the plan data
 * (cell weights, kernel samples, spectra) and the pass intermediates on
 * every call inside one fixed static device array of
 * rte_noalloc_scratch_bytes() bytes (about 5 MB), which every GPU that has
 * loaded it holds until process exit; then it applies the same FP64 passes
 * as rte_apply_K.  Arguments as rte_plan_create + rte_apply_K: x_dev, y_dev
 * are caller-owned FP64 mode fields double2 [L+1][n][n] that may not alias;
 * sigma_hat is a host array of L+1 values.  Limits: n <= 64 and L <= 4;
 * larger sizes return RTE_EUNSUPPORTED (use a plan).
 * Set-up: the first call on each device, with that device current, looks up
 * the array's device address.  Under CUDA's default lazy module loading that
 * lookup is also when the CUDA runtime loads the array onto the device, i.e.
 * when its 5 MB of device memory are taken (RTE_ENOMEM if the device is
 * full, RTE_ECUDA for another failure).  So make the first call on each device
 * at start-up, where taking that memory is allowed, and before any stream
 * capture; every later call takes no device memory.  (With
 * CUDA_MODULE_LOADING=EAGER the array is loaded with the library instead.)
 * All calls share the array and it keeps the last call's contents; calls
 * whose work overlaps on the GPU race on it, so the caller must serialise
 * them.  Asynchronous on cuda_stream.  (The paper has no counterpart of this
 * entry point.) */
rte_status rte_apply_K_noalloc(int n, double h, double mu_t, double mu_s, int L, const double* sigma_hat,
                               const void* x_dev, void* y_dev, void* cuda_stream);
long long rte_noalloc_scratch_bytes(void);

/* Free all device memory of the plan.  NULL is accepted. */
rte_status rte_destroy(rte_plan plan);

const char* rte_status_str(rte_status s);

/* Last CUDA error text seen by the library (for diagnostics). */
const char* rte_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* RTE_H */
