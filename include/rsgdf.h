/*
 * rsgdf.h -- C ABI of the GB300 (sm_103a) RSGDF library.
 *
 * Range-separated Gaussian density fitting (Ye & Berkelbach, "Fast periodic
 * Gaussian density fitting by range separation"): the periodic three-center
 * Coulomb-metric integrals j3c and two-center integrals j2c, with the Coulomb
 * kernel split (Eq. Coulomb_RS) into erfc(omega r)/r, summed over lattice
 * translations in real space (Eq. VPmunu_SR), and erf(omega r)/r, summed over
 * reciprocal vectors (Eq. VPmunu_LR).
 *
 * Definitions computed (Eqs. TAAO, JPQ, VPmunu; q = G + k12 = 0 removed):
 *   V^{k1k2}_{P mu nu} = sum_{l,d} e^{-i k12.l} e^{+i k2.d} (chi_P^l | w | phi_mu^0 phi_nu^d)
 *   J^k_{PQ}           = sum_l e^{+i k.l} (chi_P^0 | w | chi_Q^l)
 * with k12 = k2 - k1, chi^l(r) = chi(r - l), every integral over all space.
 *
 * Conventions shared by every entry point
 *   - Units: Bohr.  Basis functions are Cartesian Gaussians x^lx y^ly z^lz
 *     exp(-a r^2) in lexicographic component order (xx, xy, xz, yy, yz, zz,
 *     ...), l <= RSGDF_LMAX.  Every primitive carries the radial norm of its
 *     x^l component and each contracted shell is rescaled so that its x^l
 *     component has unit norm; `coeffs` are the raw contraction coefficients.
 *   - k-points form a Gamma-including uniform mesh kmesh[0] x kmesh[1] x
 *     kmesh[2], k = sum_i n_i/N_i b_i; index k = (n0*N1 + n1)*N2 + n2 (the
 *     last direction fastest).  BvK cells use the same index order.
 *   - Inputs described by host pointers are read during the call only; the
 *     caller keeps ownership.  Outputs are caller-owned DEVICE buffers;
 *     complex numbers are interleaved (re, im) doubles.
 *   - Work is enqueued on opts->stream (a cudaStream_t; NULL = legacy default
 *     stream) and is asynchronous with respect to the host.  Scratch memory
 *     is allocated stream-ordered on that stream and released before return.
 *   - Return value: RSGDF_OK or a negative error code; rsgdf_last_error()
 *     gives a message (thread-local).  Argument errors are detected before
 *     any work is enqueued and leave outputs untouched.
 *   - There is no CPU fallback: without a usable sm_103a device every compute
 *     entry point returns RSGDF_EDEVICE.
 */
#ifndef RSGDF_H
#define RSGDF_H

#ifdef __cplusplus
extern "C" {
#endif

#define RSGDF_OK 0
#define RSGDF_EINVAL (-1)   /* invalid argument */
#define RSGDF_ENOMEM (-2)   /* device allocation failed */
#define RSGDF_ENOTPD (-3)   /* metric not positive definite (see info_out) */
#define RSGDF_ETIMEOUT (-4) /* a bounded device wait gave up */
#define RSGDF_EDEVICE (-5)  /* CUDA error or no usable device */
#define RSGDF_ENOTIMPL (-6) /* option not implemented */

#define RSGDF_LMAX 3        /* highest angular momentum per shell */

#define RSGDF_FP64 0        /* every step in FP64 */
#define RSGDF_MIXED 1       /* split-precision G-space/k-phase products, FP32 far-field terms */

#define RSGDF_SCREEN_BOUND 0   /* the paper's estimates (Supplementary Material) */
#define RSGDF_SCREEN_LEARNED 1 /* the estimates, then the trained MLP orders/prunes work */

/* Contracted Cartesian shells (all arrays host memory). */
typedef struct {
    int nshell;
    const int *l;          /* [nshell] angular momentum, 0..RSGDF_LMAX */
    const int *nprim;      /* [nshell] primitives per shell, >= 1 */
    const int *prim_off;   /* [nshell] first primitive of the shell in exps/coeffs */
    const double *center;  /* [nshell][3] centre of the shell (Bohr) */
    const double *exps;    /* [sum nprim] exponents, > 0 */
    const double *coeffs;  /* [sum nprim] raw contraction coefficients */
} rsgdf_basis;

/* Unit cell and k-mesh. */
typedef struct {
    double a[9];    /* lattice vectors a_1, a_2, a_3 as rows (Bohr) */
    int kmesh[3];   /* Gamma-including uniform mesh, each >= 1 */
} rsgdf_cell;

/* Parameters of the range separation and of the evaluation. */
typedef struct {
    double omega;       /* > 0: range-separation parameter; <= 0: derived from gmesh and eps_lr */
    int gmesh[3];       /* all > 0 (odd): G box; any <= 0: derived from omega and eps_lr */
    double eps_screen;  /* SR screening target per integral (Supplementary Material), > 0 */
    double eps_lr;      /* cutoff of the kernel factor e^{-q^2/4 omega^2} and of pair overlaps, > 0 */
    int precision;      /* RSGDF_FP64 or RSGDF_MIXED */
    int screening;      /* RSGDF_SCREEN_BOUND or RSGDF_SCREEN_LEARNED */
    const void *mlp;    /* learned screening: handle from rsgdf_mlp_create, or NULL */
    void *stream;       /* cudaStream_t or NULL */
    double split_alpha; /* > 0: SR sums and the G = 0 term only for range-separated
                           types (compact aux shell, AO pair not both diffuse; a shell
                           is diffuse when every exponent is <= split_alpha); 0: all */
    int kernel;         /* RSGDF_KERNEL_ERF, or RSGDF_KERNEL_PLAIN (rsgdf_j3c_lr only) */
} rsgdf_opts;

#define RSGDF_KERNEL_ERF 0     /* erf(omega r)/r in the G sum (Eq. VPmunu_LR) */
#define RSGDF_KERNEL_PLAIN 1   /* 1/r in the G sum, no range separation (Eq. VPmunu_FT) */

/*
 * j2c (Eq. JPQ with the split of Eq. Coulomb_RS, "readily adapted" to the
 * two-center case): for each requested k,
 *   J^k = sum_l e^{ik.l} (chi_P^0|erfc|chi_Q^l) - delta_{k,0} pi/(Omega omega^2) S_P S_Q
 *       + 4 pi/Omega sum_{q != 0} e^{-q^2/4 omega^2}/q^2 conj(chi^_P(q)) chi^_Q(q)
 * and, when L_out != NULL, its Cholesky factor J^k = L L^H (lower, FP64).
 *   nk, kidx : requested k indices (host, nk >= 1)
 *   J_out    : device complex [nk][naux][naux], overwritten
 *   L_out    : device complex [nk][naux][naux] or NULL; upper triangle zeroed
 *   info_out : device int [nk] or NULL; -1 when the factorisation succeeded,
 *              else the first non-positive pivot (L_out then holds a partial
 *              factor).  The call itself still returns RSGDF_OK: the pivot is
 *              known only on the device.
 */
int rsgdf_j2c(const rsgdf_cell *cell, const rsgdf_basis *aux, const rsgdf_opts *opts,
              int nk, const int *kidx, double *J_out, double *L_out, int *info_out);

/*
 * SR part of j3c (Eq. VPmunu_SR): the double lattice sum of erfc-attenuated
 * integrals, screened by the Supplementary Material's rules, folded onto BvK
 * cells (Eq. BvK_latsum_LR) and contracted with the phases, minus the G = 0
 * correction pi/(Omega omega^2) S_P S^k_{mu nu} on pairs with k1 = k2.
 *   npair, kpairs : host int [npair][2] = (k1, k2) mesh indices
 *   s0, s1        : aux SHELL range [s0, s1); nP = functions of those shells
 *   V_out         : device complex [npair][nP][nao][nao], OVERWRITTEN
 */
int rsgdf_j3c_sr(const rsgdf_cell *cell, const rsgdf_basis *ao, const rsgdf_basis *aux,
                 const rsgdf_opts *opts, int npair, const int *kpairs, int s0, int s1,
                 double *V_out);

/*
 * LR part of j3c (Eqs. VPmunu_LR and AFT_pairden): analytic Fourier transforms
 * of the AO pair densities on the G box, weighted by the transformed aux
 * functions and 4 pi/Omega e^{-q^2/4 omega^2}/q^2, q = G + k12 != 0.  With
 * opts->kernel = RSGDF_KERNEL_PLAIN the weight is 4 pi/Omega 1/q^2: the whole
 * Coulomb integral in reciprocal space on that box (Eq. VPmunu_FT), the route
 * of the diffuse integral types of the compact/diffuse split.
 * Same arguments as rsgdf_j3c_sr; the result is ADDED to V_out.
 */
int rsgdf_j3c_lr(const rsgdf_cell *cell, const rsgdf_basis *ao, const rsgdf_basis *aux,
                 const rsgdf_opts *opts, int npair, const int *kpairs, int s0, int s1,
                 double *V_out);

/* SR + G=0 + LR in one call with a single phase contraction; overwrites V_out. */
int rsgdf_j3c(const rsgdf_cell *cell, const rsgdf_basis *ao, const rsgdf_basis *aux,
              const rsgdf_opts *opts, int npair, const int *kpairs, int s0, int s1,
              double *V_out);

/*
 * Batched j3c (SR + G=0 + LR, all aux shells) over many cells at once.  A
 * handle holds every cell's plan, device tables and buffers, so a run only
 * issues kernels: the SR lattice sums of all cells go out as ONE persistent
 * launch per angular-momentum class (lP + lmu + lnu), whose warps draw work
 * items of every cell from one queue; the G-space and phase steps follow per
 * cell.  Flags:
 *   RSGDF_BATCH_GRAPH    : the first run captures the launch sequence into a
 *                          CUDA graph; later runs with the same V_out pointers
 *                          replay it (other pointers: captured anew).  With
 *                          stream NULL the graph runs on an internal stream
 *                          ordered after and before the legacy stream.
 *   RSGDF_BATCH_AUTOTUNE : before the first run, each class launch is timed
 *                          on the real items over its tile choices (bin chunk
 *                          = BvK cells held per warp, items per queue grab)
 *                          and the fastest is kept for the handle's life.
 * Arguments: probs[nprob] (cell, AO, aux; host, read during create only),
 * opts as for rsgdf_j3c (opts->mlp, if used, must outlive the handle),
 * npair[nprob], kpairs = the cells' (k1, k2) lists concatenated
 * ([sum npair][2]).  V_out[p]: device complex [npair[p]][naux_p][nao_p][nao_p],
 * overwritten.  Device memory is allocated stream-ordered on opts->stream at
 * create and released by destroy, which first waits for the device.  Errors
 * as for rsgdf_j3c; create reports the failing cell in rsgdf_last_error.
 */
typedef struct {
    const rsgdf_cell *cell;
    const rsgdf_basis *ao, *aux;
} rsgdf_problem;
#define RSGDF_BATCH_GRAPH 1
#define RSGDF_BATCH_AUTOTUNE 2
typedef struct rsgdf_batch rsgdf_batch;
int rsgdf_j3c_batch_create(int nprob, const rsgdf_problem *probs, const rsgdf_opts *opts, const int *npair,
                           const int *kpairs, int flags, rsgdf_batch **out);
int rsgdf_j3c_batch_run(rsgdf_batch *b, double *const *V_out, void *stream);
int rsgdf_j3c_batch_destroy(rsgdf_batch *b);
/* per class L = 0..9 of the SR launches: CTAs, bin chunk, items per grab
 * (0 where the class has no work); each pointer may be NULL */
int rsgdf_j3c_batch_tiles(const rsgdf_batch *b, int *grid, int *bc, int *grab);
/* one-shot form: create (no flags), run, destroy */
int rsgdf_j3c_batch(int nprob, const rsgdf_problem *probs, const rsgdf_opts *opts, const int *npair,
                    const int *kpairs, double *const *V_out);

/*
 * Bloch-phase contraction of folded lattice sums (Eq. BvK_latsum_LR):
 *   V[pair][i] = sum_{lt, dt} e^{-i k12.lt} e^{+i k2.dt} X[lt][dt][i]
 *   X      : device double [Nk][Nk][m] (BvK cells lt, dt in mesh order)
 *   m      : elements per (lt, dt) block, >= 1
 *   V_out  : device complex [npair][m], overwritten
 *   stream : cudaStream_t or NULL
 */
int rsgdf_kphase(const rsgdf_cell *cell, const double *X, long long m, int npair,
                 const int *kpairs, double *V_out, void *stream);

/*
 * rsgdf_kphase without any device allocation (no counterpart in the paper;
 * same arguments, result and ordering as rsgdf_kphase).
 *
 * For callers that must not allocate device memory while they run:
 * applications that own all device memory through their own pool and forbid
 * libraries from calling cudaMalloc; steady-state loops that must not risk an
 * allocation failure (or an allocator synchronisation) half way through a step.
 *
 * Scratch (the phase table, the k-pair lists and the intermediate T, about
 * 16 Nk m bytes) lives in one static device array of RSGDF_NOALLOC_SCRATCH_BYTES
 * that every GPU loading this library keeps until the process exits.  Calls
 * whose scratch would not fit return RSGDF_EINVAL before doing anything: split
 * m (columns of X) or the k-pair list.  Nothing in the scratch needs to start
 * at zero (every byte used is written first).  All calls share the array, so
 * calls whose work overlaps on the GPU (other streams, other host threads)
 * race; serialise them on one stream.  The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress); make that first call before
 * any stream capture.  Allocates nothing: no cudaMalloc, cudaFree or
 * allocating library routine.
 */
#define RSGDF_NOALLOC_SCRATCH_BYTES (64LL << 20)
int rsgdf_kphase_noalloc(const rsgdf_cell *cell, const double *X, long long m, int npair,
                         const int *kpairs, double *V_out, void *stream);

/*
 * Learned screening of SR work items (no counterpart in the paper, whose
 * screening is the Supplementary Material's estimates alone).  A work item
 * is one (aux shell, AO shell pair, lattice vector d) of the SR double
 * lattice sum that the estimates keep.  A 3 x 64 tanh network predicts
 * log10 of the largest contracted block the item adds; with
 * opts.screening = RSGDF_SCREEN_LEARNED and opts.mlp set, rsgdf_j3c /
 * rsgdf_j3c_sr skip items whose prediction (network output, plus the base
 * feature when one is set) plus the model's margin is below
 * log10(eps_screen) - 1.  The estimates remain the outer filter (the network
 * can only remove items they keep).  Parameters live on the device: FP32
 * master copy and Adam moments, FP16 working copy; activations FP16, dot
 * products FP32.  Features per item (RSGDF_MLP_NFEAT): lP, lmu, lnu, ln of
 * the three most diffuse exponents, R12, the distance of the pair centre to
 * the nearest aux image, log10 of the s-type SR integral of that nearest
 * term summed over the primitive combinations and scaled by the image sum
 * of the diffuse s-type kernel within the screening radius, ln Rc_cut.
 */
#define RSGDF_MLP_NFEAT 10
typedef struct rsgdf_mlp rsgdf_mlp;

/* params: host float[rsgdf_mlp_nparams(nfeat)] in the packing W1 [64 x F],
 * b1, W2 [64 x 64], b2, W3 [64 x 64], b3, w4 [64], b4 [1]; mean, stdv: host
 * float[nfeat] input normalisation.  The handle owns device memory on the
 * current device until rsgdf_mlp_destroy. */
int rsgdf_mlp_nparams(int nfeat);
int rsgdf_mlp_create(int nfeat, const float *params, const float *mean, const float *stdv, rsgdf_mlp **out);
int rsgdf_mlp_destroy(rsgdf_mlp *m);
int rsgdf_mlp_get_params(const rsgdf_mlp *m, float *params_out /* host */);
/* margin >= 0 (log10 units) added to the prediction before the cut */
int rsgdf_mlp_set_margin(rsgdf_mlp *m, float margin);
/* Screening prediction = network output + X[feature] clamped to [lo, hi]
 * when feature >= 0 (residual model on a physical estimate), or the network
 * output alone when feature = -1 (the default).  With a base feature an item
 * of class L = lP + lmu + lnu (features 0..2) is skipped only if, in
 * addition, X[feature] + guard[L] is below the cut: the estimate with its
 * own calibrated margin must agree, so the network cannot drop an item the
 * estimate calls large (guard[L] = +inf: never skip class L).  guard: host
 * float[10], NULL = all 0.  Used by j3c only; rsgdf_mlp_forward returns the
 * bare network output.  EINVAL if lo > hi or a guard entry is NaN. */
int rsgdf_mlp_set_base(rsgdf_mlp *m, int feature, float lo, float hi, const float *guard);
/* y[n] = network(X[n][nfeat]) (device pointers) */
int rsgdf_mlp_forward(const rsgdf_mlp *m, const float *X, long long n, float *y, void *stream);
/* Expectile loss over (X, t): L = (1/n) sum_s w_s (y_s - t_s)^2 with
 * w = 2 tau where y < t and 2 (1 - tau) elsewhere (tau = 1/2: mean squared
 * error; tau near 1 fits an upper envelope), and its gradient w.r.t. the
 * packed parameters, both returned to host memory (grad may be NULL);
 * EINVAL unless 0 < tau < 1; synchronises */
int rsgdf_mlp_loss_grad(rsgdf_mlp *m, const float *X, const float *t, long long n, float tau, float *loss_out,
                        float *grad_out, void *stream);
/* Adam training of that loss on device data: epochs over shuffled
 * mini-batches of size batch; loss_out (host) = mean loss of the last epoch;
 * synchronises */
int rsgdf_mlp_train(rsgdf_mlp *m, const float *X, const float *t, long long n, int epochs, int batch, float lr,
                    float tau, unsigned seed, float *loss_out, void *stream);

/* SR work items of a j3c problem (the planner's order): count, features
 * (device float[n][RSGDF_MLP_NFEAT], may be NULL) and, when mag_out is not
 * NULL, log10 of the largest block each item adds, measured by running the
 * FP64 SR kernels ("magnitude mode"; -30 for items that add nothing). */
int rsgdf_sr_items(const rsgdf_cell *cell, const rsgdf_basis *ao, const rsgdf_basis *aux, const rsgdf_opts *opts,
                   int s0, int s1, long long *n_items, float *feat_out, float *mag_out);

/* Statistics of the last j3c/j2c call on this thread (host values, valid
 * after the call returns): SR lattice terms (aux shell, AO shell pair, l, d)
 * kept by the screening, the Cartesian integrals they carry, and the omega
 * and G box actually used. */
typedef struct {
    long long sr_terms;
    long long sr_integrals;
    long long sr_flops;      /* algorithmic FP64 flops of the SR terms (see the design notes) */
    long long aft_units;     /* (pair primitive, d, G, k12) units of the pair transforms */
    long long lr_flops;      /* 8 nP nao^2 NG per (k12, BvK cell) block of the LR contraction */
    double omega;
    int gmesh[3];
    int n_launch;            /* kernels launched by the call */
    /* device time (ms, CUDA events on the call's stream) per phase */
    double sr_ms;            /* SR lattice-sum kernels */
    double aft_ms;           /* pair and aux Fourier transforms */
    double lr_gemm_ms;       /* LR contraction GEMMs */
    double phase_ms;         /* Bloch-phase contractions and the G = 0 correction */
    double other_ms;         /* Cholesky, overlaps, aux charges */
    long long sr_terms_by_L[10];   /* SR terms per total angular momentum L = lP + lmu + lnu */
    long long sr_prim_terms;       /* SR terms times their primitive combinations */
    long long sr_items;            /* SR work items kept by the estimates */
    long long sr_items_pruned;     /* of which skipped by the learned screen */
    double sr_ms_by_L[10];         /* device time of the SR kernel of each L class */
    long long sr_prim_terms_by_L[10];   /* SR terms times their primitive combinations, per L */
    long long sr_prim_terms_skipped;    /* primitive terms dropped by the per-combination bound (not evaluated) */
} rsgdf_stats;

int rsgdf_last_stats(rsgdf_stats *out);

/* Synchronise a stream and report device-detected failures of the calls
 * enqueued on it: RSGDF_ETIMEOUT when a bounded device wait (tensor-core
 * completion barrier) gave up, in which case those results are invalid;
 * RSGDF_OK otherwise.  Clears the flag. */
int rsgdf_sync_status(void *stream);

/* Device scratch budget (no counterpart in the paper): the largest number of
 * bytes of stream-ordered scratch one call may hold at a time; 0 (the
 * default) means no limit.  A call whose scratch would exceed it returns
 * RSGDF_ENOMEM, exactly as when the device allocator fails; work it had
 * already enqueued still runs, and its outputs are then unspecified.  The
 * batch handle's own buffers and the caller's outputs do not count.
 * Process-wide; returns RSGDF_EINVAL for a negative value. */
int rsgdf_set_scratch_limit(long long bytes);

/* Self-test of the bounded device wait and of its error report (no
 * counterpart in the paper): enqueues one CTA on `stream` that waits, with
 * the same bounded poll the tensor-core contraction uses (at most `limit`
 * polls, >= 1), on a barrier that expects one arrival.  arrive != 0: the CTA
 * arrives first and the wait completes, so rsgdf_sync_status then returns
 * RSGDF_OK; arrive == 0: nothing arrives, the wait gives up, the kernel
 * returns and the next rsgdf_sync_status returns RSGDF_ETIMEOUT.  The device
 * stays usable either way. */
int rsgdf_selftest_wait(int arrive, long long limit, void *stream);

/* Range-separation parameter and G box implied by opts (host only). */
int rsgdf_params(const rsgdf_cell *cell, const rsgdf_opts *opts, double *omega_out, int *gmesh_out);

/* Message of the last error on this thread ("" if none). */
const char *rsgdf_last_error(void);

/* Measured FP64 FMA throughput of the current device in TFLOP/s (a short
 * in-bounds microbenchmark, used as the roofline denominator). */
int rsgdf_probe_fp64(double *tflops_out, void *stream);

/*
 * Density-fitting consumers of j2c and j3c (Eq. DF_eqn and the fitted ERIs of
 * Eq. ERI_aux).  All FP64; all arrays DEVICE memory, complex interleaved;
 * work enqueued on `stream` (cudaStream_t or NULL).
 *
 * rsgdf_df_metric: a fitting transform T_k of each metric J^k with
 * T_k^H T_k = (J^k)^{-1} on the part of J^k it keeps, so B = T V solves the
 * fitting equation J d = V through d = T^H B.
 *   RSGDF_FIT_CHOLESKY: J = L L^H (lower triangle of J read), T = L^{-1}
 *     (lower).  Pivot j fails when L_jj^2 <= rel * max_i J_ii (rel = 0: the
 *     plain positivity test); T_k is then zero.
 *   RSGDF_FIT_EIGEN: canonical orthogonalisation of the Hermitian part
 *     U diag(lam) U^H (lam descending, cyclic Jacobi): row r of T_k is
 *     lam_r^{-1/2} (column r of U)^H for lam_r > rel * lam_0 and zero for the
 *     rows past the kept count.  Unique up to a phase per row (and a unitary
 *     mixing of rows of equal lam): T^H T is unique.
 *   RSGDF_FIT_AUTO: Cholesky, and the eigen route on the k whose pivots fail
 *     (a singular or nearly singular metric, e.g. a linearly dependent aux
 *     set); the choice is made on the device, per k.
 *   J        : [nk][naux][naux]
 *   naux     : 1 .. RSGDF_DF_NMAX
 *   rel      : 0 <= rel < 1
 *   T_out    : [nk][naux][naux], overwritten; must not overlap J
 *   lam_out  : double [nk][naux] or NULL: eigenvalues (descending) of the k
 *              that took the eigen route, zeros for the others
 *   nkept_out: int [nk] or NULL: rows of T_k that are not zero
 *   info_out : int [nk] or NULL: 0 = Cholesky route; s >= 1 = eigen route,
 *              converged after s sweeps; RSGDF_DF_SWEEPS + 1 = eigen route
 *              still rotating after RSGDF_DF_SWEEPS sweeps (T from the last
 *              sweep); -1 - j = Cholesky route failed at pivot j (method
 *              RSGDF_FIT_CHOLESKY only).
 * Scratch: 3 nk naux^2 complex (stream-ordered, released before return).
 */
#define RSGDF_FIT_CHOLESKY 0
#define RSGDF_FIT_EIGEN 1
#define RSGDF_FIT_AUTO 2
#define RSGDF_DF_NMAX 1024
#define RSGDF_DF_SWEEPS 40
int rsgdf_df_metric(const double *J, int naux, int nk, int method, double rel, double *T_out, double *lam_out,
                    int *nkept_out, int *info_out, void *stream);

/*
 * rsgdf_df_fit: B^{k1k2} = T_{k12} V^{k1k2}, k12 = k2 - k1 on the mesh.
 *   cell   : its kmesh gives the k indices (host)
 *   T      : [Nk][naux][naux] from rsgdf_df_metric (all Nk mesh points)
 *   V      : [npair][naux][nao][nao] (the layout rsgdf_j3c writes)
 *   kpairs : host int [npair][2]
 *   B_out  : [npair][naux][nao][nao], overwritten; must not overlap V
 */
int rsgdf_df_fit(const rsgdf_cell *cell, const double *T, int naux, int nao, int npair, const int *kpairs,
                 const double *V, double *B_out, void *stream);

/*
 * rsgdf_df_jk: fitted Coulomb and exchange matrices of a closed-shell
 * density D^k (D = 2 C C^H; Hermitian per k):
 *   rho_P  = sum_{(k,k) in kpairs} sum_{mu nu} B^{kk}_{P mu nu} D^k_{nu mu}
 *   J^k    = (1/Nk) sum_P B^{kk}_P conj(rho_P)        (zero for k without a pair (k,k))
 *   K^{k1} = (1/Nk) sum_{(k1,k2) in kpairs} sum_P B^{k1k2}_P D^{k2} (B^{k1k2}_P)^H
 * so that E_J = (1/2Nk) sum_k Tr[D^k J^k] and E_K = -(1/4Nk) sum_k Tr[D^k K^k]
 * per cell; with every pair present these are the Hartree and exchange
 * energies of the fitted ERIs.
 *   B      : [npair][naux][nao][nao] from rsgdf_df_fit
 *   kpairs : host int [npair][2], no pair listed twice
 *   D      : [Nk][nao][nao]
 *   rho_in : [naux] or NULL (then rho from the listed pairs).  A caller that
 *            splits the pairs over processes sums rsgdf_df_rho over all of
 *            them and passes the total: J^k then needs only the local (k, k)
 *            pairs, and J and K are sums of the processes' results.
 *   J_out, K_out : [Nk][nao][nao] or NULL (not both), overwritten
 * Scratch: naux complex, plus a bounded chunk of B-sized intermediates.
 *
 * rsgdf_df_rho: rho_P above over the listed pairs; rho_out [naux], overwritten.
 */
int rsgdf_df_rho(const rsgdf_cell *cell, const double *B, int naux, int nao, int npair, const int *kpairs,
                 const double *D, double *rho_out, void *stream);
int rsgdf_df_jk(const rsgdf_cell *cell, const double *B, int naux, int nao, int npair, const int *kpairs,
                const double *D, const double *rho_in, double *J_out, double *K_out, void *stream);

/*
 * Spherical (pure) functions.  The paper's bases are spherical; every integral
 * here is computed over Cartesian shells and converted afterwards.  A spherical
 * function is chi_{lm} = sum_c s_{mc} chi_c over its shell's Cartesian functions,
 * s the monomial coefficients of the real regular solid harmonics in Racah
 * normalisation without the Condon-Shortley phase (C_l^m for m >= 0, S_l^|m| for
 * m < 0), ordered m = -l .. l; for l = 1 that is (y, z, x).  With the Cartesian
 * shells normalised on their x^l component (see the conventions above) every
 * spherical function has unit norm.
 *
 * rsgdf_sph_coefficients (host): s_out [(2l+1)][(l+1)(l+2)/2], 0 <= l <= RSGDF_LMAX.
 * rsgdf_sph_nfunc (host): number of spherical functions of a basis.
 * rsgdf_cart2sph_j3c: V_sph[pair][P'][mu'][nu'] = sum s s s V_cart[pair][P][mu][nu]
 *   over aux shells [s0, s1) (the layout rsgdf_j3c writes for that range);
 *   device complex arrays, V_sph must not overlap V_cart.  V_cart must hold
 *   [npair][Cartesian functions of the range][nao][nao]: the call reads it
 *   by that layout.
 * rsgdf_cart2sph_j2c: J_sph[k] = s J_cart[k] s^T; device complex [nk][naux][naux]
 *   in, [nk][nsph][nsph] out, no overlap.
 */
int rsgdf_sph_coefficients(int l, double *s_out);
int rsgdf_sph_nfunc(const rsgdf_basis *b, int *nsph_out);
int rsgdf_cart2sph_j3c(const rsgdf_basis *ao, const rsgdf_basis *aux, int s0, int s1, int npair,
                       const double *V_cart, double *V_sph, void *stream);
int rsgdf_cart2sph_j2c(const rsgdf_basis *aux, int nk, const double *J_cart, double *J_sph, void *stream);

/*
 * Compact/diffuse split (Fig. 1 of the paper; host only, no device work).
 * rsgdf_split_basis: every shell becomes a compact sub-shell (its primitives
 * with exponent > alpha_cut, raw coefficients kept) and/or a diffuse one, in
 * shell order, compact first; each sub-shell is normalised like any shell, so
 * parent function = sum over its sub-shells of weight x sub-shell function.
 *   nshell_out, nprim_total_out : sizes of the split basis (required)
 *   l_out, nprim_out, prim_off_out, parent_out, kind_out : int [nshell] or NULL
 *     (kind 0 = compact, 1 = diffuse; parent = shell of the input basis)
 *   center_out : double [nshell][3] or NULL; weight_out : double [nshell] or NULL
 *   exps_out, coeffs_out : double [nprim_total] or NULL
 * Call once with NULL arrays for the sizes.
 * rsgdf_split_combine: V_out[pair][P][mu][nu] over the input bases from two
 *   tensors over the split bases ([npair][split aux][split AO][split AO],
 *   device complex): V_rs, computed by rsgdf_j3c with opts->split_alpha =
 *   alpha_cut, supplies the (C|cc) and (C|cd) blocks, V_g, the plain-kernel
 *   rsgdf_j3c_lr on the same box, the other four; the sub-functions are summed
 *   into their parents with the split's weights.  All aux shells.  V_out must
 *   not overlap the inputs.
 * rsgdf_sr_items_split: SR work the planner keeps (opts: omega / G box and
 *   eps_screen as for rsgdf_j3c; all aux shells), n_items_out[6]: work items
 *   (aux shell, AO shell pair, d) for [0] the input bases, [1] the split bases,
 *   [2] the split bases restricted to the range-separated types (compact aux
 *   function, pair not both diffuse); [3..5] the same as candidate primitive
 *   terms (items x aux images within the triple's Rc cutoff x primitive
 *   combinations; the kernel's per-term tests drop some of them).
 */
int rsgdf_split_basis(const rsgdf_basis *b, double alpha_cut, int *nshell_out, int *nprim_total_out, int *l_out,
                      int *nprim_out, int *prim_off_out, double *center_out, double *exps_out, double *coeffs_out,
                      int *parent_out, int *kind_out, double *weight_out);
int rsgdf_sr_items_split(const rsgdf_cell *cell, const rsgdf_basis *ao, const rsgdf_basis *aux,
                         const rsgdf_opts *opts, double alpha_cut, long long *n_items_out);
int rsgdf_split_combine(const rsgdf_basis *ao, const rsgdf_basis *aux, double alpha_cut, int npair,
                        const double *V_rs, const double *V_g, double *V_out, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* RSGDF_H */
