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
} rsgdf_opts;

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
 * functions and 4 pi/Omega e^{-q^2/4 omega^2}/q^2, q = G + k12 != 0.
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
 * For callers that must not allocate device memory while they run: code that
 * records the call into a CUDA graph, where allocation calls are not allowed
 * during capture; applications that own all device memory through their own
 * pool and forbid libraries from calling cudaMalloc; steady-state loops that
 * must not risk an allocation failure half way through a step.
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
    double sr_ms_by_L[10];         /* device time of the SR kernel of each L class */
} rsgdf_stats;

int rsgdf_last_stats(rsgdf_stats *out);

/* Synchronise a stream and report device-detected failures of the calls
 * enqueued on it: RSGDF_ETIMEOUT when a bounded device wait (tensor-core
 * completion barrier) gave up, in which case those results are invalid;
 * RSGDF_OK otherwise.  Clears the flag. */
int rsgdf_sync_status(void *stream);

/* Range-separation parameter and G box implied by opts (host only). */
int rsgdf_params(const rsgdf_cell *cell, const rsgdf_opts *opts, double *omega_out, int *gmesh_out);

/* Message of the last error on this thread ("" if none). */
const char *rsgdf_last_error(void);

/* Measured FP64 FMA throughput of the current device in TFLOP/s (a short
 * in-bounds microbenchmark, used as the roofline denominator). */
int rsgdf_probe_fp64(double *tflops_out, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* RSGDF_H */
