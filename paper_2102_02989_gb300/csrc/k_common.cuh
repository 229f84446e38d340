// Device-side declarations shared by the library's CUDA translation units.
#pragma once
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "rsgdf_internal.h"

namespace rsgdf {

constexpr double KPI = 3.141592653589793238462643383279502884;
constexpr double KPI2_5 = 17.493418327624862846262821679872;  // pi^{5/2}

// Cartesian exponents (lx, ly, lz) of each component, lexicographic order
static __constant__ const signed char c_cart[LMAX + 1][NC_MAX][3] = {
    {{0, 0, 0}},
    {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}},
    {{2, 0, 0}, {1, 1, 0}, {1, 0, 1}, {0, 2, 0}, {0, 1, 1}, {0, 0, 2}},
    {{3, 0, 0}, {2, 1, 0}, {2, 0, 1}, {1, 2, 0}, {1, 1, 1}, {1, 0, 2}, {0, 3, 0}, {0, 2, 1}, {0, 1, 2}, {0, 0, 3}},
};

struct DevShells {
    const int *l, *nprim, *poff, *foff;
    const double *cen, *exps, *cn;
};

struct SRTripleDev {
    int P, mu, nu, pair;
    int nwin, win_off, nd, nsph;
    int cc_off;       // first entry of the triple's primitive combinations in SRArgs::ccon / cbnd
    double Rc_cut, amu, anu;
    long long item_off;
    double log10A, beta, eta1, eta2, aP;
};

// Geometry of one SR work item (aux shell P, AO shell pair, lattice vector d),
// one record per item, computed before the SR launches by one thread per item:
// L0 is the lattice vector nearest to (pair centre - C_P) and h the rest, R12
// the pair separation; the candidates of the item are the first nsph entries
// of the length-sorted lattice list, pre-filtered at the FP32 radius fcut.
struct SRItemGeom {
    double h[3], L0[3], R12;
    float fcut;
    int nsph;
    int l0[3];       // L0 in lattice coordinates
    int gd, dt;      // global d index, BvK cell of d
    int tri;         // the item's shell triple (index into SRArgs::tri)
    int pad[2];
};
static_assert(sizeof(SRItemGeom) == 96, "SRItemGeom is six 16-byte words");

struct SRArgs {
    DevShells ao, ax;
    const SRTripleDev *tri;
    int tri_begin, tri_end;
    long long item_begin, item_end;
    const double *win;
    const int *pair_doff, *dlist, *sph;
    const double *sphv;               // Cartesian vectors of the lattice list (FP64), [nsph][3]
    const float *sphvf;               // the same in FP32 (pre-filter)
    const float *sphlen;              // their lengths (ascending), FP32
    int ntri;                         // shell triples of the problem (items of triple t: [tri[t].item_off, + nd))
    const SRItemGeom *geom;           // [n_items] geometry of each work item
    const double *ccon;               // per (triple, combination) [4]: alpha, s, sqrt s, prefactor (d-independent)
    const float *cbnd;                // per (triple, combination): d-independent part of the log Coulomb bound
    double a[9];    // lattice vectors (rows)
    float af[9];    // the same in FP32 (pre-filter of the translations)
    double bq[9];   // b_i / 2 pi: fractional coordinates
    int nk[3];
    int Nk;
    double omega;
    double *X;
    long long s_lt, s_dt, s_P, s_mu, s_nu;
    int pfunc0;
    int bc;
    int warp_bytes;
    int ncomp_max, w_max, list_max;
    int combo_max;                    // primitive combinations of the largest triple of the launch (<= 64)
    int nbin_max;                     // BvK cells of the largest k mesh of the launch (<= NBIN_MAX): bin counters per warp
    float log_prim_cut;               // drop a primitive combination of an item whose bound is below e^this (-1e30: never)
    unsigned long long *term_count;   // [LTOT_MAX+2] or NULL
    const double *ec_tab;             // [aux primitive][(LMAX+1)^2] single-centre Hermite coefficients
    const double *ptab;               // pair entries of the SR d list
    const long long *sr_doff;         // [global d index] offset of its first entry
    float *item_mag;                  // [n_items] log10 of the item's largest block, or NULL
    const unsigned char *item_skip;   // [n_items] 1: pruned by the learned screen, or NULL
};

// BvK cell (mesh order, last index fastest) of an integer lattice vector
__host__ __device__ __forceinline__ int bvk_bin(int i, int j, int k, const int *nk)
{
    int a = i % nk[0]; if (a < 0) a += nk[0];
    int b = j % nk[1]; if (b < 0) b += nk[1];
    int c = k % nk[2]; if (c < 0) c += nk[2];
    return (a * nk[1] + b) * nk[2] + c;
}

// e^{sign i k.R} for k-mesh index k and BvK cell index R (both mesh order):
// angle = 2 pi sum_i (n_i j_i mod N_i)/N_i, reduced in integers.
__device__ __forceinline__ void bloch_phase(int k, int cell, const int *nk, int sign, double &c, double &s)
{
    int n2 = k % nk[2], n1 = (k / nk[2]) % nk[1], n0 = k / (nk[1] * nk[2]);
    int j2 = cell % nk[2], j1 = (cell / nk[2]) % nk[1], j0 = cell / (nk[1] * nk[2]);
    double f = (double)((n0 * j0) % nk[0]) / nk[0] + (double)((n1 * j1) % nk[1]) / nk[1] +
               (double)((n2 * j2) % nk[2]) / nk[2];
    sincospi(2.0 * f, &s, &c);
    s *= sign;
}

int upload_boys_table(const double *tab, cudaStream_t st);
int sr_default_bc(int L, int ncomp_max, int w_max, int nk_max);
// rows (BvK cell x primitive combination) of Hermite sums a warp holds for a bin chunk bc:
// room for up to 4 combinations at once when the chunk is small
// rows of Hermite sums per warp in the SR kernel: one per lane and the zero row of empty cells
__host__ __device__ constexpr int sr_rb_rows(int) { return 33; }
int launch_sr_item_geom(const SRArgs &A, long long n_items, SRItemGeom *out, cudaStream_t st);
size_t sr_warp_bytes(int L, int bc, int ncomp_max, int w_max, int list_max, int combo_max, int nbin);
size_t sr_launch_smem(int L, int bc, int ncomp_max, int w_max, int list_max, int combo_max, int nbin);
int sr_occupancy(int L, size_t smem);
int launch_sr_queue(int L, const SRArgs *ddesc, const long long *dcum, int ndesc, long long ntot,
                    size_t warp_bytes, unsigned long long *queue, int grid, int grab, cudaStream_t st);
__global__ void k_aux_charge(DevShells ax, int s0, int s1, int pfunc0, double *S);
__host__ __device__ void single_E(int lc, double g, double *E);
__global__ void k_g0_correct(double *V, const int *kpairs, int npair, int nP, int nao, const double *SP,
                             const double *Sf, const int *nk3, int Nk, double fac);

// Learned screening (k_mlp.cu)
constexpr int SR_NFEAT = 10;        // features per SR work item
constexpr int SR_NFEAT_MAX = 16;
int launch_sr_features(const SRArgs &A, float *feat, cudaStream_t st);
int launch_mlp_forward(int F, const __half *P16, const float *mean, const float *stdv, const float *X, long long n,
                       float *y, cudaStream_t st);
int launch_mlp_fwd_bwd(int F, const __half *P16, const float *mean, const float *stdv, const float *X, const float *t,
                       const int *idx, long long n, float inv_ntot, float tau, float *G, float *loss, cudaStream_t st);
int launch_mlp_adam(int np, float *P, __half *P16, float *G, float *m, float *v, float lr, int step, cudaStream_t st);
int launch_to_half(int n, const float *a, __half *b, cudaStream_t st);
int launch_mlp_mask(long long n, int F, const float *X, int base, float base_lo, float base_hi, const float *guard,
                    const float *pred, float margin, float log10_cut, unsigned char *skip, unsigned long long *count,
                    cudaStream_t st);
int mlp_param_count(int F);

// G-space and phase kernels (k_gspace.cu)
struct GArgs {
    const int *g;          // [NG][3] integer G coordinates
    int NG;
    double b[9];           // reciprocal vectors (rows)
    double f12[3];         // fractional coordinates of k12, in [-1/2, 1/2)
    double vol, omega;
    int full_coulomb;      // 1: no erf damping (route used only for checks)
};

int launch_aux_ft(const GArgs &G, DevShells ax, int s0, int s1, int pfunc0, int nP, double *W, double *F,
                  cudaStream_t st);
struct PairEntry {
    long long off;   // offset of the entry in the table (doubles)
    int pair, d, i, j;
};
int launch_pair_prep(DevShells ao, int nshell, const PairEntry *ent, int nent, const int *dlist, const double *a9,
                     double *tab, float *tab32, const double *b9, float2 *uph, cudaStream_t st);
int launch_aft_f32(const GArgs &G, DevShells ao, int nshell, int nao, const PairEntry *ent, int nent, const int *seg,
                   const double *tab, const float *tab32, const double *b9, const float2 *uph, float2 *ph0, int Nk,
                   float *Bp, int lmax_ao, cudaStream_t st);
int launch_aft(const GArgs &G, DevShells ao, int nshell, int nao, const PairEntry *ent, const int *seg,
               const double *tab, int Nk, double *Y, cudaStream_t st);
int launch_ovlp_fold(DevShells ao, int nshell, int nao, const PairEntry *ent, const int *seg, const double *tab,
                     int Nk, double *Sf, cudaStream_t st);
int launch_zgemm_tn(int M, int N, int K, int batch, const double *A, const double *B, long long strideB,
                    double *C, long long strideC, cudaStream_t st,
                    long long strideA = 0);
int launch_phase1(const double *X, long long m, int Nk, int ndt, int k12, const double *ph, double *T, int accumulate,
                  cudaStream_t st);
int launch_g0_outer(double *J, int n, const double *S, double fac, cudaStream_t st);
int launch_g0_fold(double *T, long long m, int Nk, int nP, int nao, const double *SP, const double *Sf, double fac,
                   cudaStream_t st);
int launch_phase2(const double *T, long long m, int Nk, const int *pair_list, const int *pair_k2, int npl,
                  const double *ph, double *V, int accumulate, cudaStream_t st);
int launch_cholesky(int n, int nk, const double *J, double *Lo, int *info, cudaStream_t st);
int launch_probe_fp64(double *out, int iters, cudaStream_t st);
int launch_zgemm_tn_tc(int M, int N, int K, int batch, const double *A, const double *B, long long strideB, double *C,
                       long long strideC, cudaStream_t st);

// Tensor-core tiles of the mixed-precision LR contraction (k_tc.cu): 64
// complex rows (128 real rows) x 64 columns per CTA, 16 complex k per chunk;
// operands split into TF32 hi/lo parts in the no-swizzle K-major core-matrix
// layout (8 rows x 16 bytes per core matrix).
constexpr int TC_M = 64;
constexpr int TC_N = 64;
constexpr int TC_KC = 16;
constexpr int TC_KR = 2 * TC_KC;
constexpr int TC_ABLK = 2 * 2 * TC_M * TC_KR;   // floats per A' block (hi, lo)
constexpr int TC_BBLK = 2 * TC_N * TC_KR;       // floats per B' block (hi, lo)

__device__ __forceinline__ uint32_t core_off(int r, int k)
{
    return (uint32_t)(((r >> 3) * (TC_KR / 4) + (k >> 2)) * 128 + (r & 7) * 16 + (k & 3) * 4);
}

__device__ __forceinline__ void split_tf32f(float f, float &hi, float &lo)
{
    uint32_t h;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(f));
    hi = __uint_as_float(h);
    uint32_t l;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(l) : "f"(f - hi));
    lo = __uint_as_float(l);
}

// B' element (column n, complex k, real part 0 / imaginary part 1) of batch b
__device__ __forceinline__ void tc_put_b(float *Bp, int nnt, int nkc, int b, int n, int k, int part, float x)
{
    const int nt = n / TC_N, r = n - nt * TC_N;
    const int kr2 = 2 * k + part;
    const int kc = kr2 / TC_KR, kr = kr2 - kc * TC_KR;
    float *blkp = Bp + (((long long)b * nnt + nt) * nkc + kc) * TC_BBLK;
    float hi, lo;
    split_tf32f(x, hi, lo);
    const uint32_t o = core_off(r, kr) >> 2;
    blkp[o] = hi;
    blkp[TC_N * TC_KR + o] = lo;
}

int launch_split_a(int M, int K, const double *A, float *Ap, cudaStream_t st);
int launch_zgemm_tc2(int M, int N, int K, int batch, const float *Ap, const float *Bp, double *C, long long strideC,
                     cudaStream_t st);
long long tc_b_floats(int N, int K, int batch);
long long tc_a_floats(int M, int K);
int tc_status_take(int *flag);
int launch_wait_selftest(int arrive, long long limit, cudaStream_t st);
// ph: double2 table for the FP64 path, float2 table when fp32 != 0
constexpr int DFT_NMAX_HOST = 16;   // longest mesh axis of the DFT path
int launch_dft_mesh(double *T, const int nk[3], long long slab, long long nrep, const double *tw, int conj,
                    cudaStream_t st);
int launch_real_to_complex(const double *X, double *Z, long long n, cudaStream_t st);
int launch_add_complex(double *T, const double *Z, long long n, cudaStream_t st);
int launch_scatter_pairs(const double *T, long long m, int Nk, int npair, const int *pk12, const int *pk2, double *V,
                         int accumulate, cudaStream_t st);
int launch_dft_mesh_df(double *T, const int nk[3], long long slab, long long nrep, const float *tw4, int conj,
                       cudaStream_t st);
int launch_real_to_df(const double *X, double *Z, long long n, cudaStream_t st);
int launch_convert_df(double *T, long long n, int to_df, cudaStream_t st);
int launch_add_df(double *T, const double *Z, long long n, cudaStream_t st);
int launch_scatter_pairs_df(const double *T, long long m, int Nk, int npair, const int *pk12, const int *pk2, double *V,
                            int accumulate, cudaStream_t st);
int launch_x_to_df(double *X, long long n, cudaStream_t st);
int launch_phase1_multi(const double *X, long long m, int Nk, int nlt, const int *k12list, int nk12, const void *ph,
                        double *T, int fp32, int accumulate, cudaStream_t st);
int launch_phase2_multi(const double *T, long long m, int Nk, const int *goff, int ngroups, const int *plist,
                        const int *pk2, const void *ph, double *V, int accumulate, int fp32, cudaStream_t st);

// Density-fitting consumers (k_df.cu)
constexpr int DF_NMAX = 1024;          // largest aux metric of the eigen / Cholesky routes
constexpr int DF_JACOBI_SWEEPS = 40;   // sweep limit of the Jacobi eigensolver
int launch_df_cholesky_route(int n, int nk, const double *J, const double *L, const int *cinfo, double rel, double *T,
                             int *info, int *nkept, cudaStream_t st);
int launch_df_eigen_route(int n, int nk, const double *J, const int *gate, double rel, double *A, double *U,
                          double *lam, int *order, double *T, int *info, int *nkept, cudaStream_t st);
// batched complex GEMM with a split contraction index (layout in k_df.cu)
struct ZGemmGen {
    int M, N, Q, S;
    long long lda, aq, as, bq, bs, bn, ldc;
    const long long *aoff, *boff, *coff;   // device arrays, one element offset per batch
    int conjA, conjB, atomic;
    double alpha;
};
int launch_zgemm_gen(const ZGemmGen &g, int batch, const double *A, const double *B, double *C, cudaStream_t st);

// Cartesian -> real solid harmonic transform (k_sph.cu)
void sph_coefficients(int l, std::vector<double> &s);
void sph_map(const std::vector<int> &ls, std::vector<int> &off, std::vector<int> &idx, std::vector<double> &coef);
struct SphMapDev {
    const int *off, *idx;   // CSR rows per spherical function
    const double *coef;
};
int launch_cart2sph(const double *in, double *out, long long nb, int n1, int n2, int n3, int c1, int c2, int c3,
                    SphMapDev m1, SphMapDev m2, SphMapDev m3, cudaStream_t st);
// compact/diffuse split (k_split.cu)
int launch_split_g0_mask(double *SP, int nP, const int *mask_ax, double *Sf, int Nk, int nao, const int *mask_ao,
                         cudaStream_t st);
int launch_split_combine(const double *Vrs, const double *Vg, double *out, long long nb, int n1, int n2, int c1,
                         int c2, SphMapDev mx, SphMapDev ma, const int *kind_x, const int *kind_a, cudaStream_t st);

}  // namespace rsgdf
