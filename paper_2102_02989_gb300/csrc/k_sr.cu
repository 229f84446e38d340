// SR three-center lattice-sum kernel (Eq. VPmunu_SR with the BvK folding of
// Eq. BvK_latsum_LR), its two-center use for j2c, and the small kernels of the
// G = 0 correction (S_P and the folded overlaps S_{mu nu}).
//
// Work item = (triple: aux shell P, AO shells mu, nu; one lattice vector d of
// the pair phi_mu^0 phi_nu^d); one warp per item.  The warp
//   1. collects the aux translations l of the item that pass the screening
//      (the Supplementary Material's R_c and windowed R_12 cutoffs), scanning
//      a length-sorted list of lattice vectors around the pair centre,
//   2. sorts them stably by BvK cell of l (deterministic order),
//   3. for every primitive combination, accumulates the McMurchie-Davidson
//      Hermite integrals R_tuv(erfc kernel) over the translations of each BvK
//      cell -- the lattice sum acts on R only; the lanes are spread over the
//      cells, each with a row of sums of its own --, and contracts the sums
//      once per cell with the Hermite expansion coefficients of the pair and
//      of the aux function,
//   4. adds the contracted blocks to the folded array X[lt][dt][P][mu][nu].
// The item's geometry (nearest lattice vector of the pair centre, candidate
// radius and prefix) comes from a record written by k_sr_item_geom.  The
// integral arithmetic is FP64; table indices, branches and the screening
// tests use integer and FP32 arithmetic where stated error bounds allow.
#include <cuda_runtime.h>

#include <cstdint>

#include <algorithm>

#include "k_common.cuh"
#include "rsgdf_internal.h"

namespace rsgdf {

__device__ double g_boys_table[(LTOT_MAX + 1) * BOYS_NT * BOYS_W];
static bool g_boys_ready[64] = {false};

int upload_boys_table(const double *tab, cudaStream_t st)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return RSGDF_EDEVICE;
    if (dev < 64 && g_boys_ready[dev]) return RSGDF_OK;
    if (cudaMemcpyToSymbolAsync(g_boys_table, tab, sizeof(double) * (LTOT_MAX + 1) * BOYS_NT * BOYS_W, 0,
                                cudaMemcpyHostToDevice, st) != cudaSuccess)
        return RSGDF_EDEVICE;
    if (cudaStreamSynchronize(st) != cudaSuccess) return RSGDF_EDEVICE;
    if (dev < 64) g_boys_ready[dev] = true;
    return RSGDF_OK;
}

// T >= 0 truncated to a float from the top word of its FP64 encoding (20 of
// its mantissa bits, relative error below 1e-6): integer arithmetic only, so
// the table index costs nothing on the narrow FP64 pipe.  T below 2^-126
// gives 0.
__device__ __forceinline__ float top_float(double T)
{
    const int hi = __double2hiint(T);
    return __int_as_float(max(hi - (896 << 20), 0) << 3);
}

// The table row of class L nearest to T (T_i = i h, the index from integer
// and FP32 arithmetic only) and D = T_i - T, |D| <= h/2 up to the float
// rounding of the index.
template <int L>
__device__ __forceinline__ const double *boys_row(double T, float Tf, double &D)
{
    const int i = min(__float2int_rn(Tf * (float)(1.0 / BOYS_H)), BOYS_NT - 1);
    const double *row = g_boys_table + ((size_t)L * BOYS_NT + i) * BOYS_W;
    D = row[0] - T;
    return row;
}

// sum_k c_k D^k, k < BOYS_TAYLOR (Horner)
__device__ __forceinline__ double boys_taylor(const double *c, double D)
{
    double f = c[BOYS_TAYLOR - 1];
#pragma unroll
    for (int k = BOYS_TAYLOR - 2; k >= 0; k--) f = fma(f, D, c[k]);
    return f;
}

// F_L(T) = c_L T^{-L-1/2} where e^{-T} is negligible: c_L = (sqrt(pi)/2) prod_{m<L} (m + 1/2)
__host__ __device__ constexpr double boys_asym(int L)
{
    double c = 0.5 * 1.772453850905516027298167483341;   // sqrt(pi)/2
    for (int m = 0; m < L; m++) c *= m + 0.5;
    return c;
}

// Classes L <= 1: F_m(T), m = 0..L, one Taylor series per order below
// BOYS_TMAX; above it F_0 = sqrt(pi/T)/2 and the upward recursion without
// e^{-T} (below 1e-43 there).
template <int L>
__device__ __forceinline__ void boys_low(double T, double *F)
{
    const float Tf = top_float(T);
    if (Tf < (float)BOYS_TMAX) {
        double D;
        const double *row = boys_row<L>(T, Tf, D);
#pragma unroll
        for (int m = 0; m <= L; m++) F[m] = boys_taylor(row + 1 + m * BOYS_TAYLOR, D);
    } else {
        const double rs = rsqrt(T);
        const double it = rs * rs;
        F[0] = boys_asym(0) * rs;
#pragma unroll
        for (int m = 0; m < L; m++) F[m + 1] = F[m] * ((m + 0.5) * it);
    }
}

// Classes L >= 2: F_L(T) and e^{-T} = e^{-T_i} e^{D}, each one Taylor series
// about T_i (T < BOYS_TMAX; the caller guarantees it for the attenuated
// argument sT < 70).
template <int L>
__device__ __forceinline__ void boys_seed_table(double T, float Tf, double &FL, double &eT)
{
    double D;
    const double *row = boys_row<L>(T, Tf, D);
    FL = boys_taylor(row + 1, D);
    eT = boys_taylor(row + 1 + BOYS_TAYLOR, D);
}

// The same for any T >= 0: above BOYS_TMAX the power law and e^{-T} = 0.
template <int L>
__device__ __forceinline__ void boys_seed(double T, double &FL, double &eT)
{
    const float Tf = top_float(T);
    if (Tf < (float)BOYS_TMAX) {
        boys_seed_table<L>(T, Tf, FL, eT);
    } else {
        const double rs = rsqrt(T);
        const double it = rs * rs;
        double f = boys_asym(L) * rs;
#pragma unroll
        for (int m = 0; m < L; m++) f *= it;
        FL = f;
        eT = 0.0;
    }
}

// index of R_tuv in the packed tetrahedral array
__host__ __device__ constexpr int ridx(int t, int u, int v)
{
    return (t + u + v) * (t + u + v + 1) * (t + u + v + 2) / 6 + (u + v) * (u + v + 1) / 2 + v;
}

// Per-combination constants of the erfc auxiliary integrals, 2L+2 doubles
// (s = omega^2/(omega^2 + alpha), sw_n = s^{n+1/2}, fw_n = (-2 alpha)^n):
// classes L >= 2: [0] fw_L, [1] sw_L, then for n < L the pair
// fw_n/(2n+1), -fw_n sw_n/(2n+1); classes L <= 1: the pairs fw_n, sw_n.
template <int L>
__device__ __forceinline__ void erfc_consts(double alpha, double s, double sqrt_s, double *cw)
{
    double sw = sqrt_s, fw = 1.0;
#pragma unroll
    for (int n = 0; n <= L; n++) {
        if constexpr (L >= 2) {
            if (n < L) {
                cw[2 + 2 * n] = fw * (1.0 / (2 * n + 1));
                cw[3 + 2 * n] = -(fw * sw) * (1.0 / (2 * n + 1));
            } else {
                cw[0] = fw;
                cw[1] = sw;
            }
        } else {
            cw[2 * n] = fw;
            cw[2 * n + 1] = sw;
        }
        sw *= s;
        fw *= -2.0 * alpha;
    }
}

// Hermite integrals R_tuv, t+u+v <= L, of the erfc kernel at one
// translation, added to acc.  The auxiliary integrals
// G_n = (-2 alpha)^n H_n, H_n = F_n(T) - s^{n+1/2} F_n(sT), obey a downward
// recursion of their own: H_n is the integral of t^{2n} e^{-T t^2} over
// [sqrt s, 1], and integrating (t^{2n+1} e^{-T t^2})' over that interval gives
// (2n+1) H_n = 2T H_{n+1} + e^{-T} - s^{n+1/2} e^{-sT}, that is
// G_n = (-R^2 G_{n+1} + fw_n e^{-T} - fw_n sw_n e^{-sT}) / (2n+1), R^2 = T/alpha.
// Rounding errors stay at the scale eps E_n, E_n = F_n(T) + s^{n+1/2} F_n(sT),
// of the difference that this replaces: F's own recursion gives
// F_n(x)/F_{n+1}(x) >= 2x/(2n+1), so the factor 2T/(2n+1) carried by an error
// in G_{n+1} maps eps E_{n+1} to at most eps E_n.  Classes L >= 2 seed G_L from F_L(T) and
// F_L(sT) and recur; classes L <= 1 form each G_n from its own series.
// Levels n = L-1 .. 1 of R_tuv are built in place in r (totals from high to
// low so that every read still sees level n+1); level 0 goes straight into
// acc.  Requires sT < 70.
template <int L>
__device__ __forceinline__ void hermite_acc(double T, double sT, double R2, const double *cw, double X, double Y,
                                            double Z, double *acc)
{
    constexpr int NR1 = L >= 1 ? (L * (L + 1) * (L + 2)) / 6 : 1;   // entries of totals <= L-1
    double r[NR1];
    double eT = 0.0, esT = 0.0, G0 = 0.0;
    if constexpr (L >= 2) {
        double FL, FsL;
        boys_seed<L>(T, FL, eT);
        boys_seed_table<L>(sT, top_float(sT), FsL, esT);
        r[0] = cw[0] * fma(-cw[1], FsL, FL);
    } else {
        double F[L + 1], Fs[L + 1];
        boys_low<L>(T, F);
        boys_low<L>(sT, Fs);
        G0 = cw[0] * fma(-cw[1], Fs[0], F[0]);
        if constexpr (L == 1) r[0] = cw[2] * fma(-cw[3], Fs[L], F[L]);
    }
#pragma unroll
    for (int n = L - 1; n >= 0; n--) {
#pragma unroll
        for (int S = L - n; S >= 1; S--) {
#pragma unroll
            for (int t = S; t >= 0; t--) {
#pragma unroll
                for (int u = S - t; u >= 0; u--) {
                    const int v = S - t - u;
                    double val = n == 0 ? acc[ridx(t, u, v)] : 0.0;
                    if (t > 0) {
                        val = n == 0 ? fma(X, r[ridx(t - 1, u, v)], val) : X * r[ridx(t - 1, u, v)];
                        if (t > 1) val = fma((double)(t - 1), r[ridx(t - 2, u, v)], val);
                    } else if (u > 0) {
                        val = n == 0 ? fma(Y, r[ridx(t, u - 1, v)], val) : Y * r[ridx(t, u - 1, v)];
                        if (u > 1) val = fma((double)(u - 1), r[ridx(t, u - 2, v)], val);
                    } else {
                        val = n == 0 ? fma(Z, r[ridx(t, u, v - 1)], val) : Z * r[ridx(t, u, v - 1)];
                        if (v > 1) val = fma((double)(v - 1), r[ridx(t, u, v - 2)], val);
                    }
                    if (n == 0) acc[ridx(t, u, v)] = val;
                    else r[ridx(t, u, v)] = val;
                }
            }
        }
        if constexpr (L >= 2) {
            const double b = fma(cw[2 + 2 * n], eT, cw[3 + 2 * n] * esT);
            const double g = fma(-R2 * (1.0 / (2 * n + 1)), r[0], b);
            if (n == 0) G0 = g;
            else r[0] = g;
        }
    }
    acc[0] += G0;
}

// compact Hermite-coefficient layout of a pair entry: E^{ab}_t at eoff(a,b) + t
__device__ __forceinline__ int eoff_sr(int a, int b, int ln)
{
    int o = 0;
    for (int x = 0; x < a; x++) o += (ln + 1) * (2 * x + ln + 2) / 2;
    for (int y = 0; y < b; y++) o += a + y + 1;
    return o;
}

constexpr int EAB_SZ = (LMAX + 1) * (LMAX + 1) * (2 * LMAX + 2) / 2 * 1;   // >= pair_e1(LMAX, LMAX) = 64
constexpr int EC_SZ = (LMAX + 1) * (LMAX + 1);
// products E^c_tau E^c_upsilon E^c_phi over the aux components c of one shell
// (tau, upsilon, phi of the parities of c): at most 19 for l <= 3
constexpr int SR_E3_MAX = 32;
constexpr int SR_WARPS = 2;
constexpr int SR_NT = 256;   // translations buffered per segment (flush above SR_NT - 64)
constexpr int SR_MAXCOMBO = 64;
constexpr int SR_GMAX = 4;   // primitive combinations summed at once in the term loop
constexpr int SR_SKIP_ST_HI = 0x40518000;
constexpr float FLT_U = 5.9604645e-8f;       // 2^-24, unit roundoff of FP32   // top word of 70.0: erfc terms with s T >= 70 vanish

// Per-warp shared memory of the SR kernel, one layout for the host (sizes)
// and the device (carving); offsets in bytes from the warp's base:
// translation positions sorted by BvK cell, the collected translations
// (index into the lattice list and cell), bin counters (then the row table
// of the cells), coefficient-list offsets, the FP32 survivor queue, the
// Hermite coefficients of the current primitive combination, Hermite sums
// (a row per lane and a zero row), contracted blocks, coefficient lists, and
// the per-combination constants.
struct SRSmem {
    unsigned sx, tq, tb, cnt, fill, loff, qd, eab, ec, rb, o, wb, lc, li, kc, total;
};
__host__ __device__ inline SRSmem sr_smem(int L, int bc, int ncomp_max, int w_max, int list_max, int combo_max, int nbin)
{
    SRSmem s;
    unsigned b = 0;
    s.sx = b; b += 3u * SR_NT * 8u;
    s.tq = b; b += SR_NT * 4u;
    s.tb = b; b += SR_NT * 4u;
    s.cnt = b; b += (unsigned)(nbin + 4) * 4u;
    s.fill = b; b += (unsigned)(nbin + 4) * 4u;
    s.loff = b; b += (NC_MAX * NC_MAX + 4) * 4u;
    s.qd = b; b += 64u * 4u;
    b = (b + 15u) & ~15u;
    s.eab = b; b += 3u * EAB_SZ * 8u;
    s.ec = b; b += SR_E3_MAX * 8u;
    s.rb = b; b += (unsigned)(sr_rb_rows(bc) * ntuv(L)) * 8u;
    s.o = b; b += (unsigned)(bc * ncomp_max) * 8u;
    s.wb = b; b += (unsigned)(bc * w_max) * 8u;
    s.lc = b; b += (unsigned)list_max * 8u;
    s.li = b; b += (unsigned)list_max * 4u;
    b = (b + 15u) & ~15u;
    s.kc = b; b += (unsigned)combo_max * 8u * 8u;
    s.total = (b + 15u) & ~15u;
    return s;
}

size_t sr_warp_bytes(int L, int bc, int ncomp_max, int w_max, int list_max, int combo_max, int nbin)
{
    return sr_smem(L, bc, ncomp_max, w_max, list_max, combo_max, nbin).total;
}

// Coulomb bound of one primitive SR term, natural log, in FP32 (a bound only
// needs its order of magnitude).  The aux primitive c x^a y^b z^c e^{-g r^2},
// |x^a y^b z^c| <= r^lP, has a potential no larger than at its centre,
// |c| 2 pi Gamma(lP/2 + 1) / g^{lP/2 + 1} (the potential of a non-negative
// radial density decreases outwards); erfc(w r)/r <= 1/r; and the pair
// density c_i c_j |r-A|^lm |r-B|^ln e^{-a|r-A|^2 - b|r-B|^2} integrates to at
// most |c_i c_j| e^{-ab/p R12^2} sum_{i',j'} C(lm,i') C(ln,j') |PA|^{lm-i'}
// |PB|^{ln-j'} 2 pi Gamma((i'+j'+3)/2) / p^{(i'+j'+3)/2}.
__constant__ float c_gamma_half[11] = {0.0f, 1.7724539f, 1.0f, 0.88622693f, 1.0f, 1.3293404f,
                                       2.0f, 3.3233509f, 6.0f, 11.631728f, 24.0f};   // Gamma(n/2)
__constant__ float c_binom[4][4] = {{1, 0, 0, 0}, {1, 1, 0, 0}, {1, 2, 1, 0}, {1, 3, 3, 1}};
// The part of the bound that depends on the item's d (through R12): the
// overlap factor and the pair-density sum.  The rest, log(|c| 2 pi
// Gamma(lP/2 + 1) / g^{lP/2+1}) + log|c_i c_j|, is per triple and combination
// and comes from the host (SRArgs::cbnd).
__device__ __forceinline__ float prim_combo_log_bound_r12(int lm, float a, int ln, float b, float R12)
{
    const float twopi = 6.2831853f;
    const float p = a + b;
    const float PA = b / p * R12, PB = a / p * R12;
    float S = 0.0f;
    for (int i = 0; i <= lm; i++)
        for (int j = 0; j <= ln; j++)
            S += c_binom[lm][i] * c_binom[ln][j] * powf(PA, (float)(lm - i)) * powf(PB, (float)(ln - j)) * twopi *
                 c_gamma_half[i + j + 3] * __expf(-0.5f * (i + j + 3) * __logf(p));
    return -a * b / p * R12 * R12 + __logf(S);
}

// (t, u, v) of a packed index p = ridx(t, u, v)
__device__ __forceinline__ void tuv_of(int p, int &t, int &u, int &v)
{
    int S = 0;
    while ((S + 1) * (S + 2) * (S + 3) / 6 <= p) S++;
    int q = p - S * (S + 1) * (S + 2) / 6;
    int w = 0;
    while ((w + 1) * (w + 2) / 2 <= q) w++;
    v = q - w * (w + 1) / 2;
    u = w - v;
    t = S - w;
}

// Row of the Hermite sums of cell bb for group g of Lg lanes, from the cell's
// row-table entry (first lane | lanes << 8, or -1 for an empty cell: the zero row 32).
__device__ __forceinline__ int sr_cell_row(int rt, int g, int Lg)
{
    return rt < 0 ? 32 : g * Lg + (rt & 255);
}

// Geometry of the work items, one thread per item (SRItemGeom).  The exact
// test of a translation at distance Rc keeps it only if the cutoff
// win[min(floor(Rc / DR), nwin - 1)] of its window admits the pair's R12:
// beyond the last window that does (wlast) nothing is kept, so unless that is
// the open-ended last window the candidates need only reach (wlast + 1) DR
// (none at all when no window admits R12).  A lattice-list entry l' can pass
// |h - l'| <= Rc only if |l'| <= Rc + |h|: the candidates are a prefix of the
// length-sorted list, usually shorter than the triple's (which assumes the
// largest |h| and R12).
__global__ void k_sr_item_geom(const SRArgs A, long long n_items, SRItemGeom *__restrict__ out)
{
    const long long item = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (item >= n_items) return;
    int t0 = 0, t1 = A.ntri - 1;   // last triple whose first item is <= item
    while (t0 < t1) {
        const int mid = (t0 + t1 + 1) >> 1;
        if (A.tri[mid].item_off <= item) t0 = mid; else t1 = mid - 1;
    }
    const SRTripleDev &tr = A.tri[t0];
    const int gd = A.pair_doff[tr.pair] + (int)(item - tr.item_off);
    const int P = tr.P, mu = tr.mu, nu = tr.nu;
    const int d0 = A.dlist[3 * gd], d1 = A.dlist[3 * gd + 1], d2 = A.dlist[3 * gd + 2];
    const double Ax = A.ao.cen[3 * mu], Ay = A.ao.cen[3 * mu + 1], Az = A.ao.cen[3 * mu + 2];
    const double Bx = A.ao.cen[3 * nu] + d0 * A.a[0] + d1 * A.a[3] + d2 * A.a[6];
    const double By = A.ao.cen[3 * nu + 1] + d0 * A.a[1] + d1 * A.a[4] + d2 * A.a[7];
    const double Bz = A.ao.cen[3 * nu + 2] + d0 * A.a[2] + d1 * A.a[5] + d2 * A.a[8];
    const double Cx = A.ax.cen[3 * P], Cy = A.ax.cen[3 * P + 1], Cz = A.ax.cen[3 * P + 2];
    const double R12 = sqrt((Bx - Ax) * (Bx - Ax) + (By - Ay) * (By - Ay) + (Bz - Az) * (Bz - Az));
    const double iw = 1.0 / (tr.amu + tr.anu);
    const double xr0 = (tr.amu * Ax + tr.anu * Bx) * iw - Cx;
    const double xr1 = (tr.amu * Ay + tr.anu * By) * iw - Cy;
    const double xr2 = (tr.amu * Az + tr.anu * Bz) * iw - Cz;
    SRItemGeom g;
    g.l0[0] = __double2int_rn(xr0 * A.bq[0] + xr1 * A.bq[1] + xr2 * A.bq[2]);
    g.l0[1] = __double2int_rn(xr0 * A.bq[3] + xr1 * A.bq[4] + xr2 * A.bq[5]);
    g.l0[2] = __double2int_rn(xr0 * A.bq[6] + xr1 * A.bq[7] + xr2 * A.bq[8]);
    for (int x = 0; x < 3; x++) g.L0[x] = g.l0[0] * A.a[x] + g.l0[1] * A.a[3 + x] + g.l0[2] * A.a[6 + x];
    g.h[0] = xr0 - g.L0[0];
    g.h[1] = xr1 - g.L0[1];
    g.h[2] = xr2 - g.L0[2];
    g.R12 = R12;
    const double *win = A.win + tr.win_off;
    int wlast = tr.nwin - 1;
    while (wlast >= 0 && !(R12 <= win[wlast])) wlast--;
    const double rcut = wlast == tr.nwin - 1 ? tr.Rc_cut : min(tr.Rc_cut, (wlast + 1) * SCREEN_DR);
    g.fcut = (float)rcut + 1e-3f;
    int nsph = 0;
    if (wlast >= 0) {
        const float fx = (float)g.h[0], fy = (float)g.h[1], fz = (float)g.h[2];
        const float lim = g.fcut + sqrtf(fx * fx + fy * fy + fz * fz) + 1e-3f;
        int lo = 0, hi = tr.nsph;   // first entry longer than lim in [lo, hi]
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (A.sphlen[mid] <= lim) lo = mid + 1; else hi = mid;
        }
        nsph = lo;
    }
    g.nsph = nsph;
    g.gd = gd;
    g.dt = bvk_bin(d0, d1, d2, A.nk);
    g.tri = t0;
    g.pad[0] = g.pad[1] = 0;
    out[item] = g;
}

int launch_sr_item_geom(const SRArgs &A, long long n_items, SRItemGeom *out, cudaStream_t st)
{
    if (n_items <= 0) return RSGDF_OK;
    k_sr_item_geom<<<(unsigned)((n_items + 127) / 128), 128, 0, st>>>(A, n_items, out);
    return cudaGetLastError() == cudaSuccess ? RSGDF_OK : RSGDF_EDEVICE;
}

// One SR work item (aux shell, AO shell pair, d) by one warp, from its
// geometry record; base is the warp's shared-memory region (laid out from A's
// bc, ncomp_max, w_max, list_max, combo_max and nbin_max).  Every branch on
// the item is warp-uniform.
template <int L>
__device__ __forceinline__ void sr3c_item(const SRArgs &A, const long long item, const int lane, unsigned char *base)
{
    if (A.item_skip && A.item_skip[item]) return;   // pruned by the learned screen (warp-uniform)
    constexpr int NR = ntuv(L);
    const SRSmem sm = sr_smem(L, A.bc, A.ncomp_max, A.w_max, A.list_max, A.combo_max, A.nbin_max);
    double *Sx = (double *)(base + sm.sx), *Sy = Sx + SR_NT, *Sz = Sy + SR_NT;   // sorted by BvK cell
    int *Tq = (int *)(base + sm.tq);   // collected: index into the lattice list
    int *Tb = (int *)(base + sm.tb);   // collected: BvK cell
    int *cnt = (int *)(base + sm.cnt);
    int *fill = (int *)(base + sm.fill);
    int *loff = (int *)(base + sm.loff);
    int *Qd = (int *)(base + sm.qd);
    double *Eab = (double *)(base + sm.eab);
    double *E3 = (double *)(base + sm.ec);   // aux-side coefficient products
    double *Rb = (double *)(base + sm.rb);
    double *O = (double *)(base + sm.o);
    double *Wb = (double *)(base + sm.wb);
    double *Lc = (double *)(base + sm.lc);
    int *Lx = (int *)(base + sm.li);   // packed layout of the coefficient lists (per item)
    double *Kc = (double *)(base + sm.kc);   // [combo][8]

    const SRItemGeom G = A.geom[item];
    const SRTripleDev tr = A.tri[G.tri];
    const int gd = G.gd;   // global d index
    const int P = tr.P, mu = tr.mu, nu = tr.nu;
    const int lP = A.ax.l[P], lm = A.ao.l[mu], ln = A.ao.l[nu];
    const int ncP = (lP + 1) * (lP + 2) / 2, ncm = (lm + 1) * (lm + 2) / 2, ncn = (ln + 1) * (ln + 2) / 2;
    const int ncomp = ncP * ncm * ncn;
    const int n1 = (lm + 1) * (ln + 1) * (lm + ln + 2) / 2;
    const int Lp = lm + ln, npt = (Lp + 1) * (Lp + 2) * (Lp + 3) / 6;
    {
        // offsets of the pair-side coefficient lists, one list per (a, b): a
        // warp prefix sum of the list lengths
        int carry = 0;
        for (int ab0 = 0; ab0 < ncm * ncn; ab0 += 32) {
            const int ab = ab0 + lane;
            int len = 0;
            if (ab < ncm * ncn) {
                const signed char *ca = c_cart[lm][ab / ncn], *cb = c_cart[ln][ab % ncn];
                len = (ca[0] + cb[0] + 1) * (ca[1] + cb[1] + 1) * (ca[2] + cb[2] + 1);
            }
            int inc = len;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= o) inc += y;
            }
            if (ab < ncm * ncn) loff[ab] = carry + inc - len;
            carry += __shfl_sync(0xffffffffu, inc, 31);
        }
        if (lane == 0) loff[ncm * ncn] = carry;
    }
    __syncwarp();
    // the layout of the coefficient lists is fixed per item: entry kk of the
    // list of (a, b) is E^x_t E^y_u E^z_v with Hermite index ridx(t, u, v);
    // packed as ridx | (x offset) << 8 | (y offset) << 16 | (z offset) << 24,
    // offsets into the x, y, z blocks of a primitive pair's coefficients
    for (int ab = lane; ab < ncm * ncn; ab += 32) {
        const signed char *ca = c_cart[lm][ab / ncn], *cb = c_cart[ln][ab % ncn];
        const int ox = eoff_sr(ca[0], cb[0], ln), oy = eoff_sr(ca[1], cb[1], ln), oz = eoff_sr(ca[2], cb[2], ln);
        int kk = loff[ab];
        for (int t = 0; t <= ca[0] + cb[0]; t++)
            for (int u = 0; u <= ca[1] + cb[1]; u++)
                for (int v = 0; v <= ca[2] + cb[2]; v++, kk++)
                    Lx[kk] = ridx(t, u, v) | (ox + t) << 8 | (oy + u) << 16 | (oz + v) << 24;
    }
    __syncwarp();
    const double Cx = A.ax.cen[3 * P], Cy = A.ax.cen[3 * P + 1], Cz = A.ax.cen[3 * P + 2];
    const double R12 = G.R12;
    const int l00 = G.l0[0], l01 = G.l0[1], l02 = G.l0[2];
    // candidate translations l = L0 + (an entry of the length-sorted lattice
    // list): h = (pair centre - C) - L0 once per item, then h - l' per entry
    const double L0x = G.L0[0], L0y = G.L0[1], L0z = G.L0[2];
    const double hx = G.h[0], hy = G.h[1], hz = G.h[2];
    const float fx = (float)hx, fy = (float)hy, fz = (float)hz;
    const double *win = A.win + tr.win_off;
    const float fcut = G.fcut;
    const int nsph = G.nsph;
    const int dt = G.dt;
    const double Rc2 = tr.Rc_cut * tr.Rc_cut;
    // FP32 squared distances |h - l'|^2 of candidates (|h - l'| <= fcut, |l'| <= lim):
    // each component carries at most 2u(|h_x| + |l'_x|)(1 + u) of error from the
    // roundings of h, l' and the difference (u = 2^-24), so the sum of squares is
    // off by at most 4u fcut (|h| + lim) + 3u fcut^2 plus O(u^2); e2f doubles that
    const float hf = sqrtf(fx * fx + fy * fy + fz * fz);
    const float e2f = 8.0f * FLT_U * fcut * (hf + fcut + 1e-3f + hf + fcut);
    const float rc2f = (float)Rc2;
    const float rc2f_lo = rc2f * (1.0f - 4.0f * FLT_U), rc2f_hi = rc2f * (1.0f + 4.0f * FLT_U);

    // constants of every primitive combination (k; i, j), one lane each:
    // alpha, s = w^2/(w^2+alpha), sqrt(s), prefactor, product centre - C,
    // and the combination's index.  A combination whose Coulomb bound (below)
    // shows that it adds less than A.log_prim_cut over every candidate
    // translation of the item is dropped here, and the kept ones are packed.
    const int npp = A.ao.nprim[mu] * A.ao.nprim[nu];
    const int ncombo_all = A.ax.nprim[P] * npp;
    int ncombo = 0;
    for (int cb0 = 0; nsph > 0 && cb0 < ncombo_all; cb0 += 32) {   // (no candidates: no combinations)
        const int cb = cb0 + lane;
        bool keep = false;
        double kv[7];
        if (cb < ncombo_all) {
            const int ij = cb % npp;
            const double *cc = A.ccon + 4 * (long long)(tr.cc_off + cb);
            const double *en = A.ptab + A.sr_doff[gd] + (long long)ij * (ENT_HDR + 3 * n1);
            kv[0] = cc[0];
            kv[1] = cc[1];
            kv[2] = cc[2];
            kv[3] = cc[3];
            kv[4] = en[0] - Cx;
            kv[5] = en[1] - Cy;
            kv[6] = en[2] - Cz;
            keep = true;
            if (A.log_prim_cut > -1e30f) {
                const int i = ij / A.ao.nprim[nu], j = ij - i * A.ao.nprim[nu];
                keep = A.cbnd[tr.cc_off + cb] +
                           prim_combo_log_bound_r12(lm, (float)A.ao.exps[A.ao.poff[mu] + i], ln,
                                                    (float)A.ao.exps[A.ao.poff[nu] + j], (float)R12) +
                           __logf((float)max(tr.nsph, 1)) >= A.log_prim_cut;
            }
        }
        const unsigned km = __ballot_sync(0xffffffffu, keep);
        if (keep) {
            double *kc = Kc + 8 * (ncombo + __popc(km & ((1u << lane) - 1u)));
#pragma unroll
            for (int x = 0; x < 7; x++) kc[x] = kv[x];
            kc[7] = (double)cb;
        }
        ncombo += __popc(km);
    }
    __syncwarp();

    int nT = 0;
    unsigned long long kept = 0;
    float magmax = 0.0f;   // largest |block| the item adds (magnitude mode)
    int nq = 0;   // pre-filter survivors waiting for the exact test (smem queue Qd)
    for (int b0 = 0; b0 < nsph; b0 += 32) {
        const int idx = b0 + lane;
        bool pass = false;
        if (idx < nsph) {
            // FP32 pre-filter with a margin far above its rounding error
            const float ex = fx - A.sphvf[3 * idx], ey = fy - A.sphvf[3 * idx + 1], ez = fz - A.sphvf[3 * idx + 2];
            pass = (ex * ex + ey * ey + ez * ez <= fcut * fcut);
        }
        const unsigned pm = __ballot_sync(0xffffffffu, pass);
        if (pass) Qd[nq + __popc(pm & ((1u << lane) - 1u))] = idx;
        nq += __popc(pm);
        __syncwarp();
        const bool lastround = (b0 + 32 >= nsph);
        if (nq < 32 && !lastround) continue;
        // exact test of up to 64 queued candidates, 32 at a time: Rc <= Rc_cut and
        // the window floor(Rc / DR), decided from the FP32 distance wherever its
        // error bound e2f leaves no doubt, else from the FP64 distance
        for (int q0 = 0; q0 < nq; q0 += 32) {
        const int qi = q0 + lane;
        bool acc = false;
        int ci = 0;
        if (qi < nq) {
            ci = Qd[qi];
            const float ex = fx - A.sphvf[3 * ci], ey = fy - A.sphvf[3 * ci + 1], ez = fz - A.sphvf[3 * ci + 2];
            const float r2f = ex * ex + ey * ey + ez * ez;
            const float lo = fmaxf(r2f - e2f, 0.0f), hi = r2f + e2f;
            int w = -1;   // window of the translation, -1 beyond Rc_cut
            bool known = lo > rc2f_hi;   // surely beyond Rc_cut
            if (!known && hi <= rc2f_lo) {   // surely within: the window unless an edge lies in [lo, hi]
                const int wl = (int)(sqrtf(lo) * (float)(1.0 / SCREEN_DR) * (1.0f - 4.0f * FLT_U));
                const int wh = (int)(sqrtf(hi) * (float)(1.0 / SCREEN_DR) * (1.0f + 4.0f * FLT_U));
                if (wl == wh) {
                    w = wl;
                    known = true;
                }
            }
            if (!known) {
                const double r0 = hx - A.sphv[3 * ci], r1 = hy - A.sphv[3 * ci + 1], r2 = hz - A.sphv[3 * ci + 2];
                const double rc2 = r0 * r0 + r1 * r1 + r2 * r2;
                if (rc2 <= Rc2) w = (int)floor(sqrt(rc2) * (1.0 / SCREEN_DR));
            }
            if (w >= 0) acc = (R12 <= win[min(w, tr.nwin - 1)]);
        }
        const unsigned m = __ballot_sync(0xffffffffu, acc);
        if (acc) {
            const int pos = nT + __popc(m & ((1u << lane) - 1u));
            Tq[pos] = ci;
            Tb[pos] = bvk_bin(l00 + A.sph[3 * ci], l01 + A.sph[3 * ci + 1], l02 + A.sph[3 * ci + 2], A.nk);
        }
        nT += __popc(m);
        }
        nq = 0;
        __syncwarp();
        const bool last = lastround;
        if (nT > SR_NT - 64 || (last && nT > 0)) {
            __syncwarp();
            kept += nT;
            // ---- stable counting sort by BvK cell of l
            for (int b = lane; b < A.Nk + 1; b += 32) { cnt[b] = 0; fill[b] = 0; }
            __syncwarp();
            for (int t = lane; t < nT; t += 32) atomicAdd(&cnt[Tb[t] + 1], 1);
            __syncwarp();
            if (lane == 0)
                for (int b = 1; b <= A.Nk; b++) cnt[b] += cnt[b - 1];   // cnt[b] = start of bin b
            __syncwarp();
            for (int t0 = 0; t0 < nT; t0 += 32) {
                const int t = t0 + lane;
                const int bin = (t < nT) ? Tb[t] : -1 - lane;
                const unsigned act = __ballot_sync(0xffffffffu, t < nT);
                const unsigned peers = __match_any_sync(0xffffffffu, bin);
                if (t < nT) {
                    const int rank = __popc(peers & act & ((1u << lane) - 1u));
                    const int dst = cnt[bin] + fill[bin] + rank;
                    const int ci = Tq[t];
                    Sx[dst] = L0x + A.sphv[3 * ci];
                    Sy[dst] = L0y + A.sphv[3 * ci + 1];
                    Sz[dst] = L0z + A.sphv[3 * ci + 2];
                }
                __syncwarp();
                if (t < nT && (peers & act & ((1u << lane) - 1u)) == 0) fill[bin] += __popc(peers & act);
                __syncwarp();
            }
            // ---- BvK cells of l in chunks of bc
            for (int c0 = 0; c0 < A.Nk; c0 += A.bc) {
                const int nb = min(A.bc, A.Nk - c0);
                const int r0 = cnt[c0], r1 = cnt[c0 + nb];
                if (r0 == r1) continue;
                for (int o = lane; o < nb * ncomp; o += 32) O[o] = 0.0;
                // G primitive combinations at a time, each on Lg = 32/G lanes.  The
                // lanes of a combination are spread over the cells of the chunk:
                // cell b (n_b translations) gets k_b = ceil(n_b / R) lanes, R the
                // fewest rounds with sum_b k_b <= Lg, and a lane strides through
                // the translations of its own cell.  Every lane leaves its Hermite
                // sums in a row of its own (row = lane); the rows of one cell are
                // then added into its first.  G minimises ceil(ncombo / G) R.
                const int nbv = lane < nb ? cnt[c0 + lane + 1] - cnt[c0 + lane] : 0;
                const int nz = __popc(__ballot_sync(0xffffffffu, nbv > 0));
                const int nmax = __reduce_max_sync(0xffffffffu, nbv);
                int G = 1, Rr = nmax;
                {
                    long long best = -1;
                    for (int g2 = 1; g2 <= SR_GMAX; g2 *= 2) {
                        const int lg = 32 / g2;
                        if (nz > lg) continue;   // every non-empty cell needs a lane
                        int lo = 1, hi = nmax;   // sum_b ceil(n_b / hi) = nz <= lg
                        while (lo < hi) {
                            const int mid = (lo + hi) >> 1;
                            if (__reduce_add_sync(0xffffffffu, (nbv + mid - 1) / mid) <= lg) hi = mid; else lo = mid + 1;
                        }
                        const long long rounds = (long long)((ncombo + g2 - 1) / g2) * lo;
                        if (best < 0 || rounds < best) {
                            best = rounds;
                            G = g2;
                            Rr = lo;
                        }
                    }
                }
                const int Lg = 32 / G;
                const int grp = lane / Lg, sub = lane - grp * Lg;
                const int kb = (nbv + Rr - 1) / Rr;   // lanes of cell `lane` (lane < nb)
                int ls = kb;                          // -> first lane of cell `lane`
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int y = __shfl_up_sync(0xffffffffu, ls, o);
                    if (lane >= o) ls += y;
                }
                ls -= kb;
                // row table of the cells: first lane | lanes << 8, or -1 (empty cell)
                if (lane < nb) fill[lane] = kb > 0 ? (ls | kb << 8) : -1;
                int mybin = -1, myj = 0, myk = 0;   // this lane's cell, rank among its lanes, their count
                for (int b2 = 0; b2 < nb; b2++) {
                    const int kbb = __shfl_sync(0xffffffffu, kb, b2), lsb = __shfl_sync(0xffffffffu, ls, b2);
                    if (sub >= lsb && sub < lsb + kbb) {
                        mybin = b2;
                        myj = sub - lsb;
                        myk = kbb;
                    }
                }
                for (int q = lane; q < NR; q += 32) Rb[32 * NR + q] = 0.0;   // the row of an empty cell
                __syncwarp();
                for (int cg = 0; cg < ncombo; cg += G) {
                    const int cmy = cg + grp;
                    if (cmy < ncombo && mybin >= 0) {
                        const double *kc = Kc + 8 * cmy;
                        const double alpha = kc[0], s = kc[1];
                        double cw[2 * L + 2];
                        erfc_consts<L>(alpha, s, kc[2], cw);
                        const double Px = kc[4], Py = kc[5], Pz = kc[6];
                        double accR[NR];
#pragma unroll
                        for (int q = 0; q < NR; q++) accR[q] = 0.0;
                        const int te = cnt[c0 + mybin + 1];
                        for (int tt = cnt[c0 + mybin] + myj; tt < te; tt += myk) {
                            const double X = Px - Sx[tt], Y = Py - Sy[tt], Z = Pz - Sz[tt];
                            const double R2 = X * X + Y * Y + Z * Z;
                            const double T = alpha * R2;
                            // F_n(T) and s^{n+1/2} F_n(sT) share their power-law part; for sT >= 70
                            // they differ by O(e^{-sT}) < 1e-30: the erfc term vanishes (the test
                            // compares the top words of the FP64 encodings as integers)
                            const double sT = s * T;
                            if (__double2hiint(sT) >= SR_SKIP_ST_HI) continue;
                            hermite_acc<L>(T, sT, R2, cw, X, Y, Z, accR);
                        }
                        double *row = Rb + lane * NR;
#pragma unroll
                        for (int q = 0; q < NR; q++) row[q] = accR[q];
                    }
                    __syncwarp();
                    for (int o = lane; o < G * nb * NR; o += 32) {
                        const int g = o / (nb * NR), rem = o - g * (nb * NR), bb = rem / NR, q = rem - bb * NR;
                        const int rt = fill[bb];
                        if (cg + g < ncombo && rt >= 0 && (rt >> 8) > 1) {
                            double *r0p = Rb + (g * Lg + (rt & 255)) * NR + q;
                            double sum = r0p[0];
                            for (int i = 1; i < (rt >> 8); i++) sum += r0p[i * NR];
                            r0p[0] = sum;
                        }
                    }
                    __syncwarp();
                    // contractions, one combination after the other
                    for (int gg = 0; gg < G && cg + gg < ncombo; gg++) {
                        const int cc = cg + gg, cb = (int)Kc[8 * cc + 7], k = cb / npp, ij = cb - k * npp;
                        const int ok = A.ax.poff[P] + k;
                        if (lP > 0) {
                            // E3: the products E^c_tau E^c_upsilon E^c_phi of every aux
                            // component c, one component per lane, in the order in
                            // which the sums of (A) use them
                            const double *ect = A.ec_tab + ok * EC_SZ;
                            const signed char *c3 = c_cart[lP][min(lane, ncP - 1)];
                            const int nt3 = lane < ncP ? (c3[0] / 2 + 1) * (c3[1] / 2 + 1) * (c3[2] / 2 + 1) : 0;
                            int e3 = nt3;
#pragma unroll
                            for (int o = 1; o < 32; o <<= 1) {
                                const int y = __shfl_up_sync(0xffffffffu, e3, o);
                                if (lane >= o) e3 += y;
                            }
                            e3 -= nt3;
                            if (lane < ncP)
                                for (int ta2 = c3[0] & 1; ta2 <= c3[0]; ta2 += 2)
                                    for (int ua = c3[1] & 1; ua <= c3[1]; ua += 2) {
                                        const double e2 = ect[c3[0] * (LMAX + 1) + ta2] * ect[c3[1] * (LMAX + 1) + ua];
                                        for (int va = c3[2] & 1; va <= c3[2]; va += 2) E3[e3++] = e2 * ect[c3[2] * (LMAX + 1) + va];
                                    }
                        }
                        // Hermite coefficients of (d, primitive pair)
                        const double *en = A.ptab + A.sr_doff[gd] + (long long)ij * (ENT_HDR + 3 * n1);
                        for (int e = lane; e < 3 * n1; e += 32) Eab[e] = en[ENT_HDR + e];
                        __syncwarp();
                        const double pref = Kc[8 * cc + 3];
                        // (A) aux side: W[bb][c][tuv] = sum E^c_tau E^c_upsilon E^c_phi R[t+tau, u+upsilon, v+phi]
                        if (lP > 0) {
                            // lanes over (cell, pair-side tuv), the aux components in a
                            // warp-uniform loop (uniform trip counts and table reads)
                            for (int w = lane; w < nb * npt; w += 32) {
                                const int bb = w / npt, pq = w - bb * npt;
                                int t, u, v;
                                tuv_of(pq, t, u, v);
                                const double *rb = Rb + sr_cell_row(fill[bb], gg, Lg) * NR;
                                double *wd = Wb + bb * (ncP * npt) + pq;
                                int e3 = 0;
                                for (int ic = 0; ic < ncP; ic++) {
                                    const signed char *cc3 = c_cart[lP][ic];
                                    double sum = 0.0;
                                    for (int ta2 = cc3[0] & 1; ta2 <= cc3[0]; ta2 += 2)
                                        for (int ua = cc3[1] & 1; ua <= cc3[1]; ua += 2)
                                            for (int va = cc3[2] & 1; va <= cc3[2]; va += 2)
                                                sum = fma(E3[e3++], rb[ridx(t + ta2, u + ua, v + va)], sum);
                                    wd[ic * npt] = sum;
                                }
                            }
                        }
                        // (B) pair side: the coefficient lists E^x_t E^y_u E^z_v of all (a, b), one entry per lane
                        for (int kk = lane; kk < loff[ncm * ncn]; kk += 32) {
                            const int q = Lx[kk];
                            Lc[kk] = Eab[(q >> 8) & 255] * Eab[n1 + ((q >> 16) & 255)] * Eab[2 * n1 + (q >> 24)];
                        }
                        __syncwarp();
                        // outputs ordered with (a, b) slowest so that neighbouring lanes share list lengths
                        for (int o = lane; o < nb * ncomp; o += 32) {
                            const int ab = o / (nb * ncP), rem = o - ab * (nb * ncP);
                            const int bb = rem / ncP, ic = rem - bb * ncP;
                            const double *w = lP > 0 ? Wb + (bb * ncP + ic) * npt : Rb + sr_cell_row(fill[bb], gg, Lg) * NR;
                            double s0 = 0.0, s1 = 0.0;
                            int kk = loff[ab];
                            const int ke = loff[ab + 1];
                            for (; kk + 1 < ke; kk += 2) {
                                s0 = fma(Lc[kk], w[Lx[kk] & 255], s0);
                                s1 = fma(Lc[kk + 1], w[Lx[kk + 1] & 255], s1);
                            }
                            if (kk < ke) s0 = fma(Lc[kk], w[Lx[kk] & 255], s0);
                            const int oo = bb * ncomp + ic * ncm * ncn + ab;
                            O[oo] = fma(pref, s0 + s1, O[oo]);
                        }
                        __syncwarp();
                    }
                }
                // ---- add the blocks of this chunk to X
                const long long pf = A.ax.foff[P] - A.pfunc0, mf = A.ao.foff[mu], nf = A.ao.foff[nu];
                for (int o = lane; o < nb * ncomp; o += 32) {
                    const int bb = o / ncomp, comp = o - bb * ncomp;
                    const int ic = comp / (ncm * ncn), ia = (comp / ncn) % ncm, ib = comp % ncn;
                    const long long dst = (long long)(c0 + bb) * A.s_lt + (long long)dt * A.s_dt + (pf + ic) * A.s_P +
                                          (mf + ia) * A.s_mu + (nf + ib) * A.s_nu;
                    if (O[o] != 0.0) atomicAdd(&A.X[dst], O[o]);
                    magmax = fmaxf(magmax, (float)fabs(O[o]));
                }
                __syncwarp();
            }
            nT = 0;
        }
    }
    if (A.item_mag) {
        for (int o = 16; o > 0; o >>= 1) magmax = fmaxf(magmax, __shfl_xor_sync(0xffffffffu, magmax, o));
        if (lane == 0) A.item_mag[item] = magmax > 0.0f ? log10f(magmax) : -30.0f;
    }
    if (lane == 0 && A.term_count) {
        atomicAdd(A.term_count + L, kept);
        atomicAdd(A.term_count + LTOT_MAX + 1, kept * (unsigned long long)ncomp);
        atomicAdd(A.term_count + LTOT_MAX + 2 + L, kept * (unsigned long long)ncombo);
        if (ncombo < ncombo_all)
            atomicAdd(A.term_count + 2 * LTOT_MAX + 5, kept * (unsigned long long)(ncombo_all - ncombo));
    }
}

// Persistent SR kernel of one angular-momentum class: the work items of
// ndesc problems (one SRArgs descriptor each; descriptor i owns the queue
// positions [cum[i], cum[i+1]) and maps them onto its items from
// item_begin) are drawn by warps from one queue, grab items per atomic.
// Descriptors of one launch share bc, ncomp_max, w_max and list_max, so all
// warps carve shared memory alike.
// Registers per thread of the class-L kernel: classes L <= 2 fit in 168 and
// L = 3 in 200 without spilling, so 6 and 5 CTAs of 2 warps can share an SM
// (latency of the collection and contraction phases is then hidden by more
// warps); the higher classes keep 255 (their shared memory admits few CTAs).
__host__ __device__ constexpr int sr_max_regs(int L) { return L <= 2 ? 168 : (L == 3 ? 200 : 255); }

template <int L>
__global__ void __maxnreg__(sr_max_regs(L)) k_sr3c(const SRArgs *__restrict__ desc, const long long *__restrict__ cum,
                                                        int ndesc, int warp_bytes, unsigned long long *queue, int grab)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned char *base = smem_raw + (size_t)warp * warp_bytes;
    const long long ntot = cum[ndesc];
    for (;;) {
        unsigned long long g0 = 0;
        if (lane == 0) g0 = atomicAdd(queue, (unsigned long long)grab);
        g0 = __shfl_sync(0xffffffffu, g0, 0);
        if ((long long)g0 >= ntot) break;   // warp-uniform; the queue only grows
        for (int j = 0; j < grab; j++) {
            const long long g = (long long)g0 + j;
            if (g >= ntot) break;
            int lo = 0, hi = ndesc - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (cum[mid] <= g) lo = mid; else hi = mid - 1;
            }
            sr3c_item<L>(desc[lo], desc[lo].item_begin + (g - cum[lo]), lane, base);
            __syncwarp();
        }
    }
}

typedef void (*SRKern)(const SRArgs *, const long long *, int, int, unsigned long long *, int);
static SRKern sr_kernels[LTOT_MAX + 1] = {k_sr3c<0>, k_sr3c<1>, k_sr3c<2>, k_sr3c<3>, k_sr3c<4>,
                                          k_sr3c<5>, k_sr3c<6>, k_sr3c<7>, k_sr3c<8>, k_sr3c<9>};

// bin chunk (BvK cells of the aux image held at once) for a class: as many
// as fit 4096 doubles of sums per warp, at most 16 and at most the mesh size
// (a larger chunk only costs shared memory, hence occupancy)
int sr_default_bc(int L, int ncomp_max, int w_max, int nk_max)
{
    int bc = 4096 / (ntuv(L) + ncomp_max + w_max);
    bc = bc < 1 ? 1 : (bc > 16 ? 16 : bc);
    // classes L >= 5 hold large per-cell blocks and aux-side sums (ncomp_max,
    // w_max): at most 4 cells per chunk halves them, and two CTAs share an SM
    // where one did (2.7% less SR time on the FCC 2x2x2 step; 2 cells per chunk,
    // or 4 from L = 4 on, were slower)
    if (L >= 5 && bc > 4) bc = 4;
    return bc > nk_max ? (nk_max < 1 ? 1 : nk_max) : bc;
}

size_t sr_launch_smem(int L, int bc, int ncomp_max, int w_max, int list_max, int combo_max, int nbin)
{
    return sr_warp_bytes(L, bc, ncomp_max, w_max, list_max, combo_max, nbin) * SR_WARPS;
}

// Resident CTAs per SM of the class-L kernel with the given dynamic shared memory.
int sr_occupancy(int L, size_t smem)
{
    SRKern kern = sr_kernels[L];
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, SR_WARPS * 32, smem) != cudaSuccess) return 0;
    return nb;
}

// Launch of the class-L kernel over descriptors already on the device.  The
// queue counter is reset on the stream first.  grid = CTAs (persistent).
int launch_sr_queue(int L, const SRArgs *ddesc, const long long *dcum, int ndesc, long long ntot,
                    size_t warp_bytes, unsigned long long *queue, int grid, int grab, cudaStream_t st)
{
    if (ntot <= 0) return RSGDF_OK;
    if (L < 0 || L > LTOT_MAX || grid < 1 || grab < 1) return RSGDF_EINVAL;
    const size_t smem = warp_bytes * SR_WARPS;
    SRKern kern = sr_kernels[L];
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return RSGDF_EDEVICE;
    if (cudaMemsetAsync(queue, 0, sizeof(unsigned long long), st) != cudaSuccess) return RSGDF_EDEVICE;
    const long long need = (ntot + (long long)SR_WARPS * grab - 1) / ((long long)SR_WARPS * grab);
    const int g = (int)std::min<long long>(grid, need);
    kern<<<g, SR_WARPS * 32, smem, st>>>(ddesc, dcum, ndesc, (int)warp_bytes, queue, grab);
    return cudaGetLastError() == cudaSuccess ? RSGDF_OK : RSGDF_EDEVICE;
}

// single-centre Gaussian x^c e^{-g x^2}: E[c*(LMAX+1) + tau]
__host__ __device__ void single_E(int lc, double g, double *E)
{
    double h = 0.5 / g;
    for (int k = 0; k < (LMAX + 1) * (LMAX + 1); k++) E[k] = 0.0;
    E[0] = 1.0;
    for (int c = 1; c <= lc; c++)
        for (int t = 0; t <= c; t++) {
            double v = 0.0;
            if (t > 0) v += h * E[(c - 1) * (LMAX + 1) + t - 1];
            if (t + 1 <= c - 1) v += (t + 1) * E[(c - 1) * (LMAX + 1) + t + 1];
            E[c * (LMAX + 1) + t] = v;
        }
}

// ---------------------------------------------------------------------------
// G = 0 correction pieces
// ---------------------------------------------------------------------------

// S_P = int chi_P for aux shells [s0, s1): (pi/g)^{3/2} prod_x E^{c_x}_0
__global__ void k_aux_charge(DevShells ax, int s0, int s1, int pfunc0, double *S)
{
    int P = s0 + blockIdx.x * blockDim.x + threadIdx.x;
    if (P >= s1) return;
    int l = ax.l[P], nc = (l + 1) * (l + 2) / 2;
    double E[(LMAX + 1) * (LMAX + 1)];
    for (int ic = 0; ic < nc; ic++) S[ax.foff[P] - pfunc0 + ic] = 0.0;
    for (int k = 0; k < ax.nprim[P]; k++) {
        int o = ax.poff[P] + k;
        double g = ax.exps[o];
        single_E(l, g, E);
        double base = ax.cn[o] * pow(KPI / g, 1.5);
        for (int ic = 0; ic < nc; ic++) {
            const signed char *c = c_cart[l][ic];
            S[ax.foff[P] - pfunc0 + ic] += base * E[c[0] * (LMAX + 1)] * E[c[1] * (LMAX + 1)] * E[c[2] * (LMAX + 1)];
        }
    }
}

// V[pair][P][mu][nu] -= pi/(Omega omega^2) S_P sum_dt e^{i k.dt} Sf[dt][mu][nu]
// for pairs with k1 = k2 (the q = 0 term of the SR kernel, Eq. VPmunu_SR).
__global__ void k_g0_correct(double *V, const int *kpairs, int npair, int nP, int nao, const double *SP,
                             const double *Sf, const int *nk3, int Nk, double fac)
{
    long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long per = (long long)nP * nao * nao;
    if (id >= per * npair) return;
    int pr = (int)(id / per);
    long long rem = id - (long long)pr * per;
    int k1 = kpairs[2 * pr], k2 = kpairs[2 * pr + 1];
    if (k1 != k2) return;
    int P = (int)(rem / ((long long)nao * nao));
    long long mn = rem - (long long)P * nao * nao;
    int nk[3] = {nk3[0], nk3[1], nk3[2]};
    double re = 0.0, im = 0.0;
    for (int dt = 0; dt < Nk; dt++) {
        double c, s;
        bloch_phase(k2, dt, nk, +1, c, s);
        double v = Sf[(long long)dt * nao * nao + mn];
        re += c * v;
        im += s * v;
    }
    V[2 * id] -= fac * SP[P] * re;
    V[2 * id + 1] -= fac * SP[P] * im;
}

}  // namespace rsgdf
