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
//      cell -- the lattice sum acts on R only --, and contracts the sums once
//      per cell with the Hermite expansion coefficients of the pair and of
//      the aux function,
//   4. adds the contracted blocks to the folded array X[lt][dt][P][mu][nu].
// Everything is FP64.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdint>

#include <algorithm>

#include "k_common.cuh"
#include "rsgdf_internal.h"

namespace rsgdf {

__device__ double g_boys_table[BOYS_NT * BOYS_ROW];
static bool g_boys_ready[64] = {false};

int upload_boys_table(const double *tab, cudaStream_t st)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return RSGDF_EDEVICE;
    if (dev < 64 && g_boys_ready[dev]) return RSGDF_OK;
    if (cudaMemcpyToSymbolAsync(g_boys_table, tab, sizeof(double) * BOYS_NT * BOYS_ROW, 0,
                                cudaMemcpyHostToDevice, st) != cudaSuccess)
        return RSGDF_EDEVICE;
    if (cudaStreamSynchronize(st) != cudaSuccess) return RSGDF_EDEVICE;
    if (dev < 64) g_boys_ready[dev] = true;
    return RSGDF_OK;
}

// F_m(T), m = 0..L: Taylor series of F_L about the nearest tabulated point,
// then downward recursion F_m = (2T F_{m+1} + e^{-T})/(2m+1) with e^{-T} =
// e^{-T_i} e^{T_i - T} (tabulated value times a short Taylor series); for T
// beyond the table F_0 = sqrt(pi/T)/2 and the upward recursion.
template <int L>
__device__ __forceinline__ void boys_f64(double T, double *F)
{
    if (T < BOYS_TMAX) {
        const int i = __double2int_rn(T * (1.0 / BOYS_H));
        const double D = i * BOYS_H - T;
        // row[m*BOYS_TAYLOR + k] = F_{m+k}(T_i)/k!, row[BOYS_NM*BOYS_TAYLOR + k] = e^{-T_i}/k!
        const double *row = g_boys_table + i * BOYS_ROW;
        if (L <= 2) {
#pragma unroll
            for (int m = 0; m <= L; m++) {
                const double *c = row + m * BOYS_TAYLOR;
                double f = c[BOYS_TAYLOR - 1];
#pragma unroll
                for (int k = BOYS_TAYLOR - 2; k >= 0; k--) f = fma(f, D, c[k]);
                F[m] = f;
            }
        } else {
            const double *c = row + L * BOYS_TAYLOR;
            double f = c[BOYS_TAYLOR - 1];
#pragma unroll
            for (int k = BOYS_TAYLOR - 2; k >= 0; k--) f = fma(f, D, c[k]);
            F[L] = f;
            const double *ce = row + BOYS_NM * BOYS_TAYLOR;
            double e = ce[BOYS_TAYLOR - 1];
#pragma unroll
            for (int k = BOYS_TAYLOR - 2; k >= 0; k--) e = fma(e, D, ce[k]);
            const double T2 = 2.0 * T;
#pragma unroll
            for (int m = L - 1; m >= 0; m--) F[m] = fma(T2, F[m + 1], e) * (1.0 / (2 * m + 1));
        }
    } else {
        // e^{-T} is below 1e-43 of F_m for T >= 100 and m <= 9
        const double e = (T < 100.0) ? exp(-T) : 0.0;
        const double rs = rsqrt(T);
        const double it = rs * rs;
        F[0] = 0.5 * sqrt(KPI) * rs;
#pragma unroll
        for (int m = 0; m < L; m++) F[m + 1] = ((2 * m + 1) * F[m] - e) * (0.5 * it);
    }
}

// index of R_tuv in the packed tetrahedral array
__host__ __device__ constexpr int ridx(int t, int u, int v)
{
    return (t + u + v) * (t + u + v + 1) * (t + u + v + 2) / 6 + (u + v) * (u + v + 1) / 2 + v;
}

// Hermite integrals R_tuv, t+u+v <= L, of the erfc kernel, in place: level n
// from L down to 0, totals from high to low so that every read still sees
// level n+1.  sw[n] = s^{n+1/2}, fw[n] = (-2 alpha)^n (per primitive
// combination), s = omega^2/(omega^2 + alpha).
template <int L>
__device__ __forceinline__ void hermite_R(double T, double s, const double *sw, const double *fw, double X, double Y,
                                          double Z, double *r)
{
    double F[L + 1], Fs[L + 1];
    boys_f64<L>(T, F);
    boys_f64<L>(s * T, Fs);
    r[0] = fw[L] * fma(-sw[L], Fs[L], F[L]);
#pragma unroll
    for (int n = L - 1; n >= 0; n--) {
#pragma unroll
        for (int S = L - n; S >= 1; S--) {
#pragma unroll
            for (int t = S; t >= 0; t--) {
#pragma unroll
                for (int u = S - t; u >= 0; u--) {
                    const int v = S - t - u;
                    double val;
                    if (t > 0) {
                        val = X * r[ridx(t - 1, u, v)];
                        if (t > 1) val = fma((double)(t - 1), r[ridx(t - 2, u, v)], val);
                    } else if (u > 0) {
                        val = Y * r[ridx(t, u - 1, v)];
                        if (u > 1) val = fma((double)(u - 1), r[ridx(t, u - 2, v)], val);
                    } else {
                        val = Z * r[ridx(t, u, v - 1)];
                        if (v > 1) val = fma((double)(v - 1), r[ridx(t, u, v - 2)], val);
                    }
                    r[ridx(t, u, v)] = val;
                }
            }
        }
        r[0] = fw[n] * fma(-sw[n], Fs[n], F[n]);
    }
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
constexpr int SR_WARPS = 2;
constexpr int SR_NT = 256;   // translations buffered per segment (flush above SR_NT - 64)
constexpr int SR_MAXCOMBO = 64;
constexpr int SR_GMAX = 4;   // primitive combinations summed at once in the term loop
constexpr double SR_SKIP_ST = 70.0;   // erfc terms with s T beyond this vanish   // primitive combinations per triple (aux x AO x AO)

// per-warp shared memory: term positions (3 doubles) and BvK cells, twice
// (collected and sorted), bin counters, Hermite coefficients of the current
// primitive combination, Hermite sums per cell and contracted blocks.
size_t sr_warp_bytes(int L, int bc, int ncomp_max, int w_max, int list_max)
{
    size_t b = 2 * SR_NT * (3 * sizeof(double) + sizeof(int)) + 2 * (NBIN_MAX + 4) * sizeof(int);
    b += (NC_MAX * NC_MAX + 4) * sizeof(int);                      // list offsets per (a, b)
    b += 64 * sizeof(int);                                        // FP32 survivor queue
    b = (b + 15) & ~(size_t)15;
    b += (3 * EAB_SZ + EC_SZ) * sizeof(double);
    b += ((size_t)sr_rb_rows(bc) * ntuv(L) + (size_t)bc * (ncomp_max + w_max)) * sizeof(double);
    b += (size_t)list_max * (sizeof(double) + sizeof(short));
    b = (b + 15) & ~(size_t)15;
    b += (size_t)SR_MAXCOMBO * 8 * sizeof(double);                    // per-combination constants
    return (b + 15) & ~(size_t)15;
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

// One SR work item (aux shell, AO shell pair, d) by one warp; base is the
// warp's shared-memory region (laid out from A's bc, ncomp_max, w_max and
// list_max).  Every branch on the item is warp-uniform.
template <int L>
__device__ __forceinline__ void sr3c_item(const SRArgs &A, const long long item, const int lane, unsigned char *base)
{
    if (A.item_skip && A.item_skip[item]) return;   // pruned by the learned screen (warp-uniform)
    constexpr int NR = ntuv(L);
    double *Tx = (double *)base;            // collected translations (Cartesian)
    double *Ty = Tx + SR_NT, *Tz = Ty + SR_NT;
    double *Sx = Tz + SR_NT, *Sy = Sx + SR_NT, *Sz = Sy + SR_NT;   // sorted by BvK cell
    int *Tb = (int *)(Sz + SR_NT);
    int *Sb = Tb + SR_NT;
    int *cnt = Sb + SR_NT;
    int *fill = cnt + NBIN_MAX + 4;
    int *loff = fill + NBIN_MAX + 4;
    int *Qd = loff + NC_MAX * NC_MAX + 4;
    double *Eab = (double *)(base + ((2 * SR_NT * (3 * sizeof(double) + sizeof(int)) + 2 * (NBIN_MAX + 4) * sizeof(int) +
                                      (NC_MAX * NC_MAX + 4) * sizeof(int) + 64 * sizeof(int) + 15) &
                                     ~(size_t)15));
    double *Ec = Eab + 3 * EAB_SZ;
    double *Rb = Ec + EC_SZ;
    double *O = Rb + sr_rb_rows(A.bc) * NR;
    double *Wb = O + A.bc * A.ncomp_max;
    double *Lc = Wb + A.bc * A.w_max;
    short *Li = (short *)(Lc + A.list_max);
    double *Kc = (double *)(((uintptr_t)(Li + A.list_max) + 15) & ~(uintptr_t)15);   // [combo][8]

    // the triple of this item: last triple with item_off <= item
    int lo = A.tri_begin, hi = A.tri_end - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (A.tri[mid].item_off <= item) lo = mid; else hi = mid - 1;
    }
    const SRTripleDev tr = A.tri[lo];
    const int gd = A.pair_doff[tr.pair] + (int)(item - tr.item_off);   // global d index
    const int P = tr.P, mu = tr.mu, nu = tr.nu;
    const int lP = A.ax.l[P], lm = A.ao.l[mu], ln = A.ao.l[nu];
    const int ncP = (lP + 1) * (lP + 2) / 2, ncm = (lm + 1) * (lm + 2) / 2, ncn = (ln + 1) * (ln + 2) / 2;
    const int ncomp = ncP * ncm * ncn;
    const int n1 = (lm + 1) * (ln + 1) * (lm + ln + 2) / 2;
    const int Lp = lm + ln, npt = (Lp + 1) * (Lp + 2) * (Lp + 3) / 6;
    if (lane == 0) {
        // offsets of the pair-side coefficient lists, one list per (a, b)
        int o = 0;
        for (int ab = 0; ab < ncm * ncn; ab++) {
            const signed char *ca = c_cart[lm][ab / ncn], *cb = c_cart[ln][ab % ncn];
            loff[ab] = o;
            o += (ca[0] + cb[0] + 1) * (ca[1] + cb[1] + 1) * (ca[2] + cb[2] + 1);
        }
        loff[ncm * ncn] = o;
    }
    __syncwarp();
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
    const int l00 = __double2int_rn(xr0 * A.bq[0] + xr1 * A.bq[1] + xr2 * A.bq[2]);
    const int l01 = __double2int_rn(xr0 * A.bq[3] + xr1 * A.bq[4] + xr2 * A.bq[5]);
    const int l02 = __double2int_rn(xr0 * A.bq[6] + xr1 * A.bq[7] + xr2 * A.bq[8]);
    const float fx = (float)xr0, fy = (float)xr1, fz = (float)xr2;
    const float fcut = (float)tr.Rc_cut + 1e-3f;
    const int dt = bvk_bin(d0, d1, d2, A.nk);
    const double *win = A.win + tr.win_off;
    const double Rc2 = tr.Rc_cut * tr.Rc_cut;
    const double omega2 = A.omega * A.omega;

    // constants of every primitive combination (k; i, j), one lane each:
    // alpha, s = w^2/(w^2+alpha), sqrt(s), prefactor, product centre - C
    const int npp = A.ao.nprim[mu] * A.ao.nprim[nu];
    const int ncombo = A.ax.nprim[P] * npp;
    for (int cb = lane; cb < ncombo; cb += 32) {
        const int k = cb / npp, ij = cb - k * npp;
        const int ok = A.ax.poff[P] + k;
        const double g = A.ax.exps[ok];
        const double *en = A.ptab + A.sr_doff[gd] + (long long)ij * (ENT_HDR + 3 * n1);
        const double p = en[5];
        const double ipg = 1.0 / (p + g);
        const double alpha = p * g * ipg;
        const double s = omega2 / (omega2 + alpha);
        double *kc = Kc + 8 * cb;
        kc[0] = alpha;
        kc[1] = s;
        kc[2] = sqrt(s);
        kc[3] = 2.0 * KPI2_5 / (p * g) * sqrt(ipg) * A.ax.cn[ok] * en[6] * ((lP & 1) ? -1.0 : 1.0);
        kc[4] = en[0] - Cx;
        kc[5] = en[1] - Cy;
        kc[6] = en[2] - Cz;
        kc[7] = 0.0;
    }
    __syncwarp();

    int nT = 0;
    unsigned long long kept = 0;
    float magmax = 0.0f;   // largest |block| the item adds (magnitude mode)
    int nq = 0;   // FP32 survivors waiting for the exact FP64 test (smem queue Qd)
    for (int b0 = 0; b0 < tr.nsph; b0 += 32) {
        const int idx = b0 + lane;
        bool pass = false;
        if (idx < tr.nsph) {
            const int li0 = l00 + A.sph[3 * idx], li1 = l01 + A.sph[3 * idx + 1], li2 = l02 + A.sph[3 * idx + 2];
            // FP32 pre-filter with a margin far above its rounding error
            const float ex = fx - (li0 * A.af[0] + li1 * A.af[3] + li2 * A.af[6]);
            const float ey = fy - (li0 * A.af[1] + li1 * A.af[4] + li2 * A.af[7]);
            const float ez = fz - (li0 * A.af[2] + li1 * A.af[5] + li2 * A.af[8]);
            pass = (ex * ex + ey * ey + ez * ez <= fcut * fcut);
        }
        const unsigned pm = __ballot_sync(0xffffffffu, pass);
        if (pass) Qd[nq + __popc(pm & ((1u << lane) - 1u))] = idx;
        nq += __popc(pm);
        __syncwarp();
        const bool lastround = (b0 + 32 >= tr.nsph);
        if (nq < 32 && !lastround) continue;
        // exact FP64 test of up to 64 queued candidates, 32 at a time
        for (int q0 = 0; q0 < nq; q0 += 32) {
        const int qi = q0 + lane;
        bool acc = false;
        int li0 = 0, li1 = 0, li2 = 0;
        double lx = 0.0, ly = 0.0, lz = 0.0;
        if (qi < nq) {
            const int ci = Qd[qi];
            li0 = l00 + A.sph[3 * ci];
            li1 = l01 + A.sph[3 * ci + 1];
            li2 = l02 + A.sph[3 * ci + 2];
            {
                lx = li0 * A.a[0] + li1 * A.a[3] + li2 * A.a[6];
                ly = li0 * A.a[1] + li1 * A.a[4] + li2 * A.a[7];
                lz = li0 * A.a[2] + li1 * A.a[5] + li2 * A.a[8];
                const double r0 = xr0 - lx, r1 = xr1 - ly, r2 = xr2 - lz;
                const double rc = sqrt(r0 * r0 + r1 * r1 + r2 * r2);
                if (rc <= tr.Rc_cut) {
                    int w = (int)floor(rc * (1.0 / SCREEN_DR));
                    if (w >= tr.nwin) w = tr.nwin - 1;
                    acc = (R12 <= win[w]);
                }
            }
        }
        (void)Rc2;
        const unsigned m = __ballot_sync(0xffffffffu, acc);
        if (acc) {
            const int pos = nT + __popc(m & ((1u << lane) - 1u));
            Tx[pos] = lx;
            Ty[pos] = ly;
            Tz[pos] = lz;
            Tb[pos] = bvk_bin(li0, li1, li2, A.nk);
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
                    Sx[dst] = Tx[t];
                    Sy[dst] = Ty[t];
                    Sz[dst] = Tz[t];
                    Sb[dst] = bin;
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
                // G primitive combinations at a time, each on 32/G lanes with its
                // own rows of Hermite sums: G minimises the warp rounds of the
                // term loop (a chunk holds ~tens of translations, fewer than 32
                // lanes per combination would leave idle)
                const int nTc = r1 - r0;
                int G = 1;
                {
                    long long best = (long long)ncombo * ((nTc + 31) >> 5);
                    for (int g2 = 2; g2 <= SR_GMAX && g2 * nb <= sr_rb_rows(A.bc); g2 *= 2) {
                        const int lg = 32 / g2;
                        const long long rounds = (long long)((ncombo + g2 - 1) / g2) * ((nTc + lg - 1) / lg);
                        if (rounds < best) {
                            best = rounds;
                            G = g2;
                        }
                    }
                }
                const int Lg = 32 / G;
                const int grp = lane / Lg, sub = lane - grp * Lg;
                for (int cg = 0; cg < ncombo; cg += G) {
                    for (int o = lane; o < G * nb * NR; o += 32) Rb[o] = 0.0;
                    __syncwarp();
                    const int cmy = cg + grp;
                    if (cmy < ncombo) {
                        const double *kc = Kc + 8 * cmy;
                        const double alpha = kc[0], s = kc[1];
                        double sw[L + 1], fw[L + 1];
                        sw[0] = kc[2];
                        fw[0] = 1.0;
#pragma unroll
                        for (int n = 1; n <= L; n++) {
                            sw[n] = sw[n - 1] * s;
                            fw[n] = fw[n - 1] * (-2.0 * alpha);
                        }
                        const double Px = kc[4], Py = kc[5], Pz = kc[6];
                        double *Rg = Rb + grp * nb * NR;
                        // contiguous slice of the sorted translations per lane of the group
                        const int per = (nTc + Lg - 1) / Lg;
                        const int ta = r0 + sub * per, tb = min(ta + per, r1);
                        double accR[NR];
#pragma unroll
                        for (int q = 0; q < NR; q++) accR[q] = 0.0;
                        int cur = -1;
                        for (int tt = ta; tt < tb; tt++) {
                            const int bn = Sb[tt];
                            if (bn != cur) {
                                if (cur >= 0) {
#pragma unroll
                                    for (int q = 0; q < NR; q++) {
                                        atomicAdd(&Rg[(cur - c0) * NR + q], accR[q]);
                                        accR[q] = 0.0;
                                    }
                                }
                                cur = bn;
                            }
                            const double X = Px - Sx[tt], Y = Py - Sy[tt], Z = Pz - Sz[tt];
                            const double T = alpha * (X * X + Y * Y + Z * Z);
                            // F_n(T) and s^{n+1/2} F_n(sT) share their power-law part; for sT >= 70
                            // they differ by O(e^{-sT}) < 1e-30: the erfc term vanishes
                            if (s * T >= SR_SKIP_ST) continue;
                            double r[NR];
                            hermite_R<L>(T, s, sw, fw, X, Y, Z, r);
#pragma unroll
                            for (int q = 0; q < NR; q++) accR[q] += r[q];
                        }
                        if (cur >= 0) {
#pragma unroll
                            for (int q = 0; q < NR; q++) atomicAdd(&Rg[(cur - c0) * NR + q], accR[q]);
                        }
                    }
                    __syncwarp();
                    // contractions, one combination after the other
                    for (int gg = 0; gg < G && cg + gg < ncombo; gg++) {
                        const int cc = cg + gg, k = cc / npp, ij = cc - k * npp;
                        const int ok = A.ax.poff[P] + k;
                        for (int e = lane; e < EC_SZ; e += 32) Ec[e] = A.ec_tab[ok * EC_SZ + e];
                        // Hermite coefficients of (d, primitive pair)
                        const double *en = A.ptab + A.sr_doff[gd] + (long long)ij * (ENT_HDR + 3 * n1);
                        for (int e = lane; e < 3 * n1; e += 32) Eab[e] = en[ENT_HDR + e];
                        __syncwarp();
                        const double pref = Kc[8 * cc + 3];
                        const double *Rg = Rb + gg * nb * NR;
                        // (A) aux side: W[bb][c][tuv] = sum E^c_tau E^c_upsilon E^c_phi R[t+tau, u+upsilon, v+phi]
                        const double *Wsrc = Rg;
                        int wstride = NR, cstride = 0;
                        if (lP > 0) {
                            for (int w = lane; w < nb * ncP * npt; w += 32) {
                                const int bb = w / (ncP * npt), rem = w - bb * (ncP * npt);
                                const int ic = rem / npt, pq = rem - ic * npt;
                                int t, u, v;
                                tuv_of(pq, t, u, v);
                                const signed char *cc3 = c_cart[lP][ic];
                                const double *rb = Rg + bb * NR;
                                double sum = 0.0;
                                for (int ta2 = cc3[0] & 1; ta2 <= cc3[0]; ta2 += 2)
                                    for (int ua = cc3[1] & 1; ua <= cc3[1]; ua += 2) {
                                        const double e2 = Ec[cc3[0] * (LMAX + 1) + ta2] * Ec[cc3[1] * (LMAX + 1) + ua];
                                        for (int va = cc3[2] & 1; va <= cc3[2]; va += 2)
                                            sum = fma(e2 * Ec[cc3[2] * (LMAX + 1) + va], rb[ridx(t + ta2, u + ua, v + va)], sum);
                                    }
                                Wb[w] = sum;
                            }
                            Wsrc = Wb;
                            wstride = ncP * npt;
                            cstride = npt;
                        }
                        // (B) pair side: one coefficient list E^x_t E^y_u E^z_v per (a, b)
                        for (int ab = lane; ab < ncm * ncn; ab += 32) {
                            const signed char *ca = c_cart[lm][ab / ncn], *cb = c_cart[ln][ab % ncn];
                            const double *ex0 = Eab + eoff_sr(ca[0], cb[0], ln);
                            const double *ey0 = Eab + n1 + eoff_sr(ca[1], cb[1], ln);
                            const double *ez0 = Eab + 2 * n1 + eoff_sr(ca[2], cb[2], ln);
                            int kk = loff[ab];
                            for (int t = 0; t <= ca[0] + cb[0]; t++)
                                for (int u = 0; u <= ca[1] + cb[1]; u++) {
                                    const double exy = ex0[t] * ey0[u];
                                    for (int v = 0; v <= ca[2] + cb[2]; v++, kk++) {
                                        Lc[kk] = exy * ez0[v];
                                        Li[kk] = (short)ridx(t, u, v);
                                    }
                                }
                        }
                        __syncwarp();
                        // outputs ordered with (a, b) slowest so that neighbouring lanes share list lengths
                        for (int o = lane; o < nb * ncomp; o += 32) {
                            const int ab = o / (nb * ncP), rem = o - ab * (nb * ncP);
                            const int bb = rem / ncP, ic = rem - bb * ncP;
                            const double *w = Wsrc + bb * wstride + ic * cstride;
                            double s0 = 0.0, s1 = 0.0;
                            int kk = loff[ab];
                            const int ke = loff[ab + 1];
                            for (; kk + 1 < ke; kk += 2) {
                                s0 = fma(Lc[kk], w[Li[kk]], s0);
                                s1 = fma(Lc[kk + 1], w[Li[kk + 1]], s1);
                            }
                            if (kk < ke) s0 = fma(Lc[kk], w[Li[kk]], s0);
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
    }
}

// Persistent SR kernel of one angular-momentum class: the work items of
// ndesc problems (one SRArgs descriptor each; descriptor i owns the queue
// positions [cum[i], cum[i+1]) and maps them onto its items from
// item_begin) are drawn by warps from one queue, grab items per atomic.
// Descriptors of one launch share bc, ncomp_max, w_max and list_max, so all
// warps carve shared memory alike.
template <int L>
__global__ void __launch_bounds__(SR_WARPS * 32) k_sr3c(const SRArgs *__restrict__ desc, const long long *__restrict__ cum,
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
    return bc > nk_max ? (nk_max < 1 ? 1 : nk_max) : bc;
}

size_t sr_launch_smem(int L, int bc, int ncomp_max, int w_max, int list_max)
{
    return sr_warp_bytes(L, bc, ncomp_max, w_max, list_max) * SR_WARPS;
}

// Resident CTAs per SM of the class-L kernel with the given dynamic shared memory.
int sr_occupancy(int L, size_t smem)
{
    if (cudaFuncSetAttribute(sr_kernels[L], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, sr_kernels[L], SR_WARPS * 32, smem) != cudaSuccess) return 0;
    return nb;
}

// Launch of the class-L kernel over descriptors already on the device.  The
// queue counter is reset on the stream first.  grid = CTAs (persistent).
int launch_sr_queue(int L, const SRArgs *ddesc, const long long *dcum, int ndesc, long long ntot, size_t warp_bytes,
                    unsigned long long *queue, int grid, int grab, cudaStream_t st)
{
    if (ntot <= 0) return RSGDF_OK;
    if (L < 0 || L > LTOT_MAX || grid < 1 || grab < 1) return RSGDF_EINVAL;
    const size_t smem = warp_bytes * SR_WARPS;
    if (cudaFuncSetAttribute(sr_kernels[L], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return RSGDF_EDEVICE;
    if (cudaMemsetAsync(queue, 0, sizeof(unsigned long long), st) != cudaSuccess) return RSGDF_EDEVICE;
    const long long need = (ntot + (long long)SR_WARPS * grab - 1) / ((long long)SR_WARPS * grab);
    const int g = (int)std::min<long long>(grid, need);
    sr_kernels[L]<<<g, SR_WARPS * 32, smem, st>>>(ddesc, dcum, ndesc, (int)warp_bytes, queue, grab);
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
