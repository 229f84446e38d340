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

#include "k_common.cuh"
#include "rsgdf_internal.h"

namespace rsgdf {

__device__ double g_boys_table[BOYS_NT * BOYS_NM];
static bool g_boys_ready[64] = {false};

int upload_boys_table(const double *tab, cudaStream_t st)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return RSGDF_EDEVICE;
    if (dev < 64 && g_boys_ready[dev]) return RSGDF_OK;
    if (cudaMemcpyToSymbolAsync(g_boys_table, tab, sizeof(double) * BOYS_NT * BOYS_NM, 0,
                                cudaMemcpyHostToDevice, st) != cudaSuccess)
        return RSGDF_EDEVICE;
    if (cudaStreamSynchronize(st) != cudaSuccess) return RSGDF_EDEVICE;
    if (dev < 64) g_boys_ready[dev] = true;
    return RSGDF_OK;
}

// F_m(T), m = 0..L: Taylor series of F_L about the nearest tabulated point,
// then downward recursion F_m = (2T F_{m+1} + e^{-T})/(2m+1); for T beyond the
// table F_0 = sqrt(pi/T)/2 and the upward recursion.
template <int L>
__device__ __forceinline__ void boys_f64(double T, double *F)
{
    if (T < BOYS_TMAX) {
        int i = __double2int_rn(T * (1.0 / BOYS_H));
        double D = i * BOYS_H - T;
        const double *row = g_boys_table + i * BOYS_NM + L;
        double f = row[BOYS_TAYLOR - 1];
#pragma unroll
        for (int k = BOYS_TAYLOR - 2; k >= 0; k--) f = fma(f, D * (1.0 / (k + 1)), row[k]);
        F[L] = f;
        double e = exp(-T);
#pragma unroll
        for (int m = L - 1; m >= 0; m--) F[m] = fma(2.0 * T, F[m + 1], e) * (1.0 / (2 * m + 1));
    } else {
        double e = exp(-T);
        double it = 1.0 / T;
        F[0] = 0.5 * sqrt(KPI * it);
#pragma unroll
        for (int m = 0; m < L; m++) F[m + 1] = ((2 * m + 1) * F[m] - e) * (0.5 * it);
    }
}

// index of R_tuv in the packed tetrahedral array
__host__ __device__ constexpr int ridx(int t, int u, int v)
{
    return (t + u + v) * (t + u + v + 1) * (t + u + v + 2) / 6 + (u + v) * (u + v + 1) / 2 + v;
}

// Hermite integrals R_tuv, t+u+v <= L, of the erfc kernel, in place:
// level n from L down to 0, totals from high to low so that every read still
// sees level n+1.
template <int L>
__device__ __forceinline__ void hermite_R(double alpha, double omega2, double T, double X, double Y, double Z,
                                          double *r)
{
    double F[L + 1], Fs[L + 1];
    double s = omega2 / (omega2 + alpha);
    boys_f64<L>(T, F);
    boys_f64<L>(s * T, Fs);
    double g[L + 1];
    double sp = sqrt(s), m2a = -2.0 * alpha, fac = 1.0;
#pragma unroll
    for (int n = 0; n <= L; n++) {
        g[n] = fac * (F[n] - sp * Fs[n]);
        sp *= s;
        fac *= m2a;
    }
    r[0] = g[L];
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
        r[0] = g[n];
    }
}

// Hermite expansion coefficients of the 1D product x_A^i x_B^j e^{-a xA^2 - b xB^2}:
// E[(i*(lb+1)+j)*EMT + t], EMT = 2*LMAX+1.
constexpr int EMT = 2 * LMAX + 1;
constexpr int EAB_SZ = (LMAX + 1) * (LMAX + 1) * EMT;

__device__ void pair_E(int la, int lb, double a, double b, double Ax, double Bx, double *E)
{
    double p = a + b;
    double Px = (a * Ax + b * Bx) / p;
    double XPA = Px - Ax, XPB = Px - Bx, XAB = Ax - Bx;
    double h = 0.5 / p;
    for (int k = 0; k < EAB_SZ; k++) E[k] = 0.0;
#define EE(i, j, t) E[((i) * (LMAX + 1) + (j)) * EMT + (t)]
    EE(0, 0, 0) = exp(-(a * b / p) * XAB * XAB);
    for (int i = 0; i <= la; i++)
        for (int j = 0; j <= lb; j++) {
            if (i == 0 && j == 0) continue;
            for (int t = 0; t <= i + j; t++) {
                double v;
                if (i > 0) {
                    v = XPA * EE(i - 1, j, t);
                    if (t > 0) v += h * EE(i - 1, j, t - 1);
                    if (t + 1 <= i - 1 + j) v += (t + 1) * EE(i - 1, j, t + 1);
                } else {
                    v = XPB * EE(i, j - 1, t);
                    if (t > 0) v += h * EE(i, j - 1, t - 1);
                    if (t + 1 <= i + j - 1) v += (t + 1) * EE(i, j - 1, t + 1);
                }
                EE(i, j, t) = v;
            }
        }
#undef EE
}

// single-centre Gaussian x^c e^{-g x^2}: E[c*(LMAX+1) + tau]
__device__ void single_E(int lc, double g, double *E)
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

constexpr int SR_WARPS = 2;
constexpr int SR_NT = 256;   // translations buffered per segment

size_t sr_warp_bytes(int L, int bc, int ncomp_max)
{
    size_t b = 2 * SR_NT * sizeof(int4) + 2 * (NBIN_MAX + 4) * sizeof(int);
    b = (b + 15) & ~(size_t)15;
    b += (3 * EAB_SZ + 3 * (LMAX + 1) * (LMAX + 1)) * sizeof(double);
    b += (size_t)bc * (ntuv(L) + ncomp_max) * sizeof(double);
    return (b + 15) & ~(size_t)15;
}

template <int L>
__global__ void __launch_bounds__(SR_WARPS * 32) k_sr3c(SRArgs A)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long item = A.item_begin + (long long)blockIdx.x * SR_WARPS + warp;
    if (item >= A.item_end) return;  // warp-uniform
    unsigned char *base = smem_raw + (size_t)warp * A.warp_bytes;
    int4 *Tl = (int4 *)base;
    int4 *Ts = Tl + SR_NT;
    int *cnt = (int *)(Ts + SR_NT);
    int *fill = cnt + NBIN_MAX + 4;
    double *Eab = (double *)(base + (((2 * SR_NT * sizeof(int4) + 2 * (NBIN_MAX + 4) * sizeof(int)) + 15) & ~(size_t)15));
    double *Ec = Eab + 3 * EAB_SZ;
    double *Rb = Ec + 3 * (LMAX + 1) * (LMAX + 1);
    double *O = Rb + A.bc * ntuv(L);
    constexpr int NR = ntuv(L);

    // the triple of this item: last triple with item_off <= item
    int lo = A.tri_begin, hi = A.tri_end - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (A.tri[mid].item_off <= item) lo = mid; else hi = mid - 1;
    }
    const SRTripleDev tr = A.tri[lo];
    const int di = (int)(item - tr.item_off);
    const int P = tr.P, mu = tr.mu, nu = tr.nu;
    const int lP = A.ax.l[P], lm = A.ao.l[mu], ln = A.ao.l[nu];
    const int ncP = (lP + 1) * (lP + 2) / 2, ncm = (lm + 1) * (lm + 2) / 2, ncn = (ln + 1) * (ln + 2) / 2;
    const int ncomp = ncP * ncm * ncn;
    const int *dv = A.dlist + 3 * (A.pair_doff[tr.pair] + di);
    const int d0 = dv[0], d1 = dv[1], d2 = dv[2];
    double Av[3], Bv[3], Cv[3], xr[3];
#pragma unroll
    for (int x = 0; x < 3; x++) {
        Av[x] = A.ao.cen[3 * mu + x];
        Bv[x] = A.ao.cen[3 * nu + x] + d0 * A.a[x] + d1 * A.a[3 + x] + d2 * A.a[6 + x];
        Cv[x] = A.ax.cen[3 * P + x];
    }
    double R12 = sqrt((Bv[0] - Av[0]) * (Bv[0] - Av[0]) + (Bv[1] - Av[1]) * (Bv[1] - Av[1]) +
                      (Bv[2] - Av[2]) * (Bv[2] - Av[2]));
    const double wsum = tr.amu + tr.anu;
#pragma unroll
    for (int x = 0; x < 3; x++) xr[x] = (tr.amu * Av[x] + tr.anu * Bv[x]) / wsum - Cv[x];
    int l0[3];
#pragma unroll
    for (int i = 0; i < 3; i++)
        l0[i] = __double2int_rn(xr[0] * A.bq[3 * i] + xr[1] * A.bq[3 * i + 1] + xr[2] * A.bq[3 * i + 2]);
    const int dt = bvk_bin(d0, d1, d2, A.nk);
    const double *win = A.win + tr.win_off;
    const double omega2 = A.omega * A.omega;

    int nT = 0;
    unsigned long long kept = 0;
    for (int b0 = 0; b0 < tr.nsph; b0 += 32) {
        const int idx = b0 + lane;
        bool acc = false;
        int li0 = 0, li1 = 0, li2 = 0;
        if (idx < tr.nsph) {
            li0 = l0[0] + A.sph[3 * idx];
            li1 = l0[1] + A.sph[3 * idx + 1];
            li2 = l0[2] + A.sph[3 * idx + 2];
            double r0 = xr[0] - (li0 * A.a[0] + li1 * A.a[3] + li2 * A.a[6]);
            double r1 = xr[1] - (li0 * A.a[1] + li1 * A.a[4] + li2 * A.a[7]);
            double r2 = xr[2] - (li0 * A.a[2] + li1 * A.a[5] + li2 * A.a[8]);
            double rc = sqrt(r0 * r0 + r1 * r1 + r2 * r2);
            if (rc <= tr.Rc_cut) {
                int w = (int)floor(rc * (1.0 / SCREEN_DR));
                if (w >= tr.nwin) w = tr.nwin - 1;
                acc = (R12 <= win[w]);
            }
        }
        const unsigned m = __ballot_sync(0xffffffffu, acc);
        if (acc) {
            int pos = nT + __popc(m & ((1u << lane) - 1u));
            Tl[pos] = make_int4(li0, li1, li2, bvk_bin(li0, li1, li2, A.nk));
        }
        nT += __popc(m);
        const bool last = (b0 + 32 >= tr.nsph);
        if (nT > SR_NT - 32 || (last && nT > 0)) {
            __syncwarp();
            kept += nT;
            // ---- stable counting sort by BvK cell of l
            for (int b = lane; b < A.Nk + 1; b += 32) { cnt[b] = 0; fill[b] = 0; }
            __syncwarp();
            for (int t = lane; t < nT; t += 32) atomicAdd(&cnt[Tl[t].w + 1], 1);
            __syncwarp();
            if (lane == 0)
                for (int b = 1; b <= A.Nk; b++) cnt[b] += cnt[b - 1];   // cnt[b] = start of bin b
            __syncwarp();
            for (int t0 = 0; t0 < nT; t0 += 32) {
                const int t = t0 + lane;
                const int bin = (t < nT) ? Tl[t].w : -1 - lane;
                const unsigned act = __ballot_sync(0xffffffffu, t < nT);
                const unsigned peers = __match_any_sync(0xffffffffu, bin);
                if (t < nT) {
                    int rank = __popc(peers & act & ((1u << lane) - 1u));
                    Ts[cnt[bin] + fill[bin] + rank] = Tl[t];
                }
                __syncwarp();
                if (t < nT && (peers & act & ((1u << lane) - 1u)) == 0) fill[bin] += __popc(peers & act);
                __syncwarp();
            }
            // ---- bins in chunks of bc
            for (int c0 = 0; c0 < A.Nk; c0 += A.bc) {
                const int nb = min(A.bc, A.Nk - c0);
                const int r0 = cnt[c0], r1 = cnt[c0 + nb];
                if (r0 == r1) continue;
                for (int o = lane; o < nb * ncomp; o += 32) O[o] = 0.0;
                for (int k = 0; k < A.ax.nprim[P]; k++)
                    for (int i = 0; i < A.ao.nprim[mu]; i++)
                        for (int j = 0; j < A.ao.nprim[nu]; j++) {
                            const int ok = A.ax.poff[P] + k, oi = A.ao.poff[mu] + i, oj = A.ao.poff[nu] + j;
                            const double g = A.ax.exps[ok], ea = A.ao.exps[oi], eb = A.ao.exps[oj];
                            if (lane < 3) pair_E(lm, ln, ea, eb, Av[lane], Bv[lane], Eab + lane * EAB_SZ);
                            else if (lane < 6) single_E(lP, g, Ec + (lane - 3) * (LMAX + 1) * (LMAX + 1));
                            for (int o = lane; o < nb * NR; o += 32) Rb[o] = 0.0;
                            const double p = ea + eb;
                            const double alpha = p * g / (p + g);
                            double Pc[3];
#pragma unroll
                            for (int x = 0; x < 3; x++) Pc[x] = (ea * Av[x] + eb * Bv[x]) / p - Cv[x];
                            __syncwarp();
                            // contiguous slice of the sorted translations per lane
                            const int per = (r1 - r0 + 31) >> 5;
                            const int ta = r0 + lane * per, tb = min(ta + per, r1);
                            double accR[NR];
#pragma unroll
                            for (int q = 0; q < NR; q++) accR[q] = 0.0;
                            int cur = -1;
                            for (int tt = ta; tt < tb; tt++) {
                                const int4 e = Ts[tt];
                                if (e.w != cur) {
                                    if (cur >= 0) {
#pragma unroll
                                        for (int q = 0; q < NR; q++) {
                                            atomicAdd(&Rb[(cur - c0) * NR + q], accR[q]);
                                            accR[q] = 0.0;
                                        }
                                    }
                                    cur = e.w;
                                }
                                const double X = Pc[0] - (e.x * A.a[0] + e.y * A.a[3] + e.z * A.a[6]);
                                const double Y = Pc[1] - (e.x * A.a[1] + e.y * A.a[4] + e.z * A.a[7]);
                                const double Z = Pc[2] - (e.x * A.a[2] + e.y * A.a[5] + e.z * A.a[8]);
                                const double T = alpha * (X * X + Y * Y + Z * Z);
                                double r[NR];
                                hermite_R<L>(alpha, omega2, T, X, Y, Z, r);
#pragma unroll
                                for (int q = 0; q < NR; q++) accR[q] += r[q];
                            }
                            if (cur >= 0) {
#pragma unroll
                                for (int q = 0; q < NR; q++) atomicAdd(&Rb[(cur - c0) * NR + q], accR[q]);
                            }
                            __syncwarp();
                            const double pref = 2.0 * KPI2_5 / (p * g * sqrt(p + g)) * A.ax.cn[ok] * A.ao.cn[oi] *
                                                A.ao.cn[oj] * ((lP & 1) ? -1.0 : 1.0);
                            for (int o = lane; o < nb * ncomp; o += 32) {
                                const int bb = o / ncomp, comp = o - bb * ncomp;
                                const int ic = comp / (ncm * ncn), ia = (comp / ncn) % ncm, ib = comp % ncn;
                                const signed char *cc = c_cart[lP][ic], *ca = c_cart[lm][ia], *cb = c_cart[ln][ib];
                                const double *rb = Rb + bb * NR;
                                double sum = 0.0;
                                for (int t = 0; t <= ca[0] + cb[0]; t++) {
                                    const double ex = Eab[(ca[0] * (LMAX + 1) + cb[0]) * EMT + t];
                                    for (int u = 0; u <= ca[1] + cb[1]; u++) {
                                        const double exy = ex * Eab[EAB_SZ + (ca[1] * (LMAX + 1) + cb[1]) * EMT + u];
                                        for (int v = 0; v <= ca[2] + cb[2]; v++) {
                                            const double e = exy * Eab[2 * EAB_SZ + (ca[2] * (LMAX + 1) + cb[2]) * EMT + v];
                                            for (int ta2 = cc[0] & 1; ta2 <= cc[0]; ta2 += 2) {
                                                const double e1 = e * Ec[cc[0] * (LMAX + 1) + ta2];
                                                for (int ua = cc[1] & 1; ua <= cc[1]; ua += 2) {
                                                    const double e2 = e1 * Ec[(LMAX + 1) * (LMAX + 1) + cc[1] * (LMAX + 1) + ua];
                                                    for (int va = cc[2] & 1; va <= cc[2]; va += 2) {
                                                        const double e3 = e2 * Ec[2 * (LMAX + 1) * (LMAX + 1) + cc[2] * (LMAX + 1) + va];
                                                        sum = fma(e3, rb[ridx(t + ta2, u + ua, v + va)], sum);
                                                    }
                                                }
                                            }
                                        }
                                    }
                                }
                                O[o] = fma(pref, sum, O[o]);
                            }
                            __syncwarp();
                        }
                // ---- add the blocks of this chunk to X
                const long long pf = A.ax.foff[P] - A.pfunc0, mf = A.ao.foff[mu], nf = A.ao.foff[nu];
                for (int o = lane; o < nb * ncomp; o += 32) {
                    const int bb = o / ncomp, comp = o - bb * ncomp;
                    const int ic = comp / (ncm * ncn), ia = (comp / ncn) % ncm, ib = comp % ncn;
                    const long long dst = (long long)(c0 + bb) * A.s_lt + (long long)dt * A.s_dt + (pf + ic) * A.s_P +
                                          (mf + ia) * A.s_mu + (nf + ib) * A.s_nu;
                    if (O[o] != 0.0) atomicAdd(&A.X[dst], O[o]);
                }
                __syncwarp();
            }
            nT = 0;
        }
    }
    if (lane == 0 && A.term_count) {
        atomicAdd(A.term_count + L, kept);
        atomicAdd(A.term_count + LTOT_MAX + 1, kept * (unsigned long long)ncomp);
    }
}

typedef void (*SRKern)(SRArgs);
static SRKern sr_kernels[LTOT_MAX + 1] = {k_sr3c<0>, k_sr3c<1>, k_sr3c<2>, k_sr3c<3>, k_sr3c<4>,
                                          k_sr3c<5>, k_sr3c<6>, k_sr3c<7>, k_sr3c<8>, k_sr3c<9>};

int launch_sr(int L, SRArgs args, int ncomp_max, cudaStream_t st)
{
    long long n = args.item_end - args.item_begin;
    if (n <= 0) return RSGDF_OK;
    int bc = 3072 / (ntuv(L) + ncomp_max);
    bc = bc < 1 ? 1 : (bc > 16 ? 16 : bc);
    args.bc = bc;
    size_t wb = sr_warp_bytes(L, bc, ncomp_max);
    args.warp_bytes = (int)wb;
    size_t smem = wb * SR_WARPS;
    if (cudaFuncSetAttribute(sr_kernels[L], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return RSGDF_EDEVICE;
    long long grid = (n + SR_WARPS - 1) / SR_WARPS;
    while (grid > 0) {
        long long g = grid > 2000000000LL ? 2000000000LL : grid;
        sr_kernels[L]<<<(unsigned)g, SR_WARPS * 32, smem, st>>>(args);
        if (cudaGetLastError() != cudaSuccess) return RSGDF_EDEVICE;
        args.item_begin += g * SR_WARPS;
        grid -= g;
    }
    return RSGDF_OK;
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
