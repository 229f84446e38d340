// Reciprocal-space part of RSGDF (Eqs. VPmunu_LR and AFT_pairden), the Bloch
// phase contractions of folded lattice sums (Eq. BvK_latsum_LR), the FP64
// Cholesky factorisation of j2c, and the FP64 throughput probe.
#include <cuda_runtime.h>

#include <algorithm>

#include "k_common.cuh"

namespace rsgdf {

constexpr int EMT = 2 * LMAX + 1;
constexpr int EAB_SZ = (LMAX + 1) * (LMAX + 1) * EMT;

__device__ static void pair_E_g(int la, int lb, double a, double b, double Ax, double Bx, double *E)
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

__device__ __forceinline__ void qvec(const GArgs &G, int ig, double q[3])
{
    double n0 = G.g[3 * ig] + G.f12[0], n1 = G.g[3 * ig + 1] + G.f12[1], n2 = G.g[3 * ig + 2] + G.f12[2];
#pragma unroll
    for (int x = 0; x < 3; x++) q[x] = n0 * G.b[x] + n1 * G.b[3 + x] + n2 * G.b[6 + x];
}

// W[G][P] = 4 pi/Omega e^{-q^2/4w^2}/q^2 conj(chi^_P(q)) (0 at q = 0) and,
// when F != NULL, F[G][P] = chi^_P(q).  chi^ of x^c e^{-g r^2} at C:
// (pi/g)^{3/2} e^{-q^2/4g} e^{-iq.C} prod_x sum_tau E^{c_x}_tau (-i q_x)^tau.
__global__ void k_aux_ft(GArgs G, DevShells ax, int s0, int s1, int pfunc0, int nP, double *W, double *F)
{
    int ig = blockIdx.x * blockDim.x + threadIdx.x;
    int P = s0 + blockIdx.y;
    if (ig >= G.NG || P >= s1) return;
    double q[3];
    qvec(G, ig, q);
    double q2 = q[0] * q[0] + q[1] * q[1] + q[2] * q[2];
    double w = 0.0;
    if (q2 >= 1e-14) {
        w = 4.0 * KPI / G.vol / q2;
        if (!G.full_coulomb) w *= exp(-q2 / (4.0 * G.omega * G.omega));
    }
    int l = ax.l[P], nc = (l + 1) * (l + 2) / 2;
    double re[NC_MAX], im[NC_MAX];
    for (int c = 0; c < nc; c++) { re[c] = 0.0; im[c] = 0.0; }
    const double *C = ax.cen + 3 * P;
    double qC = q[0] * C[0] + q[1] * C[1] + q[2] * C[2];
    double sc, cc;
    sincos(qC, &sc, &cc);
    for (int k = 0; k < ax.nprim[P]; k++) {
        int o = ax.poff[P] + k;
        double g = ax.exps[o];
        double E[(LMAX + 1) * (LMAX + 1)];
        double h = 0.5 / g;
        for (int z = 0; z < (LMAX + 1) * (LMAX + 1); z++) E[z] = 0.0;
        E[0] = 1.0;
        for (int c = 1; c <= l; c++)
            for (int t = 0; t <= c; t++) {
                double v = 0.0;
                if (t > 0) v += h * E[(c - 1) * (LMAX + 1) + t - 1];
                if (t + 1 <= c - 1) v += (t + 1) * E[(c - 1) * (LMAX + 1) + t + 1];
                E[c * (LMAX + 1) + t] = v;
            }
        // 1D polynomials f_x(c) = sum_tau E^c_tau (-i q_x)^tau
        double pr[3][LMAX + 1], pi[3][LMAX + 1];
        for (int x = 0; x < 3; x++)
            for (int c = 0; c <= l; c++) {
                double ar = 0.0, ai = 0.0, wr = 1.0, wi = 0.0;
                for (int t = 0; t <= c; t++) {
                    double e = E[c * (LMAX + 1) + t];
                    ar += e * wr;
                    ai += e * wi;
                    double nr = wi * q[x], ni = -wr * q[x];   // times (-i q)
                    wr = nr;
                    wi = ni;
                }
                pr[x][c] = ar;
                pi[x][c] = ai;
            }
        double base = ax.cn[o] * pow(KPI / g, 1.5) * exp(-q2 / (4.0 * g));
        for (int ic = 0; ic < nc; ic++) {
            const signed char *c = c_cart[l][ic];
            double ar = pr[0][c[0]], ai = pi[0][c[0]];
            double br = ar * pr[1][c[1]] - ai * pi[1][c[1]], bi = ar * pi[1][c[1]] + ai * pr[1][c[1]];
            double cr = br * pr[2][c[2]] - bi * pi[2][c[2]], ci = br * pi[2][c[2]] + bi * pr[2][c[2]];
            re[ic] += base * cr;
            im[ic] += base * ci;
        }
    }
    int pf = ax.foff[P] - pfunc0;
    for (int ic = 0; ic < nc; ic++) {
        // times e^{-i q.C}
        double vr = re[ic] * cc + im[ic] * sc, vi = im[ic] * cc - re[ic] * sc;
        long long o = (long long)ig * nP + pf + ic;
        W[2 * o] = w * vr;
        W[2 * o + 1] = -w * vi;
        if (F) {
            F[2 * o] = vr;
            F[2 * o + 1] = vi;
        }
    }
}

int launch_aux_ft(const GArgs &G, DevShells ax, int s0, int s1, int pfunc0, int nP, double *W, double *F,
                  cudaStream_t st)
{
    (void)nP;
    dim3 grid((G.NG + 127) / 128, s1 - s0);
    k_aux_ft<<<grid, 128, 0, st>>>(G, ax, s0, s1, pfunc0, nP, W, F);
    return cudaGetLastError() == cudaSuccess ? RSGDF_OK : RSGDF_EDEVICE;
}

// ---------------------------------------------------------------------------
// Pair transforms (Eq. AFT_pairden) folded on the BvK cells of d.
//
// Entry = (AO shell pair, d, primitive pair): its Hermite coefficients, centre
// and constants do not depend on G or k12 and are written once per call by
// k_pair_prep.  Entry layout (doubles, compact per shell pair):
//   [0..2] P (product centre), [3] 1/(4p), [4] c_i c_j (pi/p)^{3/2}, [5] p,
//   [6] c_i c_j, [7] unused, then for x, y, z: E^{ab}_t for a <= lm, b <= ln, t <= a+b, packed by
//   (a, b) with offset eoff(a, b) = sum of (a'+b'+1) over earlier (a', b').
// Entries of one (pair, BvK cell) are contiguous and ordered by primitive pair.
// ---------------------------------------------------------------------------
__host__ __device__ inline int pair_e1(int lm, int ln) { return (lm + 1) * (ln + 1) * (lm + ln + 2) / 2; }

__device__ __forceinline__ int eoff(int a, int b, int ln)
{
    // sum over (a', b') < (a, b) in row-major order of (a' + b' + 1)
    int o = 0;
    for (int x = 0; x < a; x++) o += (ln + 1) * (2 * x + ln + 2) / 2;
    for (int y = 0; y < b; y++) o += a + y + 1;
    return o;
}

__global__ void k_pair_prep(DevShells ao, int nshell, const PairEntry *ent, int nent, const int *dlist,
                            const double *a9, double *tab, float *tab32, const double *b9, float2 *uph)
{
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nent) return;
    const PairEntry en = ent[e];
    const int mu = en.pair / nshell, nu = en.pair % nshell;
    const int lm = ao.l[mu], ln = ao.l[nu];
    const int oi = ao.poff[mu] + en.i, oj = ao.poff[nu] + en.j;
    const double a = ao.exps[oi], b = ao.exps[oj], p = a + b;
    const int d0 = dlist[3 * en.d], d1 = dlist[3 * en.d + 1], d2 = dlist[3 * en.d + 2];
    double *out = tab + en.off;
    double E[EAB_SZ];
    const int n1 = pair_e1(lm, ln);
    for (int x = 0; x < 3; x++) {
        const double Ax = ao.cen[3 * mu + x];
        const double Bx = ao.cen[3 * nu + x] + d0 * a9[x] + d1 * a9[3 + x] + d2 * a9[6 + x];
        out[x] = (a * Ax + b * Bx) / p;
        pair_E_g(lm, ln, a, b, Ax, Bx, E);
        double *o = out + ENT_HDR + x * n1;
        int k = 0;
        for (int ia = 0; ia <= lm; ia++)
            for (int ib = 0; ib <= ln; ib++)
                for (int t = 0; t <= ia + ib; t++) o[k++] = E[(ia * (LMAX + 1) + ib) * EMT + t];
    }
    out[3] = 0.25 / p;
    out[4] = ao.cn[oi] * ao.cn[oj] * KPI * sqrt(KPI) / (p * sqrt(p));
    out[5] = p;
    out[6] = ao.cn[oi] * ao.cn[oj];
    out[7] = 0.0;
    if (tab32) {
        // FP32 copy (same offsets) for the mixed-precision transforms
        float *o32 = tab32 + en.off;
        for (int k = 0; k < ENT_HDR + 3 * n1; k++) o32[k] = (float)out[k];
        // unit phasors e^{-i b_j.P}, argument reduced in FP64
        for (int j = 0; j < 3; j++) {
            const double ph = b9[3 * j] * out[0] + b9[3 * j + 1] * out[1] + b9[3 * j + 2] * out[2];
            const double r = ph - 2.0 * KPI * rint(ph * (0.5 / KPI));
            double s, c;
            sincos(r, &s, &c);
            uph[3 * e + j] = make_float2((float)c, (float)-s);
        }
    }
}

int launch_pair_prep(DevShells ao, int nshell, const PairEntry *ent, int nent, const int *dlist, const double *a9,
                     double *tab, float *tab32, const double *b9, float2 *uph, cudaStream_t st)
{
    if (nent <= 0) return RSGDF_OK;
    k_pair_prep<<<(nent + 127) / 128, 128, 0, st>>>(ao, nshell, ent, nent, dlist, a9, tab, tab32, b9, uph);
    return cudaGetLastError() == cudaSuccess ? RSGDF_OK : RSGDF_EDEVICE;
}

// Y[dt][G][mu][nu] = sum over the entries of (pair, dt) of
//   c e^{-q^2/4p} e^{-i q.P} prod_x sum_t E^x_t (-i q_x)^t
constexpr int AFT_THREADS = 128;

__global__ void __launch_bounds__(AFT_THREADS) k_aft(GArgs G, DevShells ao, int nshell, int nao, const PairEntry *ent,
                                                     const int *seg, const double *tab, int Nk, double *Y)
{
    const int ig = blockIdx.x * AFT_THREADS + threadIdx.x;
    const int dt = blockIdx.y, pr = blockIdx.z;
    if (ig >= G.NG) return;
    const int mu = pr / nshell, nu = pr % nshell;
    const int lm = ao.l[mu], ln = ao.l[nu];
    const int ncm = (lm + 1) * (lm + 2) / 2, ncn = (ln + 1) * (ln + 2) / 2;
    const int n1 = pair_e1(lm, ln);
    double q[3];
    qvec(G, ig, q);
    const double q2 = q[0] * q[0] + q[1] * q[1] + q[2] * q[2];
    // powers q_x^t, t <= 2 LMAX
    double qp[3][EMT];
    for (int x = 0; x < 3; x++) {
        qp[x][0] = 1.0;
        for (int t = 1; t <= lm + ln; t++) qp[x][t] = qp[x][t - 1] * q[x];
    }
    double accr[NC_MAX * NC_MAX], acci[NC_MAX * NC_MAX];
    for (int z = 0; z < ncm * ncn; z++) { accr[z] = 0.0; acci[z] = 0.0; }
    double last_inv4p = -1.0, gauss = 0.0;
    const int e0 = seg[pr * Nk + dt], e1 = seg[pr * Nk + dt + 1];
    for (int e = e0; e < e1; e++) {
        const double *en = tab + ent[e].off;
        const double inv4p = en[3];
        if (inv4p != last_inv4p) {
            gauss = exp(-q2 * inv4p);
            last_inv4p = inv4p;
        }
        double sp, cp;
        sincos(q[0] * en[0] + q[1] * en[1] + q[2] * en[2], &sp, &cp);
        const double base = en[4] * gauss;
        const double br = base * cp, bi = -base * sp;   // base e^{-i q.P}
        // f_x(a, b) = sum_t E_t (-i q_x)^t: even t real, odd t imaginary
        double fr[3][(LMAX + 1) * (LMAX + 1)], fi[3][(LMAX + 1) * (LMAX + 1)];
        for (int x = 0; x < 3; x++) {
            const double *Ex = en + ENT_HDR + x * n1;
            int k = 0;
            for (int a = 0; a <= lm; a++)
                for (int b = 0; b <= ln; b++) {
                    double re = 0.0, im = 0.0;
                    for (int t = 0; t <= a + b; t++, k++) {
                        // (-i)^t = 1, -i, -1, i
                        const double v = Ex[k] * qp[x][t];
                        switch (t & 3) {
                        case 0: re += v; break;
                        case 1: im -= v; break;
                        case 2: re -= v; break;
                        default: im += v; break;
                        }
                    }
                    fr[x][a * (LMAX + 1) + b] = re;
                    fi[x][a * (LMAX + 1) + b] = im;
                }
        }
        for (int ia = 0; ia < ncm; ia++)
            for (int ib = 0; ib < ncn; ib++) {
                const signed char *ca = c_cart[lm][ia], *cb = c_cart[ln][ib];
                const int i0 = ca[0] * (LMAX + 1) + cb[0], i1 = ca[1] * (LMAX + 1) + cb[1], i2 = ca[2] * (LMAX + 1) + cb[2];
                const double xr = fr[0][i0] * fr[1][i1] - fi[0][i0] * fi[1][i1];
                const double xi = fr[0][i0] * fi[1][i1] + fi[0][i0] * fr[1][i1];
                const double yr = xr * fr[2][i2] - xi * fi[2][i2];
                const double yi = xr * fi[2][i2] + xi * fr[2][i2];
                accr[ia * ncn + ib] += yr * br - yi * bi;
                acci[ia * ncn + ib] += yr * bi + yi * br;
            }
    }
    const int mf = ao.foff[mu], nf = ao.foff[nu];
    for (int ia = 0; ia < ncm; ia++)
        for (int ib = 0; ib < ncn; ib++) {
            long long o = (((long long)dt * G.NG + ig) * nao + mf + ia) * nao + nf + ib;
            Y[2 * o] = accr[ia * ncn + ib];
            Y[2 * o + 1] = acci[ia * ncn + ib];
        }
}

int launch_aft(const GArgs &G, DevShells ao, int nshell, int nao, const PairEntry *ent, const int *seg,
               const double *tab, int Nk, double *Y, cudaStream_t st)
{
    dim3 grid((G.NG + AFT_THREADS - 1) / AFT_THREADS, Nk, nshell * nshell);
    k_aft<<<grid, AFT_THREADS, 0, st>>>(G, ao, nshell, nao, ent, seg, tab, Nk, Y);
    return cudaGetLastError() == cudaSuccess ? RSGDF_OK : RSGDF_EDEVICE;
}

// e^{-i f12.(b.P)} per entry for one k12 (argument in FP64, reduced)
__global__ void k_aft_phase0(const PairEntry *ent, int nent, const double *tab, double f0, double f1, double f2,
                             const double *b9, float2 *ph0)
{
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nent) return;
    const double *en = tab + ent[e].off;
    double th = 0.0;
    const double f[3] = {f0, f1, f2};
    for (int j = 0; j < 3; j++) th += f[j] * (b9[3 * j] * en[0] + b9[3 * j + 1] * en[1] + b9[3 * j + 2] * en[2]);
    const double r = th - 2.0 * KPI * rint(th * (0.5 / KPI));
    double s, c;
    sincos(r, &s, &c);
    ph0[e] = make_float2((float)c, (float)-s);
}

__device__ __forceinline__ float2 cmulf(float2 a, float2 b) { return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }

// integer power z^n of a unit phasor, |n| small (conjugate for n < 0)
__device__ __forceinline__ float2 cpowf(float2 z, int n)
{
    float2 r = make_float2(1.0f, 0.0f);
    const int a = n < 0 ? -n : n;
    for (int k = 0; k < a; k++) r = cmulf(r, z);
    if (n < 0) r.y = -r.y;
    return r;
}

// Mixed-precision pair transforms: FP32 arithmetic; e^{-i q.P} =
// e^{-i f.(b.P)} prod_j (e^{-i b_j.P})^{n_j} from FP64-accurate phasors.
// One (G point, BvK cell dt, AO shell pair) of the mixed pair transform, for
// the angular momenta LM, LN as compile-time constants: the accumulators and
// the per-axis polynomial factors then live in registers.
template <int LM, int LN>
__device__ __forceinline__ void aft_f32_body(const GArgs &G, const DevShells &ao, int nao, int mu, int nu, int ig,
                                             int dt, int pr, const PairEntry *ent, const int *seg, const float *tab32,
                                             const float2 *uph, const float2 *ph0, int Nk, float *Bp, int nnt, int nkc)
{
    constexpr int ncm = (LM + 1) * (LM + 2) / 2, ncn = (LN + 1) * (LN + 2) / 2;
    constexpr int n1 = (LM + 1) * (LN + 1) * (LM + LN + 2) / 2;
    const int gn[3] = {G.g[3 * ig], G.g[3 * ig + 1], G.g[3 * ig + 2]};
    float q[3];
    for (int x = 0; x < 3; x++)
        q[x] = (float)((gn[0] + G.f12[0]) * G.b[x] + (gn[1] + G.f12[1]) * G.b[3 + x] + (gn[2] + G.f12[2]) * G.b[6 + x]);
    const float q2 = q[0] * q[0] + q[1] * q[1] + q[2] * q[2];
    float qp[3][LM + LN + 1];
#pragma unroll
    for (int x = 0; x < 3; x++) {
        qp[x][0] = 1.0f;
#pragma unroll
        for (int t = 1; t <= LM + LN; t++) qp[x][t] = qp[x][t - 1] * q[x];
    }
    float accr[ncm * ncn], acci[ncm * ncn];
#pragma unroll
    for (int z = 0; z < ncm * ncn; z++) { accr[z] = 0.0f; acci[z] = 0.0f; }
    float last_inv4p = -1.0f, gauss = 0.0f;
    const int e0 = seg[pr * Nk + dt], e1 = seg[pr * Nk + dt + 1];
    for (int e = e0; e < e1; e++) {
        const float *en = tab32 + ent[e].off;
        const float inv4p = en[3];
        if (inv4p != last_inv4p) {
            gauss = expf(-q2 * inv4p);
            last_inv4p = inv4p;
        }
        float2 ph = ph0[e];
        ph = cmulf(ph, cpowf(uph[3 * e], gn[0]));
        ph = cmulf(ph, cpowf(uph[3 * e + 1], gn[1]));
        ph = cmulf(ph, cpowf(uph[3 * e + 2], gn[2]));
        const float base = en[4] * gauss;
        const float br = base * ph.x, bi = base * ph.y;
        // per axis and (a, b): sum_t E^{ab}_t (-i q)^t
        float fr[3][(LM + 1) * (LN + 1)], fi[3][(LM + 1) * (LN + 1)];
#pragma unroll
        for (int x = 0; x < 3; x++) {
            const float *Ex = en + ENT_HDR + x * n1;
            int k = 0;
#pragma unroll
            for (int a = 0; a <= LM; a++)
#pragma unroll
                for (int b = 0; b <= LN; b++) {
                    float re = 0.0f, im = 0.0f;
#pragma unroll
                    for (int t = 0; t <= a + b; t++, k++) {
                        const float v = Ex[k] * qp[x][t];
                        if ((t & 3) == 0) re += v;
                        else if ((t & 3) == 1) im -= v;
                        else if ((t & 3) == 2) re -= v;
                        else im += v;
                    }
                    fr[x][a * (LN + 1) + b] = re;
                    fi[x][a * (LN + 1) + b] = im;
                }
        }
#pragma unroll
        for (int ia = 0; ia < ncm; ia++)
#pragma unroll
            for (int ib = 0; ib < ncn; ib++) {
                const signed char *ca = c_cart[LM][ia], *cb = c_cart[LN][ib];
                const int i0 = ca[0] * (LN + 1) + cb[0], i1 = ca[1] * (LN + 1) + cb[1], i2 = ca[2] * (LN + 1) + cb[2];
                const float xr = fr[0][i0] * fr[1][i1] - fi[0][i0] * fi[1][i1];
                const float xi = fr[0][i0] * fi[1][i1] + fi[0][i0] * fr[1][i1];
                const float yr = xr * fr[2][i2] - xi * fi[2][i2];
                const float yi = xr * fi[2][i2] + xi * fr[2][i2];
                accr[ia * ncn + ib] += yr * br - yi * bi;
                acci[ia * ncn + ib] += yr * bi + yi * br;
            }
    }
    // written straight into the split-TF32 operand tiles of the tensor-core contraction
    const int mf = ao.foff[mu], nf = ao.foff[nu];
#pragma unroll
    for (int ia = 0; ia < ncm; ia++)
#pragma unroll
        for (int ib = 0; ib < ncn; ib++) {
            const int n = (mf + ia) * nao + nf + ib;
            tc_put_b(Bp, nnt, nkc, dt, n, ig, 0, accr[ia * ncn + ib]);
            tc_put_b(Bp, nnt, nkc, dt, n, ig, 1, acci[ia * ncn + ib]);
        }
}

// Pairs whose shells both have l <= 2: one instantiation per (lm, ln), chosen
// per block (the pair is uniform over a block).  Pairs with an f shell are
// left to k_aft_f32_f.
__global__ void __launch_bounds__(AFT_THREADS) k_aft_f32(GArgs G, DevShells ao, int nshell, int nao,
                                                         const PairEntry *ent, const int *seg, const float *tab32,
                                                         const float2 *uph, const float2 *ph0, int Nk, float *Bp,
                                                         int nnt, int nkc)
{
    const int ig = blockIdx.x * AFT_THREADS + threadIdx.x;
    const int dt = blockIdx.y, pr = blockIdx.z;
    if (ig >= G.NG) return;
    const int mu = pr / nshell, nu = pr % nshell;
#define AFT_CASE(a, b)                                                                                          \
    case (a) * (LMAX + 1) + (b):                                                                                \
        aft_f32_body<a, b>(G, ao, nao, mu, nu, ig, dt, pr, ent, seg, tab32, uph, ph0, Nk, Bp, nnt, nkc);    \
        break;
    switch (ao.l[mu] * (LMAX + 1) + ao.l[nu]) {
        AFT_CASE(0, 0) AFT_CASE(0, 1) AFT_CASE(0, 2)
        AFT_CASE(1, 0) AFT_CASE(1, 1) AFT_CASE(1, 2)
        AFT_CASE(2, 0) AFT_CASE(2, 1) AFT_CASE(2, 2)
        default: break;
    }
#undef AFT_CASE
}

// Pairs with an f shell: the same transform with runtime loop bounds.
__global__ void __launch_bounds__(AFT_THREADS) k_aft_f32_f(GArgs G, DevShells ao, int nshell, int nao,
                                                           const PairEntry *ent, const int *seg, const float *tab32,
                                                           const float2 *uph, const float2 *ph0, int Nk, float *Bp,
                                                           int nnt, int nkc)
{
    const int ig = blockIdx.x * AFT_THREADS + threadIdx.x;
    const int dt = blockIdx.y, pr = blockIdx.z;
    if (ig >= G.NG) return;
    const int mu = pr / nshell, nu = pr % nshell;
    const int lm = ao.l[mu], ln = ao.l[nu];
    if (lm < 3 && ln < 3) return;
    const int ncm = (lm + 1) * (lm + 2) / 2, ncn = (ln + 1) * (ln + 2) / 2;
    const int n1 = pair_e1(lm, ln);
    const int gn[3] = {G.g[3 * ig], G.g[3 * ig + 1], G.g[3 * ig + 2]};
    float q[3];
    for (int x = 0; x < 3; x++)
        q[x] = (float)((gn[0] + G.f12[0]) * G.b[x] + (gn[1] + G.f12[1]) * G.b[3 + x] + (gn[2] + G.f12[2]) * G.b[6 + x]);
    const float q2 = q[0] * q[0] + q[1] * q[1] + q[2] * q[2];
    float qp[3][EMT];
    for (int x = 0; x < 3; x++) {
        qp[x][0] = 1.0f;
        for (int t = 1; t <= lm + ln; t++) qp[x][t] = qp[x][t - 1] * q[x];
    }
    float accr[NC_MAX * NC_MAX], acci[NC_MAX * NC_MAX];
    for (int z = 0; z < ncm * ncn; z++) { accr[z] = 0.0f; acci[z] = 0.0f; }
    float last_inv4p = -1.0f, gauss = 0.0f;
    const int e0 = seg[pr * Nk + dt], e1 = seg[pr * Nk + dt + 1];
    for (int e = e0; e < e1; e++) {
        const float *en = tab32 + ent[e].off;
        const float inv4p = en[3];
        if (inv4p != last_inv4p) {
            gauss = expf(-q2 * inv4p);
            last_inv4p = inv4p;
        }
        float2 ph = ph0[e];
        ph = cmulf(ph, cpowf(uph[3 * e], gn[0]));
        ph = cmulf(ph, cpowf(uph[3 * e + 1], gn[1]));
        ph = cmulf(ph, cpowf(uph[3 * e + 2], gn[2]));
        const float base = en[4] * gauss;
        const float br = base * ph.x, bi = base * ph.y;
        float fr[3][(LMAX + 1) * (LMAX + 1)], fi[3][(LMAX + 1) * (LMAX + 1)];
        for (int x = 0; x < 3; x++) {
            const float *Ex = en + ENT_HDR + x * n1;
            int k = 0;
            for (int a = 0; a <= lm; a++)
                for (int b = 0; b <= ln; b++) {
                    float re = 0.0f, im = 0.0f;
                    for (int t = 0; t <= a + b; t++, k++) {
                        const float v = Ex[k] * qp[x][t];
                        switch (t & 3) {
                        case 0: re += v; break;
                        case 1: im -= v; break;
                        case 2: re -= v; break;
                        default: im += v; break;
                        }
                    }
                    fr[x][a * (LMAX + 1) + b] = re;
                    fi[x][a * (LMAX + 1) + b] = im;
                }
        }
        for (int ia = 0; ia < ncm; ia++)
            for (int ib = 0; ib < ncn; ib++) {
                const signed char *ca = c_cart[lm][ia], *cb = c_cart[ln][ib];
                const int i0 = ca[0] * (LMAX + 1) + cb[0], i1 = ca[1] * (LMAX + 1) + cb[1], i2 = ca[2] * (LMAX + 1) + cb[2];
                const float xr = fr[0][i0] * fr[1][i1] - fi[0][i0] * fi[1][i1];
                const float xi = fr[0][i0] * fi[1][i1] + fi[0][i0] * fr[1][i1];
                const float yr = xr * fr[2][i2] - xi * fi[2][i2];
                const float yi = xr * fi[2][i2] + xi * fr[2][i2];
                accr[ia * ncn + ib] += yr * br - yi * bi;
                acci[ia * ncn + ib] += yr * bi + yi * br;
            }
    }
    const int mf = ao.foff[mu], nf = ao.foff[nu];
    for (int ia = 0; ia < ncm; ia++)
        for (int ib = 0; ib < ncn; ib++) {
            const int n = (mf + ia) * nao + nf + ib;
            tc_put_b(Bp, nnt, nkc, dt, n, ig, 0, accr[ia * ncn + ib]);
            tc_put_b(Bp, nnt, nkc, dt, n, ig, 1, acci[ia * ncn + ib]);
        }
}

int launch_aft_f32(const GArgs &G, DevShells ao, int nshell, int nao, const PairEntry *ent, int nent, const int *seg,
                   const double *tab, const float *tab32, const double *b9, const float2 *uph, float2 *ph0, int Nk,
                   float *Bp, int lmax_ao, cudaStream_t st)
{
    const int nnt = (nao * nao + TC_N - 1) / TC_N, nkc = (G.NG + TC_KC - 1) / TC_KC;
    k_aft_phase0<<<(nent + 127) / 128, 128, 0, st>>>(ent, nent, tab, G.f12[0], G.f12[1], G.f12[2], b9, ph0);
    dim3 grid((G.NG + AFT_THREADS - 1) / AFT_THREADS, Nk, nshell * nshell);
    k_aft_f32<<<grid, AFT_THREADS, 0, st>>>(G, ao, nshell, nao, ent, seg, tab32, uph, ph0, Nk, Bp, nnt, nkc);
    if (lmax_ao >= 3)
        k_aft_f32_f<<<grid, AFT_THREADS, 0, st>>>(G, ao, nshell, nao, ent, seg, tab32, uph, ph0, Nk, Bp, nnt, nkc);
    return cudaGetLastError() == cudaSuccess ? RSGDF_OK : RSGDF_EDEVICE;
}

// Folded overlaps Sf[dt][mu][nu] = sum over the entries of (pair, dt) of
// c prod_x E^x_0 (the transform at q = 0); one thread per (pair, dt).
__global__ void k_ovlp_fold(DevShells ao, int nshell, int nao, const PairEntry *ent, const int *seg,
                            const double *tab, int Nk, double *Sf)
{
    int id = blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= nshell * nshell * Nk) return;
    const int pr = id / Nk, dt = id % Nk;
    const int mu = pr / nshell, nu = pr % nshell;
    const int lm = ao.l[mu], ln = ao.l[nu], ncm = (lm + 1) * (lm + 2) / 2, ncn = (ln + 1) * (ln + 2) / 2;
    const int n1 = pair_e1(lm, ln);
    double acc[NC_MAX * NC_MAX];
    for (int z = 0; z < ncm * ncn; z++) acc[z] = 0.0;
    for (int e = seg[pr * Nk + dt]; e < seg[pr * Nk + dt + 1]; e++) {
        const double *en = tab + ent[e].off;
        for (int ia = 0; ia < ncm; ia++)
            for (int ib = 0; ib < ncn; ib++) {
                const signed char *ca = c_cart[lm][ia], *cb = c_cart[ln][ib];
                double v = en[4];
                for (int x = 0; x < 3; x++) v *= en[ENT_HDR + x * n1 + eoff(ca[x], cb[x], ln)];
                acc[ia * ncn + ib] += v;
            }
    }
    const int mf = ao.foff[mu], nf = ao.foff[nu];
    for (int ia = 0; ia < ncm; ia++)
        for (int ib = 0; ib < ncn; ib++) Sf[((long long)dt * nao + mf + ia) * nao + nf + ib] = acc[ia * ncn + ib];
}

int launch_ovlp_fold(DevShells ao, int nshell, int nao, const PairEntry *ent, const int *seg, const double *tab,
                     int Nk, double *Sf, cudaStream_t st)
{
    int n = nshell * nshell * Nk;
    k_ovlp_fold<<<(n + 127) / 128, 128, 0, st>>>(ao, nshell, nao, ent, seg, tab, Nk, Sf);
    return cudaGetLastError() == cudaSuccess ? RSGDF_OK : RSGDF_EDEVICE;
}

// C[b][m][n] += sum_k A[k][m] B[b][k][n], complex FP64 (interleaved).
constexpr int GB_M = 32, GB_N = 32, GB_K = 16;

__global__ void __launch_bounds__(256) k_zgemm_tn(int M, int N, int K, const double2 *A, long long strideA,
                                                  const double2 *B, long long strideB, double2 *C, long long strideC)
{
    __shared__ double2 As[GB_K][GB_M];
    __shared__ double2 Bs[GB_K][GB_N];
    const int b = blockIdx.z;
    A += b * strideA;
    const double2 *Bb = B + b * strideB;
    double2 *Cb = C + b * strideC;
    const int m0 = blockIdx.y * GB_M, n0 = blockIdx.x * GB_N;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    double cr[2][2] = {{0, 0}, {0, 0}}, ci[2][2] = {{0, 0}, {0, 0}};
    for (int k0 = 0; k0 < K; k0 += GB_K) {
        for (int e = threadIdx.x; e < GB_K * GB_M; e += 256) {
            int kk = e / GB_M, mm = e % GB_M;
            int gk = k0 + kk, gm = m0 + mm;
            As[kk][mm] = (gk < K && gm < M) ? A[(long long)gk * M + gm] : make_double2(0.0, 0.0);
        }
        for (int e = threadIdx.x; e < GB_K * GB_N; e += 256) {
            int kk = e / GB_N, nn = e % GB_N;
            int gk = k0 + kk, gn = n0 + nn;
            Bs[kk][nn] = (gk < K && gn < N) ? Bb[(long long)gk * N + gn] : make_double2(0.0, 0.0);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GB_K; kk++) {
            double2 a0 = As[kk][ty * 2], a1 = As[kk][ty * 2 + 1];
            double2 b0 = Bs[kk][tx * 2], b1 = Bs[kk][tx * 2 + 1];
            double2 av[2] = {a0, a1}, bv[2] = {b0, b1};
#pragma unroll
            for (int i = 0; i < 2; i++)
#pragma unroll
                for (int j = 0; j < 2; j++) {
                    cr[i][j] = fma(av[i].x, bv[j].x, fma(-av[i].y, bv[j].y, cr[i][j]));
                    ci[i][j] = fma(av[i].x, bv[j].y, fma(av[i].y, bv[j].x, ci[i][j]));
                }
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 2; i++)
#pragma unroll
        for (int j = 0; j < 2; j++) {
            int gm = m0 + ty * 2 + i, gn = n0 + tx * 2 + j;
            if (gm < M && gn < N) {
                double2 c = Cb[(long long)gm * N + gn];
                c.x += cr[i][j];
                c.y += ci[i][j];
                Cb[(long long)gm * N + gn] = c;
            }
        }
}

int launch_zgemm_tn(int M, int N, int K, int batch, const double *A, const double *B, long long strideB, double *C,
                    long long strideC, cudaStream_t st, long long strideA)
{
    if (M <= 0 || N <= 0 || K <= 0 || batch <= 0) return RSGDF_OK;
    dim3 grid((N + GB_N - 1) / GB_N, (M + GB_M - 1) / GB_M, batch);
    k_zgemm_tn<<<grid, 256, 0, st>>>(M, N, K, (const double2 *)A, strideA / 2, (const double2 *)B, strideB / 2,
                                     (double2 *)C, strideC / 2);
    return cudaGetLastError() == cudaSuccess ? RSGDF_OK : RSGDF_EDEVICE;
}

// T[dt][i] (=|+=) sum_lt conj(ph[k12][lt]) X[lt][dt][i] for dt < ndt;
// ph[k][cell] = e^{i k.cell}
__global__ void k_phase1(const double *X, long long m, int Nk, int ndt, int k12, const double2 *ph, double2 *T,
                         int accumulate)
{
    long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= (long long)ndt * m) return;
    int dt = (int)(id / m);
    long long i = id - (long long)dt * m;
    double re = 0.0, im = 0.0;
    for (int lt = 0; lt < Nk; lt++) {
        double2 p = ph[(long long)k12 * Nk + lt];
        double x = X[((long long)lt * ndt + dt) * m + i];
        re = fma(p.x, x, re);
        im = fma(-p.y, x, im);
    }
    if (accumulate) {
        double2 t = T[id];
        t.x += re;
        t.y += im;
        T[id] = t;
    } else {
        T[id] = make_double2(re, im);
    }
}

int launch_phase1(const double *X, long long m, int Nk, int ndt, int k12, const double *ph, double *T, int accumulate,
                  cudaStream_t st)
{
    long long n = (long long)ndt * m;
    k_phase1<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(X, m, Nk, ndt, k12, (const double2 *)ph, (double2 *)T,
                                                         accumulate);
    return cudaGetLastError() == cudaSuccess ? RSGDF_OK : RSGDF_EDEVICE;
}

// J[P][Q] -= fac S_P S_Q  (the q = 0 term of the SR kernel at k = 0)
__global__ void k_g0_outer(double2 *J, int n, const double *S, double fac)
{
    long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= (long long)n * n) return;
    int P = (int)(id / n), Q = (int)(id % n);
    J[id].x -= fac * S[P] * S[Q];
}

int launch_g0_outer(double *J, int n, const double *S, double fac, cudaStream_t st)
{
    long long tot = (long long)n * n;
    k_g0_outer<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>((double2 *)J, n, S, fac);
    return cudaGetLastError() == cudaSuccess ? RSGDF_OK : RSGDF_EDEVICE;
}

// T[dt][P][mu][nu] -= fac S_P Sf[dt][mu][nu]  (k12 = 0 only)
__global__ void k_g0_fold(double2 *T, long long m, int Nk, int nP, int nao, const double *SP, const double *Sf,
                          double fac)
{
    long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= (long long)Nk * m) return;
    int dt = (int)(id / m);
    long long i = id - (long long)dt * m;
    long long nn = (long long)nao * nao;
    int P = (int)(i / nn);
    long long mn = i - (long long)P * nn;
    T[id].x -= fac * SP[P] * Sf[(long long)dt * nn + mn];
}

int launch_g0_fold(double *T, long long m, int Nk, int nP, int nao, const double *SP, const double *Sf, double fac,
                   cudaStream_t st)
{
    long long n = (long long)Nk * m;
    k_g0_fold<<<(unsigned)((n + 255) / 256), 256, 0, st>>>((double2 *)T, m, Nk, nP, nao, SP, Sf, fac);
    return cudaGetLastError() == cudaSuccess ? RSGDF_OK : RSGDF_EDEVICE;
}

// V[pair][i] (=|+=) sum_dt ph[k2][dt] T[dt][i] for the pairs of one k12
__global__ void k_phase2(const double2 *T, long long m, int Nk, const int *pair_list, const int *pair_k2, int npl,
                         const double2 *ph, double2 *V, int accumulate)
{
    long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= (long long)npl * m) return;
    int j = (int)(id / m);
    long long i = id - (long long)j * m;
    int k2 = pair_k2[j];
    double re = 0.0, im = 0.0;
    for (int dt = 0; dt < Nk; dt++) {
        double2 p = ph[(long long)k2 * Nk + dt];
        double2 t = T[(long long)dt * m + i];
        re = fma(p.x, t.x, fma(-p.y, t.y, re));
        im = fma(p.x, t.y, fma(p.y, t.x, im));
    }
    long long o = (long long)pair_list[j] * m + i;
    if (accumulate) {
        double2 v = V[o];
        v.x += re;
        v.y += im;
        V[o] = v;
    } else {
        V[o] = make_double2(re, im);
    }
}

int launch_phase2(const double *T, long long m, int Nk, const int *pair_list, const int *pair_k2, int npl,
                  const double *ph, double *V, int accumulate, cudaStream_t st)
{
    long long n = (long long)npl * m;
    if (n <= 0) return RSGDF_OK;
    k_phase2<<<(unsigned)((n + 255) / 256), 256, 0, st>>>((const double2 *)T, m, Nk, pair_list, pair_k2, npl,
                                                         (const double2 *)ph, (double2 *)V, accumulate);
    return cudaGetLastError() == cudaSuccess ? RSGDF_OK : RSGDF_EDEVICE;
}

// Right-looking Cholesky J = L L^H of one Hermitian matrix per block (lower
// triangle used).  info[k] = -1 on success, else the first pivot whose
// Schur complement is not positive.
__global__ void __launch_bounds__(1024) k_cholesky(int n, const double2 *J, double2 *Lo, int *info)
{
    const int kk = blockIdx.x;
    const double2 *A = J + (long long)kk * n * n;
    double2 *Lk = Lo + (long long)kk * n * n;
    __shared__ int bad;
    __shared__ double piv;
    for (long long e = threadIdx.x; e < (long long)n * n; e += blockDim.x) {
        int i = (int)(e / n), j = (int)(e % n);
        Lk[e] = (j <= i) ? A[e] : make_double2(0.0, 0.0);
    }
    if (threadIdx.x == 0) bad = -1;
    __syncthreads();
    for (int j = 0; j < n; j++) {
        if (threadIdx.x == 0) {
            double d = Lk[(long long)j * n + j].x;
            if (!(d > 0.0)) {
                bad = j;
                piv = 1.0;
            } else {
                piv = sqrt(d);
                Lk[(long long)j * n + j] = make_double2(piv, 0.0);
            }
        }
        __syncthreads();
        if (bad >= 0) break;
        const double inv = 1.0 / piv;
        for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) {
            double2 v = Lk[(long long)i * n + j];
            Lk[(long long)i * n + j] = make_double2(v.x * inv, v.y * inv);
        }
        __syncthreads();
        // trailing update of the lower triangle: L[i][c] -= L[i][j] conj(L[c][j]), j < c <= i
        const int m = n - j - 1;
        const long long tot = (long long)m * (m + 1) / 2;
        for (long long e = threadIdx.x; e < tot; e += blockDim.x) {
            // e -> (r, c) with 0 <= c <= r < m
            int r = (int)((sqrt(8.0 * (double)e + 1.0) - 1.0) * 0.5);
            while ((long long)(r + 1) * (r + 2) / 2 <= e) r++;
            while ((long long)r * (r + 1) / 2 > e) r--;
            int c = (int)(e - (long long)r * (r + 1) / 2);
            int i = j + 1 + r, cc = j + 1 + c;
            double2 a = Lk[(long long)i * n + j], b = Lk[(long long)cc * n + j];
            double2 t = Lk[(long long)i * n + cc];
            t.x -= a.x * b.x + a.y * b.y;
            t.y -= a.y * b.x - a.x * b.y;
            Lk[(long long)i * n + cc] = t;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0 && info) info[kk] = bad;
}

int launch_cholesky(int n, int nk, const double *J, double *Lo, int *info, cudaStream_t st)
{
    k_cholesky<<<nk, 1024, 0, st>>>(n, (const double2 *)J, (double2 *)Lo, info);
    return cudaGetLastError() == cudaSuccess ? RSGDF_OK : RSGDF_EDEVICE;
}

// FP64 FMA throughput probe: independent chains, no memory traffic.
__global__ void k_probe_fp64(double *out, int iters, double a, double b)
{
    double x[8];
#pragma unroll
    for (int i = 0; i < 8; i++) x[i] = threadIdx.x * 1e-3 + i;
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int i = 0; i < 8; i++) x[i] = fma(x[i], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < 8; i++) s += x[i];
    out[(long long)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

int launch_probe_fp64(double *out, int iters, cudaStream_t st)
{
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    k_probe_fp64<<<nsm * 8, 256, 0, st>>>(out, iters, 0.999999, 1e-7);
    return cudaGetLastError() == cudaSuccess ? RSGDF_OK : RSGDF_EDEVICE;
}

}  // namespace rsgdf

namespace rsgdf {

// ---------------------------------------------------------------------------
// Bloch-phase contractions for a batch of k12 values (Eq. BvK_latsum_LR):
//   T[j][dt][i] = sum_lt e^{-i k12_j.lt} X[lt][dt][i]        (phase1)
//   V[pair][i]  = sum_dt e^{+i k2.dt} T[j(pair)][dt][i]        (phase2)
// Register-blocked over KB k12 values (phase1) and PB pairs (phase2) so X and
// T are read a few times only.  R = double: the FP64 path.  The mixed path
// runs the same sums in double-float arithmetic on the FP32 pipes (below).
// ---------------------------------------------------------------------------
template <typename R> struct PhT;
template <> struct PhT<double> { typedef double2 type; enum { KB = 8, PB = 8 }; };

template <typename R>
__global__ void __launch_bounds__(256) k_phase1_multi(const double *__restrict__ X, long long m, int Nk, int nlt,
                                                      const int *__restrict__ k12list, int nk12,
                                                      const typename PhT<R>::type *__restrict__ ph,
                                                      double2 *__restrict__ T, int accumulate)
{
    const long long n = (long long)Nk * m;
    for (long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x; id < n; id += (long long)gridDim.x * blockDim.x) {
        const int dt = (int)(id / m);
        const long long i = id - (long long)dt * m;
        constexpr int KB = PhT<R>::KB;
        for (int j0 = 0; j0 < nk12; j0 += KB) {
            R ar[KB], ai[KB];
#pragma unroll
            for (int j = 0; j < KB; j++) { ar[j] = 0; ai[j] = 0; }
            for (int lt = 0; lt < nlt; lt++) {
                const R x = (R)X[((long long)lt * Nk + dt) * m + i];
#pragma unroll
                for (int j = 0; j < KB; j++) {
                    if (j0 + j < nk12) {
                        const auto p = __ldg(&ph[(long long)k12list[j0 + j] * Nk + lt]);
                        ar[j] += p.x * x;
                        ai[j] -= p.y * x;
                    }
                }
            }
#pragma unroll
            for (int j = 0; j < KB; j++)
                if (j0 + j < nk12) {
                    double2 *t = &T[((long long)(j0 + j) * Nk + dt) * m + i];
                    if (accumulate) {
                        double2 v = *t;
                        v.x += (double)ar[j];
                        v.y += (double)ai[j];
                        *t = v;
                    } else {
                        *t = make_double2((double)ar[j], (double)ai[j]);
                    }
                }
        }
    }
}

template <typename R>
__global__ void __launch_bounds__(256) k_phase2_multi(const double2 *__restrict__ T, long long m, int Nk,
                                                      const int *__restrict__ goff, int ngroups,
                                                      const int *__restrict__ plist, const int *__restrict__ pk2,
                                                      const typename PhT<R>::type *__restrict__ ph,
                                                      double2 *__restrict__ V, int accumulate)
{
    const int g = blockIdx.y;
    const int p0 = goff[g], p1 = goff[g + 1];
    const double2 *Tg = T + (long long)g * Nk * m;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (long long)gridDim.x * blockDim.x) {
        constexpr int PB = PhT<R>::PB;
        for (int q0 = p0; q0 < p1; q0 += PB) {
            R ar[PB], ai[PB];
#pragma unroll
            for (int j = 0; j < PB; j++) { ar[j] = 0; ai[j] = 0; }
            for (int dt = 0; dt < Nk; dt++) {
                const double2 t = Tg[(long long)dt * m + i];
                const R tr = (R)t.x, ti = (R)t.y;
#pragma unroll
                for (int j = 0; j < PB; j++) {
                    if (q0 + j < p1) {
                        const auto p = __ldg(&ph[(long long)pk2[q0 + j] * Nk + dt]);
                        ar[j] += p.x * tr - p.y * ti;
                        ai[j] += p.x * ti + p.y * tr;
                    }
                }
            }
#pragma unroll
            for (int j = 0; j < PB; j++) {
                if (q0 + j < p1) {
                    const long long o = (long long)plist[q0 + j] * m + i;
                    if (accumulate) {
                        double2 v = V[o];
                        v.x += (double)ar[j];
                        v.y += (double)ai[j];
                        V[o] = v;
                    } else {
                        V[o] = make_double2((double)ar[j], (double)ai[j]);
                    }
                }
            }
        }
    }
}

static int grid_for(long long n)
{
    long long g = (n + 255) / 256;
    if (g > 152LL * 64) g = 152LL * 64;
    return (int)(g < 1 ? 1 : g);
}

// ---------------------------------------------------------------------------
// Mixed path: the same contractions in double-float arithmetic.  A
// double-float is an unevaluated sum h + l of two floats; a product takes the
// exact rounding error of h1*h2 from one FMA (Dekker's product with a fused
// multiply-add), a sum takes it from Knuth's TwoSum, so each operation keeps
// about 44 bits while every instruction runs on the FP32 pipes.  Only the
// conversions from and to FP64 (once per X element, per T element read and
// per output) use the FP64 pipe.  The explicit _rn intrinsics keep the
// compiler from fusing the error-free steps into other FMAs.
// ---------------------------------------------------------------------------
struct dflt {
    float h, l;
};
__device__ __forceinline__ dflt df_from(double x)
{
    const float h = (float)x;
    return {h, (float)(x - (double)h)};
}
__device__ __forceinline__ double df_to(dflt a) { return (double)a.h + (double)a.l; }
__device__ __forceinline__ dflt df_mul(dflt a, dflt b)
{
    const float p = __fmul_rn(a.h, b.h);
    float e = fmaf(a.h, b.h, -p);   // exact: h1*h2 - p
    e = fmaf(a.h, b.l, e);
    e = fmaf(a.l, b.h, e);
    const float s = __fadd_rn(p, e);
    return {s, __fsub_rn(e, __fsub_rn(s, p))};
}
__device__ __forceinline__ dflt df_add(dflt a, dflt b)
{
    const float s = __fadd_rn(a.h, b.h);
    const float bb = __fsub_rn(s, a.h);
    float e = __fadd_rn(__fsub_rn(a.h, __fsub_rn(s, bb)), __fsub_rn(b.h, bb));   // exact: a.h + b.h - s
    e = __fadd_rn(e, __fadd_rn(a.l, b.l));
    const float r = __fadd_rn(s, e);
    return {r, __fsub_rn(e, __fsub_rn(r, s))};
}
__device__ __forceinline__ dflt df_neg(dflt a) { return {-a.h, -a.l}; }

// X (FP64) -> double-float pairs, in place (same 8 bytes per element).
__global__ void k_x_to_df(double *X, long long n)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const dflt d = df_from(X[i]);
        reinterpret_cast<float2 *>(X)[i] = make_float2(d.h, d.l);
    }
}

// phase tables as float4 (cos hi, cos lo, sin hi, sin lo)
constexpr int DF_KB = 8, DF_PB = 8;

__global__ void __launch_bounds__(256) k_phase1_df(const float2 *__restrict__ X, long long m, int Nk, int nlt,
                                                   const int *__restrict__ k12list, int nk12,
                                                   const float4 *__restrict__ ph, double2 *__restrict__ T,
                                                   int accumulate)
{
    const long long n = (long long)Nk * m;
    for (long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x; id < n; id += (long long)gridDim.x * blockDim.x) {
        const int dt = (int)(id / m);
        const long long i = id - (long long)dt * m;
        for (int j0 = 0; j0 < nk12; j0 += DF_KB) {
            dflt ar[DF_KB], ai[DF_KB];
#pragma unroll
            for (int j = 0; j < DF_KB; j++) { ar[j] = {0.0f, 0.0f}; ai[j] = {0.0f, 0.0f}; }
            for (int lt = 0; lt < nlt; lt++) {
                const float2 xv = X[((long long)lt * Nk + dt) * m + i];
                const dflt x = {xv.x, xv.y};
#pragma unroll
                for (int j = 0; j < DF_KB; j++) {
                    if (j0 + j < nk12) {
                        const float4 p = __ldg(&ph[(long long)k12list[j0 + j] * Nk + lt]);
                        ar[j] = df_add(ar[j], df_mul({p.x, p.y}, x));
                        ai[j] = df_add(ai[j], df_neg(df_mul({p.z, p.w}, x)));   // e^{-i k12.lt}
                    }
                }
            }
#pragma unroll
            for (int j = 0; j < DF_KB; j++)
                if (j0 + j < nk12) {
                    double2 *t = &T[((long long)(j0 + j) * Nk + dt) * m + i];
                    if (accumulate) {
                        double2 v = *t;
                        v.x += df_to(ar[j]);
                        v.y += df_to(ai[j]);
                        *t = v;
                    } else {
                        *t = make_double2(df_to(ar[j]), df_to(ai[j]));
                    }
                }
        }
    }
}

__global__ void __launch_bounds__(256) k_phase2_df(const double2 *__restrict__ T, long long m, int Nk,
                                                   const int *__restrict__ goff, int ngroups,
                                                   const int *__restrict__ plist, const int *__restrict__ pk2,
                                                   const float4 *__restrict__ ph, double2 *__restrict__ V,
                                                   int accumulate)
{
    const int g = blockIdx.y;
    const int p0 = goff[g], p1 = goff[g + 1];
    const double2 *Tg = T + (long long)g * Nk * m;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (long long)gridDim.x * blockDim.x) {
        for (int q0 = p0; q0 < p1; q0 += DF_PB) {
            dflt ar[DF_PB], ai[DF_PB];
#pragma unroll
            for (int j = 0; j < DF_PB; j++) { ar[j] = {0.0f, 0.0f}; ai[j] = {0.0f, 0.0f}; }
            for (int dt = 0; dt < Nk; dt++) {
                const double2 t = Tg[(long long)dt * m + i];
                const dflt tr = df_from(t.x), ti = df_from(t.y);
#pragma unroll
                for (int j = 0; j < DF_PB; j++) {
                    if (q0 + j < p1) {
                        const float4 p = __ldg(&ph[(long long)pk2[q0 + j] * Nk + dt]);
                        const dflt c = {p.x, p.y}, sn = {p.z, p.w};
                        // (c + i s)(tr + i ti)
                        ar[j] = df_add(ar[j], df_add(df_mul(c, tr), df_neg(df_mul(sn, ti))));
                        ai[j] = df_add(ai[j], df_add(df_mul(c, ti), df_mul(sn, tr)));
                    }
                }
            }
#pragma unroll
            for (int j = 0; j < DF_PB; j++) {
                if (q0 + j < p1) {
                    const long long o = (long long)plist[q0 + j] * m + i;
                    if (accumulate) {
                        double2 v = V[o];
                        v.x += df_to(ar[j]);
                        v.y += df_to(ai[j]);
                        V[o] = v;
                    } else {
                        V[o] = make_double2(df_to(ar[j]), df_to(ai[j]));
                    }
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Bloch-phase contractions as separable DFTs over the k mesh.  When every k12
// (phase 1) or every k2 (phase 2) is wanted, sum_{c} e^{-+i k.c} f(c) over the
// BvK cells c = (c0, c1, c2) factorises into three passes of length-N_d DFTs
// along the mesh axes: N0 + N1 + N2 complex multiply-adds per output instead
// of N0 N1 N2.  Each pass is in place on complex FP64 data laid out as
// [rep][j0][j1][j2][slab]; a thread transforms one line.  tw[q N + n] =
// e^{+2 pi i q n / N} (host table, exact angle reduction), conj = 1 for the
// negative exponent.
// ---------------------------------------------------------------------------
constexpr int DFT_NMAX = 16;

// NT > 0: the line length as a compile-time constant (the line stays in
// registers); NT = 0: any length up to DFT_NMAX, given at run time.
template <int NT>
__global__ void __launch_bounds__(256) k_dft_axis(double2 *__restrict__ T, long long S, long long nouter, int Nrt,
                                                  const double2 *__restrict__ tw, int conj)
{
    const int N = NT > 0 ? NT : Nrt;
    constexpr int NV = NT > 0 ? NT : DFT_NMAX;
    const long long nl = nouter * S;
    for (long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x; id < nl; id += (long long)gridDim.x * blockDim.x) {
        const long long outer = id / S, inner = id - outer * S;
        double2 *line = T + outer * N * S + inner;
        double2 v[NV];
#pragma unroll
        for (int n = 0; n < N; n++) v[n] = line[n * S];
#pragma unroll
        for (int q = 0; q < N; q++) {
            double re = 0.0, im = 0.0;
#pragma unroll
            for (int n = 0; n < N; n++) {
                const double2 w = __ldg(&tw[q * N + n]);
                const double wy = conj ? -w.y : w.y;
                re = fma(w.x, v[n].x, fma(-wy, v[n].y, re));
                im = fma(w.x, v[n].y, fma(wy, v[n].x, im));
            }
            line[q * S] = make_double2(re, im);
        }
    }
}

__global__ void k_real_to_complex(const double *__restrict__ X, double2 *__restrict__ Z, long long n)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        Z[i] = make_double2(X[i], 0.0);
}

__global__ void k_add_complex(double2 *__restrict__ T, const double2 *__restrict__ Z, long long n)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        double2 t = T[i];
        const double2 z = Z[i];
        t.x += z.x;
        t.y += z.y;
        T[i] = t;
    }
}

// V[p][i] (+)= T[k12(p)][k2(p)][i]
__global__ void k_scatter_pairs(const double2 *__restrict__ T, long long m, int Nk, const int *__restrict__ pk12,
                                const int *__restrict__ pk2, double2 *__restrict__ V, int accumulate)
{
    const int p = blockIdx.y;
    const double2 *src = T + ((long long)pk12[p] * Nk + pk2[p]) * m;
    double2 *dst = V + (long long)p * m;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (long long)gridDim.x * blockDim.x) {
        double2 v = src[i];
        if (accumulate) {
            const double2 o = dst[i];
            v.x += o.x;
            v.y += o.y;
        }
        dst[i] = v;
    }
}

// In-place 3-D DFT over the mesh index of T[rep][j0][j1][j2][slab] (complex).
int launch_dft_mesh(double *T, const int nk[3], long long slab, long long nrep, const double *tw, int conj,
                    cudaStream_t st)
{
    long long inner = slab;
    for (int d = 2; d >= 0; d--) {
        const int N = nk[d];
        if (N > DFT_NMAX) return RSGDF_EINVAL;
        long long outer = nrep;
        for (int e = 0; e < d; e++) outer *= nk[e];
        if (N > 1) {
            const long long nl = outer * inner;
            const double2 *twd = (const double2 *)tw + d * DFT_NMAX * DFT_NMAX;
            switch (N) {
#define DFT_CASE(n) case n: k_dft_axis<n><<<grid_for(nl), 256, 0, st>>>((double2 *)T, inner, outer, N, twd, conj); break;
                DFT_CASE(2) DFT_CASE(3) DFT_CASE(4) DFT_CASE(5) DFT_CASE(6) DFT_CASE(7) DFT_CASE(8)
#undef DFT_CASE
                default: k_dft_axis<0><<<grid_for(nl), 256, 0, st>>>((double2 *)T, inner, outer, N, twd, conj);
            }
            if (cudaGetLastError() != cudaSuccess) return RSGDF_EDEVICE;
        }
        inner *= N;
    }
    return RSGDF_OK;
}

int launch_real_to_complex(const double *X, double *Z, long long n, cudaStream_t st)
{
    k_real_to_complex<<<grid_for(n), 256, 0, st>>>(X, (double2 *)Z, n);
    return cudaGetLastError() == cudaSuccess ? RSGDF_OK : RSGDF_EDEVICE;
}

int launch_add_complex(double *T, const double *Z, long long n, cudaStream_t st)
{
    k_add_complex<<<grid_for(n), 256, 0, st>>>((double2 *)T, (const double2 *)Z, n);
    return cudaGetLastError() == cudaSuccess ? RSGDF_OK : RSGDF_EDEVICE;
}

int launch_scatter_pairs(const double *T, long long m, int Nk, int npair, const int *pk12, const int *pk2, double *V,
                         int accumulate, cudaStream_t st)
{
    if (npair <= 0) return RSGDF_OK;
    dim3 grid((unsigned)std::min<long long>((m + 255) / 256, 1024), npair);
    k_scatter_pairs<<<grid, 256, 0, st>>>((const double2 *)T, m, Nk, pk12, pk2, (double2 *)V, accumulate);
    return cudaGetLastError() == cudaSuccess ? RSGDF_OK : RSGDF_EDEVICE;
}

// Mixed path: the same DFT passes in double-float arithmetic; complex values
// stored as float4 (re hi, re lo, im hi, im lo) in the same 16 bytes as a
// double2, so the format changes in place.
__device__ __forceinline__ float4 df4_from(double2 v)
{
    const dflt r = df_from(v.x), i = df_from(v.y);
    return make_float4(r.h, r.l, i.h, i.l);
}

template <int NT>
__global__ void __launch_bounds__(256) k_dft_axis_df(float4 *__restrict__ T, long long S, long long nouter, int Nrt,
                                                     const float4 *__restrict__ tw, int conj)
{
    const int N = NT > 0 ? NT : Nrt;
    constexpr int NV = NT > 0 ? NT : DFT_NMAX;
    const long long nl = nouter * S;
    for (long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x; id < nl; id += (long long)gridDim.x * blockDim.x) {
        const long long outer = id / S, inner = id - outer * S;
        float4 *line = T + outer * N * S + inner;
        float4 v[NV];
#pragma unroll
        for (int n = 0; n < N; n++) v[n] = line[n * S];
#pragma unroll
        for (int q = 0; q < N; q++) {
            dflt re = {0.0f, 0.0f}, im = {0.0f, 0.0f};
#pragma unroll
            for (int n = 0; n < N; n++) {
                const float4 w = __ldg(&tw[q * N + n]);
                const dflt c = {w.x, w.y};
                const dflt sn = conj ? dflt{-w.z, -w.w} : dflt{w.z, w.w};
                const dflt vr = {v[n].x, v[n].y}, vi = {v[n].z, v[n].w};
                re = df_add(re, df_add(df_mul(c, vr), df_neg(df_mul(sn, vi))));
                im = df_add(im, df_add(df_mul(c, vi), df_mul(sn, vr)));
            }
            line[q * S] = make_float4(re.h, re.l, im.h, im.l);
        }
    }
}

__global__ void k_real_to_df(const double *__restrict__ X, float4 *__restrict__ Z, long long n)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        Z[i] = df4_from(make_double2(X[i], 0.0));
}

// dir = 1: double2 -> double-float in place; dir = 0: back
__global__ void k_convert_df(double2 *T, long long n, int dir)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        if (dir) {
            const double2 v = T[i];
            reinterpret_cast<float4 *>(T)[i] = df4_from(v);
        } else {
            const float4 v = reinterpret_cast<const float4 *>(T)[i];
            T[i] = make_double2(df_to({v.x, v.y}), df_to({v.z, v.w}));
        }
    }
}

__global__ void k_add_df(double2 *__restrict__ T, const float4 *__restrict__ Z, long long n)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        double2 t = T[i];
        const float4 z = Z[i];
        t.x += df_to({z.x, z.y});
        t.y += df_to({z.z, z.w});
        T[i] = t;
    }
}

__global__ void k_scatter_pairs_df(const float4 *__restrict__ T, long long m, int Nk, const int *__restrict__ pk12,
                                   const int *__restrict__ pk2, double2 *__restrict__ V, int accumulate)
{
    const int p = blockIdx.y;
    const float4 *src = T + ((long long)pk12[p] * Nk + pk2[p]) * m;
    double2 *dst = V + (long long)p * m;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (long long)gridDim.x * blockDim.x) {
        const float4 z = src[i];
        double2 v = make_double2(df_to({z.x, z.y}), df_to({z.z, z.w}));
        if (accumulate) {
            const double2 o = dst[i];
            v.x += o.x;
            v.y += o.y;
        }
        dst[i] = v;
    }
}

int launch_dft_mesh_df(double *T, const int nk[3], long long slab, long long nrep, const float *tw4, int conj,
                       cudaStream_t st)
{
    long long inner = slab;
    for (int d = 2; d >= 0; d--) {
        const int N = nk[d];
        if (N > DFT_NMAX) return RSGDF_EINVAL;
        long long outer = nrep;
        for (int e = 0; e < d; e++) outer *= nk[e];
        if (N > 1) {
            const long long nl = outer * inner;
            const float4 *twd = (const float4 *)tw4 + d * DFT_NMAX * DFT_NMAX;
            switch (N) {
#define DFT_CASE(n) case n: k_dft_axis_df<n><<<grid_for(nl), 256, 0, st>>>((float4 *)T, inner, outer, N, twd, conj); break;
                DFT_CASE(2) DFT_CASE(3) DFT_CASE(4) DFT_CASE(5) DFT_CASE(6) DFT_CASE(7) DFT_CASE(8)
#undef DFT_CASE
                default: k_dft_axis_df<0><<<grid_for(nl), 256, 0, st>>>((float4 *)T, inner, outer, N, twd, conj);
            }
            if (cudaGetLastError() != cudaSuccess) return RSGDF_EDEVICE;
        }
        inner *= N;
    }
    return RSGDF_OK;
}

int launch_real_to_df(const double *X, double *Z, long long n, cudaStream_t st)
{
    k_real_to_df<<<grid_for(n), 256, 0, st>>>(X, (float4 *)Z, n);
    return cudaGetLastError() == cudaSuccess ? RSGDF_OK : RSGDF_EDEVICE;
}

int launch_convert_df(double *T, long long n, int to_df, cudaStream_t st)
{
    k_convert_df<<<grid_for(n), 256, 0, st>>>((double2 *)T, n, to_df);
    return cudaGetLastError() == cudaSuccess ? RSGDF_OK : RSGDF_EDEVICE;
}

int launch_add_df(double *T, const double *Z, long long n, cudaStream_t st)
{
    k_add_df<<<grid_for(n), 256, 0, st>>>((double2 *)T, (const float4 *)Z, n);
    return cudaGetLastError() == cudaSuccess ? RSGDF_OK : RSGDF_EDEVICE;
}

int launch_scatter_pairs_df(const double *T, long long m, int Nk, int npair, const int *pk12, const int *pk2, double *V,
                            int accumulate, cudaStream_t st)
{
    if (npair <= 0) return RSGDF_OK;
    dim3 grid((unsigned)std::min<long long>((m + 255) / 256, 1024), npair);
    k_scatter_pairs_df<<<grid, 256, 0, st>>>((const float4 *)T, m, Nk, pk12, pk2, (double2 *)V, accumulate);
    return cudaGetLastError() == cudaSuccess ? RSGDF_OK : RSGDF_EDEVICE;
}

int launch_x_to_df(double *X, long long n, cudaStream_t st)
{
    if (n <= 0) return RSGDF_OK;
    k_x_to_df<<<grid_for(n), 256, 0, st>>>(X, n);
    return cudaGetLastError() == cudaSuccess ? RSGDF_OK : RSGDF_EDEVICE;
}

// fp32 = 1: X already in double-float pairs (launch_x_to_df), ph = float4 table;
// accumulate = 1: T += (the LR part is already there)
int launch_phase1_multi(const double *X, long long m, int Nk, int nlt, const int *k12list, int nk12, const void *ph,
                        double *T, int fp32, int accumulate, cudaStream_t st)
{
    const long long n = (long long)Nk * m;
    if (fp32)
        k_phase1_df<<<grid_for(n), 256, 0, st>>>((const float2 *)X, m, Nk, nlt, k12list, nk12, (const float4 *)ph,
                                                 (double2 *)T, accumulate);
    else
        k_phase1_multi<double><<<grid_for(n), 256, 0, st>>>(X, m, Nk, nlt, k12list, nk12, (const double2 *)ph,
                                                             (double2 *)T, accumulate);
    return cudaGetLastError() == cudaSuccess ? RSGDF_OK : RSGDF_EDEVICE;
}

int launch_phase2_multi(const double *T, long long m, int Nk, const int *goff, int ngroups, const int *plist,
                        const int *pk2, const void *ph, double *V, int accumulate, int fp32, cudaStream_t st)
{
    dim3 grid((unsigned)std::min<long long>((m + 255) / 256, 4096), ngroups);
    if (fp32)
        k_phase2_df<<<grid, 256, 0, st>>>((const double2 *)T, m, Nk, goff, ngroups, plist, pk2, (const float4 *)ph,
                                          (double2 *)V, accumulate);
    else
        k_phase2_multi<double><<<grid, 256, 0, st>>>((const double2 *)T, m, Nk, goff, ngroups, plist, pk2,
                                                    (const double2 *)ph, (double2 *)V, accumulate);
    return cudaGetLastError() == cudaSuccess ? RSGDF_OK : RSGDF_EDEVICE;
}

}  // namespace rsgdf
