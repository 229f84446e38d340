/*
 * RSGDF oracle: a plain, slow FP64 CPU implementation of the periodic
 * three-center (j3c) and two-center (j2c) Coulomb-metric integrals of
 * range-separated Gaussian density fitting (Ye & Berkelbach, "Fast periodic
 * Gaussian density fitting by range separation").
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or constant generator with the CUDA library; it is written
 * for readability, not speed: every integral is evaluated term by term with
 * the McMurchie-Davidson (Hermite) scheme, no blocking, no caching beyond
 * what the formulas name.
 *
 * Conventions (the paper leaves them open; the readings are listed with the
 * design notes of the project):
 *   - Cartesian Gaussians x^lx y^ly z^lz exp(-a r^2), components ordered
 *     lexicographically (xx,xy,xz,yy,yz,zz,...).  Every primitive carries the
 *     radial norm of its x^l component and every contracted shell is
 *     rescaled so that its x^l component has unit norm.
 *   - Periodic integrals (Eqs. TAAO, JPQ, VPmunu):
 *       V^{k1k2}_{P mu nu} = sum_{l,d} e^{-i k12.l} e^{+i k2.d}
 *                            (chi_P^l | w | phi_mu^0 phi_nu^d),  k12 = k2-k1
 *       J^k_{PQ}           = sum_l e^{+i k.l} (chi_P^0 | w | chi_Q^l)
 *     with the q = G + k12 = 0 component removed (McClain convention).
 *   - Range separation (Eq. Coulomb_RS): w = erfc(w r)/r + erf(w r)/r.
 *     SR part: real-space lattice sums (Eq. VPmunu_SR) with the G=0
 *     correction -pi/(Omega omega^2) S_P S_{mu nu}; LR part: reciprocal-space
 *     sum (Eq. VPmunu_LR) with the prefactor 4 pi / Omega.
 *   - Route R2 ("full G", Eq. VPmunu_FT): 4 pi/Omega sum_{q != 0}
 *     conj(chi^(q)) rho^(q) / |q|^2 with a large G box; used only to check
 *     route R1 on tiny cells.
 *   - Screening of the SR double lattice sum follows the Supplementary
 *     Material "Conditions for prescreening the double lattice summation"
 *     (Eqs. bound_Rc, S_h, Ncell, bound_R12_FF, bound_R12, R12cutmin).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <complex.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_LMAX 4           /* per shell */
#define OR_LTOT (3 * OR_LMAX)
#define OR_NC(l) (((l) + 1) * ((l) + 2) / 2)

static const double OR_PI = 3.14159265358979323846264338327950288;

/* ------------------------------------------------------------------ */
/* Instrumented operation counter                                      */
/* ------------------------------------------------------------------ */

/* When switched on for a thread (or_flops_begin), the FP64 operations of one
 * SR primitive integral are tallied by category as the code below performs
 * them.  The categories separate what depends on the lattice translation of
 * a term (the separation and T, the erfc auxiliary function G_n, the Hermite
 * seeds and recursion) from what depends only on the primitive combination
 * (s, sqrt s, the (-2 alpha)^n factors).  Boys evaluations are counted as
 * calls with their highest order: the series used here is written for
 * clarity, not economy, so its own operation count is not the method's. */
enum {
    OR_FL_SEP_T,      /* P - C - l and T = alpha |P - C - l|^2 */
    OR_FL_BOYS_CALL,  /* Boys evaluations (calls) */
    OR_FL_BOYS_ORD,   /* sum over calls of the highest order requested */
    OR_FL_COMBINE,    /* s T and G_n = F_n(T) - s^{n+1/2} F_n(sT), n = 0..L */
    OR_FL_SEED,       /* R^n_000 = (-2 alpha)^n G_n */
    OR_FL_HERMITE,    /* R^n_{tuv} recursion */
    OR_FL_COMBO,      /* per primitive combination: s, sqrt s, (-2 alpha)^n */
    OR_FL_N
};
static _Thread_local long long or_fl[OR_FL_N];
static _Thread_local int or_fl_on;
#define OR_FL(k, n) do { if (or_fl_on) or_fl[k] += (n); } while (0)

void or_flops_begin(void)
{
    memset(or_fl, 0, sizeof(or_fl));
    or_fl_on = 1;
}

void or_flops_end(long long *out /* [OR_FL_N] */)
{
    or_fl_on = 0;
    for (int k = 0; k < OR_FL_N; k++) out[k] = or_fl[k];
}

int or_flops_ncat(void) { return OR_FL_N; }

typedef struct {
    int nshell;
    const int *l;         /* [nshell] angular momentum */
    const int *nprim;     /* [nshell] primitives per shell */
    const int *prim_off;  /* [nshell] offset into exps/coeffs */
    const double *center; /* [nshell][3] Bohr */
    const double *exps;   /* [nprim_total] */
    const double *coeffs; /* [nprim_total] raw contraction coefficients */
} or_basis;

/* ------------------------------------------------------------------ */
/* Boys function F_m(T) = int_0^1 t^{2m} exp(-T t^2) dt                */
/* ------------------------------------------------------------------ */

/* For T < 30 every order comes from the convergent series
 *   F_m(T) = e^{-T} sum_k (2T)^k / ((2m+1)(2m+3)...(2m+2k+1)),
 * all of whose terms are positive.  For T >= 30 start from
 *   F_0(T) = sqrt(pi/T)/2 erf(sqrt(T))
 * and recur upward F_{m+1} = ((2m+1) F_m - e^{-T}) / (2T), which is stable
 * for m < T. */
void or_boys(int mmax, double T, double *F)
{
    OR_FL(OR_FL_BOYS_CALL, 1);
    OR_FL(OR_FL_BOYS_ORD, mmax);
    if (T < 30.0) {
        double eT = exp(-T);
        for (int m = 0; m <= mmax; m++) {
            double term = 1.0 / (2 * m + 1), sum = term;
            for (int k = 1; k < 2000; k++) {
                term *= 2.0 * T / (2 * m + 2 * k + 1);
                sum += term;
                if (term < 1e-18 * sum) break;
            }
            F[m] = eT * sum;
        }
    } else {
        double eT = exp(-T);
        F[0] = 0.5 * sqrt(OR_PI / T) * erf(sqrt(T));
        for (int m = 0; m < mmax; m++)
            F[m + 1] = ((2 * m + 1) * F[m] - eT) / (2.0 * T);
    }
}

/* Kernel-specific auxiliary function G_n, so that the Hermite integral
 * R^n_000 = (-2 alpha)^n G_n.  kernel: 0 = 1/r, 1 = erf(omega r)/r,
 * 2 = erfc(omega r)/r.  For erf the effective exponent is s*alpha with
 * s = omega^2/(omega^2+alpha), which gives G_n = s^{n+1/2} F_n(sT). */
static void kernel_G(int kernel, double omega, int L, double alpha, double T, double *G)
{
    double F[OR_LTOT + 2], Fs[OR_LTOT + 2];
    if (kernel == 0) {
        or_boys(L, T, G);
        return;
    }
    double s = omega * omega / (omega * omega + alpha);
    OR_FL(OR_FL_COMBO, 4);
    or_boys(L, s * T, Fs);
    OR_FL(OR_FL_COMBINE, 1);
    double sp = sqrt(s);
    OR_FL(OR_FL_COMBO, 1);
    if (kernel == 1) {
        for (int n = 0; n <= L; n++) { G[n] = sp * Fs[n]; sp *= s; }
    } else {
        or_boys(L, T, F);
        for (int n = 0; n <= L; n++) { G[n] = F[n] - sp * Fs[n]; sp *= s; OR_FL(OR_FL_COMBINE, 3); }
    }
}

/* ------------------------------------------------------------------ */
/* Cartesian components and normalisation                             */
/* ------------------------------------------------------------------ */

static void cart_list(int l, int (*c)[3])
{
    int n = 0;
    for (int lx = l; lx >= 0; lx--)
        for (int ly = l - lx; ly >= 0; ly--) {
            c[n][0] = lx; c[n][1] = ly; c[n][2] = l - lx - ly; n++;
        }
}

static double dfact(int n) /* n!! with (-1)!! = 1 */
{
    double r = 1.0;
    for (int k = n; k > 1; k -= 2) r *= k;
    return r;
}

/* radial norm of the x^l component of a primitive */
static double prim_norm(double a, int l)
{
    return sqrt(pow(2.0 * a / OR_PI, 1.5) * pow(4.0 * a, l) / dfact(2 * l - 1));
}

/* Effective coefficients c'_i so that the shell's x^l component,
 * sum_i c'_i x^l exp(-a_i r^2), has unit norm. */
void or_norm_coeffs(const or_basis *b, double *out)
{
    for (int s = 0; s < b->nshell; s++) {
        int l = b->l[s], o = b->prim_off[s], np = b->nprim[s];
        double ov = 0.0;
        for (int i = 0; i < np; i++)
            for (int j = 0; j < np; j++) {
                double ai = b->exps[o + i], aj = b->exps[o + j];
                double ci = b->coeffs[o + i] * prim_norm(ai, l);
                double cj = b->coeffs[o + j] * prim_norm(aj, l);
                double p = ai + aj;
                ov += ci * cj * dfact(2 * l - 1) / pow(2.0 * p, l) * pow(OR_PI / p, 1.5);
            }
        double nc = 1.0 / sqrt(ov);
        for (int i = 0; i < np; i++)
            out[o + i] = nc * b->coeffs[o + i] * prim_norm(b->exps[o + i], l);
    }
}

static int basis_nfunc(const or_basis *b)
{
    int n = 0;
    for (int s = 0; s < b->nshell; s++) n += OR_NC(b->l[s]);
    return n;
}

static void basis_offsets(const or_basis *b, int *off)
{
    int n = 0;
    for (int s = 0; s < b->nshell; s++) { off[s] = n; n += OR_NC(b->l[s]); }
}

/* ------------------------------------------------------------------ */
/* McMurchie-Davidson building blocks                                  */
/* ------------------------------------------------------------------ */

/* Hermite expansion of the 1D product x_A^i x_B^j e^{-a x_A^2} e^{-b x_B^2}
 * = sum_t E[i][j][t] Lambda_t with Lambda_t = d^t/dP^t e^{-p (x-P)^2}.
 * E is stored as E[(i*(lb+1)+j)*(la+lb+1)+t]. */
static void herm_E(int la, int lb, double a, double b, double Ax, double Bx, double *E)
{
    int nt = la + lb + 1;
    double p = a + b, mu = (p > 0) ? a * b / p : 0.0;
    double Px = (p > 0) ? (a * Ax + b * Bx) / p : Ax;
    double XPA = Px - Ax, XPB = Px - Bx, XAB = Ax - Bx;
    double h = 0.5 / p;
    memset(E, 0, sizeof(double) * (la + 1) * (lb + 1) * nt);
#define EI(i, j, t) E[((i) * (lb + 1) + (j)) * nt + (t)]
    EI(0, 0, 0) = exp(-mu * XAB * XAB);
    for (int i = 0; i <= la; i++)
        for (int j = 0; j <= lb; j++) {
            if (i == 0 && j == 0) continue;
            for (int t = 0; t <= i + j; t++) {
                double v = 0.0;
                if (i > 0) {
                    if (t > 0) v += h * EI(i - 1, j, t - 1);
                    if (t <= i - 1 + j) v += XPA * EI(i - 1, j, t);
                    if (t + 1 <= i - 1 + j) v += (t + 1) * EI(i - 1, j, t + 1);
                } else {
                    if (t > 0) v += h * EI(i, j - 1, t - 1);
                    if (t <= i + j - 1) v += XPB * EI(i, j - 1, t);
                    if (t + 1 <= i + j - 1) v += (t + 1) * EI(i, j - 1, t + 1);
                }
                EI(i, j, t) = v;
            }
        }
#undef EI
}

/* Hermite Coulomb-type integrals R_{tuv} = R^0_{tuv} for t+u+v <= L from
 * R^n_000 = (-2 alpha)^n G_n and the recurrence
 *   R^n_{t+1,u,v} = t R^{n+1}_{t-1,u,v} + X R^{n+1}_{t,u,v}  (same for u, v).
 * Output R[(t*(L+1)+u)*(L+1)+v]. */
static void herm_R(int L, double alpha, double X, double Y, double Z, const double *G, double *R)
{
    int D = L + 1;
    double *W = (double *)malloc(sizeof(double) * D * D * D * D);
#define RI(n, t, u, v) W[(((n) * D + (t)) * D + (u)) * D + (v)]
    double f = 1.0;
    for (int n = 0; n <= L; n++) {
        RI(n, 0, 0, 0) = f * G[n];
        f *= -2.0 * alpha;
        OR_FL(OR_FL_SEED, 1);
        OR_FL(OR_FL_COMBO, 2);
    }
    for (int s = 1; s <= L; s++)
        for (int t = 0; t <= s; t++)
            for (int u = 0; u <= s - t; u++) {
                int v = s - t - u;
                for (int n = 0; n <= L - s; n++) {
                    double r;
                    if (t > 0) {
                        r = X * RI(n + 1, t - 1, u, v);
                        OR_FL(OR_FL_HERMITE, 1);
                        if (t > 1) { r += (t - 1) * RI(n + 1, t - 2, u, v); OR_FL(OR_FL_HERMITE, 2); }
                    } else if (u > 0) {
                        r = Y * RI(n + 1, t, u - 1, v);
                        OR_FL(OR_FL_HERMITE, 1);
                        if (u > 1) { r += (u - 1) * RI(n + 1, t, u - 2, v); OR_FL(OR_FL_HERMITE, 2); }
                    } else {
                        r = Z * RI(n + 1, t, u, v - 1);
                        OR_FL(OR_FL_HERMITE, 1);
                        if (v > 1) { r += (v - 1) * RI(n + 1, t, u, v - 2); OR_FL(OR_FL_HERMITE, 2); }
                    }
                    RI(n, t, u, v) = r;
                }
            }
    for (int t = 0; t <= L; t++)
        for (int u = 0; u <= L - t; u++)
            for (int v = 0; v <= L - t - u; v++) R[(t * D + u) * D + v] = RI(0, t, u, v);
#undef RI
    free(W);
}

/* Primitive three-center integral block (c | w | a b) over unnormalised
 * Cartesian primitives: c at C (exponent g, l = lc), a at A, b at B.
 * out[(ic*nca + ia)*ncb + ib]. */
void or_prim3c(int kernel, double omega, int lc, double g, const double *C,
               int la, double a, const double *A, int lb, double b, const double *B, double *out)
{
    int L = lc + la + lb, D = L + 1;
    double p = a + b;
    double Pc[3];
    for (int x = 0; x < 3; x++) Pc[x] = (a * A[x] + b * B[x]) / p;
    int nab = la + lb + 1;
    double *Eab[3], *Ec[3];
    for (int x = 0; x < 3; x++) {
        Eab[x] = (double *)malloc(sizeof(double) * (la + 1) * (lb + 1) * nab);
        Ec[x] = (double *)malloc(sizeof(double) * (lc + 1) * (lc + 1));
        herm_E(la, lb, a, b, A[x], B[x], Eab[x]);
        herm_E(lc, 0, g, 0.0, C[x], C[x], Ec[x]);
    }
    double alpha = p * g / (p + g);
    double X = Pc[0] - C[0], Y = Pc[1] - C[1], Z = Pc[2] - C[2];
    double T = alpha * (X * X + Y * Y + Z * Z);
    OR_FL(OR_FL_SEP_T, 9);
    double G[OR_LTOT + 2];
    kernel_G(kernel, omega, L, alpha, T, G);
    double *R = (double *)malloc(sizeof(double) * D * D * D);
    herm_R(L, alpha, X, Y, Z, G, R);
    double pref = 2.0 * pow(OR_PI, 2.5) / (p * g * sqrt(p + g));
    int cc[OR_NC(OR_LMAX)][3], ca[OR_NC(OR_LMAX)][3], cb[OR_NC(OR_LMAX)][3];
    cart_list(lc, cc); cart_list(la, ca); cart_list(lb, cb);
    int ncc = OR_NC(lc), nca = OR_NC(la), ncb = OR_NC(lb);
    for (int ic = 0; ic < ncc; ic++)
        for (int ia = 0; ia < nca; ia++)
            for (int ib = 0; ib < ncb; ib++) {
                double sum = 0.0;
                int ax = ca[ia][0], ay = ca[ia][1], az = ca[ia][2];
                int bx = cb[ib][0], by = cb[ib][1], bz = cb[ib][2];
                int cx = cc[ic][0], cy = cc[ic][1], cz = cc[ic][2];
                for (int t = 0; t <= ax + bx; t++)
                    for (int u = 0; u <= ay + by; u++)
                        for (int v = 0; v <= az + bz; v++) {
                            double eab = Eab[0][(ax * (lb + 1) + bx) * nab + t] *
                                         Eab[1][(ay * (lb + 1) + by) * nab + u] *
                                         Eab[2][(az * (lb + 1) + bz) * nab + v];
                            if (eab == 0.0) continue;
                            for (int tau = 0; tau <= cx; tau++)
                                for (int nu = 0; nu <= cy; nu++)
                                    for (int phi = 0; phi <= cz; phi++) {
                                        double ec = Ec[0][cx * (lc + 1) + tau] *
                                                    Ec[1][cy * (lc + 1) + nu] *
                                                    Ec[2][cz * (lc + 1) + phi];
                                        if (ec == 0.0) continue;
                                        double sg = ((tau + nu + phi) & 1) ? -1.0 : 1.0;
                                        sum += eab * sg * ec * R[((t + tau) * D + (u + nu)) * D + (v + phi)];
                                    }
                        }
                out[(ic * nca + ia) * ncb + ib] = pref * sum;
            }
    for (int x = 0; x < 3; x++) { free(Eab[x]); free(Ec[x]); }
    free(R);
}

/* Primitive two-center block (c | w | d): a Gaussian times the constant
 * function 1 (an s primitive of exponent 0) is the Gaussian itself, so this
 * is the three-center block with a unit partner on the d side. */
void or_prim2c(int kernel, double omega, int lc, double g, const double *C,
               int ld, double e, const double *Dc, double *out)
{
    or_prim3c(kernel, omega, lc, g, C, ld, e, Dc, 0, 0.0, Dc, out);
}

/* Primitive overlap block (a | b) = prod_x E^{ab}_0 (pi/p)^{3/2} */
void or_prim_ovlp(int la, double a, const double *A, int lb, double b, const double *B, double *out)
{
    int nab = la + lb + 1;
    double *E[3];
    for (int x = 0; x < 3; x++) {
        E[x] = (double *)malloc(sizeof(double) * (la + 1) * (lb + 1) * nab);
        herm_E(la, lb, a, b, A[x], B[x], E[x]);
    }
    double pf = pow(OR_PI / (a + b), 1.5);
    int ca[OR_NC(OR_LMAX)][3], cb[OR_NC(OR_LMAX)][3];
    cart_list(la, ca); cart_list(lb, cb);
    for (int ia = 0; ia < OR_NC(la); ia++)
        for (int ib = 0; ib < OR_NC(lb); ib++) {
            double v = pf;
            for (int x = 0; x < 3; x++) v *= E[x][(ca[ia][x] * (lb + 1) + cb[ib][x]) * nab + 0];
            out[ia * OR_NC(lb) + ib] = v;
        }
    for (int x = 0; x < 3; x++) free(E[x]);
}

/* Fourier transform of a primitive product,
 *   int x_A^.. x_B^.. e^{-a rA^2} e^{-b rB^2} e^{-i q.r} dr
 *   = sum_{tuv} E_{tuv} (-i qx)^t (-i qy)^u (-i qz)^v (pi/p)^{3/2} e^{-q^2/4p} e^{-i q.P}.
 * With b = 0 this is the transform of a single Gaussian.  out[ia*ncb+ib]. */
void or_prim_ft(int la, double a, const double *A, int lb, double b, const double *B,
                const double *q, double complex *out)
{
    int nab = la + lb + 1;
    double p = a + b;
    double *E[3];
    double Pc[3];
    for (int x = 0; x < 3; x++) {
        E[x] = (double *)malloc(sizeof(double) * (la + 1) * (lb + 1) * nab);
        herm_E(la, lb, a, b, A[x], B[x], E[x]);
        Pc[x] = (a * A[x] + b * B[x]) / p;
    }
    double q2 = q[0] * q[0] + q[1] * q[1] + q[2] * q[2];
    double qP = q[0] * Pc[0] + q[1] * Pc[1] + q[2] * Pc[2];
    double complex base = pow(OR_PI / p, 1.5) * exp(-q2 / (4.0 * p)) * cexp(-I * qP);
    int ca[OR_NC(OR_LMAX)][3], cb[OR_NC(OR_LMAX)][3];
    cart_list(la, ca); cart_list(lb, cb);
    for (int ia = 0; ia < OR_NC(la); ia++)
        for (int ib = 0; ib < OR_NC(lb); ib++) {
            double complex v = base;
            for (int x = 0; x < 3; x++) {
                double complex f = 0.0;
                double complex mq = -I * q[x], pw = 1.0;
                int i = ca[ia][x], j = cb[ib][x];
                for (int t = 0; t <= i + j; t++) {
                    f += E[x][(i * (lb + 1) + j) * nab + t] * pw;
                    pw *= mq;
                }
                v *= f;
            }
            out[ia * OR_NC(lb) + ib] = v;
        }
    for (int x = 0; x < 3; x++) free(E[x]);
}

/* ------------------------------------------------------------------ */
/* Contracted blocks                                                   */
/* ------------------------------------------------------------------ */

/* (P | w | mu nu) for shells with centres shifted by sP and sNu (Bohr). */
static void shell3c(int kernel, double omega, const or_basis *aux, const double *caux, int P,
                    const double *sP, const or_basis *ao, const double *cao, int mu, int nu,
                    const double *sNu, double *out)
{
    int lP = aux->l[P], lm = ao->l[mu], ln = ao->l[nu];
    int n = OR_NC(lP) * OR_NC(lm) * OR_NC(ln);
    double buf[OR_NC(OR_LMAX) * OR_NC(OR_LMAX) * OR_NC(OR_LMAX)];
    double C[3], A[3], B[3];
    for (int x = 0; x < 3; x++) {
        C[x] = aux->center[3 * P + x] + sP[x];
        A[x] = ao->center[3 * mu + x];
        B[x] = ao->center[3 * nu + x] + sNu[x];
    }
    memset(out, 0, sizeof(double) * n);
    for (int k = 0; k < aux->nprim[P]; k++)
        for (int i = 0; i < ao->nprim[mu]; i++)
            for (int j = 0; j < ao->nprim[nu]; j++) {
                int ok = aux->prim_off[P] + k, oi = ao->prim_off[mu] + i, oj = ao->prim_off[nu] + j;
                or_prim3c(kernel, omega, lP, aux->exps[ok], C, lm, ao->exps[oi], A, ln, ao->exps[oj], B, buf);
                double c = caux[ok] * cao[oi] * cao[oj];
                for (int e = 0; e < n; e++) out[e] += c * buf[e];
            }
}

/* ------------------------------------------------------------------ */
/* Lattice helpers                                                     */
/* ------------------------------------------------------------------ */

typedef struct {
    double a[3][3];  /* rows: lattice vectors */
    double b[3][3];  /* rows: reciprocal vectors, a_i . b_j = 2 pi delta_ij */
    double vol;
    int nk[3];
    int Nk;
} or_lattice;

static void lattice_init(or_lattice *L, const double *a9, const int *kmesh)
{
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) L->a[i][j] = a9[3 * i + j];
    double (*a)[3] = L->a;
    double det = a[0][0] * (a[1][1] * a[2][2] - a[1][2] * a[2][1]) -
                 a[0][1] * (a[1][0] * a[2][2] - a[1][2] * a[2][0]) +
                 a[0][2] * (a[1][0] * a[2][1] - a[1][1] * a[2][0]);
    L->vol = fabs(det);
    /* b_i = 2 pi (a_j x a_k) / det */
    for (int i = 0; i < 3; i++) {
        int j = (i + 1) % 3, k = (i + 2) % 3;
        L->b[i][0] = 2 * OR_PI * (a[j][1] * a[k][2] - a[j][2] * a[k][1]) / det;
        L->b[i][1] = 2 * OR_PI * (a[j][2] * a[k][0] - a[j][0] * a[k][2]) / det;
        L->b[i][2] = 2 * OR_PI * (a[j][0] * a[k][1] - a[j][1] * a[k][0]) / det;
    }
    for (int i = 0; i < 3; i++) L->nk[i] = kmesh[i];
    L->Nk = kmesh[0] * kmesh[1] * kmesh[2];
}

static double norm3(const double *v) { return sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]); }

static void lat_vec(const or_lattice *L, const int *m, double *r)
{
    for (int x = 0; x < 3; x++) r[x] = m[0] * L->a[0][x] + m[1] * L->a[1][x] + m[2] * L->a[2][x];
}

/* integer box of lattice coordinates covering the ball |m.a - c| <= rad */
static void lat_box(const or_lattice *L, const double *c, double rad, int *lo, int *hi)
{
    for (int i = 0; i < 3; i++) {
        double f = (c[0] * L->b[i][0] + c[1] * L->b[i][1] + c[2] * L->b[i][2]) / (2 * OR_PI);
        double e = rad * norm3(L->b[i]) / (2 * OR_PI);
        lo[i] = (int)floor(f - e) - 1;
        hi[i] = (int)ceil(f + e) + 1;
    }
}

static int imod(int a, int n) { int r = a % n; return r < 0 ? r + n : r; }

static int bvk_index(const or_lattice *L, const int *m)
{
    return (imod(m[0], L->nk[0]) * L->nk[1] + imod(m[1], L->nk[1])) * L->nk[2] + imod(m[2], L->nk[2]);
}

static void k_frac(const or_lattice *L, int kidx, int *n)
{
    n[2] = kidx % L->nk[2];
    n[1] = (kidx / L->nk[2]) % L->nk[1];
    n[0] = kidx / (L->nk[1] * L->nk[2]);
}

/* e^{i k.m} for k = sum n_i/N_i b_i and m = sum m_i a_i: the angle is
 * 2 pi sum_i (n_i m_i mod N_i)/N_i, reduced exactly in integers. */
static double complex k_phase(const or_lattice *L, const int *n, const int *m)
{
    double frac = 0.0;
    for (int i = 0; i < 3; i++) frac += (double)imod(n[i] * m[i], L->nk[i]) / L->nk[i];
    double ang = 2 * OR_PI * frac;
    return cos(ang) + I * sin(ang);
}

/* ------------------------------------------------------------------ */
/* Screening of the SR double lattice sum (Supplementary Material)      */
/* ------------------------------------------------------------------ */

#define OR_EPS_PRIME 1e-4
#define OR_DR 1.0
#define OR_MAXWIN 512

typedef struct {
    double Rc_cut;
    int nwin;
    double R12_cut[OR_MAXWIN];
    double R12_max;
    double amu, anu;   /* most diffuse exponents, for the pair centre */
} or_sr_bound;

static int min_exp_index(const or_basis *b, int s)
{
    int o = b->prim_off[s], best = o;
    for (int i = 1; i < b->nprim[s]; i++)
        if (b->exps[o + i] < b->exps[best]) best = o + i;
    return best;
}

/* the most diffuse primitive of a shell treated as a normalised 1s */
static double coef_1s(const or_basis *b, const double *cn, int s, int idx)
{
    double a = b->exps[idx];
    return fabs(cn[idx]) * pow(2.0 * a / OR_PI, 0.75) / prim_norm(a, b->l[s]);
}

static int count_nf_cells(const or_lattice *L)
{
    double rad = 3.0 * cbrt(L->vol);
    double z[3] = {0, 0, 0};
    int lo[3], hi[3], n = 0;
    lat_box(L, z, rad, lo, hi);
    for (int i = lo[0]; i <= hi[0]; i++)
        for (int j = lo[1]; j <= hi[1]; j++)
            for (int k = lo[2]; k <= hi[2]; k++) {
                int m[3] = {i, j, k};
                double r[3];
                lat_vec(L, m, r);
                if (norm3(r) <= rad) n++;
            }
    return n;
}

/* Eq. Ncell: cells in the shell [R, R+dR] */
static double ncell_shell(const or_lattice *L, double R, int nnf)
{
    double R0 = sqrt(nnf * L->vol / (8 * OR_PI * OR_DR)) - OR_DR;
    if (R > R0) return 4 * OR_PI / L->vol * 2.0 * (R + OR_DR) * (R + OR_DR) * OR_DR;
    return nnf;
}

/* f(R; omega) = [erf(eta1 R) - erf(eta2 R)]/R, limit 2(eta1-eta2)/sqrt(pi) at 0 */
static double f_rc(double R, double e1, double e2)
{
    if (R < 1e-8) return 2.0 * (e1 - e2) / sqrt(OR_PI);
    return (erf(e1 * R) - erf(e2 * R)) / R;
}

/* lattice sum of h(R12) = e^{-beta R12^2} over images n with h >= eps',
 * restricted to R12 > rmin; never smaller than the largest single term. */
/* polynomial growth of a Cartesian pair of degrees (lm, ln) at separation R12,
 * relative to the 1s treatment (1 for s functions) */
static double ang_r12(int lm, int ln, double am, double an, double R)
{
    double p = am + an;
    return pow(1.0 + sqrt(4.0 * am) * an / p * R, lm) * pow(1.0 + sqrt(4.0 * an) * am / p * R, ln);
}

/* polynomial growth of the erfc tail seen by functions of degree lP (aux)
 * and lm + ln (pair) at aux-pair distance R, relative to the 1s treatment */
static double ang_rc(int lP, int lpair, double aP, double p, double eta2, double R)
{
    double x = 2.0 * eta2 * eta2 * R;
    return pow(1.0 + x / sqrt(aP), lP) * pow(1.0 + x / sqrt(p), lpair);
}

static double hsum(const or_lattice *L, const double *d0, double beta, double rmin, double *hmax_out,
                   int lm, int ln, double am, double an)
{
    double rad = sqrt(-log(OR_EPS_PRIME) / beta);
    int lo[3], hi[3];
    double nd[3] = {-d0[0], -d0[1], -d0[2]};
    lat_box(L, nd, rad, lo, hi);
    double s = 0.0, hmax = 0.0;
    for (int i = lo[0]; i <= hi[0]; i++)
        for (int j = lo[1]; j <= hi[1]; j++)
            for (int k = lo[2]; k <= hi[2]; k++) {
                int m[3] = {i, j, k};
                double r[3];
                lat_vec(L, m, r);
                for (int x = 0; x < 3; x++) r[x] += d0[x];
                double R = norm3(r);
                double h0 = exp(-beta * R * R);
                double h = h0 * ang_r12(lm, ln, am, an, R);
                if (R > rmin && h0 >= OR_EPS_PRIME) s += h;
                if (R > rmin && h > hmax) hmax = h;
            }
    if (hmax_out) *hmax_out = hmax;
    return s;
}

/* Bounds for one (aux shell P, AO shell mu, AO shell nu) triple. */
static void sr_bounds(const or_lattice *L, int nnf, double omega, double eps,
                      const or_basis *aux, const double *caux, int P,
                      const or_basis *ao, const double *cao, int mu, int nu, or_sr_bound *out)
{
    int iP = min_exp_index(aux, P), im = min_exp_index(ao, mu), in = min_exp_index(ao, nu);
    double aP = aux->exps[iP], am = ao->exps[im], an = ao->exps[in];
    double p = am + an, beta = am * an / p;
    double eta1 = 1.0 / sqrt(1.0 / aP + 1.0 / p);
    double eta2 = 1.0 / sqrt(1.0 / (eta1 * eta1) + 1.0 / (omega * omega));
    /* Decay rates (beta, eta1, eta2) come from the most diffuse primitives.
     * The prefactor is the textbook s-type one, pi^3 C_P C_mu C_nu /
     * (a_P p)^{3/2} (the printed (pi/4)^3 is read as pi^3), summed over all
     * primitive combinations of the contractions, each primitive treated as a
     * normalised 1s: a compact primitive pair with a large weight carries most
     * of the pair's charge even though it does not set the decay. */
    double sP = 0.0, sA = 0.0;
    for (int k = 0; k < aux->nprim[P]; k++) {
        int o = aux->prim_off[P] + k;
        sP += coef_1s(aux, caux, P, o) / pow(aux->exps[o], 1.5);
    }
    for (int i = 0; i < ao->nprim[mu]; i++)
        for (int j = 0; j < ao->nprim[nu]; j++) {
            int oi = ao->prim_off[mu] + i, oj = ao->prim_off[nu] + j;
            sA += coef_1s(ao, cao, mu, oi) * coef_1s(ao, cao, nu, oj) / pow(ao->exps[oi] + ao->exps[oj], 1.5);
        }
    double A = OR_PI * OR_PI * OR_PI * sP * sA;
    double d0[3];
    for (int x = 0; x < 3; x++) d0[x] = ao->center[3 * nu + x] - ao->center[3 * mu + x];
    int lP = aux->l[P], lm = ao->l[mu], ln = ao->l[nu];
    double hmax;
    double Sh = hsum(L, d0, beta, -1.0, &hmax, lm, ln, am, an);
    if (Sh < hmax) Sh = hmax;
    out->amu = am; out->anu = an;
    /* Eq. bound_Rc: smallest Rc with g(Rc) < eps; g decreases monotonically */
    double c0 = A * Sh * 4 * OR_PI / L->vol / sqrt(OR_PI) / (2 * eta2 * eta2 * eta2);
#define OR_GRC(R) (c0 / (R) * exp(-eta2 * eta2 * (R) * (R)) * ang_rc(lP, lm + ln, aP, p, eta2, (R)))
    double lo = 1e-6, hi = 1e-6;
    while (OR_GRC(hi) >= eps && hi < 1e4) hi *= 2;
    if (hi > lo) {
        for (int it = 0; it < 200; it++) {
            double mid = 0.5 * (lo + hi);
            if (OR_GRC(mid) >= eps) lo = mid; else hi = mid;
        }
    }
#undef OR_GRC
    out->Rc_cut = hi;
    /* Eq. R12cutmin: smallest x at which the continuum estimate
     * (4 pi/Omega) x/(2 beta) e^{-beta x^2} is no smaller than the
     * eps'-truncated lattice sum of h beyond x */
    double xmax = sqrt(-log(OR_EPS_PRIME) / beta) + OR_DR;
    double r12min = xmax;
    for (double x = 0.0; x <= xmax; x += 0.01) {
        double est = 4 * OR_PI / L->vol * x / (2 * beta) * exp(-beta * x * x) * ang_r12(lm, ln, am, an, x);
        double sum = hsum(L, d0, beta, x, NULL, lm, ln, am, an);
        if (est >= sum) { r12min = x; break; }
    }
    /* Eq. bound_R12_FF per window [w dR, (w+1) dR], then Eq. bound_R12 */
    int nw = (int)floor(out->Rc_cut / OR_DR) + 1;
    if (nw > OR_MAXWIN) nw = OR_MAXWIN;
    out->nwin = nw;
    out->R12_max = 0.0;
    double x0 = 1.0 / sqrt(2 * beta);
    for (int w = 0; w < nw; w++) {
        double R = w * OR_DR;
        double c1 = A * ncell_shell(L, R, nnf) * f_rc(R, eta1, eta2) * ang_rc(lP, lm + ln, aP, p, eta2, R) *
                    4 * OR_PI / L->vol / (2 * beta);
#define OR_GR12(x) (c1 * (x) * exp(-beta * (x) * (x)) * ang_r12(lm, ln, am, an, (x)))
        double x;
        /* the estimate rises to a maximum and then falls: bracket the outer root */
        double xm = x0, vm = OR_GR12(x0);
        for (double t = 0.0; t < x0 + 10.0 / sqrt(beta); t += 0.05 / sqrt(beta))
            if (OR_GR12(t) > vm) { vm = OR_GR12(t); xm = t; }
        if (vm < eps) {
            x = 0.0;
        } else {
            double a = xm, b = xm + 1e-3;
            while (OR_GR12(b) >= eps && b < 1e4) b *= 2;
            for (int it = 0; it < 200; it++) {
                double mid = 0.5 * (a + b);
                if (OR_GR12(mid) >= eps) a = mid; else b = mid;
            }
            x = b;
        }
#undef OR_GR12
        out->R12_cut[w] = x > r12min ? x : r12min;
        if (out->R12_cut[w] > out->R12_max) out->R12_max = out->R12_cut[w];
    }
}

/* j2c SR screening: the three-center bound with the pair replaced by the
 * second aux function (S_h = 1): keep |D + l - C| <= Rc_cut. */
static double sr2_bound(const or_lattice *L, double omega, double eps,
                        const or_basis *aux, const double *caux, int P, int Q)
{
    int iP = min_exp_index(aux, P), iQ = min_exp_index(aux, Q);
    double aP = aux->exps[iP], aQ = aux->exps[iQ];
    double eta1 = 1.0 / sqrt(1.0 / aP + 1.0 / aQ);
    double eta2 = 1.0 / sqrt(1.0 / (eta1 * eta1) + 1.0 / (omega * omega));
    double sP = 0.0, sQ = 0.0;
    for (int k = 0; k < aux->nprim[P]; k++) {
        int o = aux->prim_off[P] + k;
        sP += coef_1s(aux, caux, P, o) / pow(aux->exps[o], 1.5);
    }
    for (int k = 0; k < aux->nprim[Q]; k++) {
        int o = aux->prim_off[Q] + k;
        sQ += coef_1s(aux, caux, Q, o) / pow(aux->exps[o], 1.5);
    }
    double A = OR_PI * OR_PI * OR_PI * sP * sQ;
    double c0 = A * 4 * OR_PI / L->vol / sqrt(OR_PI) / (2 * eta2 * eta2 * eta2);
    double lo = 1e-6, hi = 1e-6;
    while (c0 / hi * exp(-eta2 * eta2 * hi * hi) >= eps && hi < 1e4) hi *= 2;
    for (int it = 0; it < 200; it++) {
        double mid = 0.5 * (lo + hi);
        if (c0 / mid * exp(-eta2 * eta2 * mid * mid) >= eps) lo = mid; else hi = mid;
    }
    return hi;
}

/* exported for the tests: bounds of one triple */
int or_sr_bounds(const double *a9, const int *kmesh, double omega, double eps,
                 const or_basis *aux, int P, const or_basis *ao, int mu, int nu,
                 double *Rc_cut, double *R12_cut /*[OR_MAXWIN]*/, int *nwin)
{
    or_lattice L;
    lattice_init(&L, a9, kmesh);
    int naux_p = aux->prim_off[aux->nshell - 1] + aux->nprim[aux->nshell - 1];
    int nao_p = ao->prim_off[ao->nshell - 1] + ao->nprim[ao->nshell - 1];
    double *caux = malloc(sizeof(double) * naux_p), *cao = malloc(sizeof(double) * nao_p);
    or_norm_coeffs(aux, caux); or_norm_coeffs(ao, cao);
    or_sr_bound b;
    sr_bounds(&L, count_nf_cells(&L), omega, eps, aux, caux, P, ao, cao, mu, nu, &b);
    *Rc_cut = b.Rc_cut; *nwin = b.nwin;
    for (int w = 0; w < b.nwin; w++) R12_cut[w] = b.R12_cut[w];
    free(caux); free(cao);
    return 0;
}

/* Keep-rule of the pair density for the AFT and the overlaps: some
 * primitive pair with |c_i c_j| (pi/p)^{3/2} e^{-a b/p R12^2} >= eps_lr. */
static int pair_kept(const or_basis *ao, const double *cao, int mu, int nu, double R12, double eps)
{
    for (int i = 0; i < ao->nprim[mu]; i++)
        for (int j = 0; j < ao->nprim[nu]; j++) {
            int oi = ao->prim_off[mu] + i, oj = ao->prim_off[nu] + j;
            double a = ao->exps[oi], b = ao->exps[oj], p = a + b;
            double v = fabs(cao[oi] * cao[oj]) * pow(OR_PI / p, 1.5) * exp(-a * b / p * R12 * R12);
            if (v >= eps) return 1;
        }
    return 0;
}

/* radius beyond which pair_kept() fails for every primitive pair */
static double pair_radius(const or_basis *ao, const double *cao, int mu, int nu, double eps)
{
    double rmax = 0.0;
    for (int i = 0; i < ao->nprim[mu]; i++)
        for (int j = 0; j < ao->nprim[nu]; j++) {
            int oi = ao->prim_off[mu] + i, oj = ao->prim_off[nu] + j;
            double a = ao->exps[oi], b = ao->exps[oj], p = a + b;
            double c = fabs(cao[oi] * cao[oj]) * pow(OR_PI / p, 1.5);
            if (c >= eps) {
                double r = sqrt(log(c / eps) / (a * b / p));
                if (r > rmax) rmax = r;
            }
        }
    return rmax;
}

/* ------------------------------------------------------------------ */
/* j3c, route R1 (range separation)                                    */
/* ------------------------------------------------------------------ */

typedef struct {
    double omega, eps_sr, eps_lr;
    int gmesh[3];
    int do_sr, do_g0, do_lr;
    int direct_phase;   /* 1: apply phases per lattice term (no BvK folding) */
} or_opts;

/* G-vector list of the box mesh n_i in [-(N_i-1)/2, (N_i-1)/2] */
static int gbox(const int *gm, int (*g)[3])
{
    int n = 0;
    for (int i = -(gm[0] - 1) / 2; i <= (gm[0] - 1) / 2; i++)
        for (int j = -(gm[1] - 1) / 2; j <= (gm[1] - 1) / 2; j++)
            for (int k = -(gm[2] - 1) / 2; k <= (gm[2] - 1) / 2; k++) {
                if (g) { g[n][0] = i; g[n][1] = j; g[n][2] = k; }
                n++;
            }
    return n;
}

/* fractional coordinates of k12 = k2 - k1 folded to [-1/2, 1/2) */
static void k12_frac(const or_lattice *L, const int *n1, const int *n2, double *f)
{
    for (int i = 0; i < 3; i++) {
        int d = imod(n2[i] - n1[i], L->nk[i]);
        double x = (double)d / L->nk[i];
        if (x >= 0.5) x -= 1.0;
        f[i] = x;
    }
}

static void frac_to_cart(const or_lattice *L, const double *f, const int *g, double *q)
{
    for (int x = 0; x < 3; x++)
        q[x] = (g[0] + f[0]) * L->b[0][x] + (g[1] + f[1]) * L->b[1][x] + (g[2] + f[2]) * L->b[2][x];
}

/* Counting SR lattice terms (P shell, mu shell, nu shell, l, d). */
typedef struct { long long terms; long long integrals; } or_count;

/*
 * SR part of Eq. VPmunu_SR.  Output V[pair][iP][imu][inu] (complex),
 * aux shells [s0, s1).  Terms are folded into BvK bins X[lt][dt] (Eq.
 * BvK_latsum_LR) and then contracted with the phases; with direct_phase
 * every term is multiplied by its phases instead.
 */
static void j3c_sr(const or_lattice *L, const or_opts *o, const or_basis *ao, const double *cao,
                   const or_basis *aux, const double *caux, int s0, int s1, int npair,
                   const int *kpairs, double complex *V, or_count *cnt)
{
    int nao = basis_nfunc(ao);
    int *aoff = malloc(sizeof(int) * ao->nshell), *xoff = malloc(sizeof(int) * aux->nshell);
    basis_offsets(ao, aoff); basis_offsets(aux, xoff);
    int nP = 0;
    for (int s = s0; s < s1; s++) nP += OR_NC(aux->l[s]);
    int Nk = L->Nk;
    int nnf = count_nf_cells(L);
    long long terms = 0, ints = 0;
    int ntrip = (s1 - s0) * ao->nshell * ao->nshell;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : terms, ints)
    for (int tr = 0; tr < ntrip; tr++) {
        int P = s0 + tr / (ao->nshell * ao->nshell);
        int mu = (tr / ao->nshell) % ao->nshell, nu = tr % ao->nshell;
        int lP = aux->l[P], lm = ao->l[mu], ln = ao->l[nu];
        int ncP = OR_NC(lP), ncm = OR_NC(lm), ncn = OR_NC(ln), nblk = ncP * ncm * ncn;
        int pofs = xoff[P] - xoff[s0];
        or_sr_bound bd;
        sr_bounds(L, nnf, o->omega, o->eps_sr, aux, caux, P, ao, cao, mu, nu, &bd);
        double *X = NULL;
        if (!o->direct_phase) X = calloc((size_t)Nk * Nk * nblk, sizeof(double));
        double blk[OR_NC(OR_LMAX) * OR_NC(OR_LMAX) * OR_NC(OR_LMAX)];
        const double *A = &ao->center[3 * mu], *B = &ao->center[3 * nu], *C = &aux->center[3 * P];
        double dcen[3];
        for (int x = 0; x < 3; x++) dcen[x] = A[x] - B[x];
        int dlo[3], dhi[3];
        lat_box(L, dcen, bd.R12_max, dlo, dhi);
        for (int d0 = dlo[0]; d0 <= dhi[0]; d0++)
            for (int d1 = dlo[1]; d1 <= dhi[1]; d1++)
                for (int d2 = dlo[2]; d2 <= dhi[2]; d2++) {
                    int dm[3] = {d0, d1, d2};
                    double dv[3], Bd[3], Rc0[3];
                    lat_vec(L, dm, dv);
                    for (int x = 0; x < 3; x++) Bd[x] = B[x] + dv[x];
                    double r12v[3] = {Bd[0] - A[0], Bd[1] - A[1], Bd[2] - A[2]};
                    double R12 = norm3(r12v);
                    if (R12 > bd.R12_max) continue;
                    for (int x = 0; x < 3; x++)
                        Rc0[x] = (bd.amu * A[x] + bd.anu * Bd[x]) / (bd.amu + bd.anu) - C[x];
                    int llo[3], lhi[3];
                    lat_box(L, Rc0, bd.Rc_cut, llo, lhi);
                    int dt = bvk_index(L, dm);
                    for (int l0 = llo[0]; l0 <= lhi[0]; l0++)
                        for (int l1 = llo[1]; l1 <= lhi[1]; l1++)
                            for (int l2 = llo[2]; l2 <= lhi[2]; l2++) {
                                int lm_[3] = {l0, l1, l2};
                                double lv[3], rc[3];
                                lat_vec(L, lm_, lv);
                                for (int x = 0; x < 3; x++) rc[x] = Rc0[x] - lv[x];
                                double Rc = norm3(rc);
                                if (Rc > bd.Rc_cut) continue;
                                int w = (int)floor(Rc / OR_DR);
                                if (w >= bd.nwin) w = bd.nwin - 1;
                                if (R12 > bd.R12_cut[w]) continue;
                                shell3c(2, o->omega, aux, caux, P, lv, ao, cao, mu, nu, dv, blk);
                                terms++;
                                ints += nblk;
                                if (!o->direct_phase) {
                                    int lt = bvk_index(L, lm_);
                                    double *dst = X + ((size_t)lt * Nk + dt) * nblk;
                                    for (int e = 0; e < nblk; e++) dst[e] += blk[e];
                                } else {
                                    for (int pr = 0; pr < npair; pr++) {
                                        int n1[3], n2[3], n12[3];
                                        k_frac(L, kpairs[2 * pr], n1); k_frac(L, kpairs[2 * pr + 1], n2);
                                        for (int x = 0; x < 3; x++) n12[x] = n2[x] - n1[x];
                                        /* e^{-i k12.l} e^{+i k2.d} */
                                        double complex ph = conj(k_phase(L, n12, lm_)) * k_phase(L, n2, dm);
                                        for (int ic = 0; ic < ncP; ic++)
                                            for (int ia = 0; ia < ncm; ia++)
                                                for (int ib = 0; ib < ncn; ib++) {
                                                    size_t idx = (((size_t)pr * nP + pofs + ic) * nao + aoff[mu] + ia) * nao + aoff[nu] + ib;
                                                    V[idx] += ph * blk[(ic * ncm + ia) * ncn + ib];
                                                }
                                    }
                                }
                            }
                }
        if (!o->direct_phase) {
            for (int pr = 0; pr < npair; pr++) {
                int n1[3], n2[3], n12[3];
                k_frac(L, kpairs[2 * pr], n1); k_frac(L, kpairs[2 * pr + 1], n2);
                for (int x = 0; x < 3; x++) n12[x] = n2[x] - n1[x];
                for (int lt = 0; lt < Nk; lt++)
                    for (int dt = 0; dt < Nk; dt++) {
                        int ml[3], md[3];
                        k_frac(L, lt, ml); k_frac(L, dt, md); /* BvK cell j_i in mesh order */
                        double complex ph = conj(k_phase(L, n12, ml)) * k_phase(L, n2, md);
                        const double *src = X + ((size_t)lt * Nk + dt) * nblk;
                        for (int ic = 0; ic < ncP; ic++)
                            for (int ia = 0; ia < ncm; ia++)
                                for (int ib = 0; ib < ncn; ib++) {
                                    size_t idx = (((size_t)pr * nP + pofs + ic) * nao + aoff[mu] + ia) * nao + aoff[nu] + ib;
                                    V[idx] += ph * src[(ic * ncm + ia) * ncn + ib];
                                }
                    }
            }
            free(X);
        }
    }
    if (cnt) { cnt->terms = terms; cnt->integrals = ints; }
    free(aoff); free(xoff);
}

/* aux integrals S_P = int chi_P (per aux function of shells [s0,s1)) */
static void aux_charge(const or_basis *aux, const double *caux, int s0, int s1, double *S)
{
    int n = 0;
    for (int P = s0; P < s1; P++) {
        int lP = aux->l[P], nc = OR_NC(lP);
        double blk[OR_NC(OR_LMAX)];
        memset(blk, 0, sizeof(blk));
        const double *C = &aux->center[3 * P];
        for (int k = 0; k < aux->nprim[P]; k++) {
            int ok = aux->prim_off[P] + k;
            double tmp[OR_NC(OR_LMAX)];
            /* overlap with the constant function 1 */
            or_prim_ovlp(lP, aux->exps[ok], C, 0, 0.0, C, tmp);
            for (int e = 0; e < nc; e++) blk[e] += caux[ok] * tmp[e];
        }
        for (int e = 0; e < nc; e++) S[n + e] = blk[e];
        n += nc;
    }
}

/* S^k_{mu nu} = sum_d e^{i k.d} (phi_mu^0 | phi_nu^d), out[k-list][mu][nu] */
static void ao_ovlp_k(const or_lattice *L, double eps, const or_basis *ao, const double *cao,
                      int nk, const int *klist, double complex *S)
{
    int nao = basis_nfunc(ao);
    int *aoff = malloc(sizeof(int) * ao->nshell);
    basis_offsets(ao, aoff);
    memset(S, 0, sizeof(double complex) * nk * nao * nao);
#pragma omp parallel for schedule(dynamic, 1)
    for (int pr = 0; pr < ao->nshell * ao->nshell; pr++) {
        int mu = pr / ao->nshell, nu = pr % ao->nshell;
        int lm = ao->l[mu], ln = ao->l[nu], ncm = OR_NC(lm), ncn = OR_NC(ln);
        const double *A = &ao->center[3 * mu], *B = &ao->center[3 * nu];
        double rad = pair_radius(ao, cao, mu, nu, eps);
        double dcen[3] = {A[0] - B[0], A[1] - B[1], A[2] - B[2]};
        int lo[3], hi[3];
        lat_box(L, dcen, rad, lo, hi);
        for (int i = lo[0]; i <= hi[0]; i++)
            for (int j = lo[1]; j <= hi[1]; j++)
                for (int k = lo[2]; k <= hi[2]; k++) {
                    int dm[3] = {i, j, k};
                    double dv[3], Bd[3];
                    lat_vec(L, dm, dv);
                    for (int x = 0; x < 3; x++) Bd[x] = B[x] + dv[x];
                    double r[3] = {Bd[0] - A[0], Bd[1] - A[1], Bd[2] - A[2]};
                    if (!pair_kept(ao, cao, mu, nu, norm3(r), eps)) continue;
                    double blk[OR_NC(OR_LMAX) * OR_NC(OR_LMAX)], tmp[OR_NC(OR_LMAX) * OR_NC(OR_LMAX)];
                    memset(blk, 0, sizeof(blk));
                    for (int a = 0; a < ao->nprim[mu]; a++)
                        for (int b = 0; b < ao->nprim[nu]; b++) {
                            int oa = ao->prim_off[mu] + a, ob = ao->prim_off[nu] + b;
                            or_prim_ovlp(lm, ao->exps[oa], A, ln, ao->exps[ob], Bd, tmp);
                            for (int e = 0; e < ncm * ncn; e++) blk[e] += cao[oa] * cao[ob] * tmp[e];
                        }
                    for (int kk = 0; kk < nk; kk++) {
                        int n[3];
                        k_frac(L, klist[kk], n);
                        double complex ph = k_phase(L, n, dm);
                        for (int ia = 0; ia < ncm; ia++)
                            for (int ib = 0; ib < ncn; ib++)
                                S[((size_t)kk * nao + aoff[mu] + ia) * nao + aoff[nu] + ib] += ph * blk[ia * ncn + ib];
                    }
                }
    }
    free(aoff);
}

/* chi^_P(q) for aux functions of shells [s0,s1) */
static void aux_ft(const or_basis *aux, const double *caux, int s0, int s1, const double *q, double complex *out)
{
    int n = 0;
    for (int P = s0; P < s1; P++) {
        int lP = aux->l[P], nc = OR_NC(lP);
        double complex tmp[OR_NC(OR_LMAX)];
        for (int e = 0; e < nc; e++) out[n + e] = 0;
        const double *C = &aux->center[3 * P];
        for (int k = 0; k < aux->nprim[P]; k++) {
            int ok = aux->prim_off[P] + k;
            or_prim_ft(lP, aux->exps[ok], C, 0, 0.0, C, q, tmp);
            for (int e = 0; e < nc; e++) out[n + e] += caux[ok] * tmp[e];
        }
        n += nc;
    }
}

/*
 * LR part (Eq. VPmunu_LR, prefactor 4 pi/Omega) or, with full_coulomb, the
 * whole integral in reciprocal space (Eq. VPmunu_FT).  The pair transform
 * rho^{k1k2}(q) = sum_d e^{i k2.d} FT[phi_mu^0 phi_nu^d](q) (Eq.
 * AFT_pairden) is accumulated per BvK bin of d and then phased.
 */
static void j3c_recip(const or_lattice *L, const or_opts *o, int full_coulomb, const int *gmesh,
                      const or_basis *ao, const double *cao, const or_basis *aux, const double *caux,
                      int s0, int s1, int npair, const int *kpairs, double complex *V)
{
    int nao = basis_nfunc(ao);
    int *aoff = malloc(sizeof(int) * ao->nshell);
    basis_offsets(ao, aoff);
    int nP = 0;
    for (int s = s0; s < s1; s++) nP += OR_NC(aux->l[s]);
    int NG = gbox(gmesh, NULL);
    int (*g)[3] = malloc(sizeof(int) * 3 * NG);
    gbox(gmesh, g);
    int Nk = L->Nk;
    /* distinct k12 among the requested pairs */
    int *k12id = malloc(sizeof(int) * npair);
    int *k12rep = malloc(sizeof(int) * 2 * npair);
    int nk12 = 0;
    for (int pr = 0; pr < npair; pr++) {
        int n1[3], n2[3];
        k_frac(L, kpairs[2 * pr], n1); k_frac(L, kpairs[2 * pr + 1], n2);
        int key = 0;
        for (int x = 0; x < 3; x++) key = key * L->nk[x] + imod(n2[x] - n1[x], L->nk[x]);
        int f = -1;
        for (int j = 0; j < nk12; j++) if (k12rep[2 * j] == key) f = j;
        if (f < 0) { f = nk12; k12rep[2 * nk12] = key; k12rep[2 * nk12 + 1] = pr; nk12++; }
        k12id[pr] = f;
    }
    for (int kq = 0; kq < nk12; kq++) {
        int pr0 = k12rep[2 * kq + 1];
        int n1[3], n2[3];
        k_frac(L, kpairs[2 * pr0], n1); k_frac(L, kpairs[2 * pr0 + 1], n2);
        double f12[3];
        k12_frac(L, n1, n2, f12);
        /* Y[dt][G][mu][nu] */
        double complex *Y = calloc((size_t)Nk * NG * nao * nao, sizeof(double complex));
        double complex *W = calloc((size_t)NG * nP, sizeof(double complex));
#pragma omp parallel for schedule(dynamic, 1)
        for (int ig = 0; ig < NG; ig++) {
            double q[3];
            frac_to_cart(L, f12, g[ig], q);
            double q2 = q[0] * q[0] + q[1] * q[1] + q[2] * q[2];
            if (q2 < 1e-14) continue; /* the q = 0 term is excluded */
            double w = 4 * OR_PI / L->vol / q2;
            if (!full_coulomb) w *= exp(-q2 / (4 * o->omega * o->omega));
            aux_ft(aux, caux, s0, s1, q, &W[(size_t)ig * nP]);
            for (int e = 0; e < nP; e++) W[(size_t)ig * nP + e] *= w;
        }
#pragma omp parallel for schedule(dynamic, 1)
        for (int pr = 0; pr < ao->nshell * ao->nshell; pr++) {
            int mu = pr / ao->nshell, nu = pr % ao->nshell;
            int lm = ao->l[mu], ln = ao->l[nu], ncm = OR_NC(lm), ncn = OR_NC(ln);
            const double *A = &ao->center[3 * mu], *B = &ao->center[3 * nu];
            double rad = pair_radius(ao, cao, mu, nu, o->eps_lr);
            double dcen[3] = {A[0] - B[0], A[1] - B[1], A[2] - B[2]};
            int lo[3], hi[3];
            lat_box(L, dcen, rad, lo, hi);
            double complex tmp[OR_NC(OR_LMAX) * OR_NC(OR_LMAX)];
            for (int i = lo[0]; i <= hi[0]; i++)
                for (int j = lo[1]; j <= hi[1]; j++)
                    for (int k = lo[2]; k <= hi[2]; k++) {
                        int dm[3] = {i, j, k};
                        double dv[3], Bd[3];
                        lat_vec(L, dm, dv);
                        for (int x = 0; x < 3; x++) Bd[x] = B[x] + dv[x];
                        double r[3] = {Bd[0] - A[0], Bd[1] - A[1], Bd[2] - A[2]};
                        if (!pair_kept(ao, cao, mu, nu, norm3(r), o->eps_lr)) continue;
                        int dt = bvk_index(L, dm);
                        for (int ig = 0; ig < NG; ig++) {
                            double q[3];
                            frac_to_cart(L, f12, g[ig], q);
                            double complex *dst = &Y[((size_t)dt * NG + ig) * nao * nao];
                            for (int a = 0; a < ao->nprim[mu]; a++)
                                for (int b = 0; b < ao->nprim[nu]; b++) {
                                    int oa = ao->prim_off[mu] + a, ob = ao->prim_off[nu] + b;
                                    or_prim_ft(lm, ao->exps[oa], A, ln, ao->exps[ob], Bd, q, tmp);
                                    double c = cao[oa] * cao[ob];
                                    for (int ia = 0; ia < ncm; ia++)
                                        for (int ib = 0; ib < ncn; ib++)
                                            dst[(aoff[mu] + ia) * nao + aoff[nu] + ib] += c * tmp[ia * ncn + ib];
                                }
                        }
                    }
        }
        /* V[pair] += sum_G conj(W_P(q)) sum_dt e^{i k2.dt} Y[dt](G) */
        for (int pr = 0; pr < npair; pr++) {
            if (k12id[pr] != kq) continue;
            int m1[3], m2[3];
            k_frac(L, kpairs[2 * pr], m1); k_frac(L, kpairs[2 * pr + 1], m2);
            double complex *ph = malloc(sizeof(double complex) * Nk);
            for (int dt = 0; dt < Nk; dt++) {
                int md[3];
                k_frac(L, dt, md);
                ph[dt] = k_phase(L, m2, md);
            }
#pragma omp parallel for schedule(static)
            for (int iP = 0; iP < nP; iP++) {
                for (int ig = 0; ig < NG; ig++) {
                    double complex wc = conj(W[(size_t)ig * nP + iP]);
                    if (wc == 0) continue;
                    for (int dt = 0; dt < Nk; dt++) {
                        double complex f = wc * ph[dt];
                        const double complex *src = &Y[((size_t)dt * NG + ig) * nao * nao];
                        double complex *dst = &V[((size_t)pr * nP + iP) * nao * nao];
                        for (int e = 0; e < nao * nao; e++) dst[e] += f * src[e];
                    }
                }
            }
            free(ph);
        }
        free(Y); free(W);
    }
    free(g); free(k12id); free(k12rep); free(aoff);
}

static int basis_nprim_total(const or_basis *b)
{
    return b->prim_off[b->nshell - 1] + b->nprim[b->nshell - 1];
}

/*
 * Route R1: V = SR (Eq. VPmunu_SR, incl. the G=0 correction) + LR (Eq.
 * VPmunu_LR).  V is overwritten: [npair][nP][nao][nao] complex.
 * counts[0] = SR lattice terms, counts[1] = SR Cartesian integrals.
 */
int or_j3c(const double *a9, const int *kmesh, const or_basis *ao, const or_basis *aux,
           const or_opts *o, int s0, int s1, int npair, const int *kpairs,
           double complex *V, long long *counts)
{
    or_lattice L;
    lattice_init(&L, a9, kmesh);
    double *cao = malloc(sizeof(double) * basis_nprim_total(ao));
    double *caux = malloc(sizeof(double) * basis_nprim_total(aux));
    or_norm_coeffs(ao, cao); or_norm_coeffs(aux, caux);
    int nao = basis_nfunc(ao), nP = 0;
    for (int s = s0; s < s1; s++) nP += OR_NC(aux->l[s]);
    memset(V, 0, sizeof(double complex) * (size_t)npair * nP * nao * nao);
    or_count cnt = {0, 0};
    if (o->do_sr) j3c_sr(&L, o, ao, cao, aux, caux, s0, s1, npair, kpairs, V, &cnt);
    if (o->do_g0) {
        /* -pi/(Omega omega^2) S_P S^k_{mu nu} on pairs with k1 = k2 */
        double *SP = malloc(sizeof(double) * nP);
        aux_charge(aux, caux, s0, s1, SP);
        double complex *Sk = malloc(sizeof(double complex) * nao * nao);
        for (int pr = 0; pr < npair; pr++) {
            if (kpairs[2 * pr] != kpairs[2 * pr + 1]) continue;
            ao_ovlp_k(&L, o->eps_lr, ao, cao, 1, &kpairs[2 * pr], Sk);
            double f = OR_PI / (L.vol * o->omega * o->omega);
            for (int iP = 0; iP < nP; iP++)
                for (int e = 0; e < nao * nao; e++)
                    V[((size_t)pr * nP + iP) * nao * nao + e] -= f * SP[iP] * Sk[e];
        }
        free(SP); free(Sk);
    }
    if (o->do_lr) j3c_recip(&L, o, 0, o->gmesh, ao, cao, aux, caux, s0, s1, npair, kpairs, V);
    if (counts) { counts[0] = cnt.terms; counts[1] = cnt.integrals; }
    free(cao); free(caux);
    return 0;
}

/* Route R2: the whole integral in reciprocal space on the G box gmesh. */
int or_j3c_fullG(const double *a9, const int *kmesh, const or_basis *ao, const or_basis *aux,
                 const or_opts *o, const int *gmesh, int s0, int s1, int npair, const int *kpairs,
                 double complex *V)
{
    or_lattice L;
    lattice_init(&L, a9, kmesh);
    double *cao = malloc(sizeof(double) * basis_nprim_total(ao));
    double *caux = malloc(sizeof(double) * basis_nprim_total(aux));
    or_norm_coeffs(ao, cao); or_norm_coeffs(aux, caux);
    int nao = basis_nfunc(ao), nP = 0;
    for (int s = s0; s < s1; s++) nP += OR_NC(aux->l[s]);
    memset(V, 0, sizeof(double complex) * (size_t)npair * nP * nao * nao);
    j3c_recip(&L, o, 1, gmesh, ao, cao, aux, caux, s0, s1, npair, kpairs, V);
    free(cao); free(caux);
    return 0;
}

/* ------------------------------------------------------------------ */
/* j2c                                                                 */
/* ------------------------------------------------------------------ */

/*
 * J^k_{PQ} = sum_l e^{i k.l} (chi_P^0 | erfc | chi_Q^l)
 *          - delta_{k,0} pi/(Omega omega^2) S_P S_Q
 *          + 4 pi/Omega sum_{q != 0} e^{-q^2/4 omega^2}/q^2 conj(chi^_P(q)) chi^_Q(q)
 * (route R1; full_coulomb = 1 gives route R2 on gmesh2).  J[nk][naux][naux].
 */
static int j2c_any(const double *a9, const int *kmesh, const or_basis *aux, const or_opts *o,
                   int full, const int *gmesh2, int nk, const int *klist, double complex *J)
{
    or_lattice L;
    lattice_init(&L, a9, kmesh);
    double *caux = malloc(sizeof(double) * basis_nprim_total(aux));
    or_norm_coeffs(aux, caux);
    int naux = basis_nfunc(aux);
    int *xoff = malloc(sizeof(int) * aux->nshell);
    basis_offsets(aux, xoff);
    memset(J, 0, sizeof(double complex) * nk * naux * naux);
    if (!full) {
        if (o->do_sr) {
#pragma omp parallel for schedule(dynamic, 1)
            for (int pq = 0; pq < aux->nshell * aux->nshell; pq++) {
                int P = pq / aux->nshell, Q = pq % aux->nshell;
                int lP = aux->l[P], lQ = aux->l[Q], ncP = OR_NC(lP), ncQ = OR_NC(lQ);
                double Rcut = sr2_bound(&L, o->omega, o->eps_sr, aux, caux, P, Q);
                const double *C = &aux->center[3 * P], *D = &aux->center[3 * Q];
                double cen[3] = {C[0] - D[0], C[1] - D[1], C[2] - D[2]};
                int lo[3], hi[3];
                lat_box(&L, cen, Rcut, lo, hi);
                double blk[OR_NC(OR_LMAX) * OR_NC(OR_LMAX)], tmp[OR_NC(OR_LMAX) * OR_NC(OR_LMAX)];
                for (int i = lo[0]; i <= hi[0]; i++)
                    for (int j = lo[1]; j <= hi[1]; j++)
                        for (int k = lo[2]; k <= hi[2]; k++) {
                            int lm[3] = {i, j, k};
                            double lv[3], Dl[3];
                            lat_vec(&L, lm, lv);
                            for (int x = 0; x < 3; x++) Dl[x] = D[x] + lv[x];
                            double r[3] = {Dl[0] - C[0], Dl[1] - C[1], Dl[2] - C[2]};
                            if (norm3(r) > Rcut) continue;
                            memset(blk, 0, sizeof(blk));
                            for (int a = 0; a < aux->nprim[P]; a++)
                                for (int b = 0; b < aux->nprim[Q]; b++) {
                                    int oa = aux->prim_off[P] + a, ob = aux->prim_off[Q] + b;
                                    or_prim2c(2, o->omega, lP, aux->exps[oa], C, lQ, aux->exps[ob], Dl, tmp);
                                    for (int e = 0; e < ncP * ncQ; e++) blk[e] += caux[oa] * caux[ob] * tmp[e];
                                }
                            for (int kk = 0; kk < nk; kk++) {
                                int n[3];
                                k_frac(&L, klist[kk], n);
                                double complex ph = k_phase(&L, n, lm);
                                for (int a = 0; a < ncP; a++)
                                    for (int b = 0; b < ncQ; b++)
                                        J[((size_t)kk * naux + xoff[P] + a) * naux + xoff[Q] + b] += ph * blk[a * ncQ + b];
                            }
                        }
            }
        }
        if (o->do_g0) {
            double *S = malloc(sizeof(double) * naux);
            aux_charge(aux, caux, 0, aux->nshell, S);
            double f = OR_PI / (L.vol * o->omega * o->omega);
            for (int kk = 0; kk < nk; kk++) {
                if (klist[kk] != 0) continue;
                for (int a = 0; a < naux; a++)
                    for (int b = 0; b < naux; b++) J[((size_t)kk * naux + a) * naux + b] -= f * S[a] * S[b];
            }
            free(S);
        }
    }
    if (full || o->do_lr) {
        const int *gm = full ? gmesh2 : o->gmesh;
        int NG = gbox(gm, NULL);
        int (*g)[3] = malloc(sizeof(int) * 3 * NG);
        gbox(gm, g);
        for (int kk = 0; kk < nk; kk++) {
            int n[3], z[3] = {0, 0, 0};
            k_frac(&L, klist[kk], n);
            double f[3];
            k12_frac(&L, z, n, f);
#pragma omp parallel
            {
                double complex *acc = calloc((size_t)naux * naux, sizeof(double complex));
                double complex *ch = malloc(sizeof(double complex) * naux);
#pragma omp for schedule(dynamic, 4)
                for (int ig = 0; ig < NG; ig++) {
                    double q[3];
                    frac_to_cart(&L, f, g[ig], q);
                    double q2 = q[0] * q[0] + q[1] * q[1] + q[2] * q[2];
                    if (q2 < 1e-14) continue;
                    double w = 4 * OR_PI / L.vol / q2;
                    if (!full) w *= exp(-q2 / (4 * o->omega * o->omega));
                    aux_ft(aux, caux, 0, aux->nshell, q, ch);
                    for (int a = 0; a < naux; a++)
                        for (int b = 0; b < naux; b++) acc[a * naux + b] += w * conj(ch[a]) * ch[b];
                }
#pragma omp critical
                for (int e = 0; e < naux * naux; e++) J[(size_t)kk * naux * naux + e] += acc[e];
                free(acc); free(ch);
            }
        }
        free(g);
    }
    free(caux); free(xoff);
    return 0;
}

int or_j2c(const double *a9, const int *kmesh, const or_basis *aux, const or_opts *o,
           int nk, const int *klist, double complex *J)
{
    return j2c_any(a9, kmesh, aux, o, 0, NULL, nk, klist, J);
}

int or_j2c_fullG(const double *a9, const int *kmesh, const or_basis *aux, const or_opts *o,
                 const int *gmesh, int nk, const int *klist, double complex *J)
{
    return j2c_any(a9, kmesh, aux, o, 1, gmesh, nk, klist, J);
}

/* Textbook Cholesky J = L L^H of a Hermitian matrix (column by column).
 * Returns 0, or 1 + the index of the first non-positive pivot. */
int or_cholesky(int n, const double complex *A, double complex *Lo)
{
    memset(Lo, 0, sizeof(double complex) * n * n);
    for (int j = 0; j < n; j++) {
        double d = creal(A[j * n + j]);
        for (int k = 0; k < j; k++) d -= creal(Lo[j * n + k] * conj(Lo[j * n + k]));
        if (!(d > 0.0)) return 1 + j;
        double djj = sqrt(d);
        Lo[j * n + j] = djj;
        for (int i = j + 1; i < n; i++) {
            double complex s = A[i * n + j];
            for (int k = 0; k < j; k++) s -= Lo[i * n + k] * conj(Lo[j * n + k]);
            Lo[i * n + j] = s / djj;
        }
    }
    return 0;
}

/* helpers exported for the tests */
void or_aux_charge(const or_basis *aux, double *S)
{
    double *c = malloc(sizeof(double) * basis_nprim_total(aux));
    or_norm_coeffs(aux, c);
    aux_charge(aux, c, 0, aux->nshell, S);
    free(c);
}

int or_count_nf_cells(const double *a9)
{
    or_lattice L;
    int km[3] = {1, 1, 1};
    lattice_init(&L, a9, km);
    return count_nf_cells(&L);
}

int or_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void or_set_num_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}
