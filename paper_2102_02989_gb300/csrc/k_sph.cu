// Cartesian -> real solid harmonic transform of integral tensors.
//
// A spherical function of shell l and order m is chi_{lm} = sum_c s_{mc} chi_c
// over the shell's Cartesian functions (lexicographic components), with s the
// monomial coefficients of the Racah-normalised real regular solid harmonics
// (no Condon-Shortley phase), order m = -l..l:
//   C_l^m = N_lm Re[(x + i y)^m Q_lm],  S_l^m = N_lm Im[(x + i y)^m Q_lm],
//   Q_lm  = sum_k a_k z^{l-m-2k} r^{2k},
//   a_k   = 2^{-l} (-1)^k binom(l,k) binom(2l-2k,l) (l-2k)!/(l-2k-m)!,
//   N_lm  = sqrt((2 - delta_m0) (l-m)!/(l+m)!),
// i.e. r^l P_l^m(cos theta) e^{i m phi} written out from the Rodrigues form of
// P_l and (x + i y)^m = (r sin theta e^{i phi})^m, with r^{2k} expanded by the
// multinomial theorem.  Because every Cartesian shell carries the norm of its
// x^l component and the angular integrals of |C_l^m|^2 and x^{2l} agree, the
// spherical functions come out unit-normalised.
//
// The transform of a tensor is a sparse gather: each output element sums the
// products of the (at most 4 per index for l <= 3) nonzero coefficients of its
// three indices.  HBM-bound; one thread per output element.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "k_common.cuh"

namespace rsgdf {

static double fact(int n)
{
    double f = 1.0;
    for (int i = 2; i <= n; i++) f *= i;
    return f;
}

static double binom(int n, int k) { return (k < 0 || k > n) ? 0.0 : fact(n) / (fact(k) * fact(n - k)); }

// s[(m + l) * ncart + c], components c in lexicographic order (lx descending, then ly descending)
void sph_coefficients(int l, std::vector<double> &s)
{
    const int nc = (l + 1) * (l + 2) / 2;
    s.assign((size_t)(2 * l + 1) * nc, 0.0);
    auto comp = [l](int lx, int ly) {   // lexicographic index of (lx, ly, l - lx - ly)
        const int a = l - lx;           // components before lx: sum_{t < a} (t + 1)
        return a * (a + 1) / 2 + (a - ly);
    };
    for (int am = 0; am <= l; am++) {
        const double N = std::sqrt((am == 0 ? 1.0 : 2.0) * fact(l - am) / fact(l + am));
        for (int k = 0; 2 * k <= l - am; k++) {
            const double ak = std::ldexp(1.0, -l) * ((k & 1) ? -1.0 : 1.0) * binom(l, k) * binom(2 * l - 2 * k, l) *
                              fact(l - 2 * k) / fact(l - 2 * k - am);
            // (x + i y)^am: term j carries x^{am-j} y^j i^j
            for (int j = 0; j <= am; j++) {
                const double bj = binom(am, j);
                const bool imag = j & 1;
                const double sgn = ((j / 2) & 1) ? -1.0 : 1.0;   // i^j = sgn (j even) or sgn i (j odd)
                // r^{2k} = sum_{p+q+t=k} k!/(p! q! t!) x^{2p} y^{2q} z^{2t}
                for (int p = 0; p <= k; p++)
                    for (int q = 0; p + q <= k; q++) {
                        const int t = k - p - q;
                        const double mult = fact(k) / (fact(p) * fact(q) * fact(t));
                        const int lx = am - j + 2 * p, ly = j + 2 * q;
                        const double v = N * ak * bj * sgn * mult;
                        (void)t;
                        const int c = comp(lx, ly);
                        if (!imag) s[(size_t)(am + l) * nc + c] += v;            // C_l^am at m = +am
                        else if (am > 0) s[(size_t)(l - am) * nc + c] += v;      // S_l^am at m = -am
                    }
            }
        }
    }
}

// CSR map of a basis (shells with momenta ls, Cartesian offsets in shell order):
// row r (spherical function) lists (Cartesian index, coefficient).
void sph_map(const std::vector<int> &ls, std::vector<int> &off, std::vector<int> &idx, std::vector<double> &coef)
{
    off.assign(1, 0);
    idx.clear();
    coef.clear();
    int c0 = 0;
    std::vector<double> s;
    for (int l : ls) {
        const int nc = (l + 1) * (l + 2) / 2;
        sph_coefficients(l, s);
        for (int m = 0; m < 2 * l + 1; m++) {
            for (int c = 0; c < nc; c++) {
                const double v = s[(size_t)m * nc + c];
                if (std::fabs(v) > 1e-15) {
                    idx.push_back(c0 + c);
                    coef.push_back(v);
                }
            }
            off.push_back((int)idx.size());
        }
        c0 += nc;
    }
}

// out[b][i][j][t] = sum c1 c2 c3 in[b][p][q][r] over the nonzeros of rows i, j, t
__global__ void __launch_bounds__(256) k_cart2sph(const double2 *__restrict__ in, double2 *__restrict__ out, long long nb,
                                                  int n1, int n2, int n3, int c1, int c2, int c3, SphMapDev m1,
                                                  SphMapDev m2, SphMapDev m3)
{
    const long long tot = nb * n1 * n2 * n3;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
        long long r = e;
        const int t = (int)(r % n3);
        r /= n3;
        const int j = (int)(r % n2);
        r /= n2;
        const int i = (int)(r % n1);
        const long long b = r / n1;
        const double2 *src = in + b * c1 * c2 * c3;
        double re = 0.0, im = 0.0;
        for (int u = m1.off[i]; u < m1.off[i + 1]; u++) {
            const double w1 = m1.coef[u];
            const double2 *s1 = src + (long long)m1.idx[u] * c2 * c3;
            for (int v = m2.off[j]; v < m2.off[j + 1]; v++) {
                const double w12 = w1 * m2.coef[v];
                const double2 *s2 = s1 + (long long)m2.idx[v] * c3;
                for (int w = m3.off[t]; w < m3.off[t + 1]; w++) {
                    const double f = w12 * m3.coef[w];
                    const double2 x = s2[m3.idx[w]];
                    re = fma(f, x.x, re);
                    im = fma(f, x.y, im);
                }
            }
        }
        out[e] = make_double2(re, im);
    }
}

int launch_cart2sph(const double *in, double *out, long long nb, int n1, int n2, int n3, int c1, int c2, int c3,
                    SphMapDev m1, SphMapDev m2, SphMapDev m3, cudaStream_t st)
{
    const long long tot = nb * n1 * n2 * n3;
    if (tot <= 0) return RSGDF_OK;
    int dev = 0, nsm = 148;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const long long blocks = std::min<long long>((tot + 255) / 256, (long long)nsm * 16);
    k_cart2sph<<<(unsigned)blocks, 256, 0, st>>>((const double2 *)in, (double2 *)out, nb, n1, n2, n3, c1, c2, c3, m1,
                                                 m2, m3);
    return cudaGetLastError() == cudaSuccess ? RSGDF_OK : RSGDF_EDEVICE;
}

}  // namespace rsgdf
