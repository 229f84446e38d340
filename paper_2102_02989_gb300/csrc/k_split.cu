// Compact/diffuse split of j3c (Fig. 1 of the paper, Eq. VPmunu_FT): the
// problem runs on sub-shell bases (every shell cut at alpha_cut into a compact
// and a diffuse sub-shell); the range-separated route supplies the (C|cc) and
// (C|cd) blocks, the plain-kernel reciprocal sum the other four types, and the
// sub-functions are summed back into the parent functions.
#include <cuda_runtime.h>

#include <algorithm>

#include "k_common.cuh"

namespace rsgdf {

// G = 0 term restricted to the range-separated types: S_P = 0 for functions of
// diffuse aux shells, S_{mu nu} = 0 where both AO functions are diffuse.
__global__ void k_split_g0_mask(double *SP, int nP, const int *__restrict__ mask_ax, double *Sf, int Nk, int nao,
                                const int *__restrict__ mask_ao)
{
    const long long nn = (long long)nao * nao, tot = (long long)Nk * nn;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < tot + nP;
         e += (long long)gridDim.x * blockDim.x) {
        if (e < nP) {
            if (mask_ax[e]) SP[e] = 0.0;
        } else {
            const long long f = e - nP, r = f % nn;
            const int a = (int)(r / nao), b = (int)(r - (long long)a * nao);
            if (mask_ao[a] && mask_ao[b]) Sf[f] = 0.0;
        }
    }
}

int launch_split_g0_mask(double *SP, int nP, const int *mask_ax, double *Sf, int Nk, int nao, const int *mask_ao,
                         cudaStream_t st)
{
    const long long tot = (long long)Nk * nao * nao + nP;
    const long long blocks = std::min<long long>((tot + 255) / 256, 4096);
    k_split_g0_mask<<<(unsigned)blocks, 256, 0, st>>>(SP, nP, mask_ax, Sf, Nk, nao, mask_ao);
    return cudaGetLastError() == cudaSuccess ? RSGDF_OK : RSGDF_EDEVICE;
}

// out[b][i][j][t] = sum over the sub-functions (p, q, r) of parents (i, j, t)
// of w_p w_q w_r X[b][p][q][r], X = Vrs where kind_x[p] == 0 and not
// (kind_a[q] == 1 and kind_a[r] == 1), else Vg (kind 1 = diffuse).
__global__ void __launch_bounds__(256) k_split_combine(const double2 *__restrict__ Vrs, const double2 *__restrict__ Vg,
                                                       double2 *__restrict__ out, long long nb, int n1, int n2,
                                                       int c1, int c2, SphMapDev mx, SphMapDev ma,
                                                       const int *__restrict__ kind_x, const int *__restrict__ kind_a)
{
    const long long tot = nb * n1 * n2 * n2;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
        long long r = e;
        const int t = (int)(r % n2);
        r /= n2;
        const int j = (int)(r % n2);
        r /= n2;
        const int i = (int)(r % n1);
        const long long b = r / n1;
        const long long base = b * c1 * c2 * c2;
        double re = 0.0, im = 0.0;
        for (int u = mx.off[i]; u < mx.off[i + 1]; u++) {
            const int p = mx.idx[u];
            const double w1 = mx.coef[u];
            const bool cx = kind_x[p] == 0;
            for (int v = ma.off[j]; v < ma.off[j + 1]; v++) {
                const int q = ma.idx[v];
                const double w12 = w1 * ma.coef[v];
                for (int w = ma.off[t]; w < ma.off[t + 1]; w++) {
                    const int s = ma.idx[w];
                    const long long o = base + ((long long)p * c2 + q) * c2 + s;
                    const bool rs = cx && !(kind_a[q] == 1 && kind_a[s] == 1);
                    const double2 x = rs ? Vrs[o] : Vg[o];
                    const double f = w12 * ma.coef[w];
                    re = fma(f, x.x, re);
                    im = fma(f, x.y, im);
                }
            }
        }
        out[e] = make_double2(re, im);
    }
}

int launch_split_combine(const double *Vrs, const double *Vg, double *out, long long nb, int n1, int n2, int c1,
                         int c2, SphMapDev mx, SphMapDev ma, const int *kind_x, const int *kind_a, cudaStream_t st)
{
    const long long tot = nb * n1 * n2 * n2;
    if (tot <= 0) return RSGDF_OK;
    int dev = 0, nsm = 148;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const long long blocks = std::min<long long>((tot + 255) / 256, (long long)nsm * 16);
    k_split_combine<<<(unsigned)blocks, 256, 0, st>>>((const double2 *)Vrs, (const double2 *)Vg, (double2 *)out, nb,
                                                      n1, n2, c1, c2, mx, ma, kind_x, kind_a);
    return cudaGetLastError() == cudaSuccess ? RSGDF_OK : RSGDF_EDEVICE;
}

}  // namespace rsgdf
