// Learned screening of SR work items (the project's addition to the paper's
// screening): per-item features, and a 3 x 64 tanh multilayer perceptron that
// predicts log10 of the largest block an item adds.  Hand-written kernels:
// inference, fused forward + backward over blocks of 64 samples, Adam.
// Parameters are kept in FP32 (master copy, Adam moments) and used in FP16
// (working copy); stored activations are FP16; every dot product accumulates
// in FP32.  Packing of the parameter vector: W1 [64 x F] row-major, b1 [64],
// W2 [64 x 64], b2, W3 [64 x 64], b3, w4 [64], b4 [1].
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "k_common.cuh"

namespace rsgdf {

constexpr int MH = 64;          // hidden width
constexpr int MLP_BS = 64;      // samples per training block

__host__ __device__ inline int mlp_nparams(int F) { return MH * F + MH + 2 * (MH * MH + MH) + MH + 1; }

struct MlpOff {
    int W1, b1, W2, b2, W3, b3, w4, b4;
};
__host__ __device__ inline MlpOff mlp_off(int F)
{
    MlpOff o;
    o.W1 = 0;
    o.b1 = MH * F;
    o.W2 = o.b1 + MH;
    o.b2 = o.W2 + MH * MH;
    o.W3 = o.b2 + MH;
    o.b3 = o.W3 + MH * MH;
    o.w4 = o.b3 + MH;
    o.b4 = o.w4 + MH;
    return o;
}

// ---------------------------------------------------------------------------
// Features of SR work items (same item order as the SR kernel):
//   lP, lmu, lnu, ln a_P, ln a_mu, ln a_nu (most diffuse exponents), R12,
//   distance of the pair centre to the nearest aux image, log10 of the
//   s-type SR integral of that nearest term summed over the primitive
//   combinations (exact for s shells) times the image sum of the
//   diffuse-rate s-type kernel within the screening radius relative to the
//   nearest image, ln Rc_cut.
// ---------------------------------------------------------------------------
__global__ void k_sr_features(SRArgs A, float *feat)
{
    // FP32 throughout: the features feed a network whose decisions carry a
    // calibrated margin, and FP64 issues at 1/64 of the FP32 rate here
    const long long item = A.item_begin + (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (item >= A.item_end) return;
    int lo = A.tri_begin, hi = A.tri_end - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (A.tri[mid].item_off <= item) lo = mid; else hi = mid - 1;
    }
    const SRTripleDev tr = A.tri[lo];
    const int gd = A.pair_doff[tr.pair] + (int)(item - tr.item_off);
    const int d0 = A.dlist[3 * gd], d1 = A.dlist[3 * gd + 1], d2 = A.dlist[3 * gd + 2];
    float Av[3], Bv[3], x[3];
    for (int k = 0; k < 3; k++) {
        Av[k] = (float)A.ao.cen[3 * tr.mu + k];
        Bv[k] = (float)A.ao.cen[3 * tr.nu + k] + d0 * A.af[k] + d1 * A.af[3 + k] + d2 * A.af[6 + k];
    }
    const float R12 = sqrtf((Bv[0] - Av[0]) * (Bv[0] - Av[0]) + (Bv[1] - Av[1]) * (Bv[1] - Av[1]) +
                            (Bv[2] - Av[2]) * (Bv[2] - Av[2]));
    const float amu = (float)tr.amu, anu = (float)tr.anu;
    for (int k = 0; k < 3; k++) x[k] = (amu * Av[k] + anu * Bv[k]) / (amu + anu) - (float)A.ax.cen[3 * tr.P + k];
    int l[3];
    for (int i = 0; i < 3; i++)
        l[i] = __float2int_rn(x[0] * (float)A.bq[3 * i] + x[1] * (float)A.bq[3 * i + 1] + x[2] * (float)A.bq[3 * i + 2]);
    // nearest aux image: the rounded lattice point and its 26 neighbours
    float rc2 = 3.0e38f;
    int ln[3] = {l[0], l[1], l[2]};
    for (int i = -1; i <= 1; i++)
        for (int j = -1; j <= 1; j++)
            for (int k = -1; k <= 1; k++) {
                float r2 = 0.0f;
                for (int c = 0; c < 3; c++) {
                    const float r = x[c] - ((l[0] + i) * A.af[c] + (l[1] + j) * A.af[3 + c] + (l[2] + k) * A.af[6 + c]);
                    r2 += r * r;
                }
                if (r2 < rc2) {
                    rc2 = r2;
                    ln[0] = l[0] + i;
                    ln[1] = l[1] + j;
                    ln[2] = l[2] + k;
                }
            }
    const float rc = sqrtf(rc2);
    // s-type SR integral of the nearest term summed over primitive combinations:
    // |c_P c_i c_j| (pi^2/(g p))^{3/2} e^{-ab/p R12^2} [erf(e1 R) - erf(e2 R)]/R
    float est = 0.0f;
    const float om2 = (float)(A.omega * A.omega);
    const float kpi = 3.14159265f;
    for (int k = 0; k < A.ax.nprim[tr.P]; k++) {
        const int ok = A.ax.poff[tr.P] + k;
        const float g = (float)A.ax.exps[ok];
        for (int i = 0; i < A.ao.nprim[tr.mu]; i++)
            for (int j = 0; j < A.ao.nprim[tr.nu]; j++) {
                const int oi = A.ao.poff[tr.mu] + i, oj = A.ao.poff[tr.nu] + j;
                const float ea = (float)A.ao.exps[oi], eb = (float)A.ao.exps[oj], p = ea + eb;
                float R2 = 0.0f;
                for (int c = 0; c < 3; c++) {
                    const float r = (ea * Av[c] + eb * Bv[c]) / p - (float)A.ax.cen[3 * tr.P + c] -
                                    (ln[0] * A.af[c] + ln[1] * A.af[3 + c] + ln[2] * A.af[6 + c]);
                    R2 += r * r;
                }
                const float R = sqrtf(R2);
                const float e1 = sqrtf(g * p / (g + p));
                const float e2 = e1 * sqrtf(om2 / (e1 * e1 + om2));
                const float fR = (R < 1e-4f) ? 2.0f * (e1 - e2) * 0.5641895835f : (erff(e1 * R) - erff(e2 * R)) / R;
                const float pf = kpi * kpi / (g * p);
                est += fabsf((float)A.ax.cn[ok] * (float)A.ao.cn[oi] * (float)A.ao.cn[oj]) * pf * sqrtf(pf) *
                       __expf(-ea * eb / p * R12 * R12) * fR;
            }
    }
    // every aux image inside the screening radius adds to the lattice sum: scale
    // by the image sum of the diffuse-rate s-type kernel relative to the
    // nearest image ([erf(e1 R) - erf(e2 R)]/R)
    {
        const float e1 = (float)tr.eta1, e2 = (float)tr.eta2;
        auto fk = [&](float R) {
            return (R < 1e-4f) ? 2.0f * (e1 - e2) * 0.5641895835f : (erff(e1 * R) - erff(e2 * R)) / R;
        };
        const float f0 = fk(rc);
        const float fcut = (float)tr.Rc_cut + 1e-3f;
        float sum = 0.0f;
        for (int idx = 0; idx < tr.nsph; idx++) {
            const int li0 = l[0] + A.sph[3 * idx], li1 = l[1] + A.sph[3 * idx + 1], li2 = l[2] + A.sph[3 * idx + 2];
            const float ex = x[0] - (li0 * A.af[0] + li1 * A.af[3] + li2 * A.af[6]);
            const float ey = x[1] - (li0 * A.af[1] + li1 * A.af[4] + li2 * A.af[7]);
            const float ez = x[2] - (li0 * A.af[2] + li1 * A.af[5] + li2 * A.af[8]);
            const float r = sqrtf(ex * ex + ey * ey + ez * ez);
            if (r <= fcut) sum += fk(r);
        }
        if (f0 > 0.0f && sum > f0) est *= sum / f0;
    }
    const float lest = log10f(fmaxf(est, 1e-37f));
    float *f = feat + item * SR_NFEAT;
    f[0] = (float)A.ax.l[tr.P];
    f[1] = (float)A.ao.l[tr.mu];
    f[2] = (float)A.ao.l[tr.nu];
    f[3] = logf((float)tr.aP);
    f[4] = logf((float)tr.amu);
    f[5] = logf(fmaxf((float)tr.anu, 1e-37f));
    f[6] = R12;
    f[7] = rc;
    f[8] = est > 0.0f ? lest : -300.0f;
    f[9] = logf((float)tr.Rc_cut);
}

int launch_sr_features(const SRArgs &A, float *feat, cudaStream_t st)
{
    const long long n = A.item_end - A.item_begin;
    if (n <= 0) return RSGDF_OK;
    k_sr_features<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(A, feat);
    return cudaGetLastError() == cudaSuccess ? RSGDF_OK : RSGDF_EDEVICE;
}

// ---------------------------------------------------------------------------
// Inference: one thread per sample, FP16 parameters staged in shared memory.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void load_params_smem(const __half *P, __half *sP, int np)
{
    for (int i = threadIdx.x; i < np; i += blockDim.x) sP[i] = P[i];
    __syncthreads();
}

__global__ void k_mlp_forward(int F, const __half *P16, const float *mean, const float *stdv, const float *X, long long n,
                              float *y)
{
    extern __shared__ __half sP[];
    const int np = mlp_nparams(F);
    load_params_smem(P16, sP, np);
    const MlpOff o = mlp_off(F);
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    float xin[SR_NFEAT_MAX];
    for (int f = 0; f < F; f++) xin[f] = (X[s * F + f] - mean[f]) / stdv[f];
    float h[MH], g[MH];
    for (int j = 0; j < MH; j++) {
        float a = __half2float(sP[o.b1 + j]);
        for (int f = 0; f < F; f++) a = fmaf(__half2float(sP[o.W1 + j * F + f]), xin[f], a);
        h[j] = tanhf(a);
    }
    for (int j = 0; j < MH; j++) {
        float a = __half2float(sP[o.b2 + j]);
        for (int k = 0; k < MH; k++) a = fmaf(__half2float(sP[o.W2 + j * MH + k]), h[k], a);
        g[j] = tanhf(a);
    }
    for (int j = 0; j < MH; j++) {
        float a = __half2float(sP[o.b3 + j]);
        for (int k = 0; k < MH; k++) a = fmaf(__half2float(sP[o.W3 + j * MH + k]), g[k], a);
        h[j] = tanhf(a);
    }
    float out = __half2float(sP[o.b4]);
    for (int k = 0; k < MH; k++) out = fmaf(__half2float(sP[o.w4 + k]), h[k], out);
    y[s] = out;
}

// ---------------------------------------------------------------------------
// Training: forward and backward of one block of MLP_BS samples, gradients
// of the expectile loss (1/n) sum_s w_s r_s^2, r = y - t, w = 2 tau when the
// network under-predicts (r < 0) and 2 (1 - tau) otherwise, added to G
// (FP32).  tau = 1/2 is the mean squared error.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_mlp_fwd_bwd(int F, const __half *P16, const float *mean, const float *stdv,
                                                     const float *X, const float *t, const int *idx, long long n,
                                                     float inv_ntot, float tau, float *G, float *loss)
{
    extern __shared__ unsigned char smraw[];
    const int np = mlp_nparams(F);
    const MlpOff o = mlp_off(F);
    __half *sP = (__half *)smraw;                                   // parameters
    float *xs = (float *)(smraw + ((np * 2 + 15) & ~15));          // [BS][F]
    __half *H1 = (__half *)(xs + MLP_BS * SR_NFEAT_MAX);           // [BS][MH] each
    __half *H2 = H1 + MLP_BS * MH;
    __half *H3 = H2 + MLP_BS * MH;
    float *Da = (float *)(H3 + MLP_BS * MH);                        // [BS][MH]
    float *Db = Da + MLP_BS * MH;
    float *dy = Db + MLP_BS * MH;                                   // [BS]
    load_params_smem(P16, sP, np);
    const int tid = threadIdx.x;
    const long long s0 = (long long)blockIdx.x * MLP_BS;
    const int nb = (int)min((long long)MLP_BS, n - s0);
    for (int e = tid; e < MLP_BS * F; e += blockDim.x) {
        const int s = e / F, f = e - s * F;
        float v = 0.0f;
        if (s < nb) {
            const long long src = idx ? idx[s0 + s] : (s0 + s);
            v = (X[src * F + f] - mean[f]) / stdv[f];
        }
        xs[s * SR_NFEAT_MAX + f] = v;
    }
    __syncthreads();
    // forward, one (sample, unit) pair per thread iteration
    for (int e = tid; e < MLP_BS * MH; e += blockDim.x) {
        const int s = e / MH, j = e - s * MH;
        float a = __half2float(sP[o.b1 + j]);
        for (int f = 0; f < F; f++) a = fmaf(__half2float(sP[o.W1 + j * F + f]), xs[s * SR_NFEAT_MAX + f], a);
        H1[e] = __float2half(tanhf(a));
    }
    __syncthreads();
    for (int e = tid; e < MLP_BS * MH; e += blockDim.x) {
        const int s = e / MH, j = e - s * MH;
        float a = __half2float(sP[o.b2 + j]);
        for (int k = 0; k < MH; k++) a = fmaf(__half2float(sP[o.W2 + j * MH + k]), __half2float(H1[s * MH + k]), a);
        H2[e] = __float2half(tanhf(a));
    }
    __syncthreads();
    for (int e = tid; e < MLP_BS * MH; e += blockDim.x) {
        const int s = e / MH, j = e - s * MH;
        float a = __half2float(sP[o.b3 + j]);
        for (int k = 0; k < MH; k++) a = fmaf(__half2float(sP[o.W3 + j * MH + k]), __half2float(H2[s * MH + k]), a);
        H3[e] = __float2half(tanhf(a));
    }
    __syncthreads();
    if (tid < MLP_BS) {
        float dv = 0.0f;
        if (tid < nb) {
            float yv = __half2float(sP[o.b4]);
            for (int k = 0; k < MH; k++) yv = fmaf(__half2float(sP[o.w4 + k]), __half2float(H3[tid * MH + k]), yv);
            const long long src = idx ? idx[s0 + tid] : (s0 + tid);
            const float r = yv - t[src];
            const float w = (r < 0.0f) ? 2.0f * tau : 2.0f * (1.0f - tau);
            dv = 2.0f * w * r * inv_ntot;
            atomicAdd(loss, w * r * r * inv_ntot);
        }
        dy[tid] = dv;
    }
    __syncthreads();
    // layer 4: gw4 = sum_s dy h3, gb4 = sum_s dy; d3 = dy w4 (1 - h3^2)
    for (int k = tid; k < MH; k += blockDim.x) {
        float a = 0.0f;
        for (int s = 0; s < MLP_BS; s++) a = fmaf(dy[s], __half2float(H3[s * MH + k]), a);
        atomicAdd(&G[o.w4 + k], a);
    }
    if (tid == 0) {
        float a = 0.0f;
        for (int s = 0; s < MLP_BS; s++) a += dy[s];
        atomicAdd(&G[o.b4], a);
    }
    for (int e = tid; e < MLP_BS * MH; e += blockDim.x) {
        const int s = e / MH, j = e - s * MH;
        const float h = __half2float(H3[e]);
        Da[e] = dy[s] * __half2float(sP[o.w4 + j]) * (1.0f - h * h);
    }
    __syncthreads();
    // layer 3: gW3[j][k] = sum_s d3[s][j] h2[s][k]; d2 = (d3 W3) (1 - h2^2)
    for (int e = tid; e < MH * MH; e += blockDim.x) {
        const int j = e / MH, k = e - j * MH;
        float a = 0.0f;
        for (int s = 0; s < MLP_BS; s++) a = fmaf(Da[s * MH + j], __half2float(H2[s * MH + k]), a);
        atomicAdd(&G[o.W3 + e], a);
    }
    for (int j = tid; j < MH; j += blockDim.x) {
        float a = 0.0f;
        for (int s = 0; s < MLP_BS; s++) a += Da[s * MH + j];
        atomicAdd(&G[o.b3 + j], a);
    }
    for (int e = tid; e < MLP_BS * MH; e += blockDim.x) {
        const int s = e / MH, k = e - s * MH;
        float a = 0.0f;
        for (int j = 0; j < MH; j++) a = fmaf(Da[s * MH + j], __half2float(sP[o.W3 + j * MH + k]), a);
        const float h = __half2float(H2[e]);
        Db[e] = a * (1.0f - h * h);
    }
    __syncthreads();
    // layer 2: gW2 = sum_s d2 h1; d1 = (d2 W2)(1 - h1^2)
    for (int e = tid; e < MH * MH; e += blockDim.x) {
        const int j = e / MH, k = e - j * MH;
        float a = 0.0f;
        for (int s = 0; s < MLP_BS; s++) a = fmaf(Db[s * MH + j], __half2float(H1[s * MH + k]), a);
        atomicAdd(&G[o.W2 + e], a);
    }
    for (int j = tid; j < MH; j += blockDim.x) {
        float a = 0.0f;
        for (int s = 0; s < MLP_BS; s++) a += Db[s * MH + j];
        atomicAdd(&G[o.b2 + j], a);
    }
    for (int e = tid; e < MLP_BS * MH; e += blockDim.x) {
        const int s = e / MH, k = e - s * MH;
        float a = 0.0f;
        for (int j = 0; j < MH; j++) a = fmaf(Db[s * MH + j], __half2float(sP[o.W2 + j * MH + k]), a);
        const float h = __half2float(H1[e]);
        Da[e] = a * (1.0f - h * h);
    }
    __syncthreads();
    // layer 1: gW1[j][f] = sum_s d1[s][j] x[s][f]
    for (int e = tid; e < MH * F; e += blockDim.x) {
        const int j = e / F, f = e - j * F;
        float a = 0.0f;
        for (int s = 0; s < MLP_BS; s++) a = fmaf(Da[s * MH + j], xs[s * SR_NFEAT_MAX + f], a);
        atomicAdd(&G[o.W1 + e], a);
    }
    for (int j = tid; j < MH; j += blockDim.x) {
        float a = 0.0f;
        for (int s = 0; s < MLP_BS; s++) a += Da[s * MH + j];
        atomicAdd(&G[o.b1 + j], a);
    }
}

// Adam (Kingma & Ba) on the FP32 master parameters; refreshes the FP16 copy.
__global__ void k_mlp_adam(int np, float *P, __half *P16, float *G, float *m, float *v, float lr, float b1, float b2,
                           float eps, float c1, float c2)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= np) return;
    const float g = G[i];
    const float mi = b1 * m[i] + (1.0f - b1) * g;
    const float vi = b2 * v[i] + (1.0f - b2) * g * g;
    m[i] = mi;
    v[i] = vi;
    const float p = P[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    P[i] = p;
    P16[i] = __float2half(p);
    G[i] = 0.0f;
}

__global__ void k_to_half(int n, const float *a, __half *b)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = __float2half(a[i]);
}

// Skip mask: the screening prediction is the network output plus, when
// base >= 0, the feature X[base] clamped to [base_lo, base_hi] (the network
// then models the correction to that physical estimate).  An item is skipped
// only if, in addition, the estimate itself plus its calibrated margin for
// the item's class L = lP + lmu + lnu (guard[L]) is below the cut: outside
// its training range the network alone cannot drop an item the estimate
// calls large.
struct GuardL {
    float g[LTOT_MAX + 1];
};

__global__ void k_mlp_mask(long long n, int F, const float *X, int base, float base_lo, float base_hi, GuardL guard,
                           const float *pred, float margin, float log10_cut, unsigned char *skip,
                           unsigned long long *count)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float y = pred[i];
    bool allowed = true;
    if (base >= 0) {
        const float b = X[i * F + base];
        y += fminf(fmaxf(b, base_lo), base_hi);
        // class L = lP + lmu + lnu from the first three features
        int L = __float2int_rn(X[i * F] + X[i * F + 1] + X[i * F + 2]);
        L = L < 0 ? 0 : (L > LTOT_MAX ? LTOT_MAX : L);
        allowed = (b + guard.g[L] < log10_cut);   // the physical estimate must agree
    }
    const unsigned char sk = (allowed && y + margin < log10_cut) ? 1 : 0;
    skip[i] = sk;
    if (sk) atomicAdd(count, 1ULL);
}

size_t mlp_train_smem(int F)
{
    const int np = mlp_nparams(F);
    size_t b = ((size_t)np * 2 + 15) & ~(size_t)15;
    b += (size_t)MLP_BS * SR_NFEAT_MAX * 4;
    b += 3 * (size_t)MLP_BS * MH * 2;
    b += 2 * (size_t)MLP_BS * MH * 4 + MLP_BS * 4;
    return b;
}

int launch_mlp_forward(int F, const __half *P16, const float *mean, const float *stdv, const float *X, long long n,
                       float *y, cudaStream_t st)
{
    if (n <= 0) return RSGDF_OK;
    const size_t sm = (size_t)mlp_nparams(F) * 2;
    k_mlp_forward<<<(unsigned)((n + 127) / 128), 128, sm, st>>>(F, P16, mean, stdv, X, n, y);
    return cudaGetLastError() == cudaSuccess ? RSGDF_OK : RSGDF_EDEVICE;
}

int launch_mlp_fwd_bwd(int F, const __half *P16, const float *mean, const float *stdv, const float *X, const float *t,
                       const int *idx, long long n, float inv_ntot, float tau, float *G, float *loss, cudaStream_t st)
{
    if (n <= 0) return RSGDF_OK;
    const size_t sm = mlp_train_smem(F);
    if (cudaFuncSetAttribute(k_mlp_fwd_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess)
        return RSGDF_EDEVICE;
    k_mlp_fwd_bwd<<<(unsigned)((n + MLP_BS - 1) / MLP_BS), 256, sm, st>>>(F, P16, mean, stdv, X, t, idx, n, inv_ntot, tau,
                                                                        G, loss);
    return cudaGetLastError() == cudaSuccess ? RSGDF_OK : RSGDF_EDEVICE;
}

int launch_mlp_adam(int np, float *P, __half *P16, float *G, float *m, float *v, float lr, int step, cudaStream_t st)
{
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.0f - powf(b1, (float)step), c2 = 1.0f - powf(b2, (float)step);
    k_mlp_adam<<<(np + 255) / 256, 256, 0, st>>>(np, P, P16, G, m, v, lr, b1, b2, 1e-8f, c1, c2);
    return cudaGetLastError() == cudaSuccess ? RSGDF_OK : RSGDF_EDEVICE;
}

int launch_to_half(int n, const float *a, __half *b, cudaStream_t st)
{
    k_to_half<<<(n + 255) / 256, 256, 0, st>>>(n, a, b);
    return cudaGetLastError() == cudaSuccess ? RSGDF_OK : RSGDF_EDEVICE;
}

int launch_mlp_mask(long long n, int F, const float *X, int base, float base_lo, float base_hi, const float *guard,
                    const float *pred, float margin, float log10_cut, unsigned char *skip, unsigned long long *count,
                    cudaStream_t st)
{
    if (n <= 0) return RSGDF_OK;
    GuardL gl;
    for (int L = 0; L <= LTOT_MAX; L++) gl.g[L] = guard[L];
    k_mlp_mask<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, F, X, base, base_lo, base_hi, gl, pred, margin,
                                                          log10_cut, skip, count);
    return cudaGetLastError() == cudaSuccess ? RSGDF_OK : RSGDF_EDEVICE;
}

int mlp_param_count(int F) { return mlp_nparams(F); }

}  // namespace rsgdf
