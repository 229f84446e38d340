// Density-fitting consumers of j3c (Eq. DF_eqn, Eq. ERI_aux): the fitting
// transform T_k of the aux metric J^k (j2c) with T_k^H T_k = (J^k)^{-1}, the
// fitted three-index factors B^{k1k2} = T_{k12} V^{k1k2}, and the fitted
// Coulomb and exchange matrices of a density.  Not on the integral hot path;
// every step runs here, in FP64.
//
// Metric transforms.  Cholesky route: J = L L^H (k_cholesky), T = L^{-1} by
// forward substitution, one thread per column.  Eigen route (canonical
// orthogonalisation, the fallback for a singular or nearly singular metric):
// cyclic Jacobi on the Hermitian part of J, one CTA cluster per k.  A sweep visits
// every index pair once in m - 1 steps of the round-robin (circle) ordering
// (m = n rounded up to even), so the m/2 pairs of a step are disjoint and
// their rotations commute: all column updates (A J, U J) of a step run in
// parallel, then all row updates (J^H (A J)).  For a pair (p, q) with
// a_pq = g e^{i phi}, J = D R: D scales index q by e^{-i phi} (a_pq becomes
// real), R is the real rotation annihilating it, t = tan theta the smaller
// root of t^2 + 2 tau t - 1 = 0, tau = (a_qq - a_pp) / (2 g).  A pair is
// rotated when g > max(DF_JACOBI_TOL sqrt(|a_pp a_qq|), DF_JACOBI_ABS ||A||_F):
// the relative test keeps small positive eigenvalues accurate, the absolute
// floor (a few rounding units of the matrix norm, the backward error of any
// FP64 eigensolver) stops rotations among the rounding noise of near-zero or
// negative eigenvalues of an indefinite metric.  Sweeps stop after one without
// rotations, or after DF_JACOBI_SWEEPS.  Every loop is bounded; nothing waits.
#include <cuda_runtime.h>

#include <algorithm>

#include "k_common.cuh"

namespace rsgdf {

constexpr int DF_THREADS = 256;
constexpr int JAC_THREADS = 256;
constexpr int JAC_CL = 8;   // CTAs per k (portable cluster size)
constexpr double DF_JACOBI_TOL = 1e-14;
constexpr double DF_JACOBI_ABS = 1e-15;

__device__ __forceinline__ double2 zmul(double2 a, double2 b) { return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }

// player at position x of step s of the circle ordering on m (even) players
__device__ __forceinline__ int circle_player(int x, int s, int m) { return x == 0 ? 0 : ((x - 1 + s) % (m - 1)) + 1; }

// One thread-block cluster of JAC_CL CTAs per k (the FP64 work of a step
// spread over JAC_CL SMs).  Every CTA computes the rotation parameters of all
// pairs of a step from the same values of A, so all CTAs agree bit for bit
// (and on the rotation count) without exchanging anything; the column and row
// updates are split over the cluster.  Phases are separated by hardware cluster
// barriers (every thread of every CTA reaches each one: the control flow is
// uniform, the early exit included).  A and U live in global memory.
// gate: NULL (every k) or info[k]; k with info[k] == 0 (Cholesky route taken) are skipped.
// info_out[k] = sweeps run (>= 1), or DF_JACOBI_SWEEPS + 1 when the last sweep still rotated.
__device__ __forceinline__ void cluster_barrier()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__global__ void __cluster_dims__(JAC_CL, 1, 1) __launch_bounds__(JAC_THREADS)
    k_jacobi_herm(const double2 *__restrict__ J, int n, const int *gate, double2 *Awork, double2 *Uwork, double *lam,
                  int *order, int *info_out)
{
    __shared__ double cs_c[DF_NMAX / 2], cs_s[DF_NMAX / 2];
    __shared__ double2 cs_e[DF_NMAX / 2];   // e^{i phi} of each pair
    __shared__ int pp_[DF_NMAX / 2], qq_[DF_NMAX / 2];
    __shared__ int nrot;
    __shared__ double red[JAC_THREADS];
    const int k = blockIdx.x / JAC_CL, rank = blockIdx.x % JAC_CL, tid = threadIdx.x;
    const int gtid = rank * JAC_THREADS + tid, gstride = JAC_CL * JAC_THREADS;
    if (gate && gate[k] == 0) return;   // uniform over the cluster
    const long long nn = (long long)n * n;
    const double2 *Jk = J + k * nn;
    double2 *A = Awork + k * nn, *U = Uwork + k * nn;
    // every CTA: the Frobenius norm of the Hermitian part (for the absolute floor)
    double f2 = 0.0;
    for (long long e = tid; e < nn; e += JAC_THREADS) {
        const int r = (int)(e / n), c = (int)(e - (long long)r * n);
        const double2 a = Jk[(long long)r * n + c], b = Jk[(long long)c * n + r];
        const double hx = 0.5 * (a.x + b.x), hy = 0.5 * (a.y - b.y);
        f2 += hx * hx + hy * hy;
    }
    red[tid] = f2;
    // the cluster's slice of A = (J + J^H) / 2 and U = 1
    for (long long e = gtid; e < nn; e += gstride) {
        const int r = (int)(e / n), c = (int)(e - (long long)r * n);
        const double2 a = Jk[(long long)r * n + c], b = Jk[(long long)c * n + r];
        A[e] = make_double2(0.5 * (a.x + b.x), 0.5 * (a.y - b.y));
        U[e] = make_double2(r == c ? 1.0 : 0.0, 0.0);
    }
    __syncthreads();
    for (int w = JAC_THREADS / 2; w > 0; w >>= 1) {
        if (tid < w) red[tid] += red[tid + w];
        __syncthreads();
    }
    const double gabs = DF_JACOBI_ABS * sqrt(red[0]);
    cluster_barrier();
    const int m = n + (n & 1), npair = m / 2;
    const long long nwork = (long long)npair * n;
    int sweep = 0, converged = 0;
    while (sweep < DF_JACOBI_SWEEPS && !converged) {
        if (tid == 0) nrot = 0;
        __syncthreads();
        for (int s = 0; s < m - 1; s++) {
            int my_rot = 0;
            for (int j = tid; j < npair; j += JAC_THREADS) {
                int p = circle_player(j, s, m), q = circle_player(m - 1 - j, s, m);
                if (p > q) {
                    const int t = p;
                    p = q;
                    q = t;
                }
                pp_[j] = p;
                qq_[j] = q;
                double c = 1.0, sn = 0.0;
                double2 e = make_double2(1.0, 0.0);
                if (q < n) {
                    const double2 apq = __ldcg(A + (long long)p * n + q);
                    const double g = sqrt(apq.x * apq.x + apq.y * apq.y);
                    const double app = __ldcg(A + (long long)p * n + p).x, aqq = __ldcg(A + (long long)q * n + q).x;
                    if (g > fmax(DF_JACOBI_TOL * sqrt(fabs(app * aqq)), gabs) && g > 1e-300) {
                        e = make_double2(apq.x / g, apq.y / g);
                        const double tau = (aqq - app) / (2.0 * g);
                        const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                        c = 1.0 / sqrt(1.0 + t * t);
                        sn = t * c;
                        my_rot += sn != 0.0;
                    }
                }
                cs_c[j] = c;
                cs_s[j] = sn;
                cs_e[j] = e;
            }
            if (my_rot) atomicAdd(&nrot, my_rot);
            cluster_barrier();   // every CTA has read A for the parameters
            // columns: A <- A J, U <- U J; J_pp = c, J_qp = -s e*, J_pq = s, J_qq = c e*
            for (long long w = gtid; w < nwork; w += gstride) {
                const int j = (int)(w / n), r = (int)(w - (long long)j * n);
                if (cs_s[j] == 0.0) continue;
                const int p = pp_[j], q = qq_[j];
                const double c = cs_c[j], sn = cs_s[j];
                const double2 ec = make_double2(cs_e[j].x, -cs_e[j].y);
                double2 *row = A + (long long)r * n;
                const double2 ap = __ldcg(row + p), aq = zmul(__ldcg(row + q), ec);
                row[p] = make_double2(c * ap.x - sn * aq.x, c * ap.y - sn * aq.y);
                row[q] = make_double2(sn * ap.x + c * aq.x, sn * ap.y + c * aq.y);
                double2 *ur = U + (long long)r * n;
                const double2 up = __ldcg(ur + p), uq = zmul(__ldcg(ur + q), ec);
                ur[p] = make_double2(c * up.x - sn * uq.x, c * up.y - sn * uq.y);
                ur[q] = make_double2(sn * up.x + c * uq.x, sn * up.y + c * uq.y);
            }
            cluster_barrier();
            // rows: A <- J^H A; (J^H)_pp = c, (J^H)_pq = -s e, (J^H)_qp = s, (J^H)_qq = c e
            for (long long w = gtid; w < nwork; w += gstride) {
                const int j = (int)(w / n), col = (int)(w - (long long)j * n);
                if (cs_s[j] == 0.0) continue;
                const int p = pp_[j], q = qq_[j];
                const double c = cs_c[j], sn = cs_s[j];
                const double2 ap = __ldcg(A + (long long)p * n + col), aq = zmul(__ldcg(A + (long long)q * n + col), cs_e[j]);
                A[(long long)p * n + col] = make_double2(c * ap.x - sn * aq.x, c * ap.y - sn * aq.y);
                A[(long long)q * n + col] = make_double2(sn * ap.x + c * aq.x, sn * ap.y + c * aq.y);
            }
            cluster_barrier();
        }
        sweep++;
        converged = nrot == 0;
        __syncthreads();
    }
    if (rank == 0 && tid == 0) info_out[k] = converged ? sweep : DF_JACOBI_SWEEPS + 1;
    // eigenvalues descending, ties by index, by rank counting
    double *lk = lam + (long long)k * n;
    int *ok = order + (long long)k * n;
    for (int i = gtid; i < n; i += gstride) {
        const double v = __ldcg(A + (long long)i * n + i).x;
        int rk = 0;
        for (int j = 0; j < n; j++) {
            const double u = __ldcg(A + (long long)j * n + j).x;
            rk += (u > v) || (u == v && j < i);
        }
        lk[rk] = v;
        ok[rk] = i;
    }
}

// T[k][r][P] = lam_r^{-1/2} conj(U[P][order[r]]) for lam_r > rel lam_0, else 0; nkept[k] = that count.
__global__ void k_fit_transform(int n, const int *gate, const double2 *__restrict__ U, const double *__restrict__ lam,
                                const int *__restrict__ order, double rel, double2 *__restrict__ T, int *nkept)
{
    const int k = blockIdx.y;
    if (gate && gate[k] == 0) return;
    const long long nn = (long long)n * n;
    const double *lk = lam + (long long)k * n;
    const double cut = fmax(rel * lk[0], 0.0);
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < nn; e += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(e / n), P = (int)(e - (long long)r * n);
        double2 w = make_double2(0.0, 0.0);
        if (lk[r] > cut) {
            const double2 u = U[k * nn + (long long)P * n + order[(long long)k * n + r]];
            const double f = 1.0 / sqrt(lk[r]);
            w = make_double2(u.x * f, -u.y * f);
        }
        T[k * nn + e] = w;
    }
    if (nkept && blockIdx.x == 0 && threadIdx.x == 0) {
        int c = 0;
        for (int r = 0; r < n; r++) c += lk[r] > cut;
        nkept[k] = c;
    }
}

// Cholesky route: cinfo[k] is k_cholesky's report (-1 or the first non-positive
// pivot).  The factor passes when every pivot L_jj^2 > rel max_i J_ii; then
// T = L^{-1} (lower), info[k] = 0, nkept[k] = n.  Otherwise T[k] = 0,
// info[k] = -1 - (first failing pivot), nkept[k] = 0.
__global__ void __launch_bounds__(DF_THREADS) k_tri_inverse(int n, const double2 *__restrict__ J,
                                                           const double2 *__restrict__ L, const int *cinfo, double rel,
                                                           double2 *T, int *info, int *nkept)
{
    __shared__ double red[DF_THREADS];
    __shared__ int bad;
    const int k = blockIdx.x, tid = threadIdx.x;
    const long long nn = (long long)n * n;
    const double2 *Jk = J + k * nn, *Lk = L + k * nn;
    double2 *Tk = T + k * nn;
    double mx = 0.0;
    for (int i = tid; i < n; i += DF_THREADS) mx = fmax(mx, Jk[(long long)i * n + i].x);
    red[tid] = mx;
    if (tid == 0) bad = cinfo[k] >= 0 ? cinfo[k] : n;
    __syncthreads();
    for (int w = DF_THREADS / 2; w > 0; w >>= 1) {
        if (tid < w) red[tid] = fmax(red[tid], red[tid + w]);
        __syncthreads();
    }
    const double cut = rel * red[0];
    const int lim = bad;
    for (int j = tid; j < lim; j += DF_THREADS) {
        const double d = Lk[(long long)j * n + j].x;
        if (!(d * d > cut)) atomicMin(&bad, j);
    }
    __syncthreads();
    if (bad < n) {
        for (long long e = tid; e < nn; e += DF_THREADS) Tk[e] = make_double2(0.0, 0.0);
        if (tid == 0) {
            info[k] = -1 - bad;
            if (nkept) nkept[k] = 0;
        }
        return;
    }
    // forward substitution L x = e_j, one column per thread
    for (int j = tid; j < n; j += DF_THREADS) {
        for (int i = 0; i < j; i++) Tk[(long long)i * n + j] = make_double2(0.0, 0.0);
        for (int i = j; i < n; i++) {
            double re = i == j ? 1.0 : 0.0, im = 0.0;
            const double2 *Li = Lk + (long long)i * n;
            for (int mm = j; mm < i; mm++) {
                const double2 l = Li[mm], x = Tk[(long long)mm * n + j];
                re -= l.x * x.x - l.y * x.y;
                im -= l.x * x.y + l.y * x.x;
            }
            const double d = Li[i].x;   // real positive diagonal
            Tk[(long long)i * n + j] = make_double2(re / d, im / d);
        }
    }
    if (tid == 0) {
        info[k] = 0;
        if (nkept) nkept[k] = n;
    }
}

int launch_df_cholesky_route(int n, int nk, const double *J, const double *L, const int *cinfo, double rel, double *T,
                             int *info, int *nkept, cudaStream_t st)
{
    k_tri_inverse<<<nk, DF_THREADS, 0, st>>>(n, (const double2 *)J, (const double2 *)L, cinfo, rel, (double2 *)T,
                                             info, nkept);
    return cudaGetLastError() == cudaSuccess ? RSGDF_OK : RSGDF_EDEVICE;
}

int launch_df_eigen_route(int n, int nk, const double *J, const int *gate, double rel, double *A, double *U,
                          double *lam, int *order, double *T, int *info, int *nkept, cudaStream_t st)
{
    if (n < 1 || n > DF_NMAX || nk < 1) return RSGDF_EINVAL;
    const long long nn = (long long)n * n;
    k_jacobi_herm<<<nk * JAC_CL, JAC_THREADS, 0, st>>>((const double2 *)J, n, gate, (double2 *)A, (double2 *)U, lam,
                                                       order, info);
    if (cudaGetLastError() != cudaSuccess) return RSGDF_EDEVICE;
    dim3 grid((unsigned)std::min<long long>((nn + 255) / 256, 1024), nk);
    // the gate is read before the Jacobi kernel overwrote it: eigen k now hold
    // a sweep count (>= 1), Cholesky k still 0
    k_fit_transform<<<grid, 256, 0, st>>>(n, gate, (const double2 *)U, lam, order, rel, (double2 *)T, nkept);
    return cudaGetLastError() == cudaSuccess ? RSGDF_OK : RSGDF_EDEVICE;
}

// ---------------------------------------------------------------------------
// General batched complex GEMM with a split contraction index:
//   C_b(m, n) (= | +=) alpha sum_{q < Q, s < S} opA(A_b(m, q, s)) opB(B_b(q, s, n))
//   A_b(m, q, s) = A[aoff[b] + m lda + q aq + s as]
//   B_b(q, s, n) = B[boff[b] + q bq + s bs + n bn]
//   C_b(m, n)    = C[coff[b] + m ldc + n]
// op = identity or complex conjugate; accumulation by atomics when several
// batches write the same C.  32 x 32 output tile per CTA, 2 x 2 per thread.
// ---------------------------------------------------------------------------
constexpr int GG_M = 32, GG_N = 32, GG_K = 16;

// ksplit > 1 (atomic accumulation only): blockIdx.z = batch * ksplit + part,
// each part summing its own kper-long slice of the contraction index.
__global__ void __launch_bounds__(256) k_zgemm_gen(ZGemmGen g, const double2 *__restrict__ A,
                                                   const double2 *__restrict__ B, double2 *C, int ksplit,
                                                   long long kper)
{
    __shared__ double2 As[GG_K][GG_M + 1];
    __shared__ double2 Bs[GG_K][GG_N + 1];
    const int b = blockIdx.z / ksplit, part = blockIdx.z - b * ksplit;
    const long long ao = g.aoff[b], bo = g.boff[b], co = g.coff[b];
    const int m0 = blockIdx.y * GG_M, n0 = blockIdx.x * GG_N;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const long long KT = (long long)g.Q * g.S;
    const long long kbeg = part * kper, kend = kbeg + kper < KT ? kbeg + kper : KT;
    const bool a_kfast = g.lda != 1, b_kfast = g.bn != 1;
    const double sa = g.conjA ? -1.0 : 1.0, sb = g.conjB ? -1.0 : 1.0;
    double cr[2][2] = {{0, 0}, {0, 0}}, ci[2][2] = {{0, 0}, {0, 0}};
    for (long long k0 = kbeg; k0 < kend; k0 += GG_K) {
        for (int e = threadIdx.x; e < GG_K * GG_M; e += 256) {
            const int kk = a_kfast ? e % GG_K : e / GG_M, mm = a_kfast ? e / GG_K : e % GG_M;
            const long long gk = k0 + kk;
            const int gm = m0 + mm;
            double2 v = make_double2(0.0, 0.0);
            if (gk < kend && gm < g.M) {
                const long long q = gk / g.S, s = gk - q * g.S;
                v = A[ao + gm * g.lda + q * g.aq + s * g.as];
                v.y *= sa;
            }
            As[kk][mm] = v;
        }
        for (int e = threadIdx.x; e < GG_K * GG_N; e += 256) {
            const int kk = b_kfast ? e % GG_K : e / GG_N, nn = b_kfast ? e / GG_K : e % GG_N;
            const long long gk = k0 + kk;
            const int gn = n0 + nn;
            double2 v = make_double2(0.0, 0.0);
            if (gk < kend && gn < g.N) {
                const long long q = gk / g.S, s = gk - q * g.S;
                v = B[bo + q * g.bq + s * g.bs + gn * g.bn];
                v.y *= sb;
            }
            Bs[kk][nn] = v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GG_K; kk++) {
            const double2 av[2] = {As[kk][ty * 2], As[kk][ty * 2 + 1]};
            const double2 bv[2] = {Bs[kk][tx * 2], Bs[kk][tx * 2 + 1]};
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
            const int gm = m0 + ty * 2 + i, gn = n0 + tx * 2 + j;
            if (gm < g.M && gn < g.N) {
                double *c = (double *)(C + co + gm * g.ldc + gn);
                if (g.atomic) {
                    atomicAdd(c, g.alpha * cr[i][j]);
                    atomicAdd(c + 1, g.alpha * ci[i][j]);
                } else {
                    c[0] = g.alpha * cr[i][j];
                    c[1] = g.alpha * ci[i][j];
                }
            }
        }
}

int launch_zgemm_gen(const ZGemmGen &g, int batch, const double *A, const double *B, double *C, cudaStream_t st)
{
    if (g.M <= 0 || g.N <= 0 || batch <= 0) return RSGDF_OK;
    const long long tiles = (long long)((g.N + GG_N - 1) / GG_N) * ((g.M + GG_M - 1) / GG_M);
    const long long KT = (long long)g.Q * g.S;
    // split the contraction over more CTAs when the output alone would not fill
    // two waves of the SMs (atomic accumulation only), keeping >= 4 chunks per part
    int dev = 0, nsm = 148;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    int ksplit = 1;
    if (g.atomic && tiles * batch < 2LL * nsm)
        ksplit = (int)std::max(1LL, std::min((2LL * nsm + tiles * batch - 1) / (tiles * batch), KT / (4 * GG_K)));
    const long long kper = ((KT + ksplit - 1) / ksplit + GG_K - 1) / GG_K * GG_K;
    ksplit = (int)((KT + kper - 1) / kper);
    const int bmax = 65535 / ksplit;
    for (int b0 = 0; b0 < batch; b0 += bmax) {
        ZGemmGen h = g;
        h.aoff += b0;
        h.boff += b0;
        h.coff += b0;
        dim3 grid((g.N + GG_N - 1) / GG_N, (g.M + GG_M - 1) / GG_M, std::min(bmax, batch - b0) * ksplit);
        k_zgemm_gen<<<grid, 256, 0, st>>>(h, (const double2 *)A, (const double2 *)B, (double2 *)C, ksplit, kper);
        if (cudaGetLastError() != cudaSuccess) return RSGDF_EDEVICE;
    }
    return RSGDF_OK;
}

}  // namespace rsgdf
