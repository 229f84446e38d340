// Split-precision complex GEMM on the 5th-generation tensor cores (tcgen05,
// kind::tf32, FP32 accumulators in tensor memory) for the mixed-precision LR
// contraction (Eq. VPmunu_LR):
//   C[b][m][n] += sum_k A[k][m] B[b][k][n]        (complex FP64 in and out)
//
// Complex arithmetic is embedded in one real GEMM: rows 0..63 of the 128-row
// tile give Re C, rows 64..127 give Im C, and K is doubled by interleaving the
// real and imaginary parts of every k:
//   Re C = sum_k [ Re A, -Im A ] . [ Re B, Im B ],  Im C = sum_k [ Im A, Re A ] . [ Re B, Im B ].
// Every operand value x (rounded to FP32) is split into TF32 parts hi + lo and
// each K-step issues hi*hi + hi*lo + lo*hi into the same accumulator (the
// "3xTF32" scheme: about 22 significant bits per product).  Each 16-complex-k
// chunk is summed in tensor memory, read back with tcgen05.ld and added to a
// compensated FP32 pair (TwoSum) per output, so the FP32 rounding of the long
// K sum does not accumulate.  Operands are staged through registers (the FP64
// to hi/lo conversion happens there) into shared memory in the canonical
// no-swizzle K-major layout: core matrices of 8 rows x 16 bytes.
#include <cuda_runtime.h>

#include <cstdint>

#include "k_common.cuh"

namespace rsgdf {

constexpr int TC_THREADS = 128;
constexpr long long TC_SPIN = 1LL << 26;   // bounded mbarrier wait
constexpr int TC_STAGES = 2;               // operand stages of the bulk-copy pipeline (48 KB each; 2 CTAs per SM)

__device__ int g_tc_status;      // set to 1 when a bounded wait gives up


__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr)
{
    const uint32_t lbo = 128;                  // next core matrix along K
    const uint32_t sbo = (TC_KR / 4) * 128;    // next 8-row group
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;                    // descriptor version of this architecture
    return d;                                  // no swizzle, base offset 0
}

__device__ __forceinline__ uint32_t instr_desc_tf32(int m, int n)
{
    uint32_t d = 0;
    d |= 1u << 4;                    // accumulator FP32
    d |= 2u << 7;                    // A TF32
    d |= 2u << 10;                   // B TF32
    d |= (uint32_t)(n >> 3) << 17;   // both operands K-major
    d |= (uint32_t)(m >> 4) << 24;
    return d;
}

__device__ __forceinline__ void split_tf32(double v, float &hi, float &lo)
{
    const float f = (float)v;
    uint32_t h;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(f));
    hi = __uint_as_float(h);
    uint32_t l;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(l) : "f"(f - hi));
    lo = __uint_as_float(l);
}

__device__ __forceinline__ void two_sum(float &s, float &c, float x)
{
    const float t = s + x;
    const float bp = t - s;
    c += (s - (t - bp)) + (x - bp);
    s = t;
}

__global__ void __launch_bounds__(TC_THREADS) k_zgemm_tn_tc(int M, int N, int K, const double2 *A, const double2 *B,
                                                             long long strideB, double2 *C, long long strideC)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char *sAh = smem;                                   // 128 x 32 fp32
    unsigned char *sAl = sAh + 2 * TC_M * TC_KR * 4;
    unsigned char *sBh = sAl + 2 * TC_M * TC_KR * 4;             // 64 x 32 fp32
    unsigned char *sBl = sBh + TC_N * TC_KR * 4;
    __shared__ __align__(8) unsigned long long mbar;
    __shared__ uint32_t tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int b = blockIdx.z;
    const int m0 = blockIdx.y * TC_M, n0 = blockIdx.x * TC_N;
    const double2 *Bb = B + b * strideB;
    double2 *Cb = C + b * strideC;

    if (warp == 0) {
        const uint32_t dst = (uint32_t)__cvta_generic_to_shared(&tmem_base);
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst), "r"(TC_N));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    const uint32_t mb = (uint32_t)__cvta_generic_to_shared(&mbar);
    if (tid == 0) asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mb), "r"(1));
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_base;
    const uint32_t idesc = instr_desc_tf32(2 * TC_M, TC_N);
    const uint32_t aAh = (uint32_t)__cvta_generic_to_shared(sAh), aAl = (uint32_t)__cvta_generic_to_shared(sAl);
    const uint32_t aBh = (uint32_t)__cvta_generic_to_shared(sBh), aBl = (uint32_t)__cvta_generic_to_shared(sBl);

    float sh[TC_N], sc[TC_N];
#pragma unroll
    for (int j = 0; j < TC_N; j++) { sh[j] = 0.0f; sc[j] = 0.0f; }
    bool ok = true;
    int phase = 0;
    for (int k0 = 0; k0 < K; k0 += TC_KC) {
        // ---- stage A' (128 real rows) and B' (64 rows), hi and lo parts
        for (int e = tid; e < 2 * TC_M * TC_KR; e += TC_THREADS) {
            const int r = e / TC_KR, kr = e - r * TC_KR;
            const int m = m0 + (r & (TC_M - 1)), k = k0 + (kr >> 1);
            double v = 0.0;
            if (m < M && k < K) {
                const double2 a = A[(long long)k * M + m];
                if (r < TC_M) v = (kr & 1) ? -a.y : a.x;   // Re row: [Re A, -Im A]
                else v = (kr & 1) ? a.x : a.y;             // Im row: [Im A, Re A]
            }
            float hi, lo;
            split_tf32(v, hi, lo);
            *(float *)(sAh + core_off(r, kr)) = hi;
            *(float *)(sAl + core_off(r, kr)) = lo;
        }
        for (int e = tid; e < TC_N * TC_KR; e += TC_THREADS) {
            const int kr = e / TC_N, r = e - kr * TC_N;    // consecutive threads: consecutive n
            const int n = n0 + r, k = k0 + (kr >> 1);
            double v = 0.0;
            if (n < N && k < K) {
                const double2 x = Bb[(long long)k * N + n];
                v = (kr & 1) ? x.y : x.x;
            }
            float hi, lo;
            split_tf32(v, hi, lo);
            *(float *)(sBh + core_off(r, kr)) = hi;
            *(float *)(sBl + core_off(r, kr)) = lo;
        }
        asm volatile("fence.proxy.async.shared::cta;");
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;");
        if (tid == 0) {
#pragma unroll
            for (int ks = 0; ks < TC_KR / 8; ks++) {
                const uint32_t off = ks * 256;   // two core matrices along K per MMA
                const uint64_t dah = smem_desc(aAh + off), dal = smem_desc(aAl + off);
                const uint64_t dbh = smem_desc(aBh + off), dbl = smem_desc(aBl + off);
                const uint32_t acc0 = ks > 0 ? 1u : 0u;
                asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                             "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
                             "l"(dah), "l"(dbh), "r"(idesc), "r"(acc0));
                asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                             "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
                             "l"(dah), "l"(dbl), "r"(idesc), "r"(1u));
                asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                             "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
                             "l"(dal), "l"(dbh), "r"(idesc), "r"(1u));
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mb));
        }
        // ---- wait for the chunk's MMAs (bounded)
        {
            uint32_t done = 0;
            long long it = 0;
            while (!done && it < TC_SPIN) {
                asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                             "selp.u32 %0, 1, 0, p;\n}"
                             : "=r"(done)
                             : "r"(mb), "r"(phase));
                it++;
            }
            if (!done) ok = false;
        }
        phase ^= 1;
        asm volatile("tcgen05.fence::after_thread_sync;");
        // ---- accumulator rows of this warp: TMEM lanes 32 warp .. 32 warp + 31
#pragma unroll
        for (int c0 = 0; c0 < TC_N; c0 += 8) {
            uint32_t r[8];
            const uint32_t ta = tmem + ((uint32_t)(warp * 32) << 16) + c0;
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                         : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                           "=r"(r[7])
                         : "r"(ta));
            asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
            for (int j = 0; j < 8; j++) two_sum(sh[c0 + j], sc[c0 + j], __uint_as_float(r[j]));
        }
        asm volatile("tcgen05.fence::before_thread_sync;");
        // CTA-uniform decision: every thread leaves the loop together
        const int all_ok = __syncthreads_and(ok ? 1 : 0);
        asm volatile("tcgen05.fence::after_thread_sync;");
        if (!all_ok) {
            ok = false;
            break;
        }
    }
    if (!ok && (tid & 31) == 0) atomicExch(&g_tc_status, 1);
    // ---- epilogue: row r of the real tile is Re (r < 64) or Im (r >= 64) of complex row m0 + r % 64
    const int r = warp * 32 + (tid & 31);
    const int m = m0 + (r & (TC_M - 1));
    if (ok && m < M) {
        double *Cr = (double *)(Cb + (long long)m * N) + (r >= TC_M ? 1 : 0);
#pragma unroll
        for (int j = 0; j < TC_N; j++) {
            const int n = n0 + j;
            if (n < N) Cr[2LL * n] += (double)sh[j] + (double)sc[j];
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_N));
}

size_t tc_smem_bytes() { return (size_t)(2 * 2 * TC_M + 2 * TC_N) * TC_KR * 4; }

int launch_zgemm_tn_tc(int M, int N, int K, int batch, const double *A, const double *B, long long strideB, double *C,
                       long long strideC, cudaStream_t st)
{
    if (M <= 0 || N <= 0 || K <= 0 || batch <= 0) return RSGDF_OK;
    const size_t smem = tc_smem_bytes();
    if (cudaFuncSetAttribute(k_zgemm_tn_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return RSGDF_EDEVICE;
    dim3 grid((N + TC_N - 1) / TC_N, (M + TC_M - 1) / TC_M, batch);
    k_zgemm_tn_tc<<<grid, TC_THREADS, smem, st>>>(M, N, K, (const double2 *)A, (const double2 *)B, strideB / 2,
                                                   (double2 *)C, strideC / 2);
    return cudaGetLastError() == cudaSuccess ? RSGDF_OK : RSGDF_EDEVICE;
}

int tc_status_take(int *flag)
{
    int z = 0;
    if (cudaMemcpyFromSymbol(flag, g_tc_status, sizeof(int)) != cudaSuccess) return RSGDF_EDEVICE;
    if (*flag && cudaMemcpyToSymbol(g_tc_status, &z, sizeof(int)) != cudaSuccess) return RSGDF_EDEVICE;
    return RSGDF_OK;
}

}  // namespace rsgdf

namespace rsgdf {

// ---------------------------------------------------------------------------
// Pre-split operand tiles and the pipelined GEMM.
//
// A' block (m tile, k chunk): hi then lo, each 128 real rows x 32 real k in
// the core-matrix layout above (8192 floats per block).  B' block (batch,
// n tile, k chunk): hi then lo, each 64 rows x 32 (4096 floats per block).
// The blocks are contiguous, so each chunk arrives by two bulk copies
// (cp.async.bulk, completion counted on an mbarrier).
// ---------------------------------------------------------------------------

// A'[mt][kc] from A[k][m] (complex FP64): Re rows [Re A, -Im A], Im rows [Im A, Re A]
__global__ void k_split_a(int M, int K, const double2 *A, float *Ap, int nmt, int nkc)
{
    long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long tot = (long long)nmt * nkc * 2 * TC_M * TC_KR;
    if (id >= tot) return;
    const int per = 2 * TC_M * TC_KR;
    const long long blk = id / per;
    const int e = (int)(id - blk * per);
    const int mt = (int)(blk / nkc), kc = (int)(blk - (long long)mt * nkc);
    const int r = e / TC_KR, kr = e - r * TC_KR;
    const int m = mt * TC_M + (r & (TC_M - 1)), k = kc * TC_KC + (kr >> 1);
    float v = 0.0f;
    if (m < M && k < K) {
        const double2 a = A[(long long)k * M + m];
        const double d = (r < TC_M) ? ((kr & 1) ? -a.y : a.x) : ((kr & 1) ? a.x : a.y);
        v = (float)d;
    }
    float hi, lo;
    split_tf32f(v, hi, lo);
    float *blkp = Ap + blk * TC_ABLK;
    const uint32_t o = core_off(r, kr) >> 2;
    blkp[o] = hi;
    blkp[2 * TC_M * TC_KR + o] = lo;
}

int launch_split_a(int M, int K, const double *A, float *Ap, cudaStream_t st)
{
    const int nmt = (M + TC_M - 1) / TC_M, nkc = (K + TC_KC - 1) / TC_KC;
    const long long tot = (long long)nmt * nkc * 2 * TC_M * TC_KR;
    k_split_a<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(M, K, (const double2 *)A, Ap, nmt, nkc);
    return cudaGetLastError() == cudaSuccess ? RSGDF_OK : RSGDF_EDEVICE;
}

__device__ __forceinline__ bool mbar_wait_n(uint32_t mb, int parity, long long limit)
{
    uint32_t done = 0;
    long long it = 0;
    while (!done && it < limit) {
        asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                     "selp.u32 %0, 1, 0, p;\n}"
                     : "=r"(done)
                     : "r"(mb), "r"(parity));
        it++;
    }
    return done != 0;
}

__device__ __forceinline__ bool mbar_wait(uint32_t mb, int parity) { return mbar_wait_n(mb, parity, TC_SPIN); }

// Self-test of the bounded wait and of its error report: one CTA waits on an
// mbarrier that expects one arrival.  With arrive != 0 thread 0 arrives
// first and the wait completes; with arrive == 0 nothing ever arrives, every
// thread gives up after `limit` polls and the kernel records the timeout in
// g_tc_status exactly as the tensor-core contraction does, then returns.
__global__ void k_wait_selftest(int arrive, long long limit)
{
    __shared__ __align__(8) unsigned long long bar;
    const uint32_t mb = (uint32_t)__cvta_generic_to_shared(&bar);
    if (threadIdx.x == 0) asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mb), "r"(1));
    __syncthreads();
    if (arrive && threadIdx.x == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(mb));
    const bool ok = mbar_wait_n(mb, 0, limit);
    const int all_ok = __syncthreads_and(ok ? 1 : 0);
    if (!all_ok && threadIdx.x == 0) atomicExch(&g_tc_status, 1);
}

int launch_wait_selftest(int arrive, long long limit, cudaStream_t st)
{
    if (limit < 1) return RSGDF_EINVAL;
    k_wait_selftest<<<1, 64, 0, st>>>(arrive, limit);
    return cudaGetLastError() == cudaSuccess ? RSGDF_OK : RSGDF_EDEVICE;
}

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t mb)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(mb)
                 : "memory");
}

__device__ __forceinline__ void issue_chunk_mma(uint32_t tmem_acc, uint32_t sa, uint32_t sb, uint32_t idesc)
{
    const uint32_t aAh = sa, aAl = sa + 2 * TC_M * TC_KR * 4;
    const uint32_t aBh = sb, aBl = sb + TC_N * TC_KR * 4;
#pragma unroll
    for (int ks = 0; ks < TC_KR / 8; ks++) {
        const uint32_t off = ks * 256;
        const uint64_t dah = smem_desc(aAh + off), dal = smem_desc(aAl + off);
        const uint64_t dbh = smem_desc(aBh + off), dbl = smem_desc(aBl + off);
        const uint32_t acc0 = ks > 0 ? 1u : 0u;
        asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                     "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(tmem_acc),
                     "l"(dah), "l"(dbh), "r"(idesc), "r"(acc0));
        asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                     "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(tmem_acc),
                     "l"(dah), "l"(dbl), "r"(idesc), "r"(1u));
        asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                     "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(tmem_acc),
                     "l"(dal), "l"(dbh), "r"(idesc), "r"(1u));
    }
}

// C[b][m][n] += A^T B from pre-split tiles; TC_STAGES-stage bulk-copy pipeline
// (operands requested TC_STAGES - 1 chunks ahead) and two tensor-memory
// accumulators (chunk c in accumulator c & 1).
__global__ void __launch_bounds__(TC_THREADS) k_zgemm_tc2(int M, int N, int nkc, const float *Ap, const float *Bp,
                                                          int nnt, double2 *C, long long strideC)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) unsigned long long full[TC_STAGES], done[TC_STAGES];
    __shared__ uint32_t tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int nt = blockIdx.x, mt = blockIdx.y, b = blockIdx.z;
    const int m0 = mt * TC_M, n0 = nt * TC_N;
    const int SB = (TC_ABLK + TC_BBLK) * 4;   // bytes per stage
    if (warp == 0) {
        const uint32_t dst = (uint32_t)__cvta_generic_to_shared(&tmem_base);
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst), "r"(2 * TC_N));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        for (int s = 0; s < TC_STAGES; s++) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"((uint32_t)__cvta_generic_to_shared(&full[s])), "r"(1));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"((uint32_t)__cvta_generic_to_shared(&done[s])), "r"(1));
        }
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_base;
    const uint32_t idesc = instr_desc_tf32(2 * TC_M, TC_N);
    const uint32_t s0 = (uint32_t)__cvta_generic_to_shared(smem);
    const float *Ablk = Ap + (long long)mt * nkc * TC_ABLK;
    const float *Bblk = Bp + ((long long)b * nnt + nt) * nkc * TC_BBLK;
    // chunk c lives in stage c % TC_STAGES; its barriers complete once per use
    // of the stage, so the k-th use waits on parity k & 1
    int issued = 0, landed = 0, committed = -1;   // thread 0's bookkeeping for the error path
    auto load_chunk = [&](int c) {
        const int s = c % TC_STAGES;
        const uint32_t mb = (uint32_t)__cvta_generic_to_shared(&full[s]);
        issued = c + 1;
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mb), "r"(SB));
        bulk_g2s(s0 + s * SB, Ablk + (long long)c * TC_ABLK, TC_ABLK * 4, mb);
        bulk_g2s(s0 + s * SB + TC_ABLK * 4, Bblk + (long long)c * TC_BBLK, TC_BBLK * 4, mb);
    };
    auto done_of = [&](int c) { return (uint32_t)__cvta_generic_to_shared(&done[c % TC_STAGES]); };
    float sh[TC_N], sc[TC_N];
#pragma unroll
    for (int j = 0; j < TC_N; j++) { sh[j] = 0.0f; sc[j] = 0.0f; }
    bool ok = true;
    if (tid == 0)
        for (int c = 0; c < TC_STAGES - 1 && c < nkc; c++) load_chunk(c);
    for (int c = 0; c < nkc; c++) {
        const int s = c % TC_STAGES;
        if (tid == 0) {
            // operands of chunk c have landed
            if (!mbar_wait((uint32_t)__cvta_generic_to_shared(&full[s]), (c / TC_STAGES) & 1))
                ok = false;
            else
                landed = c + 1;
            asm volatile("tcgen05.fence::after_thread_sync;");
            if (ok) issue_chunk_mma(tmem + (c & 1) * TC_N, s0 + s * SB, s0 + s * SB + TC_ABLK * 4, idesc);
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(done_of(c)));
            committed = c;
            // chunk c + STAGES - 1 goes into the stage chunk c - 1 used, free once its MMAs completed
            const int nxt = c + TC_STAGES - 1;
            if (nxt < nkc) {
                if (c >= 1 && !mbar_wait(done_of(c - 1), ((c - 1) / TC_STAGES) & 1)) ok = false;
                if (ok) load_chunk(nxt);
            }
        }
        // read out chunk c-1 (accumulator (c-1) & 1) while chunk c runs
        if (c >= 1) {
            const int ap = (c - 1) & 1;
            if (!mbar_wait(done_of(c - 1), ((c - 1) / TC_STAGES) & 1)) ok = false;
            asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll
            for (int c0 = 0; c0 < TC_N; c0 += 8) {
                uint32_t r[8];
                const uint32_t ta = tmem + ap * TC_N + ((uint32_t)(warp * 32) << 16) + c0;
                asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                             : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                               "=r"(r[7])
                             : "r"(ta));
                asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
                for (int j = 0; j < 8; j++) two_sum(sh[c0 + j], sc[c0 + j], __uint_as_float(r[j]));
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;");
        const int all_ok = __syncthreads_and(ok ? 1 : 0);
        asm volatile("tcgen05.fence::after_thread_sync;");
        if (!all_ok) {
            ok = false;
            break;
        }
    }
    if (ok && nkc >= 1) {
        const int sp = (nkc - 1) & 1;   // accumulator of the last chunk
        if (!mbar_wait(done_of(nkc - 1), ((nkc - 1) / TC_STAGES) & 1)) ok = false;
        asm volatile("tcgen05.fence::after_thread_sync;");
        if (__all_sync(0xffffffffu, ok)) {
#pragma unroll
            for (int c0 = 0; c0 < TC_N; c0 += 8) {
                uint32_t r[8];
                const uint32_t ta = tmem + sp * TC_N + ((uint32_t)(warp * 32) << 16) + c0;
                asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                             : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                               "=r"(r[7])
                             : "r"(ta));
                asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
                for (int j = 0; j < 8; j++) two_sum(sh[c0 + j], sc[c0 + j], __uint_as_float(r[j]));
            }
        } else {
            ok = false;
        }
    }
    if (!ok && (tid & 31) == 0) atomicExch(&g_tc_status, 1);
    if (!ok && tid == 0) {
        // a bounded wait gave up: let this CTA's own bulk copies and its last
        // committed MMAs finish (bounded again) before the shared and tensor
        // memory are released
        for (int c = landed; c < issued; c++) mbar_wait((uint32_t)__cvta_generic_to_shared(&full[c % TC_STAGES]), (c / TC_STAGES) & 1);
        if (committed >= 0) mbar_wait(done_of(committed), (committed / TC_STAGES) & 1);
    }
    const int r = warp * 32 + (tid & 31);
    const int m = m0 + (r & (TC_M - 1));
    if (ok && m < M) {
        double *Cr = (double *)(C + b * strideC + (long long)m * N) + (r >= TC_M ? 1 : 0);
#pragma unroll
        for (int j = 0; j < TC_N; j++) {
            const int n = n0 + j;
            if (n < N) Cr[2LL * n] += (double)sh[j] + (double)sc[j];
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * TC_N));
}

int launch_zgemm_tc2(int M, int N, int K, int batch, const float *Ap, const float *Bp, double *C, long long strideC,
                     cudaStream_t st)
{
    if (M <= 0 || N <= 0 || K <= 0 || batch <= 0) return RSGDF_OK;
    const int nkc = (K + TC_KC - 1) / TC_KC, nnt = (N + TC_N - 1) / TC_N, nmt = (M + TC_M - 1) / TC_M;
    const size_t smem = TC_STAGES * (size_t)(TC_ABLK + TC_BBLK) * 4;
    if (cudaFuncSetAttribute(k_zgemm_tc2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return RSGDF_EDEVICE;
    dim3 grid(nnt, nmt, batch);
    k_zgemm_tc2<<<grid, TC_THREADS, smem, st>>>(M, N, nkc, Ap, Bp, nnt, (double2 *)C, strideC / 2);
    return cudaGetLastError() == cudaSuccess ? RSGDF_OK : RSGDF_EDEVICE;
}

long long tc_b_floats(int N, int K, int batch)
{
    const long long nkc = (K + TC_KC - 1) / TC_KC, nnt = (N + TC_N - 1) / TC_N;
    return (long long)batch * nnt * nkc * TC_BBLK;
}

long long tc_a_floats(int M, int K)
{
    const long long nkc = (K + TC_KC - 1) / TC_KC, nmt = (M + TC_M - 1) / TC_M;
    return nmt * nkc * TC_ABLK;
}

}  // namespace rsgdf
