// C ABI of the RSGDF library: argument checks, the host planner, device
// uploads, the launch sequence of the j3c / j2c / kphase paths and the error
// and statistics reporting.  Scratch memory is allocated stream-ordered on
// the caller's stream and released before each call returns.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <memory>
#include <atomic>
#include <future>
#include <mutex>
#include <set>
#include <string>
#include <vector>

#include "k_common.cuh"
#include "rsgdf_internal.h"

namespace rsgdf {

static thread_local std::string t_err;
static thread_local rsgdf_stats t_stats;
static thread_local cudaStream_t t_stats_stream = nullptr;
static thread_local unsigned long long *t_count_host = nullptr;   // pinned [LTOT_MAX+1]
static thread_local bool t_count_valid = false;

// Per-phase device timers: an event pair around each launch group, summed
// when the statistics are read.
enum { PH_SR = 0, PH_AFT, PH_GEMM, PH_PHASE, PH_OTHER, PH_N };
struct PhaseTimer {
    // event pairs: a phase (kind >= 0) on the call's stream, or one SR class
    // (cls >= 0) on any stream; a pair with kind -1 only times its class
    struct Pair {
        cudaEvent_t b = nullptr, e = nullptr;
        int kind = -1, cls = -1;
    };
    std::vector<Pair> pairs;
    std::vector<int> open;   // pairs begun on the call's stream and not yet ended
    int side_open = -1;
    cudaStream_t st = nullptr;
    bool on = true;   // off while a graph is captured
    void reset(cudaStream_t s)
    {
        for (auto &p : pairs) {
            if (p.b) cudaEventDestroy(p.b);
            if (p.e) cudaEventDestroy(p.e);
        }
        pairs.clear();
        open.clear();
        side_open = -1;
        st = s;
        on = true;
    }
    static cudaEvent_t rec(cudaStream_t s)
    {
        cudaEvent_t e;
        cudaEventCreate(&e);
        cudaEventRecord(e, s);
        return e;
    }
    void begin(int k, int c = -1)
    {
        if (!on) return;
        Pair p;
        p.kind = k;
        p.cls = c;
        p.b = rec(st);
        pairs.push_back(p);
        open.push_back((int)pairs.size() - 1);
    }
    void end()
    {
        if (!on || open.empty()) return;
        pairs[open.back()].e = rec(st);
        open.pop_back();
    }
    void begin_on(cudaStream_t s, int c)
    {
        if (!on) return;
        Pair p;
        p.cls = c;
        p.b = rec(s);
        pairs.push_back(p);
        side_open = (int)pairs.size() - 1;
    }
    void end_on(cudaStream_t s)
    {
        if (!on || side_open < 0) return;
        pairs[side_open].e = rec(s);
        side_open = -1;
    }
    void totals(double *ms, double *cls_ms)
    {
        for (int i = 0; i < PH_N; i++) ms[i] = 0.0;
        for (int i = 0; i <= LTOT_MAX; i++) cls_ms[i] = 0.0;
        for (const Pair &p : pairs) {
            float t = 0.0f;
            if (!p.b || !p.e || cudaEventElapsedTime(&t, p.b, p.e) != cudaSuccess) continue;
            if (p.kind >= 0) ms[p.kind] += t;
            if (p.cls >= 0) cls_ms[p.cls] += t;
        }
    }
};
static thread_local PhaseTimer t_timer;

static int fail(int code, const std::string &msg)
{
    t_err = msg;
    return code;
}

#define CU(x)                                                                           \
    do {                                                                                \
        cudaError_t e_ = (x);                                                           \
        if (e_ != cudaSuccess) return fail(RSGDF_EDEVICE, std::string(#x ": ") + cudaGetErrorString(e_)); \
    } while (0)

#define RC(x)                                   \
    do {                                        \
        int r_ = (x);                           \
        if (r_ != RSGDF_OK) {                   \
            if (t_err.empty()) t_err = #x;      \
            return r_;                          \
        }                                       \
    } while (0)

// Stream-ordered device scratch released on scope exit.
// Largest device scratch one call may hold (bytes; 0 = no limit), set by
// rsgdf_set_scratch_limit.
static std::atomic<long long> g_scratch_limit{0};

// The device's default stream-ordered pool, where scratch comes from, returns
// its memory to the driver at every synchronisation unless told to keep some
// (release threshold 0), and mapping it again costs milliseconds per call.
// Once per device the threshold is raised to keep up to 8 GiB between calls
// (never lowered).
static void keep_pool_memory()
{
    static std::atomic<unsigned long long> done{0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return;
    }
    if (done.load() & (1ull << dev)) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        unsigned long long cur = 0, keep = 8ull << 30;
        if (cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &cur) == cudaSuccess && cur < keep)
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    cudaGetLastError();
    done.fetch_or(1ull << dev);
}

// Pinned staging of host-to-device uploads.  A copy from pageable memory goes
// through the driver's small staging buffers, and when the stream still holds
// queued kernels (j3c enqueues its LR work before the SR set-up) the host
// waits until the device has drained them: about 2 ms of the headline call.
// Uploads are therefore copied into a pinned arena of the calling thread and
// sent from there.  The arena is filled front to back and reused from the
// front once every copy sent from it has completed (an event per stream after
// its last copy); if it fills while copies are pending, a larger one takes
// over and the full one is freed at the next such point.  Uploads above
// 64 MiB, and uploads during a stream capture, take the pageable path.
struct PinnedArena {
    char *buf = nullptr;
    size_t cap = 0, used = 0;
    std::vector<char *> retired;                               // full arenas whose copies may still be pending
    std::vector<std::pair<cudaStream_t, cudaEvent_t>> marks;   // last copy per stream
    bool idle() const
    {
        for (const auto &m : marks)
            if (cudaEventQuery(m.second) == cudaErrorNotReady) return false;
        cudaGetLastError();
        return true;
    }
    void drain()
    {
        for (const auto &m : marks) cudaEventSynchronize(m.second);
        cudaGetLastError();
    }
    // pinned destination of n bytes for a copy on stream s, or nullptr (pageable path)
    char *take(size_t n, cudaStream_t s)
    {
        constexpr size_t MAXUP = 64ull << 20, MAXCAP = 256ull << 20;
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (n == 0 || n > MAXUP || cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
            cudaGetLastError();
            return nullptr;
        }
        n = (n + 255) & ~(size_t)255;
        if ((used > 0 || !retired.empty()) && idle()) {   // every copy sent so far has completed
            for (char *r : retired) cudaFreeHost(r);
            retired.clear();
            used = 0;
        }
        if (used + n > cap) {
            // a larger arena; the full one is freed once its copies have completed
            const size_t want = std::min(MAXCAP, std::max({(size_t)32 << 20, 2 * cap, 2 * n}));
            void *p = nullptr;
            if (want < n || cudaHostAlloc(&p, want, cudaHostAllocPortable) != cudaSuccess) {
                cudaGetLastError();
                drain();   // no larger arena: wait for the pending copies and reuse this one
                if (n > cap) return nullptr;
                used = 0;
            } else {
                if (buf) retired.push_back(buf);
                buf = (char *)p;
                cap = want;
                used = 0;
            }
        }
        char *q = buf + used;
        used += n;
        return q;
    }
    bool mark(cudaStream_t s)
    {
        for (auto &m : marks)
            if (m.first == s) return cudaEventRecord(m.second, s) == cudaSuccess;
        cudaEvent_t e;
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return false;
        marks.push_back({s, e});
        return cudaEventRecord(e, s) == cudaSuccess;
    }
};
static thread_local PinnedArena t_upload_arena;

struct Scratch {
    cudaStream_t st;
    std::vector<void *> ptrs;
    size_t held = 0;
    explicit Scratch(cudaStream_t s) : st(s) { keep_pool_memory(); }
    ~Scratch()
    {
        for (void *p : ptrs) cudaFreeAsync(p, st);
    }
    template <class T>
    int alloc(T *&p, size_t n)
    {
        p = nullptr;
        if (n == 0) n = 1;
        const long long lim = g_scratch_limit.load();
        if (lim > 0 && held + n * sizeof(T) > (size_t)lim)
            return fail(RSGDF_ENOMEM, "device scratch of " + std::to_string(held + n * sizeof(T)) +
                                          " bytes would exceed the limit of " + std::to_string(lim) + " bytes");
        void *q = nullptr;
        if (cudaMallocAsync(&q, n * sizeof(T), st) != cudaSuccess) {
            cudaGetLastError();
            return fail(RSGDF_ENOMEM, "device allocation of " + std::to_string(n * sizeof(T)) + " bytes failed");
        }
        ptrs.push_back(q);
        held += n * sizeof(T);
        p = (T *)q;
        return RSGDF_OK;
    }
    template <class T>
    int upload(T *&p, const std::vector<T> &v)
    {
        RC(alloc(p, v.size()));
        if (v.empty()) return RSGDF_OK;
        const size_t bytes = v.size() * sizeof(T);
        const void *src = v.data();
        char *pin = t_upload_arena.take(bytes, st);
        if (pin) {
            memcpy(pin, v.data(), bytes);
            src = pin;
        }
        if (cudaMemcpyAsync(p, src, bytes, cudaMemcpyHostToDevice, st) != cudaSuccess)
            return fail(RSGDF_EDEVICE, "host-to-device copy failed");
        if (pin && !t_upload_arena.mark(st)) return fail(RSGDF_EDEVICE, "event record failed");
        return RSGDF_OK;
    }
};

static int check_device()
{
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || n == 0) {
        cudaGetLastError();
        return fail(RSGDF_EDEVICE, "no CUDA device");
    }
    int dev = 0, major = 0, minor = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
    if (major * 10 + minor != 103) return fail(RSGDF_EDEVICE, "library built for sm_103a only");
    return RSGDF_OK;
}

static int upload_shells(Scratch &S, const HBasis &h, DevShells &d)
{
    int *l, *np, *po, *fo;
    double *c, *e, *cn;
    RC(S.upload(l, h.l));
    RC(S.upload(np, h.nprim));
    RC(S.upload(po, h.poff));
    RC(S.upload(fo, h.foff));
    RC(S.upload(c, h.center));
    RC(S.upload(e, h.exps));
    RC(S.upload(cn, h.cn));
    d.l = l; d.nprim = np; d.poff = po; d.foff = fo; d.cen = c; d.exps = e; d.cn = cn;
    return RSGDF_OK;
}

static int ensure_boys(cudaStream_t st)
{
    static std::vector<double> tab;
    static bool built = false;
    if (!built) {
        boys_table(tab);
        built = true;
    }
    return upload_boys_table(tab.data(), st);
}

// e^{i k.cell} for every mesh k and BvK cell, exact integer angle reduction
static void phase_table(const Lattice &L, std::vector<double> &ph)
{
    ph.assign((size_t)2 * L.Nk * L.Nk, 0.0);
    for (int k = 0; k < L.Nk; k++) {
        int n[3] = {k / (L.nk[1] * L.nk[2]), (k / L.nk[2]) % L.nk[1], k % L.nk[2]};
        for (int c = 0; c < L.Nk; c++) {
            int j[3] = {c / (L.nk[1] * L.nk[2]), (c / L.nk[2]) % L.nk[1], c % L.nk[2]};
            long double f = 0.0L;
            for (int i = 0; i < 3; i++) f += (long double)((n[i] * j[i]) % L.nk[i]) / L.nk[i];
            long double ang = 2.0L * 3.141592653589793238462643383279502884L * f;
            ph[2 * ((size_t)k * L.Nk + c)] = (double)cosl(ang);
            ph[2 * ((size_t)k * L.Nk + c) + 1] = (double)sinl(ang);
        }
    }
}

static int k12_of(const Lattice &L, int k1, int k2)
{
    int a[3] = {k1 / (L.nk[1] * L.nk[2]), (k1 / L.nk[2]) % L.nk[1], k1 % L.nk[2]};
    int b[3] = {k2 / (L.nk[1] * L.nk[2]), (k2 / L.nk[2]) % L.nk[1], k2 % L.nk[2]};
    int d[3];
    for (int i = 0; i < 3; i++) d[i] = ((b[i] - a[i]) % L.nk[i] + L.nk[i]) % L.nk[i];
    return (d[0] * L.nk[1] + d[1]) * L.nk[2] + d[2];
}

static void k12_frac(const Lattice &L, int k12, double f[3])
{
    int d[3] = {k12 / (L.nk[1] * L.nk[2]), (k12 / L.nk[2]) % L.nk[1], k12 % L.nk[2]};
    for (int i = 0; i < 3; i++) {
        double x = (double)d[i] / L.nk[i];
        if (x >= 0.5) x -= 1.0;
        f[i] = x;
    }
}

static void gbox(const int gm[3], std::vector<int> &g)
{
    g.clear();
    for (int i = -(gm[0] - 1) / 2; i <= (gm[0] - 1) / 2; i++)
        for (int j = -(gm[1] - 1) / 2; j <= (gm[1] - 1) / 2; j++)
            for (int k = -(gm[2] - 1) / 2; k <= (gm[2] - 1) / 2; k++) {
                g.push_back(i);
                g.push_back(j);
                g.push_back(k);
            }
}

static void fill_lattice(const Lattice &L, double a9[9], double bq[9], int nk[3])
{
    for (int i = 0; i < 3; i++)
        for (int x = 0; x < 3; x++) {
            a9[3 * i + x] = L.a[i][x];
            bq[3 * i + x] = L.b[i][x] / (2.0 * 3.141592653589793238462643383279502884);
        }
    for (int i = 0; i < 3; i++) nk[i] = L.nk[i];
}

static int check_opts(const rsgdf_opts *o)
{
    if (!o) return fail(RSGDF_EINVAL, "opts is NULL");
    if (!(o->eps_screen > 0.0 && o->eps_screen < 1.0)) return fail(RSGDF_EINVAL, "eps_screen must be in (0, 1)");
    if (o->precision != RSGDF_FP64 && o->precision != RSGDF_MIXED) return fail(RSGDF_EINVAL, "unknown precision mode");
    if (o->screening != RSGDF_SCREEN_BOUND && o->screening != RSGDF_SCREEN_LEARNED)
        return fail(RSGDF_EINVAL, "unknown screening mode");
    if (!(o->split_alpha >= 0.0) || !std::isfinite(o->split_alpha))
        return fail(RSGDF_EINVAL, "split_alpha must be finite and >= 0");
    if (o->kernel != RSGDF_KERNEL_ERF && o->kernel != RSGDF_KERNEL_PLAIN) return fail(RSGDF_EINVAL, "unknown kernel");
    return RSGDF_OK;
}

}  // namespace rsgdf

struct rsgdf_mlp {
    int F, np, dev;
    float *P, *G, *m, *v, *mean, *stdv;
    __half *P16;
    float margin;
    int base;                  // feature added to the network output (-1: none)
    float base_lo, base_hi;    // clamp of that feature
    float guard[rsgdf::LTOT_MAX + 1];   // per class L: skip only if feature + guard[L] < cut as well
    int step;
};

namespace rsgdf {

// ---------------------------------------------------------------------------
// SR lattice sums: per-problem setup (uploads, per-class descriptors), the
// per-problem pre-pass (pair Hermite tables, learned screen) and the class
// launches, which may cover several problems at once.
// ---------------------------------------------------------------------------
struct SRExtras {
    const rsgdf_mlp *mlp = nullptr;   // learned screen
    double log10_cut = 0.0;           // prune below this predicted log10 magnitude (after the margin)
    float *feat_out = nullptr;        // features of every item (device [n][SR_NFEAT])
    float *mag_out = nullptr;         // magnitude mode (device [n])
    bool skip_sr = false;             // features only
    float log_prim_cut = -1e31f;      // per-combination bound cut (natural log); -1e31: none
};

struct SRSetup {
    SRArgs A;                        // fields common to every class
    std::vector<SRArgs> cls;         // per class with work: triple and item ranges, list sizes
    std::vector<int> cls_L;
    DevShells ao{};
    int nshell = 0;
    PairEntry *dent = nullptr;       // SR pair entries and their Hermite table
    int nent = 0;
    int *ddl = nullptr;
    double *da9 = nullptr, *ptab = nullptr;
    const rsgdf_mlp *mlp = nullptr;
    float log10_cut = 0.0f;
    float *feat = nullptr, *pred = nullptr;
    unsigned char *skip = nullptr;
    unsigned long long *counts = nullptr;
    SRItemGeom *geom = nullptr;      // per-item geometry, written by sr_pre
    long long n_items = 0;
    int ntri = 0;
    bool skip_sr = false;
};

static int sr_setup(SRSetup &R, Scratch &S, const Lattice &L, const SRPlan &plan, const DevShells &ao,
                    const DevShells &ax, const HBasis &hao, const HBasis &hax, double omega, double *X, long long s_lt,
                    long long s_dt, long long s_P, long long s_mu, long long s_nu, int pfunc0,
                    unsigned long long *counts, const SRExtras &ex = SRExtras())
{
    memset(&R.A, 0, sizeof(R.A));
    R.cls.clear();
    R.cls_L.clear();
    R.n_items = plan.n_items;
    R.ntri = (int)plan.tri.size();
    R.counts = counts;
    R.skip_sr = ex.skip_sr;
    if (plan.tri.empty()) return RSGDF_OK;
    for (const SRTriple &t : plan.tri)
        if (hax.nprim[t.P] * hao.nprim[t.mu] * hao.nprim[t.nu] > 64)
            return fail(RSGDF_ENOTIMPL, "more than 64 primitive combinations in one shell triple");
    // per triple: the device record, its work items, and the constants of its
    // primitive combinations (k; i, j), which do not depend on the item's d:
    // alpha = p g/(p + g), s = w^2/(w^2 + alpha), sqrt s, the prefactor
    // 2 pi^{5/2}/(p g sqrt(p + g)) c_k c_i c_j (-1)^lP, and the d-independent
    // part of the log Coulomb bound of the combination
    std::vector<SRTripleDev> td(plan.tri.size());
    std::vector<double> ccon;
    std::vector<float> cbnd;
    const double om2 = omega * omega;
    const double gamma_half[11] = {0.0, 1.7724538509055160, 1.0, 0.8862269254527580, 1.0, 1.3293403881791370,
                                   2.0, 3.3233509704478426, 6.0, 11.631728396567450, 24.0};   // Gamma(n/2)
    // log |c| of every primitive and log g of every aux primitive, for the bounds
    std::vector<double> lcx(hax.exps.size()), lgx(hax.exps.size()), lco(hao.exps.size());
    for (size_t o = 0; o < lcx.size(); o++) {
        lcx[o] = std::log(std::fabs(hax.cn[o]));
        lgx[o] = std::log(hax.exps[o]);
    }
    for (size_t o = 0; o < lco.size(); o++) lco[o] = std::log(std::fabs(hao.cn[o]));
    for (size_t i = 0; i < plan.tri.size(); i++) {
        const SRTriple &t = plan.tri[i];
        td[i] = {t.P, t.mu, t.nu, t.pair, t.nwin, t.win_off, t.nd, t.nsph, (int)(ccon.size() / 4), t.Rc_cut, t.amu,
                 t.anu, t.item_off, t.log10A, t.beta, t.eta1, t.eta2, t.aP};
        const int lP = hax.l[t.P];
        const double lgam = std::log(2.0 * KPI * gamma_half[lP + 2]);
        for (int k = 0; k < hax.nprim[t.P]; k++)
            for (int ii = 0; ii < hao.nprim[t.mu]; ii++)
                for (int jj = 0; jj < hao.nprim[t.nu]; jj++) {
                    const int ok = hax.poff[t.P] + k, oi = hao.poff[t.mu] + ii, oj = hao.poff[t.nu] + jj;
                    const double g = hax.exps[ok], p = hao.exps[oi] + hao.exps[oj];
                    const double ipg = 1.0 / (p + g);
                    const double alpha = p * g * ipg;
                    const double s = om2 / (om2 + alpha);
                    ccon.push_back(alpha);
                    ccon.push_back(s);
                    ccon.push_back(std::sqrt(s));
                    ccon.push_back(2.0 * KPI2_5 / (p * g) * std::sqrt(ipg) * hax.cn[ok] * (hao.cn[oi] * hao.cn[oj]) *
                                   ((lP & 1) ? -1.0 : 1.0));
                    const double lq = lcx[ok] + lgam - 0.5 * (lP + 2) * lgx[ok] + (lco[oi] + lco[oj]);
                    cbnd.push_back((float)std::max(lq, -1e30));
                }
    }
    SRTripleDev *dtri;
    double *dwin;
    int *dpoff, *dsph;
    RC(S.upload(dtri, td));
    RC(S.upload(dwin, plan.win));
    RC(S.upload(dpoff, plan.pair_doff));
    RC(S.upload(R.ddl, plan.dlist));
    RC(S.upload(dsph, plan.sph));
    // Cartesian vectors of the lattice list, FP64 and FP32
    std::vector<double> sphv(plan.sph.size());
    std::vector<float> sphvf(plan.sph.size());
    for (size_t i = 0; i + 2 < plan.sph.size(); i += 3)
        for (int x = 0; x < 3; x++) {
            sphv[i + x] = plan.sph[i] * L.a[0][x] + plan.sph[i + 1] * L.a[1][x] + plan.sph[i + 2] * L.a[2][x];
            sphvf[i + x] = (float)sphv[i + x];
        }
    double *dsphv;
    float *dsphvf;
    RC(S.upload(dsphv, sphv));
    RC(S.upload(dsphvf, sphvf));
    std::vector<float> sphlen(plan.sph_len.begin(), plan.sph_len.end());
    float *dsphlen;
    RC(S.upload(dsphlen, sphlen));
    double *dccon;
    float *dcbnd;
    RC(S.alloc(R.geom, (size_t)std::max(plan.n_items, 1LL)));
    RC(S.upload(dccon, ccon));
    RC(S.upload(dcbnd, cbnd));
    // Hermite tables of every (pair, d, primitive pair) of the SR d lists,
    // shared by all aux shells (entries of one d contiguous, ij order)
    const int npairs = hao.nshell * hao.nshell;
    std::vector<long long> sr_doff(plan.pair_doff[npairs] + 1, 0);
    std::vector<PairEntry> ent;
    long long off = 0;
    for (int pr = 0; pr < npairs; pr++) {
        const int mu = pr / hao.nshell, nu = pr % hao.nshell;
        const long long esz = ENT_HDR + 3LL * (hao.l[mu] + 1) * (hao.l[nu] + 1) * (hao.l[mu] + hao.l[nu] + 2) / 2;
        for (int gd = plan.pair_doff[pr]; gd < plan.pair_doff[pr + 1]; gd++) {
            sr_doff[gd] = off;
            for (int i = 0; i < hao.nprim[mu]; i++)
                for (int j = 0; j < hao.nprim[nu]; j++) {
                    ent.push_back({off, pr, gd, i, j});
                    off += esz;
                }
        }
    }
    long long *dsrdoff;
    RC(S.upload(R.dent, ent));
    R.nent = (int)ent.size();
    RC(S.upload(dsrdoff, sr_doff));
    RC(S.alloc(R.ptab, (size_t)std::max(off, 1LL)));
    R.ao = ao;
    R.nshell = hao.nshell;
    {
        double a9h[9], bq_unused[9];
        int nk_unused[3];
        fill_lattice(L, a9h, bq_unused, nk_unused);
        RC(S.upload(R.da9, std::vector<double>(a9h, a9h + 9)));
    }
    // single-centre Hermite coefficients of every aux primitive
    std::vector<double> ec((size_t)hax.exps.size() * (LMAX + 1) * (LMAX + 1), 0.0);
    for (int sh = 0; sh < hax.nshell; sh++)
        for (int k = 0; k < hax.nprim[sh]; k++) {
            const int o = hax.poff[sh] + k;
            single_E_host(hax.l[sh], hax.exps[o], &ec[(size_t)o * (LMAX + 1) * (LMAX + 1)]);
        }
    double *dec;
    RC(S.upload(dec, ec));
    SRArgs &A = R.A;
    A.ao = ao;
    A.ax = ax;
    A.tri = dtri;
    A.win = dwin;
    A.pair_doff = dpoff;
    A.dlist = R.ddl;
    A.sph = dsph;
    A.log_prim_cut = ex.log_prim_cut;
    A.sphv = dsphv;
    A.sphvf = dsphvf;
    A.sphlen = dsphlen;
    A.ntri = (int)plan.tri.size();
    A.geom = R.geom;
    A.ccon = dccon;
    A.cbnd = dcbnd;
    fill_lattice(L, A.a, A.bq, A.nk);
    A.Nk = L.Nk;
    A.omega = omega;
    A.X = X;
    A.s_lt = s_lt; A.s_dt = s_dt; A.s_P = s_P; A.s_mu = s_mu; A.s_nu = s_nu;
    A.pfunc0 = pfunc0;
    A.term_count = counts;
    for (int x = 0; x < 9; x++) A.af[x] = (float)A.a[x];
    A.ec_tab = dec;
    A.ptab = R.ptab;
    A.sr_doff = dsrdoff;
    A.item_mag = ex.mag_out;
    A.tri_begin = 0;
    A.tri_end = R.ntri;
    A.item_begin = 0;
    A.item_end = plan.n_items;
    // learned screen buffers
    R.feat = ex.feat_out;
    if ((ex.mlp || R.feat) && plan.n_items > 0) {
        if (!R.feat) RC(S.alloc(R.feat, (size_t)plan.n_items * SR_NFEAT));
        if (ex.mlp) {
            R.mlp = ex.mlp;
            R.log10_cut = (float)ex.log10_cut;
            RC(S.alloc(R.pred, (size_t)plan.n_items));
            RC(S.alloc(R.skip, (size_t)plan.n_items));
            A.item_skip = R.skip;
        }
    }
    // per-class descriptors
    for (int c = 0; c <= LTOT_MAX; c++) {
        int b = plan.class_tri_begin[c], e = plan.class_tri_begin[c + 1];
        if (b >= e) continue;
        int ncmax = 0, wmax = 0, lmax_list = 0, cmax = 1;
        for (int i = b; i < e; i++) {
            const SRTriple &t = plan.tri[i];
            const int lP = hax.l[t.P], lm = hao.l[t.mu], ln = hao.l[t.nu];
            cmax = std::max(cmax, hax.nprim[t.P] * hao.nprim[t.mu] * hao.nprim[t.nu]);
            ncmax = std::max(ncmax, ncart(lP) * ncart(lm) * ncart(ln));
            if (lP > 0) wmax = std::max(wmax, ncart(lP) * ntuv(lm + ln));
            // coefficient-list length: sum over (a, b) of (ax+bx+1)(ay+by+1)(az+bz+1)
            int tot = 0;
            for (int ia = 0; ia < ncart(lm); ia++)
                for (int ib = 0; ib < ncart(ln); ib++) {
                    int ax3[3], bx3[3], n = 0;
                    for (int x = lm; x >= 0; x--)
                        for (int y = lm - x; y >= 0; y--) { if (n++ == ia) { ax3[0] = x; ax3[1] = y; ax3[2] = lm - x - y; } }
                    n = 0;
                    for (int x = ln; x >= 0; x--)
                        for (int y = ln - x; y >= 0; y--) { if (n++ == ib) { bx3[0] = x; bx3[1] = y; bx3[2] = ln - x - y; } }
                    tot += (ax3[0] + bx3[0] + 1) * (ax3[1] + bx3[1] + 1) * (ax3[2] + bx3[2] + 1);
                }
            lmax_list = std::max(lmax_list, tot);
        }
        SRArgs Ac = A;
        Ac.tri_begin = b;
        Ac.tri_end = e;
        Ac.item_begin = plan.tri[b].item_off;
        Ac.item_end = (e < (int)plan.tri.size()) ? plan.tri[e].item_off : plan.n_items;
        Ac.ncomp_max = ncmax;
        Ac.w_max = wmax;
        Ac.list_max = lmax_list;
        Ac.combo_max = cmax;
        Ac.nbin_max = A.Nk;
        R.cls.push_back(Ac);
        R.cls_L.push_back(c);
    }
    return RSGDF_OK;
}

// Pair Hermite tables, then (learned screen) features -> prediction -> mask.
static int sr_pre(const SRSetup &R, cudaStream_t st, int &nl)
{
    if (R.ntri == 0) return RSGDF_OK;
    t_timer.begin(PH_SR);
    RC(launch_pair_prep(R.ao, R.nshell, R.dent, R.nent, R.ddl, R.da9, R.ptab, nullptr, nullptr, nullptr, st));
    RC(launch_sr_item_geom(R.A, R.n_items, R.geom, st));
    t_timer.end();
    nl += 2;
    if (R.feat && R.n_items > 0) {
        t_timer.begin(PH_OTHER);
        RC(launch_sr_features(R.A, R.feat, st));
        nl++;
        if (R.mlp) {
            RC(launch_mlp_forward(R.mlp->F, R.mlp->P16, R.mlp->mean, R.mlp->stdv, R.feat, R.n_items, R.pred, st));
            RC(launch_mlp_mask(R.n_items, SR_NFEAT, R.feat, R.mlp->base, R.mlp->base_lo, R.mlp->base_hi, R.mlp->guard, R.pred,
                               R.mlp->margin, R.log10_cut, R.skip, R.counts ? R.counts + 2 * LTOT_MAX + 4 : nullptr,
                               st));
            nl += 2;
        }
        t_timer.end();
    }
    return RSGDF_OK;
}

// One launch of one class over the items of several problems.
struct SRClassLaunch {
    int L = 0;
    std::vector<SRArgs> desc;
    std::vector<long long> cum;
    SRArgs *ddesc = nullptr;
    long long *dcum = nullptr;
    int ncmax = 0, wmax = 0, lmax = 0, cmax = 1;
    int nkmax = 1;   // largest k mesh among the descriptors (bin chunks beyond it are useless)
    int bc = 1;
    size_t warp_bytes = 0;
    long long ntot = 0;
    int grid = 1, grab = 1;
};

static int g_num_sms = 0;

static int sr_set_bc(SRClassLaunch &c, int bc, cudaStream_t st)
{
    c.bc = bc;
    c.warp_bytes = sr_warp_bytes(c.L, bc, c.ncmax, c.wmax, c.lmax, c.cmax, c.nkmax);
    for (SRArgs &a : c.desc) {
        a.bc = bc;
        a.warp_bytes = (int)c.warp_bytes;
        a.ncomp_max = c.ncmax;
        a.w_max = c.wmax;
        a.list_max = c.lmax;
        a.combo_max = c.cmax;
        a.nbin_max = c.nkmax;
    }
    CU(cudaMemcpyAsync(c.ddesc, c.desc.data(), sizeof(SRArgs) * c.desc.size(), cudaMemcpyHostToDevice, st));
    const int occ = sr_occupancy(c.L, sr_launch_smem(c.L, bc, c.ncmax, c.wmax, c.lmax, c.cmax, c.nkmax));
    if (occ < 1) return fail(RSGDF_EDEVICE, "SR kernel does not fit on an SM");
    if (!g_num_sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
    }
    c.grid = occ * std::max(g_num_sms, 1);
    return RSGDF_OK;
}

// Merge the classes of several problems into one launch per class.
static int sr_merge(const std::vector<const SRSetup *> &rs, Scratch &S, cudaStream_t st,
                    std::vector<SRClassLaunch> &out)
{
    out.clear();
    for (int L = 0; L <= LTOT_MAX; L++) {
        SRClassLaunch c;
        c.L = L;
        c.cum.push_back(0);
        for (const SRSetup *r : rs) {
            if (r->skip_sr) continue;
            for (size_t i = 0; i < r->cls.size(); i++) {
                if (r->cls_L[i] != L) continue;
                const SRArgs &a = r->cls[i];
                c.desc.push_back(a);
                c.cum.push_back(c.cum.back() + (a.item_end - a.item_begin));
                c.ncmax = std::max(c.ncmax, a.ncomp_max);
                c.nkmax = std::max(c.nkmax, a.Nk);
                c.wmax = std::max(c.wmax, a.w_max);
                c.lmax = std::max(c.lmax, a.list_max);
                c.cmax = std::max(c.cmax, a.combo_max);
            }
        }
        if (c.desc.empty()) continue;
        c.ntot = c.cum.back();
        RC(S.alloc(c.ddesc, c.desc.size()));
        RC(S.upload(c.dcum, c.cum));
        RC(sr_set_bc(c, sr_default_bc(L, c.ncmax, c.wmax, c.nkmax), st));
        out.push_back(std::move(c));
    }
    return RSGDF_OK;
}

// Side streams of this host thread on the current device, one per class,
// created once: the class launches of an SR pass are independent (each adds
// its own blocks into X with atomics and owns its queue counter), so they
// run concurrently, forked from and joined to the caller's stream by events.
// A class whose items are few and long (high L) then shares the SMs with the
// many short items of the low classes instead of running its tail alone.
struct SideStreams {
    int dev = -1;
    cudaStream_t s[LTOT_MAX + 1] = {};
    cudaEvent_t fork = nullptr, join[LTOT_MAX + 1] = {};
};
static thread_local SideStreams t_side[8];

static int side_streams(SideStreams *&ss)
{
    int dev = 0;
    CU(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 8) {
        ss = nullptr;
        return RSGDF_OK;   // serial launches on the caller's stream
    }
    ss = &t_side[dev];
    if (ss->dev != dev) {
        for (int i = 0; i <= LTOT_MAX; i++) {
            CU(cudaStreamCreateWithFlags(&ss->s[i], cudaStreamNonBlocking));
            CU(cudaEventCreateWithFlags(&ss->join[i], cudaEventDisableTiming));
        }
        CU(cudaEventCreateWithFlags(&ss->fork, cudaEventDisableTiming));
        ss->dev = dev;
    }
    return RSGDF_OK;
}

static int sr_run(std::vector<SRClassLaunch> &cl, unsigned long long *dqueue, cudaStream_t st, int &nl)
{
    if (cl.empty()) return RSGDF_OK;
    SideStreams *ss = nullptr;
    RC(side_streams(ss));
    if (!ss || cl.size() == 1) {
        for (SRClassLaunch &c : cl) {
            t_timer.begin(PH_SR, c.L);
            RC(launch_sr_queue(c.L, c.ddesc, c.dcum, (int)c.desc.size(), c.ntot, c.warp_bytes, dqueue + c.L,
                               c.grid, c.grab, st));
            t_timer.end();
            nl++;
        }
        return RSGDF_OK;
    }
    t_timer.begin(PH_SR);
    CU(cudaEventRecord(ss->fork, st));
    // heaviest items first: their classes start while the SMs are empty
    std::vector<SRClassLaunch *> order;
    for (SRClassLaunch &c : cl) order.push_back(&c);
    std::sort(order.begin(), order.end(), [](const SRClassLaunch *x, const SRClassLaunch *y) { return x->L > y->L; });
    for (SRClassLaunch *c : order) {
        cudaStream_t s = ss->s[c->L];
        CU(cudaStreamWaitEvent(s, ss->fork, 0));
        t_timer.begin_on(s, c->L);
        RC(launch_sr_queue(c->L, c->ddesc, c->dcum, (int)c->desc.size(), c->ntot, c->warp_bytes, dqueue + c->L,
                           c->grid, c->grab, s));
        t_timer.end_on(s);
        CU(cudaEventRecord(ss->join[c->L], s));
        nl++;
    }
    for (SRClassLaunch *c : order) CU(cudaStreamWaitEvent(st, ss->join[c->L], 0));
    t_timer.end();
    return RSGDF_OK;
}

// Autotuner of the SR class launches: bin chunk (shared memory per warp and
// so occupancy) and items per queue grab, each candidate timed on the real
// items with events.  The launches accumulate into X: callers zero X again.
static int sr_tune(std::vector<SRClassLaunch> &cl, unsigned long long *dqueue, cudaStream_t st, float *tuned_ms)
{
    cudaEvent_t e0, e1;
    CU(cudaEventCreate(&e0));
    CU(cudaEventCreate(&e1));
    float total = 0.0f;
    for (SRClassLaunch &c : cl) {
        const int bc0 = c.bc;
        int best_bc = bc0, best_grab = 1;
        float best = 1e30f;
        const int bcs[3] = {bc0, std::max(1, bc0 / 2), std::min(std::min(16, c.nkmax), bc0 * 2)};
        const int grabs[2] = {1, 4};
        for (int ib = 0; ib < 3; ib++) {
            if (ib > 0 && bcs[ib] == bcs[0]) continue;
            if (ib == 2 && bcs[2] == bcs[1]) continue;
            if (sr_set_bc(c, bcs[ib], st) != RSGDF_OK) continue;
            for (int g : grabs) {
                c.grab = g;
                cudaEventRecord(e0, st);
                int r = launch_sr_queue(c.L, c.ddesc, c.dcum, (int)c.desc.size(), c.ntot, c.warp_bytes,
                                        dqueue + c.L, c.grid, c.grab, st);
                cudaEventRecord(e1, st);
                if (r != RSGDF_OK) break;
                float ms = 0.0f;
                if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
                    return fail(RSGDF_EDEVICE, "autotuner timing failed");
                if (ms < best) {
                    best = ms;
                    best_bc = bcs[ib];
                    best_grab = g;
                }
            }
        }
        RC(sr_set_bc(c, best_bc, st));
        c.grab = best_grab;
        total += best;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (tuned_ms) *tuned_ms = total;
    return RSGDF_OK;
}

// Whole SR pass of one problem (setup, pre-pass, class launches).
static int run_sr(Scratch &S, const Lattice &L, const SRPlan &plan, const DevShells &ao, const DevShells &ax,
                  const HBasis &hao, const HBasis &hax, double omega, double *X, long long s_lt, long long s_dt,
                  long long s_P, long long s_mu, long long s_nu, int pfunc0, unsigned long long *counts,
                  cudaStream_t st, int &nlaunch, const SRExtras &ex = SRExtras())
{
    SRSetup R;
    RC(sr_setup(R, S, L, plan, ao, ax, hao, hax, omega, X, s_lt, s_dt, s_P, s_mu, s_nu, pfunc0, counts, ex));
    RC(sr_pre(R, st, nlaunch));
    if (ex.skip_sr) return RSGDF_OK;
    std::vector<SRClassLaunch> cl;
    RC(sr_merge({&R}, S, st, cl));
    unsigned long long *dq;
    RC(S.alloc(dq, LTOT_MAX + 1));
    return sr_run(cl, dq, st, nlaunch);
}

enum { MODE_SR = 1, MODE_LR = 2 };

// One j3c problem: plan, device buffers and launch parameters.  Everything
// that allocates or copies from the host happens in j3c_prepare; the
// j3c_exec_* functions only issue kernels and memsets, so a sequence of them
// can be captured into a CUDA graph.
struct J3cProblem {
    Lattice L;
    HBasis ao, ax;
    double omega = 0.0;
    int gm[3] = {0, 0, 0};
    int s0 = 0, s1 = 0, nP = 0, pfunc0 = 0, nao = 0, Nk = 0, mode = 0;
    long long m = 0;
    DevShells dao{}, dax{};
    double *da9 = nullptr;
    const void *phk = nullptr;
    int fp32 = 0;
    std::vector<int> gkey;
    int *dplist = nullptr, *dpk2 = nullptr, *dk12 = nullptr, *dgoff = nullptr;
    // SR
    SRPlan plan;
    SRSetup sr;
    double *X = nullptr;
    int nlt = 1;   // lt slabs of X: Nk, or 1 when only k12 = 0 is asked (phase 1 is then the plain sum over lt)
    // AFT pair lists
    PairEntry *dent = nullptr;
    int nent = 0;
    int *dseg = nullptr, *dalist = nullptr;
    double *ptab = nullptr;
    float *ptab32 = nullptr;
    float2 *uph = nullptr, *ph0 = nullptr;
    double *db9 = nullptr;
    bool mixed_aft = false;
    // G = 0 correction
    double *SP = nullptr, *Sf = nullptr;
    double g0fac = 0.0;
    bool g0 = false;
    // compact/diffuse split (opts->split_alpha > 0): SR and G0 on the range-separated types only
    double split_alpha = 0.0;
    std::vector<char> ax_diffuse, ao_diffuse;          // per shell: every exponent <= split_alpha
    int *dmask_ax = nullptr, *dmask_ao = nullptr;      // per function of the aux range / the AO basis
    // G space
    int *dg = nullptr;
    int NG = 0;
    double *W = nullptr, *Y = nullptr;
    float *Apl = nullptr, *Bpl = nullptr;
    long long nbpl = 0;
    int B = 1;
    double *T = nullptr;
    std::vector<GArgs> garg;
    // separable-DFT phase contractions (every k12 present, T holds them all)
    bool dft = false;
    double *Z = nullptr, *dtw = nullptr;
    float *dtw4 = nullptr;   // double-float twiddles (mixed path)
    int *dpk12 = nullptr, *dpk2all = nullptr;
    int npair = 0;
    long long aft_units = 0, lr_flops = 0;
};

// Host-side checks and derived parameters; touches no device.
static int j3c_check(J3cProblem &P, const rsgdf_cell *cell, const rsgdf_basis *ao_in, const rsgdf_basis *aux_in,
                     const rsgdf_opts *opts, int npair, const int *kpairs, int s0, int s1)
{
    RC(check_opts(opts));
    RC(make_lattice(cell, P.L, t_err));
    RC(load_basis(ao_in, P.ao, t_err));
    RC(load_basis(aux_in, P.ax, t_err));
    if (npair < 1 || !kpairs) return fail(RSGDF_EINVAL, "need at least one k pair");
    for (int i = 0; i < 2 * npair; i++)
        if (kpairs[i] < 0 || kpairs[i] >= P.L.Nk) return fail(RSGDF_EINVAL, "k index outside the mesh");
    if (s0 < 0 || s1 > P.ax.nshell || s0 >= s1) return fail(RSGDF_EINVAL, "aux shell range is empty or out of bounds");
    RC(derive_params(P.L, opts, P.omega, P.gm, t_err));
    P.s0 = s0;
    P.s1 = s1;
    return RSGDF_OK;
}

// Plans and device buffers of a problem that passed j3c_check.
// SR plan (host screening) and its device tables; needs the k12 groups.
// SR screening plan of a problem that passed j3c_check (host only, reads
// only the lattice, the bases and the options, writes only P.plan), so it
// can run on another host thread while the LR part is prepared and enqueued.
static void j3c_plan_sr(J3cProblem &P, const rsgdf_opts *opts)
{
    if (opts->split_alpha > 0.0) {
        const double acut = opts->split_alpha;
        auto diffuse = [&](const HBasis &b, int sh) {
            for (int i = 0; i < b.nprim[sh]; i++)
                if (b.exps[b.poff[sh] + i] > acut) return false;
            return true;
        };
        std::vector<char> dx(P.ax.nshell), da(P.ao.nshell);
        for (int sh = 0; sh < P.ax.nshell; sh++) dx[sh] = diffuse(P.ax, sh);
        for (int sh = 0; sh < P.ao.nshell; sh++) da[sh] = diffuse(P.ao, sh);
        plan_sr3c(P.L, P.ao, P.ax, P.s0, P.s1, P.omega, opts->eps_screen, P.plan,
                  [&](int Q, int mu, int nu) { return !dx[Q] && !(da[mu] && da[nu]); });
    } else {
        plan_sr3c(P.L, P.ao, P.ax, P.s0, P.s1, P.omega, opts->eps_screen, P.plan);
    }
}

static int j3c_prepare_sr(J3cProblem &P, Scratch &S, const rsgdf_opts *opts, unsigned long long *dcnt,
                          bool planned = false)
{
    const Lattice &L = P.L;
    const HBasis &ao = P.ao, &ax = P.ax;
    const int Nk = P.Nk, nao = P.nao;
    const long long m = P.m;
    const double omega = P.omega;
    // SR folded sums X[lt][dt][P][mu][nu]
    if (!planned) j3c_plan_sr(P, opts);
    P.nlt = (P.gkey.size() == 1 && P.gkey[0] == 0) ? 1 : Nk;
    RC(S.alloc(P.X, (size_t)P.nlt * Nk * m));
    SRExtras ex;
    if (opts->screening == RSGDF_SCREEN_LEARNED) {
        if (!opts->mlp) return fail(RSGDF_EINVAL, "learned screening needs opts->mlp");
        ex.mlp = (const rsgdf_mlp *)opts->mlp;
        if (ex.mlp->F != SR_NFEAT) return fail(RSGDF_EINVAL, "network input width does not match the SR features");
        ex.log10_cut = std::log10(opts->eps_screen) - 1.0;
    }
    // a primitive combination whose bound stays below 1e-3 eps over every
    // candidate translation of an item is not evaluated for that item
    ex.log_prim_cut = (float)std::log(1e-3 * opts->eps_screen);
    RC(sr_setup(P.sr, S, L, P.plan, P.dao, P.dax, ao, ax, omega, P.X, P.nlt > 1 ? (long long)Nk * m : 0, m,
                (long long)nao * nao, nao, 1, P.pfunc0, dcnt, ex));
    return RSGDF_OK;
}

// with_sr = false leaves the SR plan to a later j3c_prepare_sr (so that the
// host screening can overlap device work already enqueued).
static int j3c_prepare(J3cProblem &P, Scratch &S, const rsgdf_opts *opts, int npair, const int *kpairs, int mode,
                       unsigned long long *dcnt, bool with_sr = true)
{
    const Lattice &L = P.L;
    const HBasis &ao = P.ao, &ax = P.ax;
    const int s0 = P.s0, s1 = P.s1;
    const double omega = P.omega;
    P.mode = mode;
    P.nao = ao.nfunc;
    P.pfunc0 = ax.foff[s0];
    P.nP = (s1 < ax.nshell ? ax.foff[s1] : ax.nfunc) - P.pfunc0;
    P.m = (long long)P.nP * P.nao * P.nao;
    P.Nk = L.Nk;
    const int Nk = P.Nk, nao = P.nao, nP = P.nP;
    const long long m = P.m;
    RC(upload_shells(S, ao, P.dao));
    RC(upload_shells(S, ax, P.dax));
    double a9[9], bq[9];
    int nk3[3];
    fill_lattice(L, a9, bq, nk3);
    RC(S.upload(P.da9, std::vector<double>(a9, a9 + 9)));
    std::vector<double> ph;
    phase_table(L, ph);
    // k12 groups
    std::map<int, std::vector<int>> groups;
    for (int p = 0; p < npair; p++) groups[k12_of(L, kpairs[2 * p], kpairs[2 * p + 1])].push_back(p);
    std::vector<int> plist, pk2, goff;
    P.gkey.clear();
    for (auto &kv : groups) {
        goff.push_back((int)plist.size());
        P.gkey.push_back(kv.first);
        for (int p : kv.second) {
            plist.push_back(p);
            pk2.push_back(kpairs[2 * p + 1]);
        }
    }
    goff.push_back((int)plist.size());
    RC(S.upload(P.dplist, plist));
    RC(S.upload(P.dpk2, pk2));
    RC(S.upload(P.dk12, P.gkey));
    RC(S.upload(P.dgoff, goff));
    P.fp32 = (opts->precision == RSGDF_MIXED) ? 1 : 0;
    if (P.fp32) {
        // double-float phase table: (cos hi, cos lo, sin hi, sin lo)
        std::vector<float> ph4(2 * ph.size());
        for (size_t e = 0; e < ph.size(); e++) {
            const float h = (float)ph[e];
            ph4[2 * e] = h;
            ph4[2 * e + 1] = (float)(ph[e] - (double)h);
        }
        float *dph4;
        RC(S.upload(dph4, ph4));
        P.phk = dph4;
    } else {
        double *dph;
        RC(S.upload(dph, ph));
        P.phk = dph;
    }
    if ((mode & MODE_SR) && with_sr) RC(j3c_prepare_sr(P, S, opts, dcnt));
    // AFT pair lists (also the overlaps of the G = 0 correction): entries
    // (pair, d, primitive pair) grouped by (pair, BvK cell of d)
    std::vector<int> apoff, alist;
    plan_pairs(L, ao, opts->eps_lr, apoff, alist);
    std::vector<PairEntry> ent;
    std::vector<int> seg((size_t)ao.nshell * ao.nshell * Nk + 1, 0);
    long long tab_len = 0;
    {
        std::vector<std::vector<int>> bybin(Nk);
        for (int pr = 0; pr < ao.nshell * ao.nshell; pr++) {
            int mu = pr / ao.nshell, nu = pr % ao.nshell;
            long long esz = ENT_HDR + 3LL * (ao.l[mu] + 1) * (ao.l[nu] + 1) * (ao.l[mu] + ao.l[nu] + 2) / 2;
            for (auto &v : bybin) v.clear();
            for (int di = apoff[pr]; di < apoff[pr + 1]; di++)
                bybin[bvk_bin(alist[3 * di], alist[3 * di + 1], alist[3 * di + 2], L.nk)].push_back(di);
            for (int dt = 0; dt < Nk; dt++) {
                seg[(size_t)pr * Nk + dt] = (int)ent.size();
                for (int i = 0; i < ao.nprim[mu]; i++)
                    for (int j = 0; j < ao.nprim[nu]; j++)
                        for (int di : bybin[dt]) {
                            ent.push_back({tab_len, pr, di, i, j});
                            tab_len += esz;
                        }
            }
        }
        seg[(size_t)ao.nshell * ao.nshell * Nk] = (int)ent.size();
    }
    RC(S.upload(P.dent, ent));
    P.nent = (int)ent.size();
    RC(S.upload(P.dseg, seg));
    RC(S.upload(P.dalist, alist));
    RC(S.alloc(P.ptab, (size_t)std::max(tab_len, 1LL)));
    P.mixed_aft = (opts->precision == RSGDF_MIXED) && (mode & MODE_LR);
    if (P.mixed_aft) {
        std::vector<double> b9v(9);
        for (int i = 0; i < 3; i++)
            for (int x = 0; x < 3; x++) b9v[3 * i + x] = L.b[i][x];
        RC(S.upload(P.db9, b9v));
        RC(S.alloc(P.ptab32, (size_t)std::max(tab_len, 1LL)));
        RC(S.alloc(P.uph, 3 * ent.size() + 1));
        RC(S.alloc(P.ph0, ent.size() + 1));
    }
    P.g0fac = 3.141592653589793238462643383279502884 / (L.vol * omega * omega);
    P.g0 = (mode & MODE_SR) && groups.count(0);
    if (P.g0) {
        RC(S.alloc(P.SP, nP));
        RC(S.alloc(P.Sf, (size_t)Nk * nao * nao));
    }
    P.split_alpha = opts->split_alpha;
    if (P.split_alpha > 0.0) {
        auto diffuse = [&](const HBasis &b, int sh) {
            for (int i = 0; i < b.nprim[sh]; i++)
                if (b.exps[b.poff[sh] + i] > P.split_alpha) return (char)0;
            return (char)1;
        };
        P.ax_diffuse.resize(P.ax.nshell);
        P.ao_diffuse.resize(P.ao.nshell);
        for (int sh = 0; sh < P.ax.nshell; sh++) P.ax_diffuse[sh] = diffuse(P.ax, sh);
        for (int sh = 0; sh < P.ao.nshell; sh++) P.ao_diffuse[sh] = diffuse(P.ao, sh);
        if (P.g0) {
            std::vector<int> mx(nP, 0), ma(nao, 0);
            for (int sh = P.s0; sh < P.s1; sh++)
                for (int c = 0; c < ncart(P.ax.l[sh]); c++) mx[P.ax.foff[sh] - P.pfunc0 + c] = P.ax_diffuse[sh];
            for (int sh = 0; sh < P.ao.nshell; sh++)
                for (int c = 0; c < ncart(P.ao.l[sh]); c++) ma[P.ao.foff[sh] + c] = P.ao_diffuse[sh];
            RC(S.upload(P.dmask_ax, mx));
            RC(S.upload(P.dmask_ao, ma));
        }
    }
    // G-space data
    std::vector<int> gl;
    gbox(P.gm, gl);
    P.NG = (int)(gl.size() / 3);
    const int NG = P.NG;
    if (mode & MODE_LR) {
        RC(S.upload(P.dg, gl));
        RC(S.alloc(P.W, (size_t)2 * NG * nP));
        if (opts->precision == RSGDF_MIXED) {
            // split-TF32 operand tiles; the padding of B' stays zero for every k12
            RC(S.alloc(P.Apl, (size_t)tc_a_floats(nP, NG)));
            P.nbpl = tc_b_floats(nao * nao, NG, Nk);
            RC(S.alloc(P.Bpl, (size_t)P.nbpl));
        } else {
            RC(S.alloc(P.Y, (size_t)2 * Nk * NG * nao * nao));
        }
        P.garg.clear();
        for (int k12 : P.gkey) {
            GArgs Ga;
            memset(&Ga, 0, sizeof(Ga));
            Ga.g = P.dg;
            Ga.NG = NG;
            for (int i = 0; i < 3; i++)
                for (int x = 0; x < 3; x++) Ga.b[3 * i + x] = L.b[i][x];
            k12_frac(L, k12, Ga.f12);
            Ga.vol = L.vol;
            Ga.omega = omega;
            Ga.full_coulomb = opts->kernel == RSGDF_KERNEL_PLAIN;
            P.garg.push_back(Ga);
        }
    }
    // k12 groups in batches whose T fits a fixed budget (16 GiB of the device's HBM)
    const int G = (int)P.gkey.size();
    const long long tbytes = (long long)Nk * m * 16;
    P.B = (int)std::max(1LL, std::min<long long>(G, (16LL << 30) / std::max(tbytes, 1LL)));
    RC(S.alloc(P.T, (size_t)2 * P.B * Nk * m));
    // separable DFTs for the phase contractions: every k12 group present, all
    // in T at once, a mesh large enough to gain, and most k2 per group wanted
    P.npair = npair;
    P.dft = (G == Nk) && (P.B >= G) && (Nk >= 16) && ((long long)npair * 4 >= (long long)Nk * Nk) &&
            L.nk[0] <= DFT_NMAX_HOST && L.nk[1] <= DFT_NMAX_HOST && L.nk[2] <= DFT_NMAX_HOST;
    if (P.dft) {
        std::vector<double> tw((size_t)3 * DFT_NMAX_HOST * DFT_NMAX_HOST * 2, 0.0);
        for (int d = 0; d < 3; d++) {
            const int N = L.nk[d];
            for (int q = 0; q < N; q++)
                for (int n = 0; n < N; n++) {
                    const long double ang = 2.0L * 3.141592653589793238462643383279502884L * ((q * n) % N) / N;
                    const size_t o = 2 * ((size_t)d * DFT_NMAX_HOST * DFT_NMAX_HOST + q * N + n);
                    tw[o] = (double)cosl(ang);
                    tw[o + 1] = (double)sinl(ang);
                }
        }
        RC(S.upload(P.dtw, tw));
        std::vector<float> tw4(2 * tw.size());
        for (size_t e = 0; e < tw.size(); e++) {
            const float h = (float)tw[e];
            tw4[2 * e] = h;
            tw4[2 * e + 1] = (float)(tw[e] - (double)h);
        }
        RC(S.upload(P.dtw4, tw4));
        std::vector<int> a12(npair), a2(npair);
        for (int p = 0; p < npair; p++) {
            a12[p] = k12_of(L, kpairs[2 * p], kpairs[2 * p + 1]);
            a2[p] = kpairs[2 * p + 1];
        }
        RC(S.upload(P.dpk12, a12));
        RC(S.upload(P.dpk2all, a2));
        if (mode & MODE_SR) RC(S.alloc(P.Z, (size_t)2 * Nk * Nk * m));
    }
    P.aft_units = (mode & MODE_LR) ? (long long)ent.size() * NG * (long long)G : 0;
    P.lr_flops = (mode & MODE_LR) ? 8LL * nP * nao * nao * NG * Nk * (long long)G : 0;
    return RSGDF_OK;
}

// Before the SR class launches: zero X, pair tables, learned screen.
static int j3c_exec_pre(J3cProblem &P, cudaStream_t st, int &nl)
{
    if (!(P.mode & MODE_SR)) return RSGDF_OK;
    CU(cudaMemsetAsync(P.X, 0, sizeof(double) * P.nlt * P.Nk * P.m, st));
    return sr_pre(P.sr, st, nl);
}

// Pair tables of the AFT lists (also the overlaps of the G = 0 correction),
// the G = 0 pieces, and the zero padding of the split-TF32 B' tiles.
static int j3c_exec_tables(J3cProblem &P, cudaStream_t st, int &nl)
{
    t_timer.begin(PH_AFT);
    RC(launch_pair_prep(P.dao, P.ao.nshell, P.dent, P.nent, P.dalist, P.da9, P.ptab, P.ptab32, P.db9, P.uph, st));
    t_timer.end();
    nl++;
    if (P.g0) {
        t_timer.begin(PH_OTHER);
        k_aux_charge<<<(P.s1 - P.s0 + 63) / 64, 64, 0, st>>>(P.dax, P.s0, P.s1, P.pfunc0, P.SP);
        CU(cudaGetLastError());
        RC(launch_ovlp_fold(P.dao, P.ao.nshell, P.nao, P.dent, P.dseg, P.ptab, P.Nk, P.Sf, st));
        nl += 2;
        if (P.dmask_ax) {   // the G = 0 term belongs to the range-separated types only
            RC(launch_split_g0_mask(P.SP, P.nP, P.dmask_ax, P.Sf, P.Nk, P.nao, P.dmask_ao, st));
            nl++;
        }
        t_timer.end();
    }
    if (P.Bpl) CU(cudaMemsetAsync(P.Bpl, 0, sizeof(float) * P.nbpl, st));
    return RSGDF_OK;
}

// LR contraction of k12 group g (aux transforms, pair transforms, GEMM) added to Tj.
static int j3c_exec_lr_group(J3cProblem &P, int g, double *Tj, cudaStream_t st, int &nl)
{
    const int Nk = P.Nk, nao = P.nao, nP = P.nP, NG = P.NG;
    const long long m = P.m;
    const GArgs &Ga = P.garg[g];
    t_timer.begin(PH_AFT);
    RC(launch_aux_ft(Ga, P.dax, P.s0, P.s1, P.pfunc0, nP, P.W, nullptr, st));
    if (P.mixed_aft) {
        RC(launch_split_a(nP, NG, P.W, P.Apl, st));
        RC(launch_aft_f32(Ga, P.dao, P.ao.nshell, nao, P.dent, P.nent, P.dseg, P.ptab, P.ptab32, P.db9, P.uph, P.ph0,
                          Nk, P.Bpl, P.ao.l.empty() ? 0 : *std::max_element(P.ao.l.begin(), P.ao.l.end()), st));
    } else {
        RC(launch_aft(Ga, P.dao, P.ao.nshell, nao, P.dent, P.dseg, P.ptab, Nk, P.Y, st));
    }
    t_timer.end();
    t_timer.begin(PH_GEMM);
    if (P.mixed_aft)
        RC(launch_zgemm_tc2(nP, nao * nao, NG, Nk, P.Apl, P.Bpl, Tj, 2 * m, st));
    else
        RC(launch_zgemm_tn(nP, nao * nao, NG, Nk, P.W, P.Y, (long long)2 * NG * nao * nao, Tj, 2 * m, st));
    t_timer.end();
    nl += 3;
    if (P.mixed_aft && !P.ao.l.empty() && *std::max_element(P.ao.l.begin(), P.ao.l.end()) >= 3) nl++;   // f-shell pairs
    return RSGDF_OK;
}

// Phase 1 of a batch of k12 groups (written, or added when the LR part is
// already in T), with the G = 0 correction.
static int j3c_exec_phase1(J3cProblem &P, int gb0, int nb, int accumulate, cudaStream_t st, int &nl)
{
    const int Nk = P.Nk;
    const long long m = P.m;
    t_timer.begin(PH_PHASE);
    if (P.dft) {
        // T[k12][dt] (+)= sum_lt e^{-i k12.lt} X[lt][dt]: DFT over the lt mesh axes (FP64)
        double *Zb = accumulate ? P.Z : P.T;
        const long long n = (long long)Nk * Nk * m;
        if (P.fp32) {   // double-float passes on the FP32 pipes
            RC(launch_real_to_df(P.X, Zb, n, st));
            RC(launch_dft_mesh_df(Zb, P.L.nk, (long long)Nk * m, 1, P.dtw4, 1, st));
            if (accumulate)
                RC(launch_add_df(P.T, P.Z, n, st));
            else
                RC(launch_convert_df(P.T, n, 0, st));
        } else {
            RC(launch_real_to_complex(P.X, Zb, n, st));
            RC(launch_dft_mesh(Zb, P.L.nk, (long long)Nk * m, 1, P.dtw, 1, st));
            if (accumulate) RC(launch_add_complex(P.T, P.Z, n, st));
        }
        nl += 5;
    } else {
        RC(launch_phase1_multi(P.X, m, Nk, P.nlt, P.dk12 + gb0, nb, P.phk, P.T, P.fp32, accumulate, st));
        nl++;
    }
    for (int j = 0; j < nb; j++)
        if (P.gkey[gb0 + j] == 0) {
            RC(launch_g0_fold(P.T + (size_t)2 * j * Nk * m, m, Nk, P.nP, P.nao, P.SP, P.Sf, P.g0fac, st));
            nl++;
        }
    t_timer.end();
    return RSGDF_OK;
}

static int j3c_exec_x_to_df(J3cProblem &P, cudaStream_t st, int &nl)
{
    if (P.fp32 && (P.mode & MODE_SR) && !P.dft) {
        t_timer.begin(PH_PHASE);
        RC(launch_x_to_df(P.X, (long long)P.nlt * P.Nk * P.m, st));   // X to double-float pairs, in place
        t_timer.end();
        nl++;
    }
    return RSGDF_OK;
}

// Phase 2 of a batch of k12 groups into V.
static int j3c_exec_phase2(J3cProblem &P, int gb0, int nb, double *V, cudaStream_t st, int &nl)
{
    const int acc = (P.mode == MODE_LR) ? 1 : 0;
    t_timer.begin(PH_PHASE);
    if (P.dft) {
        // V[pair] (+)= sum_dt e^{+i k2.dt} T[k12][dt]: DFT over the dt mesh axes, then the pairs
        if (P.fp32) {
            RC(launch_convert_df(P.T, (long long)P.Nk * P.Nk * P.m, 1, st));
            RC(launch_dft_mesh_df(P.T, P.L.nk, P.m, P.Nk, P.dtw4, 0, st));
            RC(launch_scatter_pairs_df(P.T, P.m, P.Nk, P.npair, P.dpk12, P.dpk2all, V, acc, st));
        } else {
            RC(launch_dft_mesh(P.T, P.L.nk, P.m, P.Nk, P.dtw, 0, st));
            RC(launch_scatter_pairs(P.T, P.m, P.Nk, P.npair, P.dpk12, P.dpk2all, V, acc, st));
        }
        nl += 5;
    } else {
        RC(launch_phase2_multi(P.T, P.m, P.Nk, P.dgoff + gb0, nb, P.dplist, P.dpk2, P.phk, V, acc, P.fp32, st));
        nl++;
    }
    t_timer.end();
    return RSGDF_OK;
}

// After the SR class launches: G = 0 pieces, phases, AFT, LR contraction.
static int j3c_exec_post(J3cProblem &P, double *V, cudaStream_t st, int &nl)
{
    const int Nk = P.Nk;
    const long long m = P.m;
    RC(j3c_exec_tables(P, st, nl));
    RC(j3c_exec_x_to_df(P, st, nl));
    const int G = (int)P.gkey.size();
    for (int gb0 = 0; gb0 < G; gb0 += P.B) {
        const int nb = std::min(P.B, G - gb0);
        if (P.mode & MODE_SR)
            RC(j3c_exec_phase1(P, gb0, nb, 0, st, nl));
        else
            CU(cudaMemsetAsync(P.T, 0, sizeof(double) * 2 * nb * Nk * m, st));
        if (P.mode & MODE_LR)
            for (int j = 0; j < nb; j++) RC(j3c_exec_lr_group(P, gb0 + j, P.T + (size_t)2 * j * Nk * m, st, nl));
        RC(j3c_exec_phase2(P, gb0, nb, V, st, nl));
    }
    CU(cudaGetLastError());
    return RSGDF_OK;
}

// LR-first order (every k12 group fits T at once): the LR contractions go
// into T before the SR plan exists, so the host screening runs while the
// device computes them; j3c_exec_post_lr_done finishes after the SR launches.
static int j3c_exec_lr_first(J3cProblem &P, cudaStream_t st, int &nl)
{
    const int G = (int)P.gkey.size();
    RC(j3c_exec_tables(P, st, nl));
    CU(cudaMemsetAsync(P.T, 0, sizeof(double) * 2 * (size_t)G * P.Nk * P.m, st));
    for (int g = 0; g < G; g++) RC(j3c_exec_lr_group(P, g, P.T + (size_t)2 * g * P.Nk * P.m, st, nl));
    return RSGDF_OK;
}

static int j3c_exec_post_lr_done(J3cProblem &P, double *V, cudaStream_t st, int &nl)
{
    const int G = (int)P.gkey.size();
    RC(j3c_exec_x_to_df(P, st, nl));
    RC(j3c_exec_phase1(P, 0, G, 1, st, nl));
    RC(j3c_exec_phase2(P, 0, G, V, st, nl));
    CU(cudaGetLastError());
    return RSGDF_OK;
}

static int stats_counts(unsigned long long *dcnt, cudaStream_t st)
{
    if (!t_count_host) CU(cudaMallocHost(&t_count_host, sizeof(unsigned long long) * (2 * LTOT_MAX + 6)));
    CU(cudaMemcpyAsync(t_count_host, dcnt, sizeof(unsigned long long) * (2 * LTOT_MAX + 6), cudaMemcpyDeviceToHost, st));
    t_count_valid = true;
    t_stats_stream = st;
    return RSGDF_OK;
}

static int j3c_impl(const rsgdf_cell *cell, const rsgdf_basis *ao_in, const rsgdf_basis *aux_in,
                    const rsgdf_opts *opts, int npair, const int *kpairs, int s0, int s1, double *V, int mode)
{
    t_err.clear();
    memset(&t_stats, 0, sizeof(t_stats));
    t_count_valid = false;
    J3cProblem P;
    RC(j3c_check(P, cell, ao_in, aux_in, opts, npair, kpairs, s0, s1));
    if (!V) return fail(RSGDF_EINVAL, "V_out is NULL");
    if (opts->kernel == RSGDF_KERNEL_PLAIN && mode != MODE_LR)
        return fail(RSGDF_EINVAL, "the plain kernel is for rsgdf_j3c_lr only");
    RC(check_device());
    // the host screening of the SR sums runs beside the LR preparation and the
    // LR device work (declared after P: an early return waits for it first)
    std::future<void> sr_plan;
    if (mode & MODE_SR) sr_plan = std::async(std::launch::async, [&P, opts] { j3c_plan_sr(P, opts); });
    cudaStream_t st = (cudaStream_t)opts->stream;
    RC(ensure_boys(st));
    t_timer.reset(st);
    Scratch S(st);
    unsigned long long *dcnt, *dq;
    RC(S.alloc(dcnt, 2 * LTOT_MAX + 6));
    RC(S.alloc(dq, LTOT_MAX + 1));
    RC(j3c_prepare(P, S, opts, npair, kpairs, mode, dcnt, false));
    int nl = 0;
    CU(cudaMemsetAsync(dcnt, 0, sizeof(unsigned long long) * (2 * LTOT_MAX + 6), st));
    const bool lr_first = (mode == (MODE_SR | MODE_LR)) && P.B >= (int)P.gkey.size();
    if (lr_first) RC(j3c_exec_lr_first(P, st, nl));   // device busy while the host plans the SR sums
    if (mode & MODE_SR) {
        sr_plan.get();
        RC(j3c_prepare_sr(P, S, opts, dcnt, true));
    }
    std::vector<SRClassLaunch> cl;
    if (mode & MODE_SR) RC(sr_merge({&P.sr}, S, st, cl));
    RC(j3c_exec_pre(P, st, nl));
    RC(sr_run(cl, dq, st, nl));
    if (lr_first)
        RC(j3c_exec_post_lr_done(P, V, st, nl));
    else
        RC(j3c_exec_post(P, V, st, nl));
    RC(stats_counts(dcnt, st));
    t_stats.sr_items = P.plan.n_items;
    t_stats.omega = P.omega;
    for (int i = 0; i < 3; i++) t_stats.gmesh[i] = P.gm[i];
    t_stats.aft_units = P.aft_units;
    t_stats.lr_flops = P.lr_flops;
    t_stats.n_launch = nl;
    return RSGDF_OK;
}

// ---------------------------------------------------------------------------
// k-phase contraction pieces shared by rsgdf_kphase and rsgdf_kphase_noalloc:
// argument checks, the grouping of the k pairs by k12, and the launches.
// ---------------------------------------------------------------------------
static int kphase_check(const rsgdf_cell *cell, const double *X, long long m, int npair, const int *kpairs,
                        const double *V_out, Lattice &L)
{
    RC(make_lattice(cell, L, t_err));
    if (!X || !V_out || m < 1) return fail(RSGDF_EINVAL, "X, V_out and m >= 1 are required");
    if (npair < 1 || !kpairs) return fail(RSGDF_EINVAL, "need at least one k pair");
    for (int i = 0; i < 2 * npair; i++)
        if (kpairs[i] < 0 || kpairs[i] >= L.Nk) return fail(RSGDF_EINVAL, "k index outside the mesh");
    return RSGDF_OK;
}

struct KphaseGroups {
    std::vector<int> plist, pk2, goff, gkey;   // pairs grouped by k12; group gi = plist[goff[gi], goff[gi+1])
};

static void kphase_groups(const Lattice &L, int npair, const int *kpairs, KphaseGroups &g)
{
    std::map<int, std::vector<int>> groups;
    for (int p = 0; p < npair; p++) groups[k12_of(L, kpairs[2 * p], kpairs[2 * p + 1])].push_back(p);
    for (auto &kv : groups) {
        g.goff.push_back((int)g.plist.size());
        g.gkey.push_back(kv.first);
        for (int p : kv.second) {
            g.plist.push_back(p);
            g.pk2.push_back(kpairs[2 * p + 1]);
        }
    }
    g.goff.push_back((int)g.plist.size());
}

static int kphase_launch(const double *X, long long m, int Nk, const KphaseGroups &g, const double *dph,
                         const int *dplist, const int *dpk2, double *T, double *V_out, cudaStream_t st)
{
    for (size_t gi = 0; gi < g.gkey.size(); gi++) {
        RC(launch_phase1(X, m, Nk, Nk, g.gkey[gi], dph, T, 0, st));
        RC(launch_phase2(T, m, Nk, dplist + g.goff[gi], dpk2 + g.goff[gi], g.goff[gi + 1] - g.goff[gi], dph, V_out,
                         0, st));
    }
    CU(cudaGetLastError());
    return RSGDF_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free k-phase contraction.  Its scratch is one file-scope device
// array; the host-side name of that array is only a stand-in, so the device
// address is looked up once per device with cudaGetSymbolAddress.
// ---------------------------------------------------------------------------
constexpr size_t NOALLOC_BYTES = (size_t)64 << 20;   // RSGDF_NOALLOC_SCRATCH_BYTES
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];
static void *g_noalloc_addr[64] = {nullptr};
static std::mutex g_noalloc_mu;

static int noalloc_scratch(void *&base)
{
    int dev = 0;
    CU(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(RSGDF_EDEVICE, "device index beyond 63");
    std::lock_guard<std::mutex> g(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void *p = nullptr;
        CU(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        g_noalloc_addr[dev] = p;
    }
    base = g_noalloc_addr[dev];
    return RSGDF_OK;
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

static int kphase_noalloc_impl(const rsgdf_cell *cell, const double *X, long long m, int npair, const int *kpairs,
                               double *V_out, void *stream)
{
    t_err.clear();
    Lattice L;
    RC(kphase_check(cell, X, m, npair, kpairs, V_out, L));
    const int Nk = L.Nk;
    const size_t b_ph = align256(sizeof(double) * 2 * (size_t)Nk * Nk);
    const size_t b_pl = align256(sizeof(int) * (size_t)npair);
    const size_t b_T = sizeof(double) * 2 * (size_t)Nk * (size_t)m;
    const size_t need = b_ph + 2 * b_pl + b_T;
    if (need > NOALLOC_BYTES)
        return fail(RSGDF_EINVAL, "kphase_noalloc needs " + std::to_string(need) + " bytes of scratch, more than the " +
                                      std::to_string(NOALLOC_BYTES) + "-byte static array: split m or the k pairs");
    RC(check_device());
    void *base = nullptr;
    RC(noalloc_scratch(base));
    cudaStream_t st = (cudaStream_t)stream;
    unsigned char *b = (unsigned char *)base;
    double *dph = (double *)b;
    int *dplist = (int *)(b + b_ph);
    int *dpk2 = (int *)(b + b_ph + b_pl);
    double *T = (double *)(b + b_ph + 2 * b_pl);
    std::vector<double> ph;
    phase_table(L, ph);
    KphaseGroups g;
    kphase_groups(L, npair, kpairs, g);
    // pageable sources: each copy has consumed its host buffer when it returns
    CU(cudaMemcpyAsync(dph, ph.data(), sizeof(double) * ph.size(), cudaMemcpyHostToDevice, st));
    CU(cudaMemcpyAsync(dplist, g.plist.data(), sizeof(int) * g.plist.size(), cudaMemcpyHostToDevice, st));
    CU(cudaMemcpyAsync(dpk2, g.pk2.data(), sizeof(int) * g.pk2.size(), cudaMemcpyHostToDevice, st));
    return kphase_launch(X, m, Nk, g, dph, dplist, dpk2, T, V_out, st);
}

}  // namespace rsgdf

struct rsgdf_batch {
    int nprob = 0;
    int flags = 0;
    cudaStream_t st0 = nullptr;   // stream of the allocations
    std::unique_ptr<rsgdf::Scratch> S;
    std::vector<std::unique_ptr<rsgdf::J3cProblem>> probs;
    std::vector<rsgdf::SRClassLaunch> cl;
    unsigned long long *dcnt = nullptr, *dq = nullptr;
    bool tuned = false;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<double *> graph_V;
    int graph_nl = 0;
    cudaStream_t own = nullptr;   // capture stream when the caller passes the legacy stream
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    long long n_items = 0, aft_units = 0, lr_flops = 0;
};

namespace rsgdf {

static int batch_exec(rsgdf_batch *b, double *const *V, cudaStream_t st, int &nl)
{
    CU(cudaMemsetAsync(b->dcnt, 0, sizeof(unsigned long long) * (2 * LTOT_MAX + 6), st));
    for (auto &P : b->probs) RC(j3c_exec_pre(*P, st, nl));
    RC(sr_run(b->cl, b->dq, st, nl));
    for (int p = 0; p < b->nprob; p++) RC(j3c_exec_post(*b->probs[p], V[p], st, nl));
    return RSGDF_OK;
}

static void batch_drop_graph(rsgdf_batch *b)
{
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
    b->graph_V.clear();
}

}  // namespace rsgdf

using namespace rsgdf;

extern "C" {

int rsgdf_j3c_batch_create(int nprob, const rsgdf_problem *probs, const rsgdf_opts *opts, const int *npair,
                           const int *kpairs, int flags, rsgdf_batch **out)
{
    t_err.clear();
    if (!out || nprob < 1 || !probs || !npair || !kpairs) return fail(RSGDF_EINVAL, "bad batch argument");
    if (flags & ~(RSGDF_BATCH_GRAPH | RSGDF_BATCH_AUTOTUNE)) return fail(RSGDF_EINVAL, "unknown batch flag");
    *out = nullptr;
    RC(check_opts(opts));
    if (opts->split_alpha > 0.0 || opts->kernel != RSGDF_KERNEL_ERF)
        return fail(RSGDF_ENOTIMPL, "the batch runs the plain range-separated path only");
    std::unique_ptr<rsgdf_batch> b(new rsgdf_batch());
    b->nprob = nprob;
    b->flags = flags;
    long long koff = 0;
    for (int p = 0; p < nprob; p++) {
        if (!probs[p].cell || !probs[p].ao || !probs[p].aux) return fail(RSGDF_EINVAL, "NULL member in probs");
        if (npair[p] < 1) return fail(RSGDF_EINVAL, "every cell needs at least one k pair");
        std::unique_ptr<J3cProblem> P(new J3cProblem());
        const int r = j3c_check(*P, probs[p].cell, probs[p].ao, probs[p].aux, opts, npair[p], kpairs + 2 * koff, 0,
                                probs[p].aux->nshell);
        if (r != RSGDF_OK) {
            t_err = "cell " + std::to_string(p) + ": " + t_err;
            return r;
        }
        koff += npair[p];
        b->probs.push_back(std::move(P));
    }
    RC(check_device());
    cudaStream_t st = (cudaStream_t)opts->stream;
    RC(ensure_boys(st));
    b->st0 = st;
    b->S.reset(new Scratch(st));
    RC(b->S->alloc(b->dcnt, 2 * LTOT_MAX + 6));
    RC(b->S->alloc(b->dq, LTOT_MAX + 1));
    koff = 0;
    std::vector<const SRSetup *> rs;
    for (int p = 0; p < nprob; p++) {
        J3cProblem &P = *b->probs[p];
        const int r = j3c_prepare(P, *b->S, opts, npair[p], kpairs + 2 * koff, MODE_SR | MODE_LR, b->dcnt);
        if (r != RSGDF_OK) {
            t_err = "cell " + std::to_string(p) + ": " + t_err;
            return r;
        }
        koff += npair[p];
        b->n_items += P.plan.n_items;
        b->aft_units += P.aft_units;
        b->lr_flops += P.lr_flops;
    }
    for (auto &P : b->probs) rs.push_back(&P->sr);
    RC(sr_merge(rs, *b->S, st, b->cl));
    CU(cudaStreamSynchronize(st));
    *out = b.release();
    return RSGDF_OK;
}

int rsgdf_j3c_batch_run(rsgdf_batch *b, double *const *V_out, void *stream)
{
    t_err.clear();
    memset(&t_stats, 0, sizeof(t_stats));
    t_count_valid = false;
    if (!b || !V_out) return fail(RSGDF_EINVAL, "bad batch argument");
    for (int p = 0; p < b->nprob; p++)
        if (!V_out[p]) return fail(RSGDF_EINVAL, "V_out has a NULL entry");
    cudaStream_t st = (cudaStream_t)stream;
    int nl = 0;
    if ((b->flags & RSGDF_BATCH_AUTOTUNE) && !b->tuned) {
        t_timer.reset(st);
        t_timer.on = false;
        for (auto &P : b->probs) RC(j3c_exec_pre(*P, st, nl));
        RC(sr_tune(b->cl, b->dq, st, nullptr));
        b->tuned = true;
        batch_drop_graph(b);
        nl = 0;
    }
    if (b->flags & RSGDF_BATCH_GRAPH) {
        cudaStream_t cs = st;
        if (st == nullptr) {
            if (!b->own) {
                CU(cudaStreamCreateWithFlags(&b->own, cudaStreamNonBlocking));
                CU(cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming));
                CU(cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming));
            }
            cs = b->own;
        }
        bool same = b->exec && (int)b->graph_V.size() == b->nprob;
        for (int p = 0; same && p < b->nprob; p++) same = (b->graph_V[p] == V_out[p]);
        if (!same) {
            batch_drop_graph(b);
            t_timer.reset(cs);
            t_timer.on = false;
            CU(cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed));
            int r = batch_exec(b, V_out, cs, nl);
            cudaGraph_t g = nullptr;
            cudaError_t e = cudaStreamEndCapture(cs, &g);
            if (r != RSGDF_OK) {
                if (g) cudaGraphDestroy(g);
                return r;
            }
            if (e != cudaSuccess) return fail(RSGDF_EDEVICE, std::string("graph capture: ") + cudaGetErrorString(e));
            b->graph = g;
            CU(cudaGraphInstantiate(&b->exec, b->graph, 0));
            b->graph_V.assign(V_out, V_out + b->nprob);
            b->graph_nl = nl;
        }
        if (cs != st) {
            CU(cudaEventRecord(b->ev_in, st));
            CU(cudaStreamWaitEvent(cs, b->ev_in, 0));
        }
        CU(cudaGraphLaunch(b->exec, cs));
        if (cs != st) {
            CU(cudaEventRecord(b->ev_out, cs));
            CU(cudaStreamWaitEvent(st, b->ev_out, 0));
        }
        nl = b->graph_nl;
    } else {
        t_timer.reset(st);
        RC(batch_exec(b, V_out, st, nl));
    }
    RC(stats_counts(b->dcnt, st));
    t_stats.sr_items = b->n_items;
    t_stats.aft_units = b->aft_units;
    t_stats.lr_flops = b->lr_flops;
    t_stats.n_launch = nl;
    return RSGDF_OK;
}

int rsgdf_j3c_batch_tiles(const rsgdf_batch *b, int *grid, int *bc, int *grab)
{
    t_err.clear();
    if (!b) return fail(RSGDF_EINVAL, "NULL batch");
    for (int L = 0; L <= LTOT_MAX; L++) {
        if (grid) grid[L] = 0;
        if (bc) bc[L] = 0;
        if (grab) grab[L] = 0;
    }
    for (const SRClassLaunch &c : b->cl) {
        if (grid) grid[c.L] = c.grid;
        if (bc) bc[c.L] = c.bc;
        if (grab) grab[c.L] = c.grab;
    }
    return RSGDF_OK;
}

int rsgdf_j3c_batch_destroy(rsgdf_batch *b)
{
    if (!b) return RSGDF_OK;
    cudaDeviceSynchronize();   // runs may be on any stream; the frees below are ordered on the allocation stream
    batch_drop_graph(b);
    if (b->own) {
        cudaStreamSynchronize(b->own);
        cudaStreamDestroy(b->own);
    }
    if (b->ev_in) cudaEventDestroy(b->ev_in);
    if (b->ev_out) cudaEventDestroy(b->ev_out);
    b->S.reset();   // stream-ordered frees on the allocation stream
    delete b;
    return RSGDF_OK;
}

int rsgdf_j3c_batch(int nprob, const rsgdf_problem *probs, const rsgdf_opts *opts, const int *npair,
                    const int *kpairs, double *const *V_out)
{
    rsgdf_batch *b = nullptr;
    RC(rsgdf_j3c_batch_create(nprob, probs, opts, npair, kpairs, 0, &b));
    const int r = rsgdf_j3c_batch_run(b, V_out, opts->stream);
    rsgdf_j3c_batch_destroy(b);
    return r;
}

int rsgdf_j3c_sr(const rsgdf_cell *cell, const rsgdf_basis *ao, const rsgdf_basis *aux, const rsgdf_opts *opts,
                 int npair, const int *kpairs, int s0, int s1, double *V_out)
{
    return j3c_impl(cell, ao, aux, opts, npair, kpairs, s0, s1, V_out, MODE_SR);
}

int rsgdf_j3c_lr(const rsgdf_cell *cell, const rsgdf_basis *ao, const rsgdf_basis *aux, const rsgdf_opts *opts,
                 int npair, const int *kpairs, int s0, int s1, double *V_out)
{
    return j3c_impl(cell, ao, aux, opts, npair, kpairs, s0, s1, V_out, MODE_LR);
}

int rsgdf_j3c(const rsgdf_cell *cell, const rsgdf_basis *ao, const rsgdf_basis *aux, const rsgdf_opts *opts,
              int npair, const int *kpairs, int s0, int s1, double *V_out)
{
    return j3c_impl(cell, ao, aux, opts, npair, kpairs, s0, s1, V_out, MODE_SR | MODE_LR);
}

int rsgdf_j2c(const rsgdf_cell *cell, const rsgdf_basis *aux_in, const rsgdf_opts *opts, int nk, const int *kidx,
              double *J_out, double *L_out, int *info_out)
{
    t_err.clear();
    memset(&t_stats, 0, sizeof(t_stats));
    t_count_valid = false;
    RC(check_opts(opts));
    Lattice L;
    HBasis ax, axu;
    RC(make_lattice(cell, L, t_err));
    RC(load_basis(aux_in, ax, t_err));
    if (nk < 1 || !kidx) return fail(RSGDF_EINVAL, "need at least one k");
    for (int i = 0; i < nk; i++)
        if (kidx[i] < 0 || kidx[i] >= L.Nk) return fail(RSGDF_EINVAL, "k index outside the mesh");
    if (!J_out) return fail(RSGDF_EINVAL, "J_out is NULL");
    double omega;
    int gm[3];
    RC(derive_params(L, opts, omega, gm, t_err));
    RC(check_device());
    cudaStream_t st = (cudaStream_t)opts->stream;
    RC(ensure_boys(st));
    t_timer.reset(st);
    Scratch S(st);
    unit_partner_basis(ax, axu);
    const int naux = ax.nfunc, Nk = L.Nk;
    int nlaunch = 0;
    DevShells dax, daxu;
    RC(upload_shells(S, ax, dax));
    RC(upload_shells(S, axu, daxu));
    std::vector<double> ph;
    phase_table(L, ph);
    double *dph;
    RC(S.upload(dph, ph));
    unsigned long long *dcnt;
    RC(S.alloc(dcnt, 2 * LTOT_MAX + 6));
    CU(cudaMemsetAsync(dcnt, 0, sizeof(unsigned long long) * (2 * LTOT_MAX + 6), st));
    // SR: X2[lt][P][Q] = sum_{l -> lt} (chi_P^l | erfc | chi_Q^0), the
    // three-center kernel with the unit function as the second pair member
    SRPlan plan;
    plan_sr2c(L, ax, axu, omega, opts->eps_screen, plan);
    const long long m = (long long)naux * naux;
    double *X2;
    RC(S.alloc(X2, (size_t)Nk * m));
    CU(cudaMemsetAsync(X2, 0, sizeof(double) * Nk * m, st));
    RC(run_sr(S, L, plan, daxu, dax, axu, ax, omega, X2, m, 0, naux, 1, 0, 0, dcnt, st, nlaunch));
    double *SP;
    RC(S.alloc(SP, naux));
    k_aux_charge<<<(ax.nshell + 63) / 64, 64, 0, st>>>(dax, 0, ax.nshell, 0, SP);
    CU(cudaGetLastError());
    nlaunch++;
    std::vector<int> gl;
    gbox(gm, gl);
    const int NG = (int)(gl.size() / 3);
    int *dg;
    double *W, *F;
    RC(S.upload(dg, gl));
    // weights and transforms of every requested k, contracted by one batched GEMM
    const long long wsz = (long long)2 * NG * naux;
    RC(S.alloc(W, (size_t)wsz * nk));
    RC(S.alloc(F, (size_t)wsz * nk));
    const double g0fac = 3.141592653589793238462643383279502884 / (L.vol * omega * omega);
    // J^k = sum_lt e^{-i k.lt} X2[lt] - [k = 0] fac S_P S_Q + W^T F
    for (int i = 0; i < nk; i++) {
        const int k = kidx[i];
        double *Jk = J_out + (size_t)2 * i * m;
        t_timer.begin(PH_PHASE);
        RC(launch_phase1(X2, m, Nk, 1, k, dph, Jk, 0, st));
        nlaunch++;
        if (k == 0) {
            RC(launch_g0_outer(Jk, naux, SP, g0fac, st));
            nlaunch++;
        }
        t_timer.end();
        GArgs G;
        memset(&G, 0, sizeof(G));
        G.g = dg;
        G.NG = NG;
        for (int a = 0; a < 3; a++)
            for (int x = 0; x < 3; x++) G.b[3 * a + x] = L.b[a][x];
        k12_frac(L, k, G.f12);
        G.vol = L.vol;
        G.omega = omega;
        t_timer.begin(PH_AFT);
        RC(launch_aux_ft(G, dax, 0, ax.nshell, 0, naux, W + i * wsz, F + i * wsz, st));
        t_timer.end();
        nlaunch++;
    }
    t_timer.begin(PH_GEMM);
    RC(launch_zgemm_tn(naux, naux, NG, nk, W, F, wsz, J_out, 2 * m, st, wsz));
    t_timer.end();
    nlaunch++;
    if (L_out) {
        t_timer.begin(PH_OTHER);
        RC(launch_cholesky(naux, nk, J_out, L_out, info_out, st));
        t_timer.end();
        nlaunch++;
    } else if (info_out) {
        CU(cudaMemsetAsync(info_out, 0xff, sizeof(int) * nk, st));
    }
    CU(cudaGetLastError());
    if (!t_count_host) CU(cudaMallocHost(&t_count_host, sizeof(unsigned long long) * (2 * LTOT_MAX + 6)));
    CU(cudaMemcpyAsync(t_count_host, dcnt, sizeof(unsigned long long) * (2 * LTOT_MAX + 6), cudaMemcpyDeviceToHost, st));
    t_count_valid = true;
    t_stats_stream = st;
    t_stats.omega = omega;
    for (int i = 0; i < 3; i++) t_stats.gmesh[i] = gm[i];
    t_stats.lr_flops = 8LL * naux * naux * NG * nk;
    t_stats.n_launch = nlaunch;
    return RSGDF_OK;
}

int rsgdf_kphase(const rsgdf_cell *cell, const double *X, long long m, int npair, const int *kpairs, double *V_out,
                 void *stream)
{
    t_err.clear();
    Lattice L;
    RC(kphase_check(cell, X, m, npair, kpairs, V_out, L));
    RC(check_device());
    cudaStream_t st = (cudaStream_t)stream;
    Scratch S(st);
    const int Nk = L.Nk;
    std::vector<double> ph;
    phase_table(L, ph);
    double *dph;
    RC(S.upload(dph, ph));
    KphaseGroups g;
    kphase_groups(L, npair, kpairs, g);
    int *dplist, *dpk2;
    RC(S.upload(dplist, g.plist));
    RC(S.upload(dpk2, g.pk2));
    double *T;
    RC(S.alloc(T, (size_t)2 * Nk * m));
    return kphase_launch(X, m, Nk, g, dph, dplist, dpk2, T, V_out, st);
}

int rsgdf_kphase_noalloc(const rsgdf_cell *cell, const double *X, long long m, int npair, const int *kpairs,
                         double *V_out, void *stream)
{
    return kphase_noalloc_impl(cell, X, m, npair, kpairs, V_out, stream);
}


int rsgdf_mlp_nparams(int nfeat) { return nfeat > 0 ? mlp_param_count(nfeat) : 0; }

int rsgdf_mlp_create(int nfeat, const float *params, const float *mean, const float *stdv, rsgdf_mlp **out)
{
    t_err.clear();
    if (!out || !params || !mean || !stdv) return fail(RSGDF_EINVAL, "NULL argument");
    if (nfeat < 1 || nfeat > SR_NFEAT_MAX) return fail(RSGDF_EINVAL, "nfeat outside 1..16");
    for (int f = 0; f < nfeat; f++)
        if (!(stdv[f] > 0.0f)) return fail(RSGDF_EINVAL, "stdv must be positive");
    RC(check_device());
    rsgdf_mlp *m = new rsgdf_mlp();
    m->F = nfeat;
    m->np = mlp_param_count(nfeat);
    m->margin = 0.0f;
    m->base = -1;
    m->base_lo = m->base_hi = 0.0f;
    for (int L = 0; L <= LTOT_MAX; L++) m->guard[L] = 0.0f;
    m->step = 0;
    cudaGetDevice(&m->dev);
    const size_t fb = sizeof(float) * m->np;
    bool ok = cudaMalloc(&m->P, fb) == cudaSuccess && cudaMalloc(&m->G, fb) == cudaSuccess &&
              cudaMalloc(&m->m, fb) == cudaSuccess && cudaMalloc(&m->v, fb) == cudaSuccess &&
              cudaMalloc(&m->P16, sizeof(__half) * m->np) == cudaSuccess &&
              cudaMalloc(&m->mean, sizeof(float) * nfeat) == cudaSuccess &&
              cudaMalloc(&m->stdv, sizeof(float) * nfeat) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        rsgdf_mlp_destroy(m);
        return fail(RSGDF_ENOMEM, "network allocation failed");
    }
    cudaMemcpy(m->P, params, fb, cudaMemcpyHostToDevice);
    cudaMemset(m->G, 0, fb);
    cudaMemset(m->m, 0, fb);
    cudaMemset(m->v, 0, fb);
    cudaMemcpy(m->mean, mean, sizeof(float) * nfeat, cudaMemcpyHostToDevice);
    cudaMemcpy(m->stdv, stdv, sizeof(float) * nfeat, cudaMemcpyHostToDevice);
    if (launch_to_half(m->np, m->P, m->P16, 0) != RSGDF_OK || cudaDeviceSynchronize() != cudaSuccess) {
        rsgdf_mlp_destroy(m);
        return fail(RSGDF_EDEVICE, "network upload failed");
    }
    *out = m;
    return RSGDF_OK;
}

int rsgdf_mlp_destroy(rsgdf_mlp *m)
{
    if (!m) return RSGDF_OK;
    cudaFree(m->P);
    cudaFree(m->G);
    cudaFree(m->m);
    cudaFree(m->v);
    cudaFree(m->P16);
    cudaFree(m->mean);
    cudaFree(m->stdv);
    delete m;
    return RSGDF_OK;
}

int rsgdf_mlp_get_params(const rsgdf_mlp *m, float *params_out)
{
    t_err.clear();
    if (!m || !params_out) return fail(RSGDF_EINVAL, "NULL argument");
    CU(cudaMemcpy(params_out, m->P, sizeof(float) * m->np, cudaMemcpyDeviceToHost));
    return RSGDF_OK;
}

int rsgdf_mlp_set_margin(rsgdf_mlp *m, float margin)
{
    t_err.clear();
    if (!m || !(margin >= 0.0f)) return fail(RSGDF_EINVAL, "margin must be >= 0");
    m->margin = margin;
    return RSGDF_OK;
}

int rsgdf_mlp_set_base(rsgdf_mlp *m, int feature, float lo, float hi, const float *guard)
{
    t_err.clear();
    if (!m || feature < -1 || feature >= m->F || !(lo <= hi)) return fail(RSGDF_EINVAL, "bad base feature or clamp");
    if (feature >= 0 && m->F < 3) return fail(RSGDF_EINVAL, "the guard needs the l features 0..2");
    for (int L = 0; L <= LTOT_MAX; L++)
        if (guard && guard[L] != guard[L]) return fail(RSGDF_EINVAL, "NaN guard");
    m->base = feature;
    m->base_lo = lo;
    m->base_hi = hi;
    for (int L = 0; L <= LTOT_MAX; L++) m->guard[L] = guard ? guard[L] : 0.0f;
    return RSGDF_OK;
}

int rsgdf_mlp_forward(const rsgdf_mlp *m, const float *X, long long n, float *y, void *stream)
{
    t_err.clear();
    if (!m || !X || !y || n < 0) return fail(RSGDF_EINVAL, "bad argument");
    RC(launch_mlp_forward(m->F, m->P16, m->mean, m->stdv, X, n, y, (cudaStream_t)stream));
    return RSGDF_OK;
}

int rsgdf_mlp_loss_grad(rsgdf_mlp *m, const float *X, const float *t, long long n, float tau, float *loss_out,
                        float *grad_out, void *stream)
{
    t_err.clear();
    if (!m || !X || !t || n < 1 || !loss_out || !(tau > 0.0f && tau < 1.0f)) return fail(RSGDF_EINVAL, "bad argument");
    cudaStream_t st = (cudaStream_t)stream;
    Scratch S(st);
    float *dl;
    RC(S.alloc(dl, 1));
    CU(cudaMemsetAsync(dl, 0, sizeof(float), st));
    CU(cudaMemsetAsync(m->G, 0, sizeof(float) * m->np, st));
    RC(launch_mlp_fwd_bwd(m->F, m->P16, m->mean, m->stdv, X, t, nullptr, n, 1.0f / (float)n, tau, m->G, dl, st));
    CU(cudaMemcpyAsync(loss_out, dl, sizeof(float), cudaMemcpyDeviceToHost, st));
    if (grad_out) CU(cudaMemcpyAsync(grad_out, m->G, sizeof(float) * m->np, cudaMemcpyDeviceToHost, st));
    CU(cudaMemsetAsync(m->G, 0, sizeof(float) * m->np, st));
    CU(cudaStreamSynchronize(st));
    return RSGDF_OK;
}

int rsgdf_mlp_train(rsgdf_mlp *m, const float *X, const float *t, long long n, int epochs, int batch, float lr,
                    float tau, unsigned seed, float *loss_out, void *stream)
{
    t_err.clear();
    if (!m || !X || !t || n < 1 || epochs < 1 || batch < 1 || !(lr > 0.0f) || !(tau > 0.0f && tau < 1.0f))
        return fail(RSGDF_EINVAL, "bad argument");
    cudaStream_t st = (cudaStream_t)stream;
    Scratch S(st);
    int *didx;
    float *dl;
    RC(S.alloc(didx, (size_t)n));
    RC(S.alloc(dl, 1));
    std::vector<int> idx((size_t)n);
    for (long long i = 0; i < n; i++) idx[i] = (int)i;
    unsigned long long state = 0x9E3779B97F4A7C15ULL ^ seed;
    auto rnd = [&]() {   // splitmix64
        state += 0x9E3779B97F4A7C15ULL;
        unsigned long long z = state;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
        return z ^ (z >> 31);
    };
    float last = 0.0f;
    for (int ep = 0; ep < epochs; ep++) {
        for (long long i = n - 1; i > 0; i--) std::swap(idx[i], idx[rnd() % (unsigned long long)(i + 1)]);
        CU(cudaMemcpyAsync(didx, idx.data(), sizeof(int) * n, cudaMemcpyHostToDevice, st));
        CU(cudaMemsetAsync(dl, 0, sizeof(float), st));
        for (long long b0 = 0; b0 < n; b0 += batch) {
            const long long nb = std::min<long long>(batch, n - b0);
            RC(launch_mlp_fwd_bwd(m->F, m->P16, m->mean, m->stdv, X, t, didx + b0, nb, 1.0f / (float)nb, tau, m->G, dl,
                                  st));
            m->step++;
            RC(launch_mlp_adam(m->np, m->P, m->P16, m->G, m->m, m->v, lr, m->step, st));
        }
        if (ep == epochs - 1) {
            float h = 0.0f;
            CU(cudaMemcpyAsync(&h, dl, sizeof(float), cudaMemcpyDeviceToHost, st));
            CU(cudaStreamSynchronize(st));
            last = h / (float)((n + batch - 1) / batch);
        }
    }
    if (loss_out) *loss_out = last;
    return RSGDF_OK;
}

int rsgdf_sr_items(const rsgdf_cell *cell, const rsgdf_basis *ao_in, const rsgdf_basis *aux_in, const rsgdf_opts *opts,
                   int s0, int s1, long long *n_items, float *feat_out, float *mag_out)
{
    t_err.clear();
    RC(check_opts(opts));
    if (!n_items) return fail(RSGDF_EINVAL, "n_items is NULL");
    Lattice L;
    HBasis ao, ax;
    RC(make_lattice(cell, L, t_err));
    RC(load_basis(ao_in, ao, t_err));
    RC(load_basis(aux_in, ax, t_err));
    if (s0 < 0 || s1 > ax.nshell || s0 >= s1) return fail(RSGDF_EINVAL, "aux shell range is empty or out of bounds");
    double omega;
    int gm[3];
    RC(derive_params(L, opts, omega, gm, t_err));
    SRPlan plan;
    plan_sr3c(L, ao, ax, s0, s1, omega, opts->eps_screen, plan);
    *n_items = plan.n_items;
    if (!feat_out && !mag_out) return RSGDF_OK;
    RC(check_device());
    cudaStream_t st = (cudaStream_t)opts->stream;
    RC(ensure_boys(st));
    t_timer.reset(st);
    Scratch S(st);
    DevShells dao, dax;
    RC(upload_shells(S, ao, dao));
    RC(upload_shells(S, ax, dax));
    const int nao = ao.nfunc, pfunc0 = ax.foff[s0];
    const int nP = (s1 < ax.nshell ? ax.foff[s1] : ax.nfunc) - pfunc0;
    const long long m = (long long)nP * nao * nao;
    double *X = nullptr;
    if (mag_out) {
        RC(S.alloc(X, (size_t)L.Nk * L.Nk * m));
        CU(cudaMemsetAsync(X, 0, sizeof(double) * L.Nk * L.Nk * m, st));
    }
    int nl = 0;
    SRExtras ex;
    ex.feat_out = feat_out;
    ex.mag_out = mag_out;
    ex.skip_sr = (mag_out == nullptr);
    RC(run_sr(S, L, plan, dao, dax, ao, ax, omega, X, (long long)L.Nk * m, m, (long long)nao * nao, nao, 1, pfunc0,
              nullptr, st, nl, ex));
    CU(cudaGetLastError());
    return RSGDF_OK;
}

int rsgdf_last_stats(rsgdf_stats *out)
{
    if (!out) return fail(RSGDF_EINVAL, "out is NULL");
    if (t_count_valid) {
        if (cudaStreamSynchronize(t_stats_stream) != cudaSuccess) return fail(RSGDF_EDEVICE, "stream sync failed");
        t_stats.sr_terms = 0;
        t_stats.sr_flops = 0;
        t_stats.sr_prim_terms = 0;
        for (int L = 0; L <= LTOT_MAX; L++) {
            t_stats.sr_terms += (long long)t_count_host[L];
            // the Hermite work is done per primitive combination of a term
            t_stats.sr_flops += (long long)t_count_host[LTOT_MAX + 2 + L] * sr_term_flops(L);
            t_stats.sr_prim_terms += (long long)t_count_host[LTOT_MAX + 2 + L];
        }
        t_stats.sr_integrals = (long long)t_count_host[LTOT_MAX + 1];
        t_stats.sr_items_pruned = (long long)t_count_host[2 * LTOT_MAX + 4];
        t_stats.sr_prim_terms_skipped = (long long)t_count_host[2 * LTOT_MAX + 5];
        double ms[PH_N];
        t_timer.totals(ms, t_stats.sr_ms_by_L);
        for (int L = 0; L <= LTOT_MAX; L++) {
            t_stats.sr_terms_by_L[L] = (long long)t_count_host[L];
            t_stats.sr_prim_terms_by_L[L] = (long long)t_count_host[LTOT_MAX + 2 + L];
        }
        t_stats.sr_ms = ms[PH_SR];
        t_stats.aft_ms = ms[PH_AFT];
        t_stats.lr_gemm_ms = ms[PH_GEMM];
        t_stats.phase_ms = ms[PH_PHASE];
        t_stats.other_ms = ms[PH_OTHER];
    }
    *out = t_stats;
    return RSGDF_OK;
}

int rsgdf_set_scratch_limit(long long bytes)
{
    if (bytes < 0) return fail(RSGDF_EINVAL, "the scratch limit must be >= 0 (0: no limit)");
    g_scratch_limit.store(bytes);
    return RSGDF_OK;
}

int rsgdf_selftest_wait(int arrive, long long limit, void *stream)
{
    t_err.clear();
    if (limit < 1) return fail(RSGDF_EINVAL, "limit must be >= 1");
    RC(check_device());
    RC(launch_wait_selftest(arrive, limit, (cudaStream_t)stream));
    return RSGDF_OK;
}

int rsgdf_sync_status(void *stream)
{
    t_err.clear();
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return fail(RSGDF_EDEVICE, "stream sync failed");
    int flag = 0;
    RC(tc_status_take(&flag));
    if (flag) return fail(RSGDF_ETIMEOUT, "a bounded device wait gave up; results of that call are invalid");
    return RSGDF_OK;
}

int rsgdf_params(const rsgdf_cell *cell, const rsgdf_opts *opts, double *omega_out, int *gmesh_out)
{
    t_err.clear();
    if (!opts || !omega_out || !gmesh_out) return fail(RSGDF_EINVAL, "NULL argument");
    Lattice L;
    RC(make_lattice(cell, L, t_err));
    double w;
    int g[3];
    RC(derive_params(L, opts, w, g, t_err));
    *omega_out = w;
    for (int i = 0; i < 3; i++) gmesh_out[i] = g[i];
    return RSGDF_OK;
}

const char *rsgdf_last_error(void) { return t_err.c_str(); }

int rsgdf_probe_fp64(double *tflops_out, void *stream)
{
    t_err.clear();
    if (!tflops_out) return fail(RSGDF_EINVAL, "NULL argument");
    RC(check_device());
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    Scratch S(st);
    double *buf;
    RC(S.alloc(buf, (size_t)nsm * 8 * 256));
    const int iters = 2000;
    RC(launch_probe_fp64(buf, iters, st));
    cudaEvent_t e0, e1;
    CU(cudaEventCreate(&e0));
    CU(cudaEventCreate(&e1));
    float best = 1e30f;
    for (int rep = 0; rep < 3; rep++) {
        CU(cudaEventRecord(e0, st));
        RC(launch_probe_fp64(buf, iters, st));
        CU(cudaEventRecord(e1, st));
        CU(cudaEventSynchronize(e1));
        float ms = 0;
        CU(cudaEventElapsedTime(&ms, e0, e1));
        best = std::min(best, ms);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    double flops = 2.0 * 8 * iters * (double)nsm * 8 * 256;
    *tflops_out = flops / (best * 1e-3) / 1e12;
    return RSGDF_OK;
}

// ---------------------------------------------------------------------------
// Density-fitting consumers (Eq. DF_eqn, Eq. ERI_aux)
// ---------------------------------------------------------------------------
static bool ranges_overlap(const void *a, const void *b, size_t bytes)
{
    const char *x = (const char *)a, *y = (const char *)b;
    return x < y + bytes && y < x + bytes;
}

int rsgdf_df_metric(const double *J, int naux, int nk, int method, double rel, double *T_out, double *lam_out,
                    int *nkept_out, int *info_out, void *stream)
{
    static_assert(RSGDF_DF_NMAX == DF_NMAX && RSGDF_DF_SWEEPS == DF_JACOBI_SWEEPS, "DF limits out of step");
    t_err.clear();
    if (!J || !T_out) return fail(RSGDF_EINVAL, "J and T_out are required");
    if (naux < 1 || naux > RSGDF_DF_NMAX) return fail(RSGDF_EINVAL, "naux outside 1..RSGDF_DF_NMAX");
    if (nk < 1) return fail(RSGDF_EINVAL, "need at least one k");
    if (method < RSGDF_FIT_CHOLESKY || method > RSGDF_FIT_AUTO) return fail(RSGDF_EINVAL, "unknown fitting method");
    if (!(rel >= 0.0 && rel < 1.0)) return fail(RSGDF_EINVAL, "rel outside [0, 1)");
    const size_t nn = (size_t)naux * naux;
    if (ranges_overlap(J, T_out, 16 * nn * nk)) return fail(RSGDF_EINVAL, "T_out overlaps J");
    RC(check_device());
    cudaStream_t st = (cudaStream_t)stream;
    Scratch S(st);
    int *info = info_out;
    if (!info) RC(S.alloc(info, nk));
    double *lam = lam_out;
    if (!lam) RC(S.alloc(lam, (size_t)naux * nk));
    CU(cudaMemsetAsync(lam, 0, sizeof(double) * naux * nk, st));
    if (method != RSGDF_FIT_EIGEN) {
        double *Lf;
        int *cinfo;
        RC(S.alloc(Lf, 2 * nn * nk));
        RC(S.alloc(cinfo, nk));
        RC(launch_cholesky(naux, nk, J, Lf, cinfo, st));
        RC(launch_df_cholesky_route(naux, nk, J, Lf, cinfo, rel, T_out, info, nkept_out, st));
    }
    if (method != RSGDF_FIT_CHOLESKY) {
        double *A, *U;
        int *order;
        RC(S.alloc(A, 2 * nn * nk));
        RC(S.alloc(U, 2 * nn * nk));
        RC(S.alloc(order, (size_t)naux * nk));
        RC(launch_df_eigen_route(naux, nk, J, method == RSGDF_FIT_AUTO ? info : nullptr, rel, A, U, lam, order, T_out,
                                 info, nkept_out, st));
    }
    CU(cudaGetLastError());
    return RSGDF_OK;
}

static int df_pairs(const rsgdf_cell *cell, int npair, const int *kpairs, Lattice &L, bool unique)
{
    RC(make_lattice(cell, L, t_err));
    if (npair < 1 || !kpairs) return fail(RSGDF_EINVAL, "need at least one k pair");
    for (int i = 0; i < 2 * npair; i++)
        if (kpairs[i] < 0 || kpairs[i] >= L.Nk) return fail(RSGDF_EINVAL, "k index outside the mesh");
    if (unique) {
        std::set<std::pair<int, int>> seen;
        for (int p = 0; p < npair; p++)
            if (!seen.insert({kpairs[2 * p], kpairs[2 * p + 1]}).second)
                return fail(RSGDF_EINVAL, "a k pair is listed twice");
    }
    return RSGDF_OK;
}

static int upload_offsets(Scratch &S, const std::vector<long long> &a, const std::vector<long long> &b,
                          const std::vector<long long> &c, ZGemmGen &g)
{
    long long *da, *db, *dc;
    RC(S.upload(da, a));
    RC(S.upload(db, b));
    RC(S.upload(dc, c));
    g.aoff = da;
    g.boff = db;
    g.coff = dc;
    return RSGDF_OK;
}

int rsgdf_df_fit(const rsgdf_cell *cell, const double *T, int naux, int nao, int npair, const int *kpairs,
                 const double *V, double *B_out, void *stream)
{
    t_err.clear();
    Lattice L;
    RC(df_pairs(cell, npair, kpairs, L, false));
    if (!T || !V || !B_out) return fail(RSGDF_EINVAL, "T, V and B_out are required");
    if (naux < 1 || nao < 1) return fail(RSGDF_EINVAL, "naux and nao must be >= 1");
    const long long n2 = (long long)nao * nao, blk = (long long)naux * n2;
    if (ranges_overlap(V, B_out, (size_t)16 * blk * npair)) return fail(RSGDF_EINVAL, "B_out overlaps V");
    RC(check_device());
    cudaStream_t st = (cudaStream_t)stream;
    Scratch S(st);
    std::vector<long long> ao(npair), bo(npair), co(npair);
    for (int p = 0; p < npair; p++) {
        ao[p] = (long long)k12_of(L, kpairs[2 * p], kpairs[2 * p + 1]) * naux * naux;
        bo[p] = co[p] = p * blk;
    }
    // B[p](r, x) = sum_P T[k12](r, P) V[p](P, x)
    ZGemmGen g{};
    g.M = naux;
    g.N = (int)n2;
    g.Q = 1;
    g.S = naux;
    g.lda = naux;
    g.as = 1;
    g.bs = n2;
    g.bn = 1;
    g.ldc = n2;
    g.alpha = 1.0;
    RC(upload_offsets(S, ao, bo, co, g));
    RC(launch_zgemm_gen(g, npair, T, V, B_out, st));
    CU(cudaGetLastError());
    return RSGDF_OK;
}

// rho(P) = sum over the diagonal pairs of sum_{mu, nu} B[p](P, mu, nu) D[k](nu, mu); overwrites rho
static int df_rho_launch(Scratch &S, const double *B, const double *D, int naux, int nao, int npair, const int *kpairs,
                         double *rho, cudaStream_t st)
{
    const long long n2 = (long long)nao * nao, blk = (long long)naux * n2;
    CU(cudaMemsetAsync(rho, 0, sizeof(double) * 2 * naux, st));
    std::vector<long long> pa, pb, pc;
    for (int p = 0; p < npair; p++)
        if (kpairs[2 * p] == kpairs[2 * p + 1]) {
            pa.push_back(p * blk);
            pb.push_back(kpairs[2 * p] * n2);
            pc.push_back(0);
        }
    if (pa.empty()) return RSGDF_OK;
    ZGemmGen g{};
    g.M = naux;
    g.N = 1;
    g.Q = nao;
    g.S = nao;
    g.lda = n2;
    g.aq = nao;
    g.as = 1;
    g.bq = 1;
    g.bs = nao;
    g.ldc = 1;
    g.atomic = 1;
    g.alpha = 1.0;
    RC(upload_offsets(S, pa, pb, pc, g));
    return launch_zgemm_gen(g, (int)pa.size(), B, D, rho, st);
}

int rsgdf_df_rho(const rsgdf_cell *cell, const double *B, int naux, int nao, int npair, const int *kpairs,
                 const double *D, double *rho_out, void *stream)
{
    t_err.clear();
    Lattice L;
    RC(df_pairs(cell, npair, kpairs, L, true));
    if (!B || !D || !rho_out) return fail(RSGDF_EINVAL, "B, D and rho_out are required");
    if (naux < 1 || nao < 1) return fail(RSGDF_EINVAL, "naux and nao must be >= 1");
    RC(check_device());
    cudaStream_t st = (cudaStream_t)stream;
    Scratch S(st);
    RC(df_rho_launch(S, B, D, naux, nao, npair, kpairs, rho_out, st));
    CU(cudaGetLastError());
    return RSGDF_OK;
}

int rsgdf_df_jk(const rsgdf_cell *cell, const double *B, int naux, int nao, int npair, const int *kpairs,
                const double *D, const double *rho_in, double *J_out, double *K_out, void *stream)
{
    t_err.clear();
    Lattice L;
    RC(df_pairs(cell, npair, kpairs, L, true));
    if (!B || !D) return fail(RSGDF_EINVAL, "B and D are required");
    if (!J_out && !K_out) return fail(RSGDF_EINVAL, "J_out and K_out are both NULL");
    if (naux < 1 || nao < 1) return fail(RSGDF_EINVAL, "naux and nao must be >= 1");
    RC(check_device());
    cudaStream_t st = (cudaStream_t)stream;
    Scratch S(st);
    const int Nk = L.Nk;
    const long long n2 = (long long)nao * nao, blk = (long long)naux * n2;
    if (J_out) {
        CU(cudaMemsetAsync(J_out, 0, sizeof(double) * 2 * Nk * n2, st));
        std::vector<long long> ja, jb, jc;
        for (int p = 0; p < npair; p++)
            if (kpairs[2 * p] == kpairs[2 * p + 1]) {
                ja.push_back(p * blk);
                jb.push_back(0);
                jc.push_back(kpairs[2 * p] * n2);
            }
        if (!ja.empty()) {
            const double *rho = rho_in;
            if (!rho) {
                double *r;
                RC(S.alloc(r, 2 * (size_t)naux));
                RC(df_rho_launch(S, B, D, naux, nao, npair, kpairs, r, st));
                rho = r;
            }
            // J[k](x) = (1/Nk) sum_P B[p](P, x) conj(rho(P))
            ZGemmGen h{};
            h.M = (int)n2;
            h.N = 1;
            h.Q = 1;
            h.S = naux;
            h.lda = 1;
            h.as = n2;
            h.bs = 1;
            h.ldc = 1;
            h.conjB = 1;
            h.alpha = 1.0 / Nk;
            RC(upload_offsets(S, ja, jb, jc, h));
            RC(launch_zgemm_gen(h, (int)ja.size(), B, rho, J_out, st));
        }
    }
    if (K_out) {
        CU(cudaMemsetAsync(K_out, 0, sizeof(double) * 2 * Nk * n2, st));
        const long long budget = 4LL << 30;
        const int cp = (int)std::max(1LL, std::min<long long>(npair, budget / (16 * blk)));
        double *Y;
        RC(S.alloc(Y, (size_t)2 * blk * cp));
        for (int c0 = 0; c0 < npair; c0 += cp) {
            const int nc = std::min(cp, npair - c0);
            std::vector<long long> a1(nc), b1(nc), c1(nc), a2(nc), b2(nc), c2(nc);
            for (int b = 0; b < nc; b++) {
                const int p = c0 + b;
                a1[b] = p * blk;
                b1[b] = kpairs[2 * p + 1] * n2;
                c1[b] = b * blk;
                a2[b] = b * blk;
                b2[b] = p * blk;
                c2[b] = kpairs[2 * p] * n2;
            }
            // Y[b]((P, mu), s) = sum_l B[p]((P, mu), l) D[k2](l, s)
            ZGemmGen g{};
            g.M = naux * nao;
            g.N = nao;
            g.Q = 1;
            g.S = nao;
            g.lda = nao;
            g.as = 1;
            g.bs = nao;
            g.bn = 1;
            g.ldc = nao;
            g.alpha = 1.0;
            RC(upload_offsets(S, a1, b1, c1, g));
            RC(launch_zgemm_gen(g, nc, B, D, Y, st));
            // K[k1](mu, nu) += (1/Nk) sum_{P, s} Y[b](P, mu, s) conj(B[p](P, nu, s))
            ZGemmGen h{};
            h.M = nao;
            h.N = nao;
            h.Q = naux;
            h.S = nao;
            h.lda = nao;
            h.aq = n2;
            h.as = 1;
            h.bq = n2;
            h.bs = 1;
            h.bn = nao;
            h.ldc = nao;
            h.conjB = 1;
            h.atomic = 1;
            h.alpha = 1.0 / Nk;
            RC(upload_offsets(S, a2, b2, c2, h));
            RC(launch_zgemm_gen(h, nc, Y, B, K_out, st));
        }
    }
    CU(cudaGetLastError());
    return RSGDF_OK;
}

// ---------------------------------------------------------------------------
// Cartesian -> real solid harmonic transforms
// ---------------------------------------------------------------------------
int rsgdf_sph_coefficients(int l, double *s_out)
{
    t_err.clear();
    if (l < 0 || l > RSGDF_LMAX) return fail(RSGDF_EINVAL, "l outside 0..RSGDF_LMAX");
    if (!s_out) return fail(RSGDF_EINVAL, "s_out is NULL");
    std::vector<double> s;
    sph_coefficients(l, s);
    std::copy(s.begin(), s.end(), s_out);
    return RSGDF_OK;
}

int rsgdf_sph_nfunc(const rsgdf_basis *b, int *nsph_out)
{
    t_err.clear();
    HBasis h;
    RC(load_basis(b, h, t_err));
    if (!nsph_out) return fail(RSGDF_EINVAL, "nsph_out is NULL");
    int n = 0;
    for (int l : h.l) n += 2 * l + 1;
    *nsph_out = n;
    return RSGDF_OK;
}

static int upload_sph_map(Scratch &S, const std::vector<int> &ls, SphMapDev &m, int &nsph, int &ncart)
{
    std::vector<int> off, idx;
    std::vector<double> coef;
    sph_map(ls, off, idx, coef);
    nsph = (int)off.size() - 1;
    ncart = 0;
    for (int l : ls) ncart += (l + 1) * (l + 2) / 2;
    int *doff, *didx;
    double *dcoef;
    RC(S.upload(doff, off));
    RC(S.upload(didx, idx));
    RC(S.upload(dcoef, coef));
    m.off = doff;
    m.idx = didx;
    m.coef = dcoef;
    return RSGDF_OK;
}

int rsgdf_cart2sph_j3c(const rsgdf_basis *ao_in, const rsgdf_basis *aux_in, int s0, int s1, int npair,
                       const double *V_cart, double *V_sph, void *stream)
{
    t_err.clear();
    HBasis ao, ax;
    RC(load_basis(ao_in, ao, t_err));
    RC(load_basis(aux_in, ax, t_err));
    if (s0 < 0 || s1 > ax.nshell || s0 >= s1) return fail(RSGDF_EINVAL, "aux shell range outside the basis");
    if (npair < 1) return fail(RSGDF_EINVAL, "need at least one k pair");
    if (!V_cart || !V_sph) return fail(RSGDF_EINVAL, "V_cart and V_sph are required");
    const std::vector<int> lx(ax.l.begin() + s0, ax.l.begin() + s1);
    int ncx = 0, nsx = 0;
    for (int l : lx) {
        ncx += (l + 1) * (l + 2) / 2;
        nsx += 2 * l + 1;
    }
    int nsa = 0;
    for (int l : ao.l) nsa += 2 * l + 1;
    const size_t in_bytes = (size_t)16 * npair * ncx * ao.nfunc * ao.nfunc;
    const size_t out_bytes = (size_t)16 * npair * nsx * nsa * nsa;
    const char *a = (const char *)V_cart, *b = (const char *)V_sph;
    if (a < b + out_bytes && b < a + in_bytes) return fail(RSGDF_EINVAL, "V_sph overlaps V_cart");
    RC(check_device());
    cudaStream_t st = (cudaStream_t)stream;
    Scratch S(st);
    SphMapDev mx, ma;
    int nsph_x, ncart_x, nsph_a, ncart_a;
    RC(upload_sph_map(S, lx, mx, nsph_x, ncart_x));
    RC(upload_sph_map(S, ao.l, ma, nsph_a, ncart_a));
    RC(launch_cart2sph(V_cart, V_sph, npair, nsph_x, nsph_a, nsph_a, ncart_x, ncart_a, ncart_a, mx, ma, ma, st));
    CU(cudaGetLastError());
    return RSGDF_OK;
}

int rsgdf_cart2sph_j2c(const rsgdf_basis *aux_in, int nk, const double *J_cart, double *J_sph, void *stream)
{
    t_err.clear();
    HBasis ax;
    RC(load_basis(aux_in, ax, t_err));
    if (nk < 1) return fail(RSGDF_EINVAL, "need at least one k");
    if (!J_cart || !J_sph) return fail(RSGDF_EINVAL, "J_cart and J_sph are required");
    int ns = 0;
    for (int l : ax.l) ns += 2 * l + 1;
    const size_t in_bytes = (size_t)16 * nk * ax.nfunc * ax.nfunc, out_bytes = (size_t)16 * nk * ns * ns;
    const char *a = (const char *)J_cart, *b = (const char *)J_sph;
    if (a < b + out_bytes && b < a + in_bytes) return fail(RSGDF_EINVAL, "J_sph overlaps J_cart");
    RC(check_device());
    cudaStream_t st = (cudaStream_t)stream;
    Scratch S(st);
    SphMapDev mx, one;
    int nsph_x, ncart_x, n1, c1;
    RC(upload_sph_map(S, ax.l, mx, nsph_x, ncart_x));
    RC(upload_sph_map(S, std::vector<int>{0}, one, n1, c1));   // identity on a trailing unit index
    RC(launch_cart2sph(J_cart, J_sph, nk, nsph_x, nsph_x, 1, ncart_x, ncart_x, 1, mx, mx, one, st));
    CU(cudaGetLastError());
    return RSGDF_OK;
}

// ---------------------------------------------------------------------------
// Compact/diffuse split (host only)
// ---------------------------------------------------------------------------
int rsgdf_split_basis(const rsgdf_basis *b, double alpha_cut, int *nshell_out, int *nprim_total_out, int *l_out,
                      int *nprim_out, int *prim_off_out, double *center_out, double *exps_out, double *coeffs_out,
                      int *parent_out, int *kind_out, double *weight_out)
{
    t_err.clear();
    if (!nshell_out || !nprim_total_out) return fail(RSGDF_EINVAL, "nshell_out and nprim_total_out are required");
    SplitBasis sb;
    RC(split_basis(b, alpha_cut, sb, t_err));
    *nshell_out = (int)sb.l.size();
    *nprim_total_out = (int)sb.exps.size();
    auto put = [](auto *dst, const auto &v) {
        if (dst) std::copy(v.begin(), v.end(), dst);
    };
    put(l_out, sb.l);
    put(nprim_out, sb.nprim);
    put(prim_off_out, sb.prim_off);
    put(center_out, sb.center);
    put(exps_out, sb.exps);
    put(coeffs_out, sb.coeffs);
    put(parent_out, sb.parent);
    put(kind_out, sb.kind);
    put(weight_out, sb.weight);
    return RSGDF_OK;
}

int rsgdf_sr_items_split(const rsgdf_cell *cell, const rsgdf_basis *ao_in, const rsgdf_basis *aux_in,
                         const rsgdf_opts *opts, double alpha_cut, long long *n_items_out)
{
    t_err.clear();
    RC(check_opts(opts));
    if (!n_items_out) return fail(RSGDF_EINVAL, "n_items_out is NULL");
    Lattice L;
    HBasis ao, ax;
    RC(make_lattice(cell, L, t_err));
    RC(load_basis(ao_in, ao, t_err));
    RC(load_basis(aux_in, ax, t_err));
    double omega;
    int gm[3];
    RC(derive_params(L, opts, omega, gm, t_err));
    SplitBasis sa, sx;
    RC(split_basis(ao_in, alpha_cut, sa, t_err));
    RC(split_basis(aux_in, alpha_cut, sx, t_err));
    const rsgdf_basis va = sa.view(), vx = sx.view();
    HBasis hsa, hsx;
    RC(load_basis(&va, hsa, t_err));
    RC(load_basis(&vx, hsx, t_err));
    SRPlan p0, p1, p2;
    plan_sr3c(L, ao, ax, 0, ax.nshell, omega, opts->eps_screen, p0);
    plan_sr3c(L, hsa, hsx, 0, hsx.nshell, omega, opts->eps_screen, p1);
    // range-separated types only: compact aux function, pair not both diffuse
    plan_sr3c(L, hsa, hsx, 0, hsx.nshell, omega, opts->eps_screen, p2, [&](int P, int mu, int nu) {
        return sx.kind[P] == 0 && !(sa.kind[mu] == 1 && sa.kind[nu] == 1);
    });
    // candidate primitive terms: d items x aux images within the triple's
    // Rc cutoff x primitive combinations (the kernel's per-term tests drop some)
    auto terms = [](const SRPlan &p, const HBasis &a, const HBasis &x) {
        long long t = 0;
        for (const SRTriple &tr : p.tri)
            t += (long long)tr.nd * tr.nsph * x.nprim[tr.P] * a.nprim[tr.mu] * a.nprim[tr.nu];
        return t;
    };
    n_items_out[0] = p0.n_items;
    n_items_out[1] = p1.n_items;
    n_items_out[2] = p2.n_items;
    n_items_out[3] = terms(p0, ao, ax);
    n_items_out[4] = terms(p1, hsa, hsx);
    n_items_out[5] = terms(p2, hsa, hsx);
    return RSGDF_OK;
}

// parent function -> (sub function, weight) CSR map and kind per sub function
static int upload_split_map(Scratch &S, const rsgdf_basis *b, const SplitBasis &sb, SphMapDev &m, int *&dkind,
                            int &nsub)
{
    std::vector<int> pf0(b->nshell + 1, 0);
    for (int s = 0; s < b->nshell; s++) pf0[s + 1] = pf0[s] + ncart(b->l[s]);
    std::vector<std::vector<std::pair<int, double>>> rows(pf0[b->nshell]);
    std::vector<int> kind;
    int f = 0;
    for (size_t j = 0; j < sb.l.size(); j++) {
        for (int c = 0; c < ncart(sb.l[j]); c++) {
            rows[pf0[sb.parent[j]] + c].push_back({f + c, sb.weight[j]});
            kind.push_back(sb.kind[j]);
        }
        f += ncart(sb.l[j]);
    }
    nsub = f;
    std::vector<int> off(1, 0), idx;
    std::vector<double> coef;
    for (auto &r : rows) {
        for (auto &e : r) {
            idx.push_back(e.first);
            coef.push_back(e.second);
        }
        off.push_back((int)idx.size());
    }
    int *doff, *didx;
    double *dcoef;
    RC(S.upload(doff, off));
    RC(S.upload(didx, idx));
    RC(S.upload(dcoef, coef));
    RC(S.upload(dkind, kind));
    m.off = doff;
    m.idx = didx;
    m.coef = dcoef;
    return RSGDF_OK;
}

int rsgdf_split_combine(const rsgdf_basis *ao_in, const rsgdf_basis *aux_in, double alpha_cut, int npair,
                        const double *V_rs, const double *V_g, double *V_out, void *stream)
{
    t_err.clear();
    HBasis ao, ax;
    RC(load_basis(ao_in, ao, t_err));
    RC(load_basis(aux_in, ax, t_err));
    if (npair < 1) return fail(RSGDF_EINVAL, "need at least one k pair");
    if (!V_rs || !V_g || !V_out) return fail(RSGDF_EINVAL, "V_rs, V_g and V_out are required");
    SplitBasis sa, sx;
    RC(split_basis(ao_in, alpha_cut, sa, t_err));
    RC(split_basis(aux_in, alpha_cut, sx, t_err));
    int nsa = 0, nsx = 0;
    for (int l : sa.l) nsa += ncart(l);
    for (int l : sx.l) nsx += ncart(l);
    const size_t in_bytes = (size_t)16 * npair * nsx * nsa * nsa;
    const size_t out_bytes = (size_t)16 * npair * ax.nfunc * ao.nfunc * ao.nfunc;
    auto overlap = [](const void *a, size_t na, const void *b, size_t nb) {
        const char *x = (const char *)a, *y = (const char *)b;
        return x < y + nb && y < x + na;
    };
    if (overlap(V_out, out_bytes, V_rs, in_bytes) || overlap(V_out, out_bytes, V_g, in_bytes))
        return fail(RSGDF_EINVAL, "V_out overlaps an input");
    RC(check_device());
    cudaStream_t st = (cudaStream_t)stream;
    Scratch S(st);
    SphMapDev mx, ma;
    int *kx, *ka, nx, na;
    RC(upload_split_map(S, aux_in, sx, mx, kx, nx));
    RC(upload_split_map(S, ao_in, sa, ma, ka, na));
    RC(launch_split_combine(V_rs, V_g, V_out, npair, ax.nfunc, ao.nfunc, nx, na, mx, ma, kx, ka, st));
    CU(cudaGetLastError());
    return RSGDF_OK;
}

}  // extern "C"
